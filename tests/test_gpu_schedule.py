"""Transform schedules of the fused 2D path (vofl_set_schedule): every
schedule computes the same operators of Eq. (2.13) within the FP32
tolerance of the FP64 oracle; the defaults per grid size are reported; a
context off its size's default schedule cannot join a batch (its bits would
differ from the batched launches')."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_util import check, gamma_of

pytestmark = pytest.mark.gpu

TOL32 = 1e-5

# (wide_cols, wide_rows, col_parts, group, fuse_forward, wide_fwd,
# row_split, col_pack): -1 / 0 = the size's default
SCHEDULES = [(-1, -1, 0, 0, -1, -1, 0, -1), (0, 0, 0, 0, 0, 0, 0, 0), (1, 1, 0, 0, -1, 1, 0, 0),
             (1, 0, 2, 6, 1, 0, 0, 0), (0, 1, 1, 3, 1, 1, 0, 0), (-1, -1, 6, 17, 0, 0, 0, 0),
             (-1, -1, 3, 4, 1, -1, 0, 0), (0, 0, 1, 1, 1, 0, 0, 0), (0, 0, 2, 17, 1, 1, 0, 0),
             # the column pass's terms dealt out over K CTAs: one CTA, a
             # wave, more CTAs than slots, several groups, the forward
             # column transform in the same kernel, wide columns
             (0, -1, 0, 0, 0, -1, 0, 1), (0, -1, 0, 0, 0, -1, 0, 152), (0, -1, 0, 0, 0, -1, 0, 5000),
             (0, -1, 0, 5, 0, -1, 0, 37), (0, -1, 0, 0, 1, -1, 0, 152), (0, -1, 0, 6, 1, -1, 0, 300),
             (1, -1, 0, 0, -1, -1, 0, 152), (1, -1, 0, 4, -1, -1, 0, 61),
             # both forward passes in one cooperative launch
             (0, -1, 0, 0, 2, 0, 0, -1), (1, 1, 0, 5, 2, -1, 0, 0), (0, 0, 3, 17, 2, 1, 0, 152)]


@pytest.mark.parametrize("n", [512, 1024])
def test_every_schedule_matches_the_oracle(V, n):
    import torch
    shape = (n, n)
    Q = S.q_lowpass(shape, 31)
    u = S.q_lowpass(shape, 32, qmin=-1.0, qmax=1.0, sigma_k=n // 8).astype(np.float32)
    M = 16
    r1, r2 = O.seismic_operators(u.astype(np.float64), gamma_of(Q), M)
    with V.Solver(shape) as s:
        s.set_q(Q)
        s.set_M(M)
        ut = torch.from_numpy(u).cuda()
        for sc in SCHEDULES:
            s.set_schedule(*sc)
            got = s.schedule()
            if sc[2] > 0:
                assert got["col_parts"] == sc[2]
            if sc[3] > 0:
                assert got["group"] == sc[3]
            if sc[7] >= 0:
                assert got["col_pack"] == sc[7]
            o1, o2 = torch.empty_like(ut), torch.empty_like(ut)
            s.apply_pair(ut, o1, o2)
            s.sync()
            check(o1.cpu().numpy(), r1, TOL32, sc)
            check(o2.cpu().numpy(), r2, TOL32, sc)


def test_default_schedules(V):
    import torch
    base = {"group": 17, "wide_cols": 0, "wide_rows": 0, "fuse_forward": 2, "wide_fwd": 0, "row_split": 1}
    want = {256: dict(base, col_parts=3, fuse_forward=1, row_split=4),
            512: dict(base, col_parts=6, wide_cols=1, wide_rows=1),
            768: dict(base, col_parts=1),
            1024: dict(base, col_parts=1, wide_rows=1)}
    for n, w in want.items():
        with V.Solver((n, n)) as s:
            got = s.schedule()
            # the column pass's terms over one CTA per SM at 512, two at 768
            pack = got.pop("col_pack")
            sms = torch.cuda.get_device_properties(0).multi_processor_count
            assert pack == {256: 0, 512: sms, 768: 2 * sms, 1024: 0}[n], (n, pack)
            assert got == w, (n, got)
            s.set_schedule(1, 1, 2, 5, 0, 0, 0, 7)
            s.set_schedule()  # back to the defaults
            assert s.schedule() == dict(w, col_pack=pack)


def test_schedule_runs_agree_and_batch_needs_one_schedule_per_size(V):
    """20 leap-frog steps on two schedules agree within the run tolerance;
    the first member of a grid size sets the batch's schedule for the size,
    and a context of that size on another schedule is refused."""
    shape = (512, 512)
    Q = S.q_lowpass(shape, 5)
    src = S.ricker_samples(20, 5e-4, 10.0)

    def run(sched):
        with V.Solver(shape) as s:
            s.set_q(Q)
            s.set_M(12)
            if sched:
                s.set_schedule(*sched)
            s.set_state(np.zeros(shape, np.float32))
            s.set_source(S.center_index(shape), src)
            s.step(20, 5e-4)
            return s.get_state().astype(np.float64)

    a = run(None)
    b = run((0, 0, 1, 4, 1))
    check(b, a, 1e-4)
    with V.Solver(shape) as s, V.Solver(shape) as s2, V.Batch() as bt:
        for x in (s, s2):
            x.set_q(Q)
            x.set_M(12)
            x.set_state(np.zeros(shape, np.float32))
        s.set_schedule(0, 0, 1, 4, 1)
        bt.add(s, 5e-4)  # the size's first member: its schedule is the batch's
        assert bt.transform(shape[0])["group"] == 4
        with pytest.raises(V.VoflError):
            bt.add(s2, 5e-4)  # the default schedule differs
        s2.set_schedule(0, 0, 1, 4, 1)
        bt.add(s2, 5e-4)
        bt.step(2)
        bt.sync()


def test_fused_forward_is_bit_identical(V):
    """The forward column transform inside the column kernel, and both
    forward passes in one cooperative launch, are the same arithmetic as
    the separate forward kernels: same bits, any grid (also over a run of
    steps, whose step counter the cooperative launch advances)."""
    import torch
    for shape in [(256, 256), (1024, 1024), (768, 768), (128, 256), (512, 512), (512, 64)]:
        Q = S.q_lowpass(shape, 41)
        u = S.q_lowpass(shape, 42, qmin=-1.0, qmax=1.0, sigma_k=16).astype(np.float32)
        outs, runs = [], []
        with V.Solver(shape) as s:
            s.set_q(Q)
            s.set_M(16)
            ut = torch.from_numpy(u).cuda()
            for ff in (0, 1, 2):
                s.set_schedule(0, -1, 0, 0, ff, 0)
                assert s.schedule()["fuse_forward"] == ff, (shape, ff, s.schedule())
                o1, o2 = torch.empty_like(ut), torch.empty_like(ut)
                s.apply_pair(ut, o1, o2)
                s.sync()
                outs.append((o1.cpu().numpy(), o2.cpu().numpy()))
                s.set_state(np.zeros(shape, np.float32))
                s.set_source(S.center_index(shape), S.ricker_samples(12, 5e-4, 10.0))
                s.step(12, 5e-4)
                runs.append(s.get_state())
        for o, r in zip(outs[1:], runs[1:]):
            assert np.array_equal(outs[0][0], o[0]) and np.array_equal(outs[0][1], o[1]), shape
            assert np.array_equal(runs[0], r), shape


@pytest.mark.parametrize("shape", [(256, 256), (128, 128), (64, 64), (128, 256)])
def test_row_split_matches_the_oracle(V, shape):
    """Rows whose terms are split over 1, 2 or 4 warps (partial Horner sums
    joined by Horner's rule), one or more Taylor groups, the seismic pair
    and the general model's one operator: all within the FP32 tolerance."""
    import torch
    Q = S.q_lowpass(shape, 51)
    u = S.q_lowpass(shape, 52, qmin=-1.0, qmax=1.0, sigma_k=16).astype(np.float32)
    M = 16
    r1, r2 = O.seismic_operators(u.astype(np.float64), gamma_of(Q), M)
    x, y = S.mesh(shape)
    order = 1.0 - 0.3 * np.cos(x) * np.sin(y)
    ro = O.matrix_free_operator(u.astype(np.float64), order, M)
    ut = torch.from_numpy(u).cuda()
    for rs in (1, 2, 4):
        for G in (0, 5):
            with V.Solver(shape) as s:
                s.set_q(Q)
                s.set_M(M)
                s.set_schedule(-1, -1, 0, G, -1, -1, rs)
                assert s.schedule()["row_split"] == rs
                o1, o2 = torch.empty_like(ut), torch.empty_like(ut)
                s.apply_pair(ut, o1, o2)
                s.sync()
                check(o1.cpu().numpy(), r1, TOL32, (shape, rs, G))
                check(o2.cpu().numpy(), r2, TOL32, (shape, rs, G))
                s.set_order(order)
                o = torch.empty_like(ut)
                s.apply(V.OP_S, ut, o)
                s.sync()
                check(o.cpu().numpy(), ro, TOL32, (shape, rs, G, "general"))


def test_batch_transform_tuning_keeps_members_equal_to_solo(V):
    """vofl_batch_tune_transform: every member takes its size's tuned
    schedule, and stepping on gives the bits of a context stepped alone on
    that schedule, within the run tolerance of the default-schedule run."""
    import synthetic as Sy
    specs = [(256, 70 + i) for i in range(3)] + [(512, 80 + i) for i in range(2)]
    nsteps, dt = 12, 5e-4

    def make(n, seed):
        s = V.Solver((n, n))
        s.set_q(Sy.q_lowpass((n, n), seed))
        s.set_M(12)
        s.set_state(np.zeros((n, n), np.float32))
        s.set_source(Sy.center_index((n, n)), Sy.ricker_samples(nsteps, dt, 10.0))
        return s

    members = [make(n, seed) for n, seed in specs]
    with V.Batch() as b:
        slots = [b.add(s, dt) for s in members]
        ms = b.tune_transform(reps=1)
        assert ms > 0
        for s, (n, _) in zip(members, specs):
            assert s.schedule() == dict(b.transform(n), fuse_forward=s.schedule()["fuse_forward"])
        b.step(nsteps)
        for slot in slots:
            b.remove(slot)
    for s, (n, seed) in zip(members, specs):
        got = s.get_state().astype(np.float64)
        sc = s.schedule()
        solo = make(n, seed)
        solo.set_schedule(sc["wide_cols"], sc["wide_rows"], sc["col_parts"], sc["group"], -1, sc["wide_fwd"],
                          sc["row_split"], sc["col_pack"])
        solo.step(nsteps, dt)
        assert np.array_equal(solo.get_state().astype(np.float64), got), (n, sc)
        solo.close()
        ref = make(n, seed)
        ref.step(nsteps, dt)
        check(got, ref.get_state().astype(np.float64), 1e-4, (n, sc))
        ref.close()
        s.close()


@pytest.mark.parametrize("n,wide,units", [(1024, 0, 130), (512, 1, 66)])
def test_pack_of_one_unit_per_cta_is_bit_identical(V, n, wide, units):
    """col_pack = the number of (column block, operator) units deals each
    CTA exactly one unit's terms: the same runs, so the same bits, as one
    CTA per unit (col_parts = 1).  1024: eight 32-element columns per CTA,
    65 blocks; 512: eight wide columns per CTA, 33 blocks; M = 16 in one
    group of 17, for the seismic pair and the general model's one operator."""
    import torch
    shape = (n, n)
    Q = S.q_lowpass(shape, 61)
    u = torch.from_numpy(S.q_lowpass(shape, 62, qmin=-1.0, qmax=1.0, sigma_k=32).astype(np.float32)).cuda()
    x, y = S.mesh(shape)
    order = 1.0 - 0.3 * np.cos(x) * np.sin(y)
    with V.Solver(shape) as s:
        s.set_q(Q)
        s.set_M(16)
        outs = {}
        for pack in (0, units):
            s.set_schedule(wide, -1, 1, 17, 0, -1, 0, pack)
            o1, o2 = torch.empty_like(u), torch.empty_like(u)
            s.apply_pair(u, o1, o2)
            s.sync()
            outs[pack] = (o1.cpu().numpy(), o2.cpu().numpy())
        assert np.array_equal(outs[0][0], outs[units][0]) and np.array_equal(outs[0][1], outs[units][1])
        s.set_order(order)
        gen = {}
        for pack in (0, units):
            s.set_schedule(wide, -1, 1, 17, 0, -1, 0, pack)
            o = torch.empty_like(u)
            s.apply(V.OP_S, u, o)
            s.sync()
            gen[pack] = o.cpu().numpy()
        assert np.array_equal(gen[0], gen[units])
