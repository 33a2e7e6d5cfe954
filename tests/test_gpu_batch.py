"""Batches of 2D simulations (vofl_batch_*): every member must end in the
same state, bit for bit, as the same context stepped alone (the batched
launches run the single-context kernel bodies), whatever the mix of sizes,
M, dt, sources, start times and schedule; one member is also checked
against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_util import gamma_of, rel_l2, check

pytestmark = pytest.mark.gpu


def _spec(n, seed, M, dt, src=True, psi=False, pulse=False):
    rng = np.random.default_rng(seed)
    shape = (n, n)
    sp = {"shape": shape, "Q": S.q_lowpass(shape, seed), "M": M, "dt": dt}
    sp["u0"] = (S.gaussian_pulse(shape, n / 16) if pulse else np.zeros(shape)).astype(np.float32)
    sp["v0"] = (0.2 * S.random_field(shape, seed + 1)).astype(np.float32) if psi else None
    if src:
        sp["idx"] = (int(rng.integers(0, n)), int(rng.integers(0, n)))
        sp["src"] = S.ricker_samples(400, dt, 10.0)
    return sp


def _solver(V, sp):
    s = V.Solver(sp["shape"])
    s.set_q(sp["Q"])
    s.set_M(sp["M"])
    s.set_state(sp["u0"], sp["v0"])
    if "src" in sp:
        s.set_source(sp["idx"], sp["src"])
    return s


def _solo(V, sp, chunks):
    with _solver(V, sp) as s:
        for c in chunks:
            s.step(c, sp["dt"])
        out = s.get_state()
        s.sync()
        return out


def test_batch_equals_solo_bitwise(V):
    """Four sizes (one with a factor 3), M from 4 to 16 (one to three Taylor
    groups), different dt, sources and a non-zero psi; steps in odd and even
    chunks (both graph parities)."""
    specs = [_spec(64, 1, 4, 2e-3), _spec(128, 2, 12, 1e-3, psi=True), _spec(256, 3, 16, 5e-4, pulse=True),
             _spec(768, 4, 8, 5e-4), _spec(128, 5, 6, 2e-3, src=False, pulse=True)]
    chunks = [3, 4, 1, 6]
    want = [_solo(V, sp, [sum(chunks)]) for sp in specs]
    with V.Batch() as b:
        solvers = [_solver(V, sp) for sp in specs]
        slots = [b.add(s, sp["dt"]) for s, sp in zip(solvers, specs)]
        assert len(b) == len(specs)
        assert b.kernels_per_step() > 0
        for c in chunks:
            b.step(c)
        b.sync()
        for s, slot in zip(solvers, slots):
            b.remove(slot)
        assert len(b) == 0
    for s, w in zip(solvers, want):
        assert s.steps_taken() == sum(chunks)
        got = s.get_state()
        s.sync()
        assert np.array_equal(got, w)
        s.close()


def test_batch_members_join_and_leave_between_steps(V):
    """A member that already ran alone, one that joins late (its Taylor start
    happens inside the batch) and one that leaves early: each equals its
    solo run of the same total length."""
    a, b_, c = _spec(128, 11, 8, 1e-3), _spec(256, 12, 10, 5e-4, psi=True), _spec(64, 13, 5, 2e-3, pulse=True)
    with V.Batch() as bt:
        sa, sb, sc = _solver(V, a), _solver(V, b_), _solver(V, c)
        sa.step(5, a["dt"])  # ran alone first
        ka = bt.add(sa, a["dt"])
        kc = bt.add(sc, c["dt"])
        bt.step(4)
        kb = bt.add(sb, b_["dt"])  # joins at its step 0
        bt.step(3)
        bt.remove(kc)  # leaves after 7 steps
        bt.step(6)
        bt.remove(ka)
        bt.remove(kb)
    got = [s.get_state() for s in (sa, sb, sc)]
    assert [s.steps_taken() for s in (sa, sb, sc)] == [18, 9, 7]
    for s in (sa, sb, sc):
        s.sync()
        s.close()
    assert np.array_equal(got[0], _solo(V, a, [18]))
    assert np.array_equal(got[1], _solo(V, b_, [9]))
    assert np.array_equal(got[2], _solo(V, c, [7]))


def test_batch_schedules_and_tuning_do_not_change_results(V):
    """Chunked, serial and tuned schedules give the same bits; tuning leaves
    every member where it was."""
    specs = [_spec(64, 20 + i, 6 + i, 1e-3, pulse=True) for i in range(5)] + \
            [_spec(256, 30 + i, 12, 5e-4) for i in range(3)]
    want = [_solo(V, sp, [9]) for sp in specs]
    for sched in ["default", (False, {64: 2, 256: 1}), (True, {64: 4}), "tune"]:
        with V.Batch() as b:
            solvers = [_solver(V, sp) for sp in specs]
            slots = [b.add(s, sp["dt"]) for s, sp in zip(solvers, specs)]
            b.step(2)
            if sched == "tune":
                ms = b.tune(reps=1)
                assert ms > 0
                par, ch = b.schedule()
                assert isinstance(par, bool)
            elif sched != "default":
                b.set_schedule(*sched)
                assert b.schedule() == (sched[0], sched[1])
            b.step(7)
            for slot in slots:
                b.remove(slot)
        for s, w in zip(solvers, want):
            got = s.get_state()
            s.sync()
            assert np.array_equal(got, w), sched
            s.close()


def test_batch_member_against_oracle(V):
    """A 128^2 member of a mixed batch against the FP64 oracle."""
    sp = _spec(128, 41, 8, 1e-3, pulse=True)
    other = _spec(256, 42, 12, 5e-4)
    with V.Batch() as b:
        s, o = _solver(V, sp), _solver(V, other)
        k1 = b.add(s, sp["dt"])
        k2 = b.add(o, other["dt"])
        b.step(40)
        b.remove(k1)
        b.remove(k2)
    g = s.get_state().astype(np.float64)
    s.sync()
    s.close()
    o.close()
    r = O.seismic_lffp(gamma_of(sp["Q"]), 1.0, 2 * np.pi, sp["u0"].astype(np.float64), None, sp["dt"], 40, sp["M"],
                       src_idx=sp["idx"], src=sp["src"])
    check(g, r, 1e-4)


def test_batch_rejects_and_locks_members(V):
    with V.Batch() as b:
        with V.Solver((128, 256)) as s:  # not square
            s.set_q(S.q_lowpass((128, 256), 1))
            s.set_state(np.zeros((128, 256), np.float32))
            with pytest.raises(V.VoflError):
                b.add(s, 1e-3)
        with V.Solver((64, 64), impl=V.IMPL_PLAIN) as s:
            s.set_q(S.q_lowpass((64, 64), 1))
            s.set_state(np.zeros((64, 64), np.float32))
            with pytest.raises(V.VoflError):
                b.add(s, 1e-3)
        with V.Solver((64, 64)) as s:
            with pytest.raises(V.VoflError):
                b.add(s, 1e-3)  # no model, no state
            s.set_q(S.q_lowpass((64, 64), 1))
            s.set_state(np.zeros((64, 64), np.float32))
            slot = b.add(s, 1e-3)
            with pytest.raises(V.VoflError):
                s.step(1, 1e-3)  # stepped by the batch
            with pytest.raises(V.VoflError):
                b.add(s, 1e-3)  # already in
            b.step(2)
            with pytest.raises(V.VoflError):
                b.remove(slot + 100)
        # the member was destroyed while in the batch: it left the batch
        assert len(b) == 0
        b.step(1)


@pytest.mark.parametrize("n", [256, 768])
def test_suggest_dt_matches_oracle(V, n):
    """The library's time-step rule against the oracle's on the batch
    workload's kind of model (the library reads c^2 eta in FP32)."""
    shape = (n, n)
    Q = S.q_lowpass(shape, 4000 + n)
    with V.Solver(shape) as s:
        s.set_q(Q)
        dt = s.suggest_dt(0.25)
    ref = O.suggested_dt(gamma_of(Q), 1.0, 2 * np.pi, shape, courant=0.25)
    assert abs(dt - ref) <= 1e-6 * ref, (dt, ref)


def test_batch_workload_members_equal_solo(V):
    """The 64-simulation workload itself (edges 256..1024 incl. 768, M = 12,
    dt by the time-step rule), autotuned, 9 steps: the first member of every
    size equals its solo run bit for bit."""
    sims = S.workload_batch()
    solvers, first = [], {}
    with V.Batch() as b:
        for i, sp in enumerate(sims):
            s = V.Solver(sp["shape"])
            s.set_q(sp["Q"])
            s.set_M(sp["M"])
            dt = s.suggest_dt(0.25)
            s.set_state(np.zeros(sp["shape"], np.float32))
            s.set_source(sp["src_idx"], S.ricker_samples(sp["nsteps"], dt, sp["f0"]))
            b.add(s, dt)
            solvers.append((s, dt))
            first.setdefault(sp["shape"][0], i)
        b.tune(reps=1)
        b.step(4)
        b.step(5)
    assert sorted(first) == [256, 512, 768, 1024]
    for n, i in first.items():
        sp = sims[i]
        s, dt = solvers[i]
        got = s.get_state()
        s.sync()
        with V.Solver(sp["shape"]) as t:
            t.set_q(sp["Q"])
            t.set_M(sp["M"])
            t.set_state(np.zeros(sp["shape"], np.float32))
            t.set_source(sp["src_idx"], S.ricker_samples(sp["nsteps"], dt, sp["f0"]))
            t.step(9, dt)
            want = t.get_state()
            t.sync()
        assert np.array_equal(got, want), n
    for s, _ in solvers:
        s.close()
