"""The general variable-order model on the GPU (vofl_set_order):
u_tt = -kappa (-Delta)^{s(x)} u + f(u), stepped by leap-frog (Eq. (3.4)).

- The paper's Table 3 (Sec. 3.2: LFFP temporal errors for Eq. (4.1) on
  [-32, 32], h = 1/64, M = 15, f(u) = u^3, reference dt = 1e-4 at t = 1) is
  reproduced by the GPU's FP64 path to the printed four digits, including
  the "unstable" cells.
- The generic operator (-Delta)^{s(x)} (s = 1 - 0.4 cos(pi x/4) cos(pi y/4),
  the shape of the paper's 2D example, M = 20) matches the FP64 oracle.
- Short general-model runs of the fused FP32 and FP64 paths match the
  oracle's stepper."""
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_util import rel_l2, check

pytestmark = pytest.mark.gpu


def _table3(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "table3_lffp_temporal_errors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[int(p[0])] = [None if v == "unstable" else float(v) for v in p[1:]]
    return rows


def _gpu_general(V, shape, s, u0, dt, nsteps, M, f3, impl, prec, lo=None, hi=None):
    ty = np.float32 if prec == V.F32 else np.float64
    with V.Solver(shape, lo, hi, prec, impl) as sv:
        sv.set_order(np.ascontiguousarray(s, dtype=np.float64), kappa=1.0, f3=f3)
        sv.set_M(M)
        sv.set_state(np.ascontiguousarray(u0, dtype=ty))
        sv.step(nsteps, dt)
        out = sv.get_state()
        sv.sync()
        return out.astype(np.float64)


@pytest.mark.parametrize("col,order", [(3, "s1"), (4, "s2")])
def test_paper_table3_on_the_gpu(V, golden_dir, col, order):
    rows = _table3(golden_dir)
    J, lo, hi = 4096, [-32.0], [32.0]
    x = S.axis(J, -32.0, 32.0)
    phi = np.exp(-x * x)
    s = 1.0 + 0.3 * np.sin(np.pi * x / 8) if order == "s1" else 1.0 + 0.2 * np.tanh(np.cos(np.pi * x / 8))
    run = lambda dt, n: _gpu_general(V, (J,), s, phi, dt, n, 15, 1.0, V.IMPL_PLAIN, V.F64, lo, hi)  # noqa: E731
    ref = run(1e-4, 10000)
    for p in range(7, 12):
        printed = rows[p][col]
        u = run(2.0 ** -p, 2 ** p)
        if printed is None:
            assert not np.all(np.isfinite(u)) or np.max(np.abs(u)) > 1e3, p
        else:
            err = O.l2_error(u, ref, [1.0 / 64])
            assert abs(err - printed) <= 0.0006 * printed, (order, p, err, printed)


def _s2d(shape, lo, hi):
    x, y = S.mesh(shape, lo, hi)
    return 1.0 - 0.4 * np.cos(np.pi * x / 4) * np.cos(np.pi * y / 4)


@pytest.mark.parametrize("impl,prec,tol", [("fused", "f32", 1e-5), ("plain", "f64", 1e-11)])
def test_generic_operator_2d(V, impl, prec, tol):
    import torch
    shape, lo, hi = (512, 512), [-8.0, -8.0], [8.0, 8.0]
    s = _s2d(shape, lo, hi)
    u = S.q_lowpass(shape, 31, qmin=-1.0, qmax=1.0, sigma_k=40.0)
    P = V.F32 if prec == "f32" else V.F64
    ty, tty = (np.float32, torch.float32) if P == V.F32 else (np.float64, torch.float64)
    im = V.IMPL_FUSED if impl == "fused" else V.IMPL_PLAIN
    uin = u.astype(ty)
    with V.Solver(shape, lo, hi, P, im) as sv:
        sv.set_order(s)
        sv.set_M(20)
        ut = torch.from_numpy(uin).cuda()
        out = torch.empty_like(ut)
        sv.apply(V.OP_S, ut, out)
        sv.sync()
        g = out.cpu().numpy().astype(np.float64)
        with pytest.raises(V.VoflError):
            sv.apply(V.OP_1PG, ut, out)  # not an operator of the general model
    r = O.matrix_free_operator(uin.astype(np.float64), s, 20, lo, hi)
    check(g, r, tol)


@pytest.mark.parametrize("n,prec,tol", [(4096, "f32", 1e-4), (2048, "f64", 1e-10)])
def test_general_run_fused_1d(V, n, prec, tol):
    """s1 of Table 3 on [-32, 32] with f(u) = u^3, 256 steps of dt = 2^-9."""
    lo, hi = [-32.0], [32.0]
    x = S.axis(n, -32.0, 32.0)
    phi = np.exp(-x * x)
    s = 1.0 + 0.3 * np.sin(np.pi * x / 8)
    P = V.F32 if prec == "f32" else V.F64
    ty = np.float32 if P == V.F32 else np.float64
    g = _gpu_general(V, (n,), s, phi, 2.0 ** -9, 256, 15, 1.0, V.IMPL_FUSED, P, lo, hi)
    r = O.general_lffp(s, 1.0, lambda u: u ** 3, phi.astype(ty).astype(np.float64), None, 2.0 ** -9, 256, 15, lo, hi)
    check(g, r, tol)


def test_general_run_fused_2d_against_oracle(V):
    """A 2D general-model run (linear, f = 0) on the fused FP32 path."""
    shape, lo, hi = (128, 128), [-8.0, -8.0], [8.0, 8.0]
    s = _s2d(shape, lo, hi)
    u0 = S.gaussian_pulse(shape, 6.0)
    g = _gpu_general(V, shape, s, u0, 2e-3, 60, 20, 0.0, V.IMPL_FUSED, V.F32, lo, hi)
    r = O.general_lffp(s, 1.0, lambda u: 0.0 * u, u0.astype(np.float32).astype(np.float64), None, 2e-3, 60, 20,
                       lo, hi)
    check(g, r, 1e-4)


def test_model_switch_and_checks(V):
    shape = (64, 64)
    with V.Solver(shape) as sv:
        with pytest.raises(V.VoflError):
            sv.set_order(np.full(shape, 2.5))  # s outside (0, 2]
        with pytest.raises(V.VoflError):
            sv.set_order(np.ones(shape), kappa=0.0)
        sv.set_order(np.full(shape, 0.8), kappa=2.0)
        dt = sv.suggest_dt(0.25)
        # constant s: omega_max = sqrt(kappa) |mu_max|^s
        mu = np.sqrt(2.0) * np.pi * 64 / (2 * np.pi)
        assert dt == pytest.approx(0.5 / (np.sqrt(2.0) * mu ** 0.8), rel=1e-6)
        sv.set_q(S.q_lowpass(shape, 1))  # back to the seismic model
        import torch
        ut = torch.zeros(shape, dtype=torch.float32, device="cuda")
        with pytest.raises(V.VoflError):
            sv.apply(V.OP_S, ut, torch.empty_like(ut))


def test_suggest_M_matches_the_oracle_rule(V):
    """The library's Taylor-power rule gives the oracle's M (seismic model of
    the headline kind, and a general model on a larger box)."""
    shape = (256, 256)
    Q = S.q_lowpass(shape, 2)
    g = np.arctan(1.0 / Q) / np.pi
    with V.Solver(shape) as sv:
        sv.set_q(Q)
        for tol in (1e-6, 1e-8, 1e-10):
            assert sv.suggest_M(tol) == O.suggested_M(1.0 + g, shape, tol=tol)
    lo, hi = [-8.0, -8.0], [8.0, 8.0]
    s = _s2d(shape, lo, hi)
    with V.Solver(shape, lo, hi) as sv:
        sv.set_order(s)
        for tol in (1e-6, 1e-10):
            assert sv.suggest_M(tol) == O.suggested_M(s, shape, lo, hi, tol)


def _table4(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "table4_tsfp2_temporal_errors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[int(p[0])] = [None if v == "unstable" else float(v) for v in p[1:]]
    return rows


def _gpu_split(V, shape, s, u0, dt, nsteps, M, f3, prec, lo=None, hi=None, v0=None, impl=None, group=0):
    ty = np.float32 if prec == V.F32 else np.float64
    with V.Solver(shape, lo, hi, prec, V.IMPL_PLAIN if impl is None else impl) as sv:
        if group:
            sv.set_schedule(group=group)
        sv.set_order(np.ascontiguousarray(np.broadcast_to(s, shape), dtype=np.float64), kappa=1.0, f3=f3)
        sv.set_M(M)
        sv.set_scheme(V.SCHEME_TSFP2)
        sv.set_state(np.ascontiguousarray(u0, dtype=ty), None if v0 is None else np.ascontiguousarray(v0, dtype=ty))
        sv.step(nsteps, dt)
        out = sv.get_state()
        sv.sync()
        return out.astype(np.float64)


@pytest.mark.parametrize("col,order", [(3, "s1"), (1, "one")])
def test_paper_table4_tsfp2_on_the_gpu(V, golden_dir, col, order):
    """Table 4 (TSFP2, Sec. 3.3) with the GPU's FP64 path: column s1 (with
    its unstable cells) and the constant-order column s = 1."""
    rows = _table4(golden_dir)
    J, lo, hi = 4096, [-32.0], [32.0]
    x = S.axis(J, -32.0, 32.0)
    phi = np.exp(-x * x)
    s = 1.0 + 0.3 * np.sin(np.pi * x / 8) if order == "s1" else np.ones(J)
    M = 15 if order == "s1" else 0
    run = lambda dt, n: _gpu_split(V, (J,), s, phi, dt, n, M, 1.0, V.F64, lo, hi)  # noqa: E731
    ref = run(1e-4, 10000)
    for p in range(7, 12):
        printed = rows[p][col]
        u = run(2.0 ** -p, 2 ** p)
        if printed is None:
            assert not np.all(np.isfinite(u)) or np.max(np.abs(u)) > 1e3, p
        else:
            err = O.l2_error(u, ref, [1.0 / 64])
            assert abs(err - printed) <= 0.0006 * printed, (order, p, err, printed)


@pytest.mark.parametrize("impl", ["plain", "fused"])
def test_tsfp2_fp32_2d_against_oracle(V, impl):
    """A 2D splitting run in FP32 with a non-zero initial velocity, on the
    cuFFT path and on the fused path (rotations on its own line transforms,
    the m >= 1 remainder on the operator kernels, the kick in their
    epilogue)."""
    shape, lo, hi = (128, 128), [-8.0, -8.0], [8.0, 8.0]
    s = _s2d(shape, lo, hi)
    u0 = S.gaussian_pulse(shape, 6.0).astype(np.float32)
    xg, yg = S.mesh(shape, lo, hi)
    v0 = (0.3 * np.sin(np.pi * xg / 4) * np.cos(np.pi * yg / 8)).astype(np.float32)
    im = V.IMPL_PLAIN if impl == "plain" else V.IMPL_FUSED
    g = _gpu_split(V, shape, s, u0, 2e-3, 50, 20, 1.0, V.F32, lo, hi, v0, impl=im)
    r = O.general_tsfp2(s, 1.0, lambda u: u ** 3, u0.astype(np.float64), v0.astype(np.float64), 2e-3, 50, 20, lo, hi)
    check(g, r, 1e-4)


@pytest.mark.parametrize("shape,M,group", [((256, 256), 12, 0), ((512, 512), 8, 3), ((768, 768), 6, 0),
                                           ((1024, 1024), 16, 0), ((256, 128), 0, 0), ((64, 64), 1, 0)])
def test_tsfp2_fused_2d_sizes(V, shape, M, group):
    """The fused splitting on every line-transform kind (32-element lines,
    wide lines at 512 and 1024, the three-stage 768-point line), several
    Taylor groups (partial sums across groups, the delta factor of the
    remainder), a rectangular grid, M = 0 (the kick alone: no remainder)
    and M = 1 (one remainder term), against the FP64 oracle.  The kick is
    explicit: dt is a quarter of 2 / |mu_max|^{max s} (the leap-frog rule;
    at 2e-3 the 768^2 and 1024^2 runs are unstable, in FP64 too)."""
    lo, hi = [-8.0, -8.0], [8.0, 8.0]
    s = _s2d(shape, lo, hi)
    xg, yg = S.mesh(shape, lo, hi)
    u0 = np.exp(-(xg ** 2 + yg ** 2) / 2.0).astype(np.float32)
    v0 = (0.2 * np.cos(np.pi * xg / 8) * np.sin(np.pi * yg / 4)).astype(np.float32)
    mu_max = np.pi * np.hypot(shape[0] / 16.0, shape[1] / 16.0)
    dt, n = 0.25 * 2.0 / mu_max ** s.max(), 6
    g = _gpu_split(V, shape, s, u0, dt, n, M, 1.0, V.F32, lo, hi, v0, impl=V.IMPL_FUSED, group=group)
    r = O.general_tsfp2(s, 1.0, lambda u: u ** 3, u0.astype(np.float64), v0.astype(np.float64), dt, n, M, lo, hi)
    check(g, r, 1e-4, (shape, M, group))


def test_tsfp2_needs_general_model_and_plain_path(V):
    shape = (64, 64)
    with V.Solver((64, 64, 64)) as sv:  # fused 3D path: no splitting
        sv.set_order(np.ones((64, 64, 64)))
        sv.set_scheme(V.SCHEME_TSFP2)
        sv.set_state(np.zeros((64, 64, 64), np.float32))
        with pytest.raises(V.VoflError):
            sv.step(1, 1e-3)
    with V.Solver(shape) as sv:  # fused 2D path, seismic model
        sv.set_q(S.q_lowpass(shape, 1))
        sv.set_scheme(V.SCHEME_TSFP2)
        sv.set_state(np.zeros(shape, np.float32))
        with pytest.raises(V.VoflError):
            sv.step(1, 1e-3)
    with V.Solver(shape, impl=V.IMPL_PLAIN) as sv:  # seismic model
        sv.set_q(S.q_lowpass(shape, 1))
        sv.set_scheme(V.SCHEME_TSFP2)
        sv.set_state(np.zeros(shape, np.float32))
        with pytest.raises(V.VoflError):
            sv.step(1, 1e-3)
        with pytest.raises(V.VoflError):
            sv.set_scheme(7)


def _table5(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "table5_tsfp2_spatial_errors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[int(p[0])] = [float(v) for v in p[1:]]
    return rows


@pytest.mark.parametrize("col,order", [(1, "one"), (3, "s1"), (4, "s2")])
def test_paper_table5_spatial_errors_on_the_gpu(V, golden_dir, col, order):
    """Table 5 (TSFP2 at dt = 1e-4, h = 1 .. 1/8 against h = 1/64) with the
    GPU's FP64 path: the printed digits at h = 1, 1/2, 1/4; the round-off
    floor at h = 1/8."""
    rows = _table5(golden_dir)
    lo, hi = [-32.0], [32.0]

    def run(J):
        x = S.axis(J, -32.0, 32.0)
        if order == "one":
            s, M = np.ones(J), 0
        elif order == "s1":
            s, M = 1.0 + 0.3 * np.sin(np.pi * x / 8), 15
        else:
            s, M = 1.0 + 0.2 * np.tanh(np.cos(np.pi * x / 8)), 15
        return _gpu_split(V, (J,), s, np.exp(-x * x), 1e-4, 10000, M, 1.0, V.F64, lo, hi)

    ref = run(4096)
    for inv_h in (1, 2, 4, 8):
        J = 64 * inv_h
        u = run(J)
        err = np.sqrt((1.0 / inv_h) * np.sum((u - ref[:: 4096 // J]) ** 2))
        printed = rows[inv_h][col]
        if inv_h < 8:
            assert abs(err - printed) <= 1e-4 * printed, (order, inv_h, err, printed)
        else:
            assert err < 1e-11, (order, err)


def _apply_s(V, shape, s, u, M, prec, lo, hi):
    import torch
    P = V.F32 if prec == "f32" else V.F64
    ty = np.float32 if P == V.F32 else np.float64
    uin = np.ascontiguousarray(u, dtype=ty)
    with V.Solver(shape, lo, hi, P, V.IMPL_FUSED) as sv:
        sv.set_order(np.ascontiguousarray(s, dtype=np.float64))
        sv.set_M(M)
        ut = torch.from_numpy(uin).cuda()
        out = torch.empty_like(ut)
        sv.apply(V.OP_S, ut, out)
        sv.sync()
        with pytest.raises(V.VoflError):
            sv.apply_pair(ut, out, torch.empty_like(ut))  # one operator: vofl_apply(VOFL_OP_S)
        return out.cpu().numpy().astype(np.float64), uin.astype(np.float64)


@pytest.mark.parametrize("M", [0, 1, 2, 7, 8, 15, 20])
def test_one_operator_split_2d(V, M):
    """The general model's terms fill both slots of the fused 2D kernels
    (terms 0..K-1 and K..M, K = ceil((M+1)/2)): every M, odd and even term
    counts, against the oracle's M-term operator."""
    shape, lo, hi = (128, 128), [-8.0, -8.0], [8.0, 8.0]
    s = _s2d(shape, lo, hi)
    u = S.q_lowpass(shape, 7, qmin=-1.0, qmax=1.0, sigma_k=20.0)
    g, uin = _apply_s(V, shape, s, u, M, "f32", lo, hi)
    r = O.matrix_free_operator(uin, s, M, lo, hi)
    check(g, r, 1e-5)


@pytest.mark.parametrize("M", [3, 8])
def test_one_operator_split_3d(V, M):
    shape, lo, hi = (64, 64, 64), [-4.0] * 3, [4.0] * 3
    xg, yg, zg = S.mesh(shape, lo, hi)
    s = 1.0 + 0.25 * np.sin(np.pi * xg / 4) * np.cos(np.pi * yg / 4) + 0.1 * np.cos(np.pi * zg / 4)
    u = S.gaussian_pulse(shape, 5.0)
    g, uin = _apply_s(V, shape, s, u, M, "f32", lo, hi)
    r = O.matrix_free_operator(uin, s, M, lo, hi)
    check(g, r, 1e-5)


@pytest.mark.parametrize("M,prec,tol", [(5, "f64", 1e-11), (12, "f64", 1e-11), (9, "f32", 1e-5)])
def test_one_operator_split_1d(V, M, prec, tol):
    n, lo, hi = 1024, [-32.0], [32.0]
    x = S.axis(n, -32.0, 32.0)
    s = 1.0 + 0.3 * np.sin(np.pi * x / 8)
    u = np.exp(-x * x) * np.cos(2.0 * x)
    g, uin = _apply_s(V, (n,), s, u, M, prec, lo, hi)
    r = O.matrix_free_operator(uin, s, M, lo, hi)
    check(g, r, tol)


def test_batches_take_seismic_contexts_only(V):
    shape = (256, 256)
    with V.Solver(shape) as sv, V.Batch() as b:
        sv.set_order(np.ones(shape))
        sv.set_state(np.zeros(shape, np.float32))
        with pytest.raises(V.VoflError):
            b.add(sv, 1e-3)


def test_tsfp2_fused_split_calls_agree(V):
    """On the fused path one vofl_step call brackets its steps by the flows
    over +dt/2 and -dt/2; a run split over several calls differs from one
    call only by those extra (exactly cancelling) flows: FP32 round-off,
    far below the run tolerance; both match the oracle."""
    shape, lo, hi = (256, 256), [-8.0, -8.0], [8.0, 8.0]
    s = _s2d(shape, lo, hi)
    xg, yg = S.mesh(shape, lo, hi)
    u0 = np.exp(-(xg ** 2 + yg ** 2) / 2.0).astype(np.float32)
    v0 = (0.2 * np.cos(np.pi * xg / 8) * np.sin(np.pi * yg / 4)).astype(np.float32)
    dt, M = 1e-3, 10
    outs = []
    for calls in ([12], [5, 7], [1] * 12):
        with V.Solver(shape, lo, hi) as sv:
            sv.set_order(s, kappa=1.0, f3=1.0)
            sv.set_M(M)
            sv.set_scheme(V.SCHEME_TSFP2)
            sv.set_state(u0, v0)
            for n in calls:
                sv.step(n, dt)
            assert sv.steps_taken() == 12
            outs.append(sv.get_state().astype(np.float64))
    r = O.general_tsfp2(s, 1.0, lambda u: u ** 3, u0.astype(np.float64), v0.astype(np.float64), dt, 12, M, lo, hi)
    for g in outs:
        check(g, r, 1e-4)
    for g in outs[1:]:
        check(g, outs[0], 1e-5)
