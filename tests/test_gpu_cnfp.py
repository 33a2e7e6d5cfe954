"""The Crank-Nicolson scheme (CNFP, Sec. 3.1) of the general model on the
GPU (vofl_set_scheme(VOFL_SCHEME_CNFP), plain path): conjugate gradients on
the normal equations of A = I + (kappa dt^2/2) L inside a fixed-point
iteration on f, with L the matrix-free operator of Eq. (2.13).

- Runs in 1D, 2D and 3D, FP64 and FP32, match the oracle (which solves each
  step's system directly) on the same inputs.
- The paper's Table 2 (J = 4096, h = 1/64, M = 15, f(u) = u^3, t = 1) is
  reproduced by the GPU's FP64 path, with the dt = 2^-12 reference that
  the printed digits and convergence rates point to.
- The scheme's preconditions, the solver settings and a solve that runs out
  of iterations come back as status codes, and the context stays usable."""
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_util import rel_l2, check

pytestmark = pytest.mark.gpu

CUBE = lambda u: u ** 3  # noqa: E731


def _gpu_cn(V, shape, s, u0, dt, nsteps, M, f3, prec, lo=None, hi=None, v0=None, tol=None, kappa=1.0):
    ty = np.float32 if prec == V.F32 else np.float64
    with V.Solver(shape, lo, hi, prec, V.IMPL_PLAIN) as sv:
        sv.set_order(np.ascontiguousarray(s, dtype=np.float64), kappa=kappa, f3=f3)
        sv.set_M(M)
        sv.set_scheme(V.SCHEME_CNFP)
        if tol is not None:
            sv.set_solver(tol)
        sv.set_state(np.ascontiguousarray(u0, dtype=ty), None if v0 is None else np.ascontiguousarray(v0, dtype=ty))
        sv.step(nsteps, dt)
        out = sv.get_state()
        sv.sync()
        stats = sv.solver_stats()
        return out.astype(np.float64), stats


@pytest.mark.parametrize("order", ["s1", "s2"])
def test_cnfp_1d_f64_matches_oracle(V, order):
    """Eq. (4.1) on [-32, 32] with h = 1/8, dt = 2^-7 to t = 1 (the largest
    step of Table 2, where A is furthest from the identity)."""
    J, lo, hi = 512, [-32.0], [32.0]
    x = S.axis(J, -32.0, 32.0)
    s = 1.0 + 0.3 * np.sin(np.pi * x / 8) if order == "s1" else 1.0 + 0.2 * np.tanh(np.cos(np.pi * x / 8))
    phi = np.exp(-x * x)
    g, (iters, solves) = _gpu_cn(V, (J,), s, phi, 2.0 ** -7, 128, 15, 1.0, V.F64, lo, hi)
    r = O.general_cnfp(s, 1.0, CUBE, phi, None, 2.0 ** -7, 128, 15, lo, hi)
    check(g, r, 1e-10)
    assert solves >= 127 and iters >= solves


def test_cnfp_1d_f64_initial_velocity(V):
    J, lo, hi = 256, [-16.0], [16.0]
    x = S.axis(J, -16.0, 16.0)
    s = 0.8 + 0.25 * np.cos(np.pi * x / 8)
    phi = np.exp(-2.0 * x * x)
    psi = 0.5 * x * np.exp(-x * x)
    g, _ = _gpu_cn(V, (J,), s, phi, 0.02, 60, 12, -1.0, V.F64, lo, hi, v0=psi)
    r = O.general_cnfp(s, 1.0, lambda u: -u ** 3, phi, psi, 0.02, 60, 12, lo, hi)
    check(g, r, 1e-10)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_cnfp_2d_matches_oracle(V, prec, tol):
    """s = 1 - 0.4 cos(pi x/4) cos(pi y/4) (the paper's 2D example shape),
    M = 20, dt = 0.3: three times the leap-frog limit 2/omega_max of this
    grid (omega_max = |mu_max|^{1.4})."""
    shape, lo, hi = (32, 32), [-8.0, -8.0], [8.0, 8.0]
    xg, yg = S.mesh(shape, lo, hi)
    s = 1.0 - 0.4 * np.cos(np.pi * xg / 4) * np.cos(np.pi * yg / 4)
    u0 = np.exp(-(xg ** 2 + yg ** 2))
    p = V.F64 if prec == "f64" else V.F32
    g, _ = _gpu_cn(V, shape, s, u0, 0.3, 20, 20, 1.0, p, lo, hi)
    r = O.general_cnfp(s, 1.0, CUBE, u0, None, 0.3, 20, 20, lo, hi)
    check(g, r, tol)


def test_cnfp_3d_f64_matches_oracle(V):
    shape, lo, hi = (8, 8, 8), [-4.0] * 3, [4.0] * 3
    xg, yg, zg = S.mesh(shape, lo, hi)
    s = 1.1 + 0.2 * np.sin(np.pi * xg / 4) * np.cos(np.pi * zg / 4)
    u0 = np.exp(-(xg ** 2 + 2 * yg ** 2 + zg ** 2))
    g, _ = _gpu_cn(V, shape, s, u0, 0.05, 12, 10, 1.0, V.F64, lo, hi)
    r = O.general_cnfp(s, 1.0, CUBE, u0, None, 0.05, 12, 10, lo, hi)
    check(g, r, 1e-10)


def _table2(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "table2_cnfp_temporal_errors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[int(p[0])] = [float(v) for v in p[1:]]
    return rows


@pytest.mark.parametrize("col,order", [(3, "s1"), (4, "s2"), (1, "one")])
def test_paper_table2_cnfp_on_the_gpu(V, golden_dir, col, order):
    """Table 2 at the paper's h = 1/64 (J = 4096) with the GPU's FP64 path;
    agreement 1e-3 relative, plus 3e-9 absolute on cells below 5e-7 (the
    oracle pin's rule: the printed values' floor at the finest steps)."""
    rows = _table2(golden_dir)
    J, lo, hi = 4096, [-32.0], [32.0]
    x = S.axis(J, -32.0, 32.0)
    phi = np.exp(-x * x)
    if order == "s1":
        s, M = 1.0 + 0.3 * np.sin(np.pi * x / 8), 15
    elif order == "s2":
        s, M = 1.0 + 0.2 * np.tanh(np.cos(np.pi * x / 8)), 15
    else:
        s, M = np.ones(J), 0
    run = lambda dt, n: _gpu_cn(V, (J,), s, phi, dt, n, M, 1.0, V.F64, lo, hi)[0]  # noqa: E731
    ref = run(2.0 ** -12, 4096)
    for p in range(7, 12):
        err = O.l2_error(run(2.0 ** -p, 2 ** p), ref, [1.0 / 64])
        printed = rows[p][col]
        floor = 3e-9 if printed < 5e-7 else 0.0
        assert abs(err - printed) <= 1e-3 * printed + floor, (order, p, err, printed)


def test_cnfp_preconditions_and_solver_limits(V):
    shape = (64,)
    x = S.axis(64, -8.0, 8.0)
    s = 1.0 + 0.3 * np.sin(np.pi * x / 8)
    with V.Solver(shape, [-8.0], [8.0], V.F64, V.IMPL_FUSED) as sv:  # fused path: no implicit scheme
        sv.set_order(s)
        sv.set_scheme(V.SCHEME_CNFP)
        sv.set_state(np.exp(-x * x))
        with pytest.raises(V.VoflError):
            sv.step(2, 0.01)
    with V.Solver(shape, [-8.0], [8.0], V.F64, V.IMPL_PLAIN) as sv:
        sv.set_q(np.full(shape, 30.0))  # seismic model: no implicit scheme
        sv.set_scheme(V.SCHEME_CNFP)
        sv.set_state(np.exp(-x * x))
        with pytest.raises(V.VoflError):
            sv.step(2, 0.01)
        sv.set_order(s, f3=1.0)
        sv.set_M(12)
        for bad in ((0.0, 10), (1.5, 10), (1e-8, 0)):
            with pytest.raises(V.VoflError):
                sv.set_solver(*bad)
        sv.set_source((32,), np.ones(4))
        sv.set_state(np.exp(-x * x))
        with pytest.raises(V.VoflError):
            sv.step(3, 0.01)
        sv.set_source((0,), [])
        # one CG chunk (4 iterations) cannot reach 1e-13 when c lambda_max
        # is about 20: the solve reports non-convergence ...
        sv.set_solver(1e-13, 1)
        sv.set_state(np.exp(-x * x))
        with pytest.raises(V.VoflError) as e:
            sv.step(3, 0.25)
        assert "ENOCONV" in str(e.value) or "converge" in str(e.value).lower() or "exhausted" in str(e.value)
        # ... and the context is still usable
        sv.set_solver(1e-13, 5000)
        sv.set_state(np.exp(-x * x))
        sv.step(3, 0.25)
        g = sv.get_state()
        sv.sync()
        it, so = sv.solver_stats()
        assert it > 0 and so >= 2
    r = O.general_cnfp(s, 1.0, CUBE, np.exp(-x * x), None, 0.25, 3, 12, [-8.0], [8.0])
    check(g, r, 1e-10)
