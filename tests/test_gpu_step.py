"""GPU parity of leap-frog runs of Eq. (1.1) against the FP64 oracle.

Tolerances: FP32 runs within 1e-4 relative L2 of the oracle at the end of
the run (the stated full-run bound); FP64 runs within 1e-9."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_util import gamma_of, gpu_run, rel_l2, check

pytestmark = pytest.mark.gpu

TOL32_RUN = 1e-4


def _oracle_run(shape, Q, u0, v0, M, dt, nsteps, src_idx=None, src=None, lo=None, hi=None, method="matrix_free"):
    return O.seismic_lffp(gamma_of(Q), 1.0, 2 * np.pi, u0, v0, dt, nsteps, M, lo, hi,
                          src_idx=src_idx, src=src, method=method)


@pytest.mark.parametrize("impl", ["fused", "plain"])
def test_run_2d_source_matches_oracle(V, impl):
    shape = (128, 128)
    Q = S.q_lowpass(shape, 2)
    nsteps, dt = 120, 5e-3
    src = S.ricker_samples(nsteps, dt, 2.0)
    idx = S.center_index(shape)
    u0 = np.zeros(shape)
    im = V.IMPL_FUSED if impl == "fused" else V.IMPL_PLAIN
    g = gpu_run(V, shape, Q, u0, None, 8, dt, nsteps, im, V.F32, idx, src)
    r = _oracle_run(shape, Q, u0, None, 8, dt, nsteps, idx, src)
    assert np.max(np.abs(r)) > 0
    check(g, r, TOL32_RUN)


def test_run_2d_pulse_with_velocity_start(V):
    """Non-zero psi exercises the Taylor start with B L2 psi."""
    shape = (256, 128)
    Q = S.q_lowpass(shape, 4)
    u0 = S.gaussian_pulse(shape, 6.0)
    x, y = S.mesh(shape)
    v0 = 0.5 * np.sin(2 * x) * np.cos(3 * y)
    nsteps, dt = 80, 4e-3
    g = gpu_run(V, shape, Q, u0.astype(np.float32), v0.astype(np.float32), 7, dt, nsteps, V.IMPL_FUSED, V.F32)
    r = _oracle_run(shape, Q, u0.astype(np.float32).astype(np.float64), v0.astype(np.float32).astype(np.float64),
                    7, dt, nsteps)
    check(g, r, TOL32_RUN)


def test_run_split_calls_equal_one_call(V):
    """Stepping in chunks (graph replays of both parities) equals one call."""
    shape = (64, 64)
    Q = S.q_lowpass(shape, 8)
    u0 = S.gaussian_pulse(shape, 3.0)
    a = gpu_run(V, shape, Q, u0, None, 6, 1e-2, 31, V.IMPL_FUSED, V.F32)
    b = gpu_run(V, shape, Q, u0, None, 6, 1e-2, 31, V.IMPL_FUSED, V.F32, chunks=[1, 4, 7, 19])
    assert np.array_equal(a, b)


@pytest.mark.parametrize("impl", ["fused", "plain"])
def test_run_fp64_1d_against_dense_operator(V, impl):
    """1D N = 256, FP64, M = 8, 200 steps of dt = 1e-3 (Q = 20 + 15 sin x,
    u0 = exp(-20 x^2)): the GPU run against the oracle stepping with the
    dense O(N^2) operator of Eq. (2.3), and with the matrix-free one."""
    w = S.workload_1d_256()
    im = V.IMPL_FUSED if impl == "fused" else V.IMPL_PLAIN
    g = gpu_run(V, w["shape"], w["Q"], w["u0"], None, w["M"], w["dt"], w["nsteps"], im, V.F64)
    r_mf = _oracle_run(w["shape"], w["Q"], w["u0"], None, w["M"], w["dt"], w["nsteps"])
    r_dense = _oracle_run(w["shape"], w["Q"], w["u0"], None, w["M"], w["dt"], w["nsteps"], method="dense")
    check(g, r_mf, 1e-11)
    # truncation of Eq. (2.9) at M = 8 on this model is far below 1e-6
    check(g, r_dense, 1e-6)


def test_run_fused_1d_fp32_source_and_velocity(V):
    """1D N = 4096 FP32 with a Ricker source and a non-zero psi, in chunks."""
    n = 4096
    Q = S.q_lowpass((n,), 9)
    x = S.axis(n)
    v0 = 0.3 * np.sin(3 * (x + np.pi))
    nsteps, dt = 150, 2e-4
    src = S.ricker_samples(nsteps, dt, 40.0)
    u0 = np.zeros(n)
    g = gpu_run(V, (n,), Q, u0, v0.astype(np.float32), 12, dt, nsteps, V.IMPL_FUSED, V.F32, (n // 3,), src,
                chunks=[1, 60, 89])
    r = _oracle_run((n,), Q, u0, v0.astype(np.float32).astype(np.float64), 12, dt, nsteps, (n // 3,), src)
    check(g, r, TOL32_RUN)


def test_run_fused_3d_matches_oracle(V):
    """3D 64^3, two-layer Q, Gaussian pulse, 30 steps (fused FP32)."""
    shape = (64, 64, 64)
    Q = S.q_two_layer_3d(64)
    u0 = S.gaussian_pulse(shape, 3.0)
    g = gpu_run(V, shape, Q, u0, None, 8, 8e-3, 30, V.IMPL_FUSED, V.F32)
    r = _oracle_run(shape, Q, u0.astype(np.float32).astype(np.float64), None, 8, 8e-3, 30)
    check(g, r, TOL32_RUN)


def test_run_fp64_3d_plain(V):
    shape = (32, 32, 32)
    Q = S.q_two_layer_3d(32)
    u0 = S.gaussian_pulse(shape, 3.0)
    g = gpu_run(V, shape, Q, u0, None, 6, 1e-2, 25, V.IMPL_PLAIN, V.F64)
    r = _oracle_run(shape, Q, u0, None, 6, 1e-2, 25)
    check(g, r, 1e-9)


def test_run_gamma_zero_is_classical_wave(V):
    """gamma = 0 (the classical acoustic wave equation, Sec. 1): one Fourier
    mode follows cos(n theta), cos(theta) = 1 - dt^2 |mu|^2 / 2."""
    shape = (64, 64)
    x, y = S.mesh(shape)
    u0 = np.cos(3 * (x + np.pi) + 2 * (y + np.pi))
    dt, n = 0.02, 50
    with V.Solver(shape) as s:
        s.set_gamma(np.zeros(shape), c0=1.0)
        s.set_M(3)
        s.set_state(u0.astype(np.float32))
        s.step(n, dt)
        g = s.get_state().astype(np.float64)
    theta = np.arccos(1 - 0.5 * dt * dt * 13)
    check(g, np.cos(n * theta) * u0.astype(np.float32), TOL32_RUN)


def test_headline_workload_short_run(V):
    """2D 1024^2, M = 16, Ricker source at the centre: the first steps of the
    headline run against the oracle."""
    w = S.workload_2d_1024(nsteps=12)
    g = gpu_run(V, w["shape"], w["Q"], w["u0"], None, w["M"], w["dt"], w["nsteps"], V.IMPL_FUSED, V.F32,
                w["src_idx"], w["src"])
    r = _oracle_run(w["shape"], w["Q"], w["u0"], None, w["M"], w["dt"], w["nsteps"], w["src_idx"], w["src"])
    check(g, r, TOL32_RUN)


def test_headline_workload_scaled_full_length(V):
    """The headline workload's recipe at 256^2 for its full 1000 steps."""
    w = S.workload_2d_1024(nsteps=1000, n=256)
    g = gpu_run(V, w["shape"], w["Q"], w["u0"], None, w["M"], w["dt"], w["nsteps"], V.IMPL_FUSED, V.F32,
                w["src_idx"], w["src"])
    r = _oracle_run(w["shape"], w["Q"], w["u0"], None, w["M"], w["dt"], w["nsteps"], w["src_idx"], w["src"])
    check(g, r, TOL32_RUN)


def test_state_errors(V):
    shape = (64, 64)
    with V.Solver(shape) as s:
        with pytest.raises(V.VoflError):
            s.step(1, 1e-3)  # no model
        s.set_q(S.q_lowpass(shape, 1))
        with pytest.raises(V.VoflError):
            s.step(1, 1e-3)  # no state
        s.set_state(np.zeros(shape, np.float32))
        s.step(2, 1e-3)
        with pytest.raises(V.VoflError):
            s.step(1, 2e-3)  # dt changed mid-run
        with pytest.raises(V.VoflError):
            s.set_q(np.zeros(shape))  # Q must be positive
        with pytest.raises(V.VoflError):
            s.set_source((64, 0), np.ones(3))


def test_headline_workload_100_steps(V):
    """The headline run (1024^2, M = 16, Ricker at the centre, dt = 5e-4)
    for its first 100 steps against the oracle, on every point."""
    w = S.workload_2d_1024(nsteps=100)
    g = gpu_run(V, w["shape"], w["Q"], w["u0"], None, w["M"], w["dt"], w["nsteps"], V.IMPL_FUSED, V.F32,
                w["src_idx"], w["src"])
    r = _oracle_run(w["shape"], w["Q"], w["u0"], None, w["M"], w["dt"], w["nsteps"], w["src_idx"], w["src"])
    check(g, r, TOL32_RUN)
