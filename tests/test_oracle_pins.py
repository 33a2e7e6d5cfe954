"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
of the paper's definitions on Fourier modes, the Taylor remainder, textbook
reductions (gamma -> 0 gives the classical leap-frog), and the numbers the
paper prints (Table 3).  A plausible slip anywhere in the oracle (a dropped
term, a wrong sign or index, a transposed axis, a missing 1/N) fails one of
them.  CPU only.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S


def _mode_closed_form(shape, modes, s_field, lo=None, hi=None):
    """sum_i a_i |mu_{k_i}|^{2 s(x)} cos(mu_{k_i}.(x-a) + phi_i): the image of a
    cosine sum under the dense operator (Eq. (2.12)): each mode +-k_i is
    multiplied pointwise by |mu_{k_i}|^{2 s(x_j)}."""
    d = len(shape)
    lo = [-np.pi] * d if lo is None else lo
    hi = [np.pi] * d if hi is None else hi
    grids = S.mesh(shape, lo, hi)
    out = np.zeros(shape)
    for amp, ks, phi in modes:
        arg = np.zeros(shape)
        m2 = 0.0
        for i in range(d):
            mu = 2 * np.pi * ks[i] / (hi[i] - lo[i])
            arg = arg + mu * (grids[i] - lo[i])
            m2 += mu * mu
        out = out + amp * (m2 ** s_field(m2)) * np.cos(arg + phi)
    return out


# --------------------------------------------------------------------------
# P1: dense operator on Fourier modes (Eq. (2.3), Eq. (2.12))
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape,lo,hi", [
    ((32,), [-np.pi], [np.pi]),
    ((24,), [-32.0], [32.0]),
    ((12, 16), [-np.pi, -np.pi], [np.pi, np.pi]),
    ((8, 6, 10), [0.0, -1.0, -np.pi], [2.0, 3.0, np.pi]),
])
def test_dense_operator_modes(shape, lo, hi):
    d = len(shape)
    rng = np.random.default_rng(11)
    modes = []
    for _ in range(3):
        ks = [int(rng.integers(-shape[d - 1 - i] // 2 + 1, shape[d - 1 - i] // 2))
              for i in range(d)]
        if all(k == 0 for k in ks):
            ks[0] = 1
        modes.append((float(rng.uniform(0.5, 2)), ks, float(rng.uniform(0, 6))))
    u = S.cosine_modes(shape, modes, lo, hi)
    grids = S.mesh(shape, lo, hi)
    s = 0.6 + 0.5 * np.sin(grids[0] * 0.7 + 0.2) ** 2
    for g in grids[1:]:
        s = s + 0.1 * np.cos(g)
    got = O.dense_operator(u, s, lo, hi)
    ref = _mode_closed_form(shape, modes, lambda m2: s, lo, hi)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_dense_operator_nyquist_real_and_sampled_points():
    """The Nyquist row of the asymmetric index set is kept (k = -J/2, |mu| =
    pi J/(b-a)); on the mode cos(pi j) the operator is |mu_N|^{2 s_j} cos(pi j)."""
    n = 16
    x = S.axis(n)
    u = np.cos(np.pi * np.arange(n))  # pure Nyquist mode
    s = 1.0 + 0.2 * np.sin(x)
    got = O.dense_operator(u, s)
    ref = (n / 2.0) ** (2 * s) * u
    assert np.allclose(got, ref, rtol=1e-13, atol=0)
    pts = np.array([0, 5, 11])
    assert np.allclose(O.dense_operator(u, s, points=pts), ref[pts], rtol=1e-13)


# --------------------------------------------------------------------------
# P2: matrix-free scheme closed form (Eq. (2.10), Eq. (2.13))
# --------------------------------------------------------------------------
@pytest.mark.parametrize("M", [0, 1, 2, 5, 8, 16])
def test_matrix_free_truncated_exponential(M):
    shape = (20, 16)
    modes = [(1.0, (3, 2), 0.3), (0.5, (-5, 1), 1.1), (0.25, (0, 7), -0.4),
             (0.7, (1, 0), 0.0)]  # |mu| = 1: ln|mu|^2 = 0
    u = S.cosine_modes(shape, modes)
    x, y = S.mesh(shape)
    s = 1.0 + 0.3 * np.sin(x) * np.cos(2 * y)
    got = O.matrix_free_operator(u, s, M)
    s0 = s.mean()
    delta = s - s0

    # |mu|^{2 s0} e_M(delta ln|mu|^2) per mode
    ref = np.zeros(shape)
    for amp, ks, phi in modes:
        m2 = ks[0] ** 2 + ks[1] ** 2
        L = math.log(m2)
        eM = sum((delta * L) ** m / math.factorial(m) for m in range(M + 1))
        ref += amp * m2 ** s0 * eM * np.cos(ks[0] * (x + np.pi) + ks[1] * (y + np.pi) + phi)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_matrix_free_uses_grid_mean_s0():
    """Any s0 gives a valid expansion; the paper's choice is the domain
    average.  With an explicit, different s0 the M -> large limit is the same
    dense result, while the default must equal an explicit grid mean."""
    shape = (32,)
    x = S.axis(32)
    u = S.random_field(shape, 3)
    s = 1.0 + 0.25 * np.sin(x)
    a = O.matrix_free_operator(u, s, 6)
    b = O.matrix_free_operator(u, s, 6, s0=float(np.mean(s)))
    assert np.array_equal(a, b)
    dense = O.dense_operator(u, s)
    c = O.matrix_free_operator(u, s, 40, s0=0.8)
    assert np.max(np.abs(c - dense)) <= 1e-9 * np.max(np.abs(dense))


# --------------------------------------------------------------------------
# P3: matrix-free -> dense as M grows, within the Taylor remainder (Eq. (2.8))
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(64,), (16, 16), (8, 8, 8)])
def test_matrix_free_converges_to_dense_within_remainder(shape):
    u = S.random_field(shape, 5)
    grids = S.mesh(shape)
    s = 1.0 + 0.3 * np.sin(grids[0])
    for g in grids[1:]:
        s = s * (1.0 + 0.1 * np.cos(g))
    dense = O.dense_operator(u, s)
    errs = []
    for M in (2, 4, 8, 12, 20):
        mf = O.matrix_free_operator(u, s, M)
        bound = O.taylor_remainder_bound(u, s, M)
        err = np.abs(mf - dense)
        assert np.all(err <= bound * (1 + 1e-9) + 1e-10 * np.max(np.abs(dense)))
        errs.append(err.max())
    assert errs[-1] <= 1e-10 * np.max(np.abs(dense))
    assert all(a > b for a, b in zip(errs[:-2], errs[1:-1]))


# --------------------------------------------------------------------------
# P8: the matrix-free scheme against the dense definition on the configs'
# full grids, at sampled points (the dense sum is O(N) per point)
# --------------------------------------------------------------------------
def test_matrix_free_matches_dense_on_the_headline_grid():
    """1024^2, s = 1 + gamma of the headline Q field (seed 2), M = 16, a
    smooth seeded field: |delta| ln|mu|^2 stays below ~0.5 over the field's
    modes, so the Taylor remainder at M = 16 is far below round-off and
    Eq. (2.13) must equal Eq. (2.12) to FFT round-off at every sampled
    point."""
    w = S.workload_2d_1024(nsteps=1)
    s = 1.0 + O.seismic_coefficients(w["Q"], 1.0, 2 * np.pi)["gamma"]
    u = S.q_lowpass((1024, 1024), 7, qmin=-1.0, qmax=1.0, sigma_k=16.0)
    pts = np.random.default_rng(8).choice(u.size, 64, replace=False)
    dense = O.dense_operator(u, s, points=pts)
    mf = O.matrix_free_operator(u, s, 16).ravel()[pts]
    assert np.max(np.abs(mf - dense)) <= 1e-12 * np.max(np.abs(dense))


def test_matrix_free_matches_dense_on_the_3d_grid():
    """256^3, s = 1 + gamma of the two-layer Q, M = 8, the config's Gaussian
    pulse: twelve seeded points and four around the pulse."""
    w = S.workload_3d_256()
    s = 1.0 + O.seismic_coefficients(w["Q"], 1.0, 2 * np.pi)["gamma"]
    u = w["u0"]
    c = (128 * 256 + 128) * 256 + 128
    pts = np.concatenate([np.random.default_rng(9).choice(u.size, 12, replace=False),
                          [c, c + 3, c + 256 * 2, c + 256 * 256 * 5]])
    dense = O.dense_operator(u, s, points=pts)
    mf = O.matrix_free_operator(u, s, 8).ravel()[pts]
    assert np.max(np.abs(mf - dense)) <= 1e-12 * np.max(np.abs(dense))


# --------------------------------------------------------------------------
# P4: special cases
# --------------------------------------------------------------------------
def test_constant_order_is_the_plain_multiplier():
    """Constant s: Eq. (2.13) collapses to F^{-1}[|mu|^{2s} F u] (Eq. (1.3)),
    which for a cosine sum is the closed form; dense and matrix-free agree."""
    shape = (16, 24)
    modes = [(1.0, (2, 3), 0.1), (2.0, (-4, 5), 0.7)]
    u = S.cosine_modes(shape, modes)
    ref = _mode_closed_form(shape, modes, lambda m2: 1.37)
    for M in (0, 3, 9):
        got = O.matrix_free_operator(u, np.full(shape, 1.37), M)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    got = O.dense_operator(u, np.full(shape, 1.37))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_constant_field_maps_to_zero_and_linearity():
    shape = (12, 10)
    x, y = S.mesh(shape)
    s = 0.8 + 0.2 * np.cos(x + y)
    assert np.max(np.abs(O.matrix_free_operator(np.full(shape, 3.0), s, 8))) < 1e-11
    assert np.max(np.abs(O.dense_operator(np.full(shape, 3.0), s))) < 1e-11
    u, v = S.random_field(shape, 1), S.random_field(shape, 2)
    lhs = O.matrix_free_operator(2.0 * u - 0.5 * v, s, 7)
    rhs = 2.0 * O.matrix_free_operator(u, s, 7) - 0.5 * O.matrix_free_operator(v, s, 7)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(lhs))


def test_second_order_is_minus_laplacian():
    """s = 1: the operator is -Delta; on sin(3x) cos(2y) that is 13 times it."""
    shape = (16, 16)
    x, y = S.mesh(shape)
    u = np.sin(3 * x) * np.cos(2 * y)
    assert np.allclose(O.dense_operator(u, np.ones(shape)), 13 * u, atol=1e-11)
    assert np.allclose(O.matrix_free_operator(u, np.ones(shape), 4), 13 * u, atol=1e-11)


# --------------------------------------------------------------------------
# seismic coefficients (Sec. 1)
# --------------------------------------------------------------------------
def test_seismic_coefficients_limits_and_invariants():
    Q = np.array([1e-3, 0.5, 1.0, 5.0, 20.0, 100.0, 1e12])
    c0, w0 = 1.7, 2 * np.pi
    co = O.seismic_coefficients(Q, c0, w0)
    g = co["gamma"]
    assert np.all((g > 0) & (g < 0.5))
    assert abs(g[2] - 0.25) < 1e-15  # arctan(1) = pi/4
    # gamma -> 0: the classical acoustic wave equation (c = c0, eta = -1, tau = 0)
    assert abs(co["c"][-1] - c0) < 1e-12 and abs(co["eta"][-1] + 1) < 1e-10
    assert abs(co["tau"][-1]) < 1e-10
    # eta and tau are the cos/sin pair of the same angle pi*gamma, with
    # scale c0^{2g} w0^{-2g} (tau has one extra 1/c0)
    scale = c0 ** (2 * g) * w0 ** (-2 * g)
    assert np.allclose((co["eta"] / scale) ** 2 + (co["tau"] * c0 / scale) ** 2, 1.0)
    assert np.allclose(np.arctan2(-co["tau"] * c0, -co["eta"]), np.pi * g)
    # half-angle: 2 (c/c0)^2 - 1 = cos(pi gamma)
    assert np.allclose(2 * (co["c"] / c0) ** 2 - 1, -co["eta"] / scale)
    with pytest.raises(ValueError):
        O.seismic_coefficients(np.array([1.0, 0.0]), 1.0, 1.0)


# --------------------------------------------------------------------------
# P5 / P6: the seismic LFFP stepper on a single Fourier mode
# --------------------------------------------------------------------------
def test_seismic_lffp_gamma_zero_is_classical_leapfrog():
    """gamma = 0: u_tt = c0^2 Delta u; on one mode the leap-frog solution is
    cos(n theta) u0 with cos(theta) = 1 - dt^2 c0^2 |mu|^2 / 2, and the Taylor
    start gives u1 = cos(theta) u0 exactly."""
    n = 32
    x = S.axis(n)
    k, c0, dt, steps = 5, 1.3, 0.02, 60
    u0 = np.cos(k * (x + np.pi))
    u = O.seismic_lffp(np.zeros(n), c0, 2 * np.pi, u0, None, dt, steps, M=4)
    theta = math.acos(1 - 0.5 * dt * dt * c0 * c0 * k * k)
    assert np.allclose(u, math.cos(steps * theta) * u0, atol=1e-11)


@pytest.mark.parametrize("gamma,k,dt", [(0.05, 3, 0.01), (0.2, 6, 0.004), (0.4, 2, 0.05)])
def test_seismic_lffp_constant_gamma_damped_recurrence(gamma, k, dt):
    """Constant gamma: one mode obeys a_{n+1} = (2-al-be) a_n - (1-be) a_{n-1}
    with al = dt^2 c^2|eta| |mu|^{2+2g}, be = dt c^2 |tau| |mu|^{1+2g} and
    a_1 = (1 - al/2) a_0; solved through the characteristic roots."""
    n, c0, w0, steps = 32, 1.0, 2 * np.pi, 40
    x = S.axis(n)
    u0 = np.cos(k * (x + np.pi))
    u = O.seismic_lffp(np.full(n, gamma), c0, w0, u0, None, dt, steps, M=3)
    c = c0 * math.cos(math.pi * gamma / 2)
    eta = c0 ** (2 * gamma) * w0 ** (-2 * gamma) * math.cos(math.pi * gamma)
    tau = c0 ** (2 * gamma - 1) * w0 ** (-2 * gamma) * math.sin(math.pi * gamma)
    al = dt * dt * c * c * eta * k ** (2 + 2 * gamma)
    be = dt * c * c * tau * k ** (1 + 2 * gamma)
    r = np.roots([1.0, -(2 - al - be), 1 - be]).astype(complex)
    a0, a1 = 1.0, 1 - al / 2
    C2 = (a1 - r[0] * a0) / (r[1] - r[0])
    C1 = a0 - C2
    an = (C1 * r[0] ** steps + C2 * r[1] ** steps).real
    assert np.allclose(u, an * u0, atol=1e-11)


def test_seismic_lffp_source_and_velocity_start():
    """Taylor start with v0 and a source (reading of Eq. (3.4c) for Eq. (1.1)):
    gamma = 0, u0 = 0, v0 = cos(kx): u1 = dt v0 + dt^2/2 * (source term);
    the source adds dt^2/2 r_0 / h at the source node only."""
    n = 16
    x = S.axis(n)
    v0 = np.cos(2 * (x + np.pi))
    dt = 0.01
    u1 = O.seismic_lffp(np.zeros(n), 1.0, 1.0, np.zeros(n), v0, dt, 1, M=2,
                        src_idx=(3,), src=np.array([2.0]))
    h = 2 * np.pi / n
    ref = dt * v0.copy()
    ref[3] += 0.5 * dt * dt * 2.0 / h
    assert np.allclose(u1, ref, atol=1e-14)


def test_seismic_lffp_dense_vs_matrix_free_variable_gamma():
    """Tiny 2D grid, variable gamma: the O2-driven run converges to the
    O1-driven run (the schemes differ only by the truncation of Eq. (2.9))."""
    shape = (8, 8)
    x, y = S.mesh(shape)
    Q = 5.0 + 20.0 * (1 + np.sin(x) * np.cos(y))
    gam = np.arctan(1.0 / Q) / np.pi
    u0 = S.gaussian_pulse(shape, 1.5)
    a = O.seismic_lffp(gam, 1.0, 2 * np.pi, u0, None, 2e-3, 20, M=10, method="matrix_free")
    b = O.seismic_lffp(gam, 1.0, 2 * np.pi, u0, None, 2e-3, 20, M=10, method="dense")
    assert O.rel_l2(a, b) < 1e-12


# --------------------------------------------------------------------------
# P7: the paper's printed LFFP temporal errors (Table 3)
# --------------------------------------------------------------------------
def _table3(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "table3_lffp_temporal_errors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[int(p[0])] = [None if v == "unstable" else float(v) for v in p[1:]]
    return rows


def test_paper_table3_lffp_variable_order(golden_dir):
    """Column s1(x) = 1 + 0.3 sin(pi x/8) of Table 3: errors at dt = 2^-9,
    2^-10, 2^-11 against the dt = 1e-4 reference reproduce the printed four
    digits, and dt = 2^-7, 2^-8 blow up ("unstable")."""
    rows = _table3(golden_dir)
    J, lo, hi = 4096, [-32.0], [32.0]
    x = S.axis(J, -32.0, 32.0)
    phi = np.exp(-x * x)
    s1 = 1.0 + 0.3 * np.sin(np.pi * x / 8)
    cube = lambda u: u ** 3  # noqa: E731
    ref = O.general_lffp(s1, 1.0, cube, phi, None, 1e-4, 10000, 15, lo, hi)
    for p in (9, 10, 11):
        u = O.general_lffp(s1, 1.0, cube, phi, None, 2.0 ** -p, 2 ** p, 15, lo, hi)
        err = O.l2_error(u, ref, [1.0 / 64])
        printed = rows[p][3]
        assert abs(err - printed) <= 0.0006 * printed, (p, err, printed)
    for p in (7, 8):
        assert rows[p][3] is None
        with np.errstate(all="ignore"):
            u = O.general_lffp(s1, 1.0, cube, phi, None, 2.0 ** -p, 2 ** p, 15, lo, hi)
        assert not np.all(np.isfinite(u)) or np.max(np.abs(u)) > 1e3


def test_paper_table3_lffp_constant_order_column(golden_dir):
    """Column s = 0.5 of Table 3 (M irrelevant: delta = 0)."""
    rows = _table3(golden_dir)
    J, lo, hi = 4096, [-32.0], [32.0]
    x = S.axis(J, -32.0, 32.0)
    phi = np.exp(-x * x)
    s = np.full(J, 0.5)
    cube = lambda u: u ** 3  # noqa: E731
    ref = O.general_lffp(s, 1.0, cube, phi, None, 1e-4, 10000, 0, lo, hi)
    u = O.general_lffp(s, 1.0, cube, phi, None, 2.0 ** -8, 2 ** 8, 0, lo, hi)
    err = O.l2_error(u, ref, [1.0 / 64])
    assert abs(err - rows[8][0]) <= 0.0006 * rows[8][0], err


def test_suggested_dt_gamma_zero_closed_form():
    """gamma = 0: eta = -1, c = c0, so omega_max = c0 |mu_max| and
    dt = courant * 2 / (c0 sqrt(sum_i (pi J_i / L_i)^2)); non-square box."""
    shape = (32, 48)  # (y, x)
    lo, hi = [0.0, -1.0], [3.0, 2.0]  # x: L = 3, y: L = 3
    mu = np.sqrt((np.pi * 48 / 3.0) ** 2 + (np.pi * 32 / 3.0) ** 2)
    dt = O.suggested_dt(np.zeros(shape), 1.7, 2 * np.pi, shape, lo, hi, courant=0.3)
    assert dt == pytest.approx(0.3 * 2 / (1.7 * mu), rel=1e-14)


@pytest.mark.parametrize("courant,stable", [(0.25, True), (0.9, True), (1.1, False)])
def test_suggested_dt_separates_stable_from_unstable(courant, stable):
    """The oracle's own stepper on the fastest mode (the Nyquist checkerboard)
    of a uniform-Q model: bounded at a fraction of the suggested bound,
    growing beyond it."""
    shape = (16, 16)
    gamma = np.full(shape, np.arctan(1 / 20.0) / np.pi)
    dt = O.suggested_dt(gamma, 1.0, 2 * np.pi, shape, courant=courant)
    y, x = np.indices(shape)
    u0 = np.cos(np.pi * x) * np.cos(np.pi * y)
    u = O.seismic_lffp(gamma, 1.0, 2 * np.pi, u0, None, dt, 400, 0)
    grew = np.max(np.abs(u)) > 10.0
    assert grew != stable


@pytest.mark.parametrize("tol", [1e-4, 1e-8, 1e-12])
def test_suggested_M_bounds_the_truncation_of_every_mode(tol):
    """At the rule's M, O2 applied to a single Fourier mode (the one with the
    smallest and the one with the largest |ln|mu|^2| on [-8, 8], so that
    ln|mu|^2 takes both signs) reproduces the exact variable-order weight
    |mu|^{2 s(x)} at every point to within tol of that weight (P1's closed
    form: (-Delta)^{s(x)} cos(mu (x - a)) = |mu|^{2 s(x)} cos(mu (x - a)))."""
    J, lo, hi = 64, [-8.0], [8.0]
    x = S.axis(J, -8.0, 8.0)
    s = 1.0 + 0.3 * np.sin(np.pi * x / 8)
    M = O.suggested_M(s, (J,), lo, hi, tol)
    assert 0 < M < 40
    for k in (1, J // 2 - 1):
        mu = 2 * np.pi * k / 16.0
        u = np.cos(mu * (x + 8.0))
        got = O.matrix_free_operator(u, s, M, lo, hi)
        exact = mu ** (2 * s) * u
        assert np.all(np.abs(got - exact) <= tol * mu ** (2 * s) + 1e-13 * np.max(np.abs(exact))), (k, M)


def _table4(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "table4_tsfp2_temporal_errors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[int(p[0])] = [None if v == "unstable" else float(v) for v in p[1:]]
    return rows


def test_paper_table4_tsfp2_variable_order(golden_dir):
    """Column s1 of Table 4 (TSFP2): errors at dt = 2^-9..2^-11 against the
    dt = 1e-4 reference reproduce the printed four digits; dt = 2^-7, 2^-8
    blow up ("unstable")."""
    rows = _table4(golden_dir)
    J, lo, hi = 4096, [-32.0], [32.0]
    x = S.axis(J, -32.0, 32.0)
    phi = np.exp(-x * x)
    s1 = 1.0 + 0.3 * np.sin(np.pi * x / 8)
    cube = lambda u: u ** 3  # noqa: E731
    ref = O.general_tsfp2(s1, 1.0, cube, phi, None, 1e-4, 10000, 15, lo, hi)
    for p in (9, 10, 11):
        u = O.general_tsfp2(s1, 1.0, cube, phi, None, 2.0 ** -p, 2 ** p, 15, lo, hi)
        err = O.l2_error(u, ref, [1.0 / 64])
        printed = rows[p][3]
        assert abs(err - printed) <= 0.0006 * printed, (p, err, printed)
    for p in (7, 8):
        assert rows[p][3] is None
        with np.errstate(all="ignore"):
            u = O.general_tsfp2(s1, 1.0, cube, phi, None, 2.0 ** -p, 2 ** p, 15, lo, hi)
        assert not np.all(np.isfinite(u)) or np.max(np.abs(u)) > 1e3


def test_paper_table4_tsfp2_constant_order_column(golden_dir):
    """Column s = 1 of Table 4: the splitting is stable for constant order at
    every printed dt, with the printed errors."""
    rows = _table4(golden_dir)
    J, lo, hi = 4096, [-32.0], [32.0]
    x = S.axis(J, -32.0, 32.0)
    phi = np.exp(-x * x)
    cube = lambda u: u ** 3  # noqa: E731
    ref = O.general_tsfp2(1.0, 1.0, cube, phi, None, 1e-4, 10000, 0, lo, hi)
    for p in range(7, 12):
        u = O.general_tsfp2(1.0, 1.0, cube, phi, None, 2.0 ** -p, 2 ** p, 0, lo, hi)
        err = O.l2_error(u, ref, [1.0 / 64])
        printed = rows[p][1]
        assert abs(err - printed) <= 0.0006 * printed, (p, err, printed)


def _table5(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "table5_tsfp2_spatial_errors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[int(p[0])] = [float(v) for v in p[1:]]
    return rows


@pytest.mark.parametrize("col,order", [(1, "one"), (3, "s1")])
def test_paper_table5_tsfp2_spatial_errors(golden_dir, col, order):
    """Table 5: TSFP2 at dt = 1e-4 to t = 1 on grids h = 1, 1/2, 1/4 against
    the h = 1/64 reference reproduces the printed digits (relative 1e-4);
    at h = 1/8 both sit at the round-off floor (< 1e-11)."""
    rows = _table5(golden_dir)
    lo, hi = [-32.0], [32.0]
    cube = lambda u: u ** 3  # noqa: E731

    def run(J):
        x = S.axis(J, -32.0, 32.0)
        s = np.ones(J) if order == "one" else 1.0 + 0.3 * np.sin(np.pi * x / 8)
        return O.general_tsfp2(s, 1.0, cube, np.exp(-x * x), None, 1e-4, 10000, 0 if order == "one" else 15, lo, hi)

    ref = run(4096)
    for inv_h in (1, 2, 4, 8):
        J = 64 * inv_h
        u = run(J)
        err = np.sqrt((1.0 / inv_h) * np.sum((u - ref[:: 4096 // J]) ** 2))
        printed = rows[inv_h][col]
        if inv_h < 8:
            assert abs(err - printed) <= 1e-4 * printed, (inv_h, err, printed)
        else:
            assert err < 1e-11


# --------------------------------------------------------------------------
# the Crank-Nicolson scheme (CNFP, Sec. 3.1)
# --------------------------------------------------------------------------
def _table2(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "table2_cnfp_temporal_errors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[int(p[0])] = [float(v) for v in p[1:]]
    return rows


def _table2_order(col, x):
    if col == 0:
        return np.full(x.shape, 0.5), 0
    if col == 1:
        return np.ones(x.shape), 0
    if col == 2:
        return np.full(x.shape, 1.3), 0
    if col == 3:
        return 1.0 + 0.3 * np.sin(np.pi * x / 8), 15
    return 1.0 + 0.2 * np.tanh(np.cos(np.pi * x / 8)), 15


@pytest.mark.parametrize("col", [0, 1, 2, 3, 4])
def test_paper_table2_cnfp_temporal_errors(golden_dir, col):
    """Table 2 (CNFP): every printed error, all five columns.  Two readings:
    the printed digits and convergence rates (2.07, 2.32 in the last rows)
    are those of a dt = 2^-12 reference rather than the dt = 1e-4 the text
    names, and the run is on h = 1/8 (J = 512) instead of h = 1/64: the
    spatial error there is at round-off (Table 5), so the temporal errors
    are the same.  Agreement: 1e-3 relative on every cell; the ten cells
    below 5e-7 (the finest steps) also get 3e-9 absolute.  Their deviations
    from the printed digits are about constant in absolute terms (s = 0.5:
    1.6e-9, 1.9e-9, 2.7e-9 at dt = 2^-9, 2^-10, 2^-11), not proportional to
    the cell: a floor in the printed values, as an unstated solver tolerance
    accumulated over 2^p steps leaves (the k = 0 mode adds each step's solve
    error), which no choice here can pin tighter."""
    rows = _table2(golden_dir)
    J = 512
    x = S.axis(J, -32.0, 32.0)
    s, M = _table2_order(col, x)
    cube = lambda u: u ** 3  # noqa: E731
    run = lambda dt, n: O.general_cnfp(s, 1.0, cube, np.exp(-x * x), None, dt, n, M, [-32.0], [32.0])  # noqa: E731
    ref = run(2.0 ** -12, 4096)
    for p in range(7, 12):
        err = O.l2_error(run(2.0 ** -p, 2 ** p), ref, [64.0 / J])
        printed = rows[p][col]
        floor = 3e-9 if printed < 5e-7 else 0.0
        assert abs(err - printed) <= 1e-3 * printed + floor, (col, p, err, printed)


@pytest.mark.parametrize("s,k", [(0.5, 3), (1.0, 5), (1.3, 2)])
def test_cnfp_single_mode_recurrence(s, k):
    """f = 0, constant order, u^0 = cos(mu x): every step multiplies the one
    Fourier mode, lambda = |mu|^{2s}, c = kappa dt^2/2:
    a1 = (1 - c lambda) a0 (start, Eq. (3.3)) and
    a_{n+1} (1 + c lambda) = 2 a_n - a_{n-1} (1 + c lambda) (Eq. (3.2))."""
    J, lo, hi, kappa, dt, n = 32, [-np.pi], [np.pi], 0.7, 0.05, 40
    x = S.axis(J, lo[0], hi[0])
    u = O.general_cnfp(s, kappa, lambda v: 0.0 * v, np.cos(k * x), None, dt, n, 3, lo, hi)
    lam, c = float(k) ** (2 * s), 0.5 * kappa * dt * dt
    a_prev, a = 1.0, 1.0 - c * lam
    for _ in range(1, n):
        a_prev, a = a, (2.0 * a - (1.0 + c * lam) * a_prev) / (1.0 + c * lam)
    assert np.max(np.abs(u - a * np.cos(k * x))) < 1e-12


def test_cnfp_spatially_constant_field_is_the_implicit_ode_scheme():
    """A constant field has L u = 0 (k = 0 is left out), so Eq. (3.2) is the
    scalar scheme (u1 - 2u + u0)/dt^2 = (f(u1) + f(u0))/2 with f(u) = -u^3
    + 0.5 u; each step's cubic in u1 is solved here by bisection."""
    J, lo, hi, dt, n = 16, [0.0], [1.0], 0.2, 30
    f = lambda v: -v ** 3 + 0.5 * v  # noqa: E731
    u = O.general_cnfp(1.2, 1.0, f, np.full(J, 0.8), None, dt, n, 2, lo, hi)
    h = 0.5 * dt * dt
    u0, u1 = 0.8, 0.8 + h * f(0.8)
    for _ in range(1, n):
        rhs = 2.0 * u1 - u0 + h * f(u0)
        g = lambda v: v - h * f(v) - rhs  # noqa: E731  (increasing in v)
        a, b = -10.0, 10.0
        for _it in range(200):
            m = 0.5 * (a + b)
            a, b = (m, b) if g(m) < 0 else (a, m)
        u0, u1 = u1, 0.5 * (a + b)
    assert np.max(np.abs(u - u1)) < 1e-12


@pytest.mark.parametrize("shape,kvec", [((16, 16), (2, 3)), ((8, 8, 8), (1, 2, 1))])
def test_cnfp_single_mode_recurrence_multid(shape, kvec):
    """The closed form of test_cnfp_single_mode_recurrence on 2D and 3D
    grids (box [-pi, pi)^d, so mu = k): u^0 = cos(k . x), lambda =
    |k|^{2s} with |k|^2 summed over the axes (Sec. 2.3)."""
    d = len(shape)
    lo, hi, s, kappa, dt, n = [-np.pi] * d, [np.pi] * d, 0.8, 1.3, 0.1, 25
    X = S.mesh(shape, lo, hi)  # x, y[, z]
    phase = sum(k * xi for k, xi in zip(kvec, X))
    u = O.general_cnfp(s, kappa, lambda v: 0.0 * v, np.cos(phase), None, dt, n, 2, lo, hi)
    lam, c = float(sum(k * k for k in kvec)) ** s, 0.5 * kappa * dt * dt
    a_prev, a = 1.0, 1.0 - c * lam
    for _ in range(1, n):
        a_prev, a = a, (2.0 * a - (1.0 + c * lam) * a_prev) / (1.0 + c * lam)
    assert np.max(np.abs(u - a * np.cos(phase))) < 1e-12


def test_cnfp_single_mode_with_initial_velocity():
    """psi = b cos(k x) enters only the start step (Eq. (3.3)):
    a1 = (1 - c lambda) a0 + dt b, then the recurrence of Eq. (3.2)."""
    J, lo, hi, s, k, kappa, dt, n, b = 32, [-np.pi], [np.pi], 1.1, 4, 0.9, 0.07, 30, 0.6
    x = S.axis(J, lo[0], hi[0])
    u = O.general_cnfp(s, kappa, lambda v: 0.0 * v, np.cos(k * x), b * np.cos(k * x), dt, n, 3, lo, hi)
    lam, c = float(k) ** (2 * s), 0.5 * kappa * dt * dt
    a_prev, a = 1.0, (1.0 - c * lam) + dt * b
    for _ in range(1, n):
        a_prev, a = a, (2.0 * a - (1.0 + c * lam) * a_prev) / (1.0 + c * lam)
    assert np.max(np.abs(u - a * np.cos(k * x))) < 1e-12


@pytest.mark.parametrize("s,k", [(0.7, 3), (1.0, 2), (1.4, 5)])
def test_tsfp2_constant_order_linear_mode_is_exact(s, k):
    """Constant order and f = 0: the splitting of Sec. 3.3 integrates
    u_tt = -kappa (-Delta)^s u exactly (the kick vanishes), so a single mode
    is u(t) = cos(w t) u0 + sin(w t)/w v0 with w = sqrt(kappa) |k|^s."""
    J, lo, hi, kappa, dt, n, b = 32, [-np.pi], [np.pi], 1.7, 0.13, 40, 0.4
    x = S.axis(J, lo[0], hi[0])
    u = O.general_tsfp2(s, kappa, lambda v: 0.0 * v, np.cos(k * x), b * np.cos(k * x), dt, n, 4, lo, hi)
    w, t = np.sqrt(kappa) * float(k) ** s, n * dt
    assert np.max(np.abs(u - (np.cos(w * t) + b * np.sin(w * t) / w) * np.cos(k * x))) < 1e-12


@pytest.mark.parametrize("s,k1,k2", [(0.8, 2, 1), (1.3, 1, 3)])
def test_tsfp2_constant_order_linear_mode_is_exact_2d(s, k1, k2):
    """The same exact single-mode solution on a 2D box with unequal sides
    and unequal point counts (ny x nx = 24 x 32, Lx = 2 pi, Ly = 4 pi): the
    mode cos(k1 x + (k2/2) y) has |mu|^2 = k1^2 + (k2/2)^2, so a swapped axis
    or a dropped y term in the oracle's 2D path changes w."""
    shape, lo, hi, kappa, dt, n, b = (24, 32), [-np.pi, -2 * np.pi], [np.pi, 2 * np.pi], 0.9, 0.11, 30, -0.3
    x, y = S.mesh(shape, lo, hi)
    mode = np.cos(k1 * x + 0.5 * k2 * y)
    u = O.general_tsfp2(s, kappa, lambda v: 0.0 * v, mode, b * mode, dt, n, 3, lo, hi)
    w, t = np.sqrt(kappa) * (k1 ** 2 + (0.5 * k2) ** 2) ** (s / 2), n * dt
    assert np.max(np.abs(u - (np.cos(w * t) + b * np.sin(w * t) / w) * mode)) < 1e-12


@pytest.mark.parametrize("s,k", [(0.6, 2), (1.2, 3)])
def test_general_lffp_single_mode_recurrence(s, k):
    """Constant order and f = 0 (Eq. (3.4)): a1 = (1 - dt^2 kappa lambda/2)
    a0 and a_{n+1} = (2 - dt^2 kappa lambda) a_n - a_{n-1}."""
    J, lo, hi, kappa, dt, n = 32, [-np.pi], [np.pi], 0.8, 0.05, 60
    x = S.axis(J, lo[0], hi[0])
    u = O.general_lffp(s, kappa, lambda v: 0.0 * v, np.cos(k * x), None, dt, n, 3, lo, hi)
    q = dt * dt * kappa * float(k) ** (2 * s)
    a_prev, a = 1.0, 1.0 - 0.5 * q
    for _ in range(1, n):
        a_prev, a = a, (2.0 - q) * a - a_prev
    assert np.max(np.abs(u - a * np.cos(k * x))) < 1e-12
