"""Oracle: plain float64 NumPy restatement of arXiv 2311.13049.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

Parity status per function (what pins it, see tests/test_oracle_*.py):
  wavenumbers / mu2                pinned (closed forms P1/P2 below)
  seismic_coefficients             pinned (gamma -> 0 limit, invariants)
  dense_operator        (O1)       pinned: cosine-mode closed form (P1)
  matrix_free_operator  (O2)       pinned: truncated-exponential closed form
                                   (P2), convergence to O1 with the Taylor
                                   remainder bound (P3), special cases (P4)
  seismic_lffp          (O3)       pinned only through single-mode closed
                                   forms (P5: gamma = 0 leap-frog, P6: constant
                                   gamma damped recurrence).  The paper prints
                                   no number for the seismic run itself, so a
                                   variable-gamma full run is "parity
                                   unpinned" beyond those reductions.
  general_lffp          (O4)       pinned: the paper's printed LFFP temporal
                                   errors (Table 3, Sec. 3.2) are reproduced (P7),
                                   and the single-mode leap-frog recurrence.
  general_tsfp2         (O4)       pinned: the paper's printed TSFP2 temporal
                                   and spatial errors (Tables 4, 5, Sec. 3.3) are
                                   reproduced, and a constant-order linear mode
                                   is integrated exactly.
  general_cnfp          (O4)       pinned: the paper's printed CNFP temporal
                                   errors (Table 2, Sec. 3.1) are reproduced,
                                   single-mode closed form (f = 0), and the
                                   scalar implicit scheme for a constant field.
  operator_matrix                  O2 applied to unit fields (pinned with O2).
  suggested_dt                     pinned: gamma = 0 closed form and the
                                   stability of the single-mode recurrence of
                                   the step on both sides of the bound.
  suggested_M                      pinned: the truncation error of O2 at the
                                   chosen M (against O2 at M = 40) is within
                                   the tolerance.

Conventions (readings of the paper where it is silent or ambiguous):
  * arrays are indexed [z][y][x] (x fastest); `lo`, `hi` are (x, y, z) ordered;
  * the frequency index set of each axis is k = -J/2 .. J/2-1 (Sec. 2, Eq. (2.2));
    mu_k = 2 pi k / (b - a); |mu_k|^2 = sum over axes (Sec. 2.3, below Eq. (2.12));
  * u_hat_k = (1/N) sum_j u_j exp(-i mu_k . (x_j - a))  (Sec. 2, under Eq. (2.2)).
"""
from __future__ import annotations

import functools
import math

import numpy as np

__all__ = [
    "grid_spacing", "wavenumbers", "mu2", "fourier_coefficients",
    "seismic_coefficients", "seismic_coefficients_from_gamma",
    "dense_operator", "matrix_free_operator", "matrix_free_terms",
    "seismic_operators", "seismic_lffp", "general_lffp",
    "l2_error", "rel_l2", "taylor_remainder_bound", "suggested_dt", "suggested_M",
    "general_tsfp2", "general_cnfp", "operator_matrix",
]


def _dims(u_shape, lo, hi):
    d = len(u_shape)
    lo = [-np.pi] * d if lo is None else [float(v) for v in lo]
    hi = [np.pi] * d if hi is None else [float(v) for v in hi]
    if len(lo) != d or len(hi) != d:
        raise ValueError("lo/hi must have one entry per dimension")
    for n in u_shape:
        if n <= 0 or n % 2:
            raise ValueError("each J_m must be a positive even integer (Sec. 2)")
    return d, lo, hi


def grid_spacing(shape, lo=None, hi=None):
    """h_m = (b_m - a_m)/J_m, returned in (x, y, z) order (Sec. 2.3)."""
    d, lo, hi = _dims(shape, lo, hi)
    return [(hi[i] - lo[i]) / shape[d - 1 - i] for i in range(d)]


def wavenumbers(J: int, a: float, b: float):
    """Signed integer index k (in DFT storage order: 0..J/2-1, -J/2..-1) and
    mu_k = 2 pi k / (b - a) of one axis (Sec. 2, definition under Eq. (2.2)).
    The Nyquist entry carries k = -J/2, as in the index set -J/2..J/2-1."""
    k = np.fft.fftfreq(J, d=1.0 / J)  # 0..J/2-1, -J/2..-1 (exact integers)
    k = np.round(k).astype(np.int64)
    return k, 2.0 * np.pi * k / (b - a)


def mu2(shape, lo=None, hi=None) -> np.ndarray:
    """|mu_k|^2 = sum_m (mu^{(m)}_{k_m})^2 on the DFT-ordered frequency grid
    (Sec. 2.3, the definition following Eq. (2.12); the paper's product sign
    in the phase is read as the dot product)."""
    d, lo, hi = _dims(shape, lo, hi)
    out = np.zeros(tuple(shape))
    for i in range(d):  # i = 0 -> x (last array axis)
        J = shape[d - 1 - i]
        _, mu = wavenumbers(J, lo[i], hi[i])
        sh = [1] * d
        sh[d - 1 - i] = J
        out = out + (mu ** 2).reshape(sh)
    return out


def fourier_coefficients(u: np.ndarray) -> np.ndarray:
    """u_hat_k = (prod 1/J_m) sum_j u_j e^{-i mu_k . (x_j - a)}, DFT order
    (Sec. 2.3, coefficient formula under Eq. (2.11)).  Since mu_k (x_j - a) =
    2 pi k j / J, this is numpy's forward DFT divided by N."""
    return np.fft.fftn(u) / u.size


# ----------------------------------------------------------------------------
# seismic model coefficients (Sec. 1, coefficients under Eq. (1.1))
# ----------------------------------------------------------------------------
def seismic_coefficients_from_gamma(gamma, c0, omega0):
    """c = c0 cos(pi gamma/2), eta = -c0^{2 gamma} omega0^{-2 gamma} cos(pi gamma),
    tau = -c0^{2 gamma - 1} omega0^{-2 gamma} sin(pi gamma)  (Sec. 1).
    c0 may be a scalar or a field (Example 3 uses a layered c0)."""
    g = np.asarray(gamma, dtype=np.float64)
    c0 = np.asarray(c0, dtype=np.float64)
    c = c0 * np.cos(np.pi * g / 2.0)
    eta = -(c0 ** (2.0 * g)) * omega0 ** (-2.0 * g) * np.cos(np.pi * g)
    tau = -(c0 ** (2.0 * g - 1.0)) * omega0 ** (-2.0 * g) * np.sin(np.pi * g)
    return dict(gamma=g, c=c, eta=eta, tau=tau)


def seismic_coefficients(Q, c0, omega0):
    """gamma = arctan(1/Q)/pi, then the coefficients above (Sec. 1)."""
    Q = np.asarray(Q, dtype=np.float64)
    if np.any(Q <= 0):
        raise ValueError("the quality factor Q must be positive (Sec. 1)")
    gamma = np.arctan(1.0 / Q) / np.pi
    return seismic_coefficients_from_gamma(gamma, c0, omega0)


# ----------------------------------------------------------------------------
# O1: the dense Fourier pseudospectral operator
# ----------------------------------------------------------------------------
def _natural_k(J):
    return np.arange(-J // 2, J // 2, dtype=np.int64)


def dense_operator(u, s, lo=None, hi=None, points=None, chunk=64):
    """(-Delta)_h^{s(x_j)} u_j = sum_{k in S_xi} |mu_k|^{2 s(x_j)} u_hat_k
    e^{i mu_k . (x_j - a)}  (Eq. (2.3) in 1D, Eq. (2.12) in d dimensions;
    S_xi excludes k = 0).

    The sum over k is carried out explicitly at every requested grid point
    (O(N) per point, O(N^2) for all points).  `points` is an optional integer
    array of flat grid indices; the default is every point.  Returns the real
    part, after checking the imaginary part is at round-off level."""
    u = np.asarray(u, dtype=np.float64)
    s = np.broadcast_to(np.asarray(s, dtype=np.float64), u.shape)
    d, lo, hi = _dims(u.shape, lo, hi)
    uhat = fourier_coefficients(u)
    # natural-order index set per axis, and the matching u_hat entries
    ks = [None] * d
    mus = [None] * d
    for i in range(d):
        J = u.shape[d - 1 - i]
        ks[i] = _natural_k(J)
        mus[i] = 2.0 * np.pi * ks[i] / (hi[i] - lo[i])
    # flattened list of all k in S_xi^0 (x fastest like the arrays)
    grids_k = np.meshgrid(*[ks[i] for i in reversed(range(d))], indexing="ij")
    kflat = [grids_k[d - 1 - i].ravel() for i in range(d)]  # x, y, z order
    mu_sq = np.zeros(kflat[0].shape)
    for i in range(d):
        mu_sq = mu_sq + (2.0 * np.pi * kflat[i] / (hi[i] - lo[i])) ** 2
    idx = tuple(kflat[d - 1 - a] % u.shape[a] for a in range(d))
    uh = uhat[idx]
    keep = mu_sq > 0  # S_xi: k != 0
    mu_sq, uh = mu_sq[keep], uh[keep]
    kflat = [k[keep] for k in kflat]
    h = grid_spacing(u.shape, lo, hi)
    if points is None:
        points = np.arange(u.size)
    points = np.asarray(points, dtype=np.int64)
    jidx = np.unravel_index(points, u.shape)  # (z, y, x) order
    out = np.empty(points.size, dtype=np.complex128)
    log_mu_sq = np.log(mu_sq)
    for p0 in range(0, points.size, chunk):
        sl = slice(p0, min(points.size, p0 + chunk))
        phase = np.zeros((sl.stop - sl.start, mu_sq.size))
        for i in range(d):
            xj_minus_a = h[i] * jidx[d - 1 - i][sl]
            phase += np.outer(xj_minus_a, 2.0 * np.pi * kflat[i] / (hi[i] - lo[i]))
        sj = s.ravel()[points[sl]]
        mult = np.exp(np.outer(sj, log_mu_sq))  # |mu|^{2 s_j} = (|mu|^2)^{s_j}
        out[sl] = (mult * np.exp(1j * phase)) @ uh
    scale = max(1.0, float(np.max(np.abs(out))))
    if np.max(np.abs(out.imag)) > 1e-9 * scale:
        raise AssertionError("dense operator produced a non-real result")
    res = out.real
    if points.size == u.size and np.all(points == np.arange(u.size)):
        return res.reshape(u.shape)
    return res


# ----------------------------------------------------------------------------
# O2: the accelerated matrix-free scheme
# ----------------------------------------------------------------------------
@functools.lru_cache(maxsize=4)
def _multiplier_tables(shape, lo, hi, s0, M):
    """P_m(k) = (ln|mu_k|^2)^m / m! * |mu_k|^{2 s0} for m = 0..M, with
    P_m(0) = 0 (k = 0 is excluded from S_xi), DFT-ordered (Eq. (2.13)).
    These do not depend on x, so one run reuses them."""
    m2 = mu2(shape, list(lo), list(hi))
    nz = m2 > 0
    L = np.zeros_like(m2)
    L[nz] = np.log(m2[nz])
    P0 = np.zeros_like(m2)
    P0[nz] = m2[nz] ** s0  # |mu|^{2 s0} = (|mu|^2)^{s0}
    tables = []
    for m in range(M + 1):
        Pm = np.zeros_like(m2)
        Pm[nz] = P0[nz] * L[nz] ** m / math.factorial(m)
        tables.append(Pm)
    return tuple(tables)


def matrix_free_terms(u, s0, M, lo=None, hi=None):
    """Inner sums of Eq. (2.10)/(2.13): for m = 0..M,
    Y_m(x_j) = sum_{k in S_xi} [(ln|mu_k|^2)^m / m!] |mu_k|^{2 s0} u_hat_k
               e^{i mu_k . (x_j - a)},
    each evaluated by one inverse DFT (numpy's ifftn times N)."""
    u = np.asarray(u, dtype=np.float64)
    d, lo, hi = _dims(u.shape, lo, hi)
    uhat = fourier_coefficients(u)
    tables = _multiplier_tables(u.shape, tuple(lo), tuple(hi), float(s0), int(M))
    return [(np.fft.ifftn(Pm * uhat) * u.size).real for Pm in tables]


def matrix_free_operator(u, s, M, lo=None, hi=None, s0=None):
    """Eq. (2.10) (1D) / Eq. (2.13) (d-dim):
    (-Delta)_h^{s(x_j)} u_j ~= sum_{m=0}^{M} [s(x_j) - s0]^m Y_m(x_j),
    with s0 the domain average of s (Eq. (2.13); on the periodic grid the
    average is the grid mean)."""
    u = np.asarray(u, dtype=np.float64)
    s = np.broadcast_to(np.asarray(s, dtype=np.float64), u.shape)
    if s0 is None:
        s0 = float(np.mean(s))
    d, lo, hi = _dims(u.shape, lo, hi)
    uhat = fourier_coefficients(u)
    tables = _multiplier_tables(u.shape, tuple(lo), tuple(hi), float(s0), int(M))
    delta = s - s0
    out = np.zeros(u.shape)
    dpow = np.ones(u.shape)  # [s(x_j) - s0]^m
    for Pm in tables:
        Y = np.fft.ifftn(Pm * uhat) * u.size
        out = out + dpow * Y.real
        dpow = dpow * delta
    return out


def taylor_remainder_bound(u, s, M, lo=None, hi=None, s0=None):
    """Per-point bound on |O2 - O1| from the Lagrange remainder of the
    Taylor expansion Eq. (2.8): |a^z - a^{z0} e_M((z-z0) ln a)| <=
    a^{z0} |(z-z0) ln a|^{M+1}/(M+1)! e^{|(z-z0) ln a|}, summed over k with
    |u_hat_k| weights."""
    u = np.asarray(u, dtype=np.float64)
    s = np.broadcast_to(np.asarray(s, dtype=np.float64), u.shape)
    if s0 is None:
        s0 = float(np.mean(s))
    uhat = np.abs(fourier_coefficients(u)).ravel()
    m2 = mu2(u.shape, lo, hi).ravel()
    nz = m2 > 0
    uhat, m2 = uhat[nz], m2[nz]
    L = np.abs(np.log(m2))
    P0 = m2 ** s0
    dl = np.abs(s.ravel() - s0)
    z = np.outer(dl, L)
    rem = (z ** (M + 1) / math.factorial(M + 1)) * np.exp(z)
    return (rem * (P0 * uhat)[None, :]).sum(axis=1).reshape(u.shape)


# ----------------------------------------------------------------------------
# the two seismic operators and the seismic leap-frog (LFFP) stepper
# ----------------------------------------------------------------------------
def seismic_operators(u, gamma, M, lo=None, hi=None, method="matrix_free"):
    """L1 u = (-Delta)^{1+gamma(x)} u and L2 u = (-Delta)^{1/2+gamma(x)} u of
    Eq. (1.1), each by O2 (Eq. (2.13)) or O1 (Eq. (2.12)).  The expansion
    centres are the grid means s0 = 1 + gamma0 and s0 = 1/2 + gamma0."""
    g = np.broadcast_to(np.asarray(gamma, dtype=np.float64), np.shape(u))
    if method == "matrix_free":
        return (matrix_free_operator(u, 1.0 + g, M, lo, hi),
                matrix_free_operator(u, 0.5 + g, M, lo, hi))
    if method == "dense":
        return dense_operator(u, 1.0 + g, lo, hi), dense_operator(u, 0.5 + g, lo, hi)
    raise ValueError(method)


def seismic_lffp(gamma, c0, omega0, u0, v0, dt, nsteps, M, lo=None, hi=None,
                 src_idx=None, src=None, method="matrix_free", return_all=False):
    """Leap-frog Fourier pseudospectral run of the seismic model Eq. (1.1)
    u_tt = c^2 [eta L1 u + tau d/dt (L2 u)] (+ a point source), L1, L2 as
    above; A = c^2 eta, B = c^2 tau.

    Readings (the paper states LFFP only for the general model Eq. (1.5);
    Sec. 3.2, Eq. (3.4)):
      step  n >= 1: u^{n+1} = 2u^n - u^{n-1}
                    + dt^2 [A L1 u^n + B (L2 u^n - L2 u^{n-1})/dt + r_n e_s / h^d]
      start n = 0 : u^1 = u^0 + dt v0 + dt^2/2 [A L1 u^0 + B L2 v0 + r_0 e_s/h^d]
                    (the Taylor start of Eq. (3.4c) with u_tt(0) from Eq. (1.1))
    where e_s is the unit vector of the source node and r_n the source sample
    at t_n.  `nsteps` counts the start step, so the result is u^{nsteps}."""
    u0 = np.asarray(u0, dtype=np.float64)
    v0 = np.zeros_like(u0) if v0 is None else np.asarray(v0, dtype=np.float64)
    coef = seismic_coefficients_from_gamma(np.broadcast_to(gamma, u0.shape), c0, omega0)
    A = coef["c"] ** 2 * coef["eta"]
    B = coef["c"] ** 2 * coef["tau"]
    h = grid_spacing(u0.shape, lo, hi)
    hd = float(np.prod(h))
    d = u0.ndim

    def source(n):
        f = np.zeros_like(u0)
        if src_idx is not None and src is not None:
            f[tuple(src_idx[d - 1 - a] for a in range(d))] = src[n] / hd
        return f

    ops = lambda w: seismic_operators(w, gamma, M, lo, hi, method)  # noqa: E731
    history = [u0.copy()]
    if nsteps <= 0:
        return (u0.copy(), history) if return_all else u0.copy()
    L1u, L2u = ops(u0)
    L2v = ops(v0)[1] if np.any(v0) else np.zeros_like(u0)
    u_prev = u0
    u = u0 + dt * v0 + 0.5 * dt * dt * (A * L1u + B * L2v + source(0))
    L2_prev = L2u
    history.append(u.copy())
    for n in range(1, nsteps):
        L1u, L2u = ops(u)
        u_next = (2.0 * u - u_prev
                  + dt * dt * (A * L1u + B * (L2u - L2_prev) / dt + source(n)))
        u_prev, u, L2_prev = u, u_next, L2u
        if return_all:
            history.append(u.copy())
    return (u, history) if return_all else u


def suggested_M(s, shape, lo=None, hi=None, tol=1e-8, M_max=40):
    """Smallest M with max_k R_M <= tol, R_M = a^{M+1}/(M+1)! e^{2a},
    a = max_x |s(x) - s0| * max_k |ln |mu_k|^2| (k != 0), s0 = grid mean.

    Reading: in Eq. (2.13) the mode k at x carries |mu_k|^{2 s0}
    exp(delta(x) ln|mu_k|^2); truncating the exponential series after the
    power M leaves at most |z|^{M+1}/(M+1)! e^{|z|} (z = delta ln|mu|^2,
    Taylor remainder), i.e. at most R_M relative to the mode's exact weight
    |mu_k|^{2s0} e^{z} >= |mu_k|^{2s0} e^{-|z|}.  The paper's indicator
    e(M, mu_k) (Sec. 2.2) assumes only |s - s0| < 1; this uses the model's
    own |delta|."""
    s = np.asarray(s, dtype=np.float64)
    d, a_lo, b_hi = _dims(shape, lo, hi)
    L = [b_hi[i] - a_lo[i] for i in range(d)]
    mu_min = min(2.0 * math.pi / Li for Li in L)
    mu_max = math.sqrt(sum((math.pi * shape[d - 1 - i] / L[i]) ** 2 for i in range(d)))
    lmax = max(abs(math.log(mu_min ** 2)), abs(math.log(mu_max ** 2)))
    a = float(np.max(np.abs(s - s.mean()))) * lmax
    term = a * math.exp(2.0 * a)  # R_0
    for M in range(M_max + 1):
        if term <= tol:
            return M
        term *= a / (M + 2)
    return M_max


def suggested_dt(gamma, c0, omega0, shape, lo=None, hi=None, courant=0.25):
    """Time step of the built-in workloads: courant * 2 / omega_max with
    omega_max = max_x c |eta|^{1/2} |mu_max|^{1 + gamma(x)}, |mu_max|^2 the
    sum over axes of the squared Nyquist wavenumbers (pi J / (b - a))^2.

    Reading: the undamped part of the step (Eq. (3.4) applied to Eq. (1.1))
    maps a Fourier mode of frequency omega by the recurrence
    u^{n+1} = (2 - (dt omega)^2) u^n - u^{n-1}, stable for dt omega < 2; the
    paper gives no time-step rule for the seismic runs, so the workloads take
    a quarter of the largest stable step at the fastest point and mode."""
    d, a, b = _dims(shape, lo, hi)
    mu_max2 = sum((math.pi * shape[d - 1 - i] / (b[i] - a[i])) ** 2 for i in range(d))
    coef = seismic_coefficients_from_gamma(np.broadcast_to(gamma, shape), c0, omega0)
    g = coef["gamma"]
    w = coef["c"] * np.sqrt(np.abs(coef["eta"])) * mu_max2 ** ((1.0 + g) / 2.0)
    return courant * 2.0 / float(np.max(w))


# ----------------------------------------------------------------------------
# O4: the general model's LFFP scheme (Eq. (1.5), Sec. 3.2, Eq. (3.4))
# ----------------------------------------------------------------------------
def general_lffp(s, kappa, f, phi, psi, dt, nsteps, M, lo=None, hi=None,
                 method="matrix_free"):
    """u^{n+1} = 2u^n - u^{n-1} + dt^2 (-kappa L_s u^n + f(u^n)),
    u^1 = phi + dt psi + dt^2/2 (-kappa L_s phi + f(phi))  (Eq. (3.4a-c)), with
    L_s the variable-order operator by O2 (default) or O1."""
    phi = np.asarray(phi, dtype=np.float64)
    psi = np.zeros_like(phi) if psi is None else np.asarray(psi, dtype=np.float64)
    if method == "matrix_free":
        op = lambda w: matrix_free_operator(w, s, M, lo, hi)  # noqa: E731
    else:
        op = lambda w: dense_operator(w, s, lo, hi)  # noqa: E731
    u_prev = phi
    u = phi + dt * psi + 0.5 * dt * dt * (-kappa * op(phi) + f(phi))
    for _ in range(1, nsteps):
        u_next = 2.0 * u - u_prev + dt * dt * (-kappa * op(u) + f(u))
        u_prev, u = u, u_next
        if not np.all(np.isfinite(u)):
            break
    return u


def operator_matrix(s, M, shape, lo=None, hi=None):
    """The N x N matrix of the M-term matrix-free operator O2 on a grid of
    `shape` (N points, flattened x fastest): column l is O2 applied to the
    l-th unit field."""
    shape = tuple(shape)
    n = int(np.prod(shape))
    cols = np.empty((n, n))
    e = np.zeros(n)
    for l in range(n):
        e[l] = 1.0
        cols[:, l] = matrix_free_operator(e.reshape(shape), s, M, lo, hi).ravel()
        e[l] = 0.0
    return cols


def general_cnfp(s, kappa, f, phi, psi, dt, nsteps, M, lo=None, hi=None, tol=1e-14, maxit=100):
    """Crank-Nicolson Fourier pseudospectral method (Sec. 3.1): u^0 = phi and
    the explicit start u^1 = phi + dt psi + dt^2/2 (-kappa L_s phi + f(phi))
    (Eq. (3.3)); then for n >= 1 u^{n+1} is the solution v of the nonlinear
    system of Eq. (3.2), the Crank-Nicolson form of Eq. (3.1),
        v + (kappa dt^2/2) L_s v - (dt^2/2) f(v)
          = 2 u^n - u^{n-1} - (kappa dt^2/2) L_s u^{n-1} + (dt^2/2) f(u^{n-1}),
    with L_s the matrix-free operator O2 as a dense matrix.  The system has
    one solution near u^n for the step sizes used here, so the oracle
    computes it by its plainest route instead of the paper's conjugate
    gradients: A = I + (kappa dt^2/2) L_s is LU-factored once, and the cubic
    term is handled by the fixed-point iteration v <- A^{-1}(rhs + (dt^2/2)
    f(v)) from v = 2 u^n - u^{n-1}, until two iterates differ by at most
    tol * max(1, |v|_inf).  Returns u^{nsteps}."""
    import scipy.linalg

    phi = np.asarray(phi, dtype=np.float64)
    shape = phi.shape
    psi = np.zeros_like(phi) if psi is None else np.asarray(psi, dtype=np.float64)
    L = operator_matrix(s, M, shape, lo, hi)
    c = 0.5 * kappa * dt * dt
    h2 = 0.5 * dt * dt
    lu = scipy.linalg.lu_factor(np.eye(L.shape[0]) + c * L)
    u_prev = phi.ravel()
    u = u_prev + dt * psi.ravel() + h2 * (-kappa * (L @ u_prev) + f(u_prev))
    if nsteps == 0:
        return phi.copy()
    for _ in range(1, nsteps):
        rhs = 2.0 * u - u_prev - c * (L @ u_prev) + h2 * f(u_prev)
        v = 2.0 * u - u_prev
        for _it in range(maxit):
            v_new = scipy.linalg.lu_solve(lu, rhs + h2 * f(v))
            done = np.max(np.abs(v_new - v)) <= tol * max(1.0, float(np.max(np.abs(v_new))))
            v = v_new
            if done:
                break
        else:
            raise RuntimeError("CNFP fixed-point iteration did not converge")
        u_prev, u = u, v
    return u.reshape(shape)


def general_tsfp2(s, kappa, f, phi, psi, dt, nsteps, M, lo=None, hi=None):
    """Second-order time-splitting Fourier pseudospectral method (Sec. 3.3,
    Strang splitting of u_t = v, v_t = -kappa (-Delta)^{s(x)} u + f(u)):
    per step, the constant-order part u_t = v, v_t = -kappa (-Delta)^{s0} u
    is integrated exactly in Fourier space over dt/2 (frequency
    w_k = sqrt(kappa) |mu_k|^{s0}; k = 0 drifts: u += t v), then the rest
    u_t = 0, v_t = -kappa [(-Delta)^{s(x)} - (-Delta)^{s0}] u + f(u) exactly
    over dt, then the first part again over dt/2.  The difference operator
    is the matrix-free sum of Eq. (2.13) without its m = 0 term (readings of
    the printed typos: |mu|^{2 s0} in the constant-order symbol, one u_hat
    factor in v_hat, no kappa inside the difference operator, the kick
    v += dt (-kappa (...) + f(u)), and steps n = 0, 1, ...).  Returns
    u^{nsteps}; u^0 = phi, v^0 = psi exactly."""
    u = np.asarray(phi, dtype=np.float64).copy()
    v = np.zeros_like(u) if psi is None else np.asarray(psi, dtype=np.float64).copy()
    s = np.broadcast_to(np.asarray(s, dtype=np.float64), u.shape)
    s0 = float(np.mean(s))
    delta = s - s0
    w = np.sqrt(kappa) * mu2(u.shape, lo, hi) ** (s0 / 2.0)
    moving = w > 0
    wsafe = np.where(moving, w, 1.0)

    def linear(u, v, t):
        uh, vh = np.fft.fftn(u), np.fft.fftn(v)
        c, sn = np.cos(w * t), np.sin(w * t)
        uh2 = np.where(moving, uh * c + vh * sn / wsafe, uh + t * vh)
        vh2 = np.where(moving, -wsafe * uh * sn + vh * c, vh)
        return np.fft.ifftn(uh2).real, np.fft.ifftn(vh2).real

    for _ in range(nsteps):
        u, v = linear(u, v, 0.5 * dt)
        terms = matrix_free_terms(u, s0, M, lo, hi)
        diff = np.zeros_like(u)
        dpow = np.ones_like(u)
        for m in range(1, M + 1):
            dpow = dpow * delta
            diff = diff + dpow * terms[m]
        v = v + dt * (-kappa * diff + f(u))
        u, v = linear(u, v, 0.5 * dt)
        if not np.all(np.isfinite(u)):
            break
    return u


# ----------------------------------------------------------------------------
# norms
# ----------------------------------------------------------------------------
def l2_error(a, b, h):
    """Discrete l2 norm sqrt(prod(h) sum |a-b|^2) used for the paper's error
    tables (the norm is unstated there; this is the reading)."""
    h = np.atleast_1d(h)
    return float(np.sqrt(np.prod(h) * np.sum((np.asarray(a) - np.asarray(b)) ** 2)))


def rel_l2(x, ref):
    """||x - ref||_2 / ||ref||_2 over all points."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref.ravel())
    return float(np.linalg.norm((x - ref).ravel()) / (den if den > 0 else 1.0))
