"""Seeded synthetic workloads for the variable-order fractional wave solver.

This module only *builds input data*: quality-factor fields Q(x), initial
wavefields, source positions and source-time samples.  It holds none of the
solver's arithmetic (no fractional operator, no coefficient model, no time
stepping), so both the CPU oracle and the CUDA library can consume its output
without sharing any computation.

Every generator is deterministic given its arguments (numpy PCG64 seeds).
Grids follow the paper's periodic discretisation: x_j = a + j h, h = (b-a)/J,
J even, j = 0..J-1 (Section 2, grid definition above Eq. (2.2)); arrays are
indexed [z][y][x] (x fastest) for 3D, [y][x] for 2D.
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


# ----------------------------------------------------------------------------
# grids
# ----------------------------------------------------------------------------
def axis(n: int, lo: float = -np.pi, hi: float = np.pi) -> np.ndarray:
    """Grid points a + j h, j = 0..n-1, of a periodic axis [lo, hi)."""
    if n <= 0 or n % 2:
        raise ValueError("grid size must be a positive even integer")
    h = (hi - lo) / n
    return lo + h * np.arange(n, dtype=np.float64)


def mesh(shape, lo=None, hi=None):
    """Coordinate arrays (x, y[, z]) for a grid of `shape` given as
    (nx,), (ny, nx) or (nz, ny, nx); returned in x, y, z order, each with the
    full grid shape."""
    d = len(shape)
    lo = [-np.pi] * d if lo is None else list(lo)
    hi = [np.pi] * d if hi is None else list(hi)
    # lo/hi are given in (x, y, z) order
    axes = [axis(shape[d - 1 - i], lo[i], hi[i]) for i in range(d)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")  # (z, y, x) order
    return tuple(grids[::-1])


# ----------------------------------------------------------------------------
# quality-factor fields
# ----------------------------------------------------------------------------
def q_sine_1d(n: int) -> np.ndarray:
    """Q(x) = 20 + 15 sin(x) on [-pi, pi) (the 1D N=256 workload)."""
    x = axis(n)
    return 20.0 + 15.0 * np.sin(x)


def q_lowpass(shape, seed: int, qmin: float = 5.0, qmax: float = 100.0,
              sigma_k: float = 8.0) -> np.ndarray:
    """Smooth random Q field: PCG64(seed) white N(0,1) noise, low-passed by a
    Gaussian exp(-|k|^2 / (2 sigma_k^2)) in integer wavenumbers, then mapped
    affinely so that min -> qmin and max -> qmax."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal(tuple(shape))
    ks = [np.fft.fftfreq(n, d=1.0 / n) for n in shape]
    kk = np.zeros(tuple(shape))
    for i, k in enumerate(ks):
        sh = [1] * len(shape)
        sh[i] = -1
        kk = kk + k.reshape(sh) ** 2
    f = np.fft.ifftn(np.fft.fftn(w) * np.exp(-kk / (2.0 * sigma_k ** 2))).real
    f = (f - f.min()) / (f.max() - f.min())
    return qmin + (qmax - qmin) * f


def q_two_layer_3d(n: int, q_top: float = 10.0, q_bottom: float = 80.0,
                   width_cells: float = 2.0) -> np.ndarray:
    """Two-layer Q on a periodic [-pi,pi)^3 grid: q_top for z > 0 and
    q_bottom for z < 0, blended across both (periodic) interfaces with a tanh
    of width ~`width_cells` cells: Q = q_b + (q_t - q_b)(1 + tanh(beta sin z))/2,
    beta = 1/(width_cells * h_z)."""
    z = axis(n)
    h = TWO_PI / n
    beta = 1.0 / (width_cells * h)
    qz = q_bottom + (q_top - q_bottom) * 0.5 * (1.0 + np.tanh(beta * np.sin(z)))
    return np.broadcast_to(qz[:, None, None], (n, n, n)).copy()


def q_constant(shape, q: float) -> np.ndarray:
    return np.full(tuple(shape), float(q))


# ----------------------------------------------------------------------------
# initial wavefields
# ----------------------------------------------------------------------------
def gauss_1d(n: int, a: float = 20.0) -> np.ndarray:
    """u0(x) = exp(-a x^2) on [-pi, pi)."""
    x = axis(n)
    return np.exp(-a * x * x)


def gaussian_pulse(shape, sigma_cells: float, center=None) -> np.ndarray:
    """Gaussian bump of width sigma_cells grid cells centred at the grid index
    `center` (default: shape//2 in each axis) on [-pi,pi)^d."""
    d = len(shape)
    grids = mesh(shape)
    h = [TWO_PI / shape[d - 1 - i] for i in range(d)]
    if center is None:
        center = [shape[d - 1 - i] // 2 for i in range(d)]  # x, y, z order
    r2 = np.zeros(tuple(shape))
    for i in range(d):
        c = -np.pi + h[i] * center[i]
        r2 = r2 + ((grids[i] - c) / (sigma_cells * h[i])) ** 2
    return np.exp(-0.5 * r2)


def cosine_modes(shape, modes, lo=None, hi=None) -> np.ndarray:
    """u(x) = sum_i a_i cos(k_i . (x - a) * 2pi/L + phi_i) for modes given as
    (a_i, (kx, ky, ...), phi_i) with integer wave numbers."""
    d = len(shape)
    lo = [-np.pi] * d if lo is None else list(lo)
    hi = [np.pi] * d if hi is None else list(hi)
    grids = mesh(shape, lo, hi)
    u = np.zeros(tuple(shape))
    for amp, ks, phi in modes:
        arg = np.zeros(tuple(shape))
        for i in range(d):
            arg = arg + TWO_PI * ks[i] * (grids[i] - lo[i]) / (hi[i] - lo[i])
        u = u + amp * np.cos(arg + phi)
    return u


def random_field(shape, seed: int) -> np.ndarray:
    """Seeded white N(0,1) field (stress input for operator parity)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(tuple(shape))


# ----------------------------------------------------------------------------
# sources
# ----------------------------------------------------------------------------
def ricker_samples(nsteps: int, dt: float, f0: float, t0: float | None = None,
                   amp: float = 1.0) -> np.ndarray:
    """Samples r(t_n), t_n = n dt, n = 0..nsteps-1, of a Ricker wavelet
    amp (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2), t0 = 1/f0 by
    default.  This is source-time input data, passed to both sides."""
    if t0 is None:
        t0 = 1.0 / f0
    t = dt * np.arange(nsteps, dtype=np.float64) - t0
    a = (np.pi * f0 * t) ** 2
    return amp * (1.0 - 2.0 * a) * np.exp(-a)


def center_index(shape):
    """Grid index (x, y, z order) of the domain centre."""
    return tuple(shape[len(shape) - 1 - i] // 2 for i in range(len(shape)))


def random_index(shape, seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    return tuple(int(rng.integers(0, shape[len(shape) - 1 - i]))
                 for i in range(len(shape)))


# ----------------------------------------------------------------------------
# named workloads (the shapes of the paper's problems and of the configs)
# ----------------------------------------------------------------------------
def workload_1d_256():
    """1D periodic [-pi,pi), N=256, Q = 20 + 15 sin x, c0 = 1, omega0 = 2pi,
    M = 8, u0 = exp(-20 x^2), u_t = 0, 200 steps of dt = 1e-3, no source."""
    n = 256
    return dict(shape=(n,), Q=q_sine_1d(n), c0=1.0, omega0=TWO_PI, M=8,
                u0=gauss_1d(n), v0=np.zeros(n), nsteps=200, dt=1e-3,
                src_idx=None, src=None)


def workload_2d_1024(nsteps: int = 1000, n: int = 1024, M: int = 16, seed: int = 2):
    """2D periodic [-pi,pi)^2, 1024^2, Q low-passed noise in [5,100] (seed 2),
    Ricker source f0 = 10 at the centre, u0 = u_t = 0, dt = 5e-4, M = 16."""
    shape = (n, n)
    dt = 5e-4
    return dict(shape=shape, Q=q_lowpass(shape, seed), c0=1.0, omega0=TWO_PI,
                M=M, u0=np.zeros(shape), v0=np.zeros(shape), nsteps=nsteps,
                dt=dt, src_idx=center_index(shape),
                src=ricker_samples(nsteps, dt, 10.0))


def workload_3d_256(nsteps: int = 500, n: int = 256, M: int = 8):
    """3D periodic [-pi,pi)^3, 256^3, two-layer Q (10 above z=0, 80 below),
    Gaussian pulse sigma = 4 cells at the centre, u_t = 0, dt = 2e-3, M = 8."""
    shape = (n, n, n)
    return dict(shape=shape, Q=q_two_layer_3d(n), c0=1.0, omega0=TWO_PI, M=M,
                u0=gaussian_pulse(shape, 4.0), v0=np.zeros(shape),
                nsteps=nsteps, dt=2e-3, src_idx=None, src=None)


def workload_batch(n_sims: int = 64, seed: int = 4, nsteps: int = 300, M: int = 12,
                   sizes=(256, 512, 768, 1024)):
    """Independent 2D simulations on [-pi,pi)^2: edge lengths drawn uniformly
    from `sizes` (PCG64(seed)), Q low-passed noise in [5,100] (seeds
    1000*seed + i), a Ricker source f0 = 10 at a seeded random node (seeds
    1000*seed + 500 + i), u0 = u_t = 0, M = 12, 300 steps.  The time step is
    not part of the input: each consumer derives it from the model (a quarter
    of the leap-frog bound at the fastest point and mode).  Source samples
    are generated by the consumer once dt is known (ricker_samples)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    edges = rng.choice(np.asarray(sizes), size=n_sims)
    sims = []
    for i, n in enumerate(edges):
        shape = (int(n), int(n))
        sims.append(dict(shape=shape, Q=q_lowpass(shape, 1000 * seed + i), c0=1.0, omega0=TWO_PI, M=M,
                         nsteps=nsteps, f0=10.0, src_idx=random_index(shape, 1000 * seed + 500 + i)))
    return sims


SERVE_KINDS = ((4096,), (512, 512), (1024, 1024), (128, 128, 128))


def serve_requests(n_requests: int = 600, seed: int = 5, rate: float = 200.0, kinds=SERVE_KINDS,
                   steps=(100, 2000), M=(8, 16)):
    """A request stream: Poisson arrivals (mean `rate` per second, PCG64
    (seed)), grid shape drawn uniformly from `kinds`, step count uniform in
    [steps[0], steps[1]], M uniform in [M[0], M[1]].  Each request's model
    and source node are seeded by its index (Q: low-passed noise in
    [5, 100], seed 1000*seed + i; Ricker f0 = 10 at a random node, seed
    1000*seed + 500 + i); generate them with serve_inputs().  Domain
    [-pi,pi)^d, c0 = 1, omega0 = 2 pi, u0 = u_t = 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    kind = rng.integers(0, len(kinds), size=n_requests)
    nst = rng.integers(steps[0], steps[1] + 1, size=n_requests)
    ms = rng.integers(M[0], M[1] + 1, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    return [dict(id=i, arrival=float(t[i]), shape=tuple(kinds[kind[i]]), nsteps=int(nst[i]), M=int(ms[i]),
                 c0=1.0, omega0=TWO_PI, f0=10.0, seed=seed) for i in range(n_requests)]


def serve_inputs(req):
    """Q field and source node of one request of serve_requests()."""
    i, seed, shape = req["id"], req["seed"], req["shape"]
    return q_lowpass(shape, 1000 * seed + i), random_index(shape, 1000 * seed + 500 + i)
