"""GPU parity of one operator application (Eq. (2.13)) against the FP64
oracle, element by element, on the same (FP32-rounded) input.

Tolerance: relative L2 error <= 1e-5 per FP32 apply (the stated bound for
one operator application); FP64 plain path <= 1e-11.  Inputs are seeded
synthetic fields of the workloads' kind (low-passed Q in [5,100], smooth and
white wavefields)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_util import gpu_apply_pair, gamma_of, rel_l2, check

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-11


def _case(shape, seed):
    Q = S.q_lowpass(shape, seed)
    u = S.q_lowpass(shape, seed + 100, qmin=-1.0, qmax=1.0, sigma_k=max(shape) / 8)
    return Q, u


@pytest.mark.parametrize("shape", [(64, 64), (128, 128), (256, 256), (512, 512), (768, 768), (1024, 1024),
                                   (128, 256), (256, 128), (64, 512), (512, 64), (256, 1024)])
def test_fused_apply_matches_oracle_sizes(V, shape):
    Q, u = _case(shape, 7)
    M = 8
    g1, g2, uin = gpu_apply_pair(V, shape, Q, u, M, V.IMPL_FUSED, V.F32)
    r1, r2 = O.seismic_operators(uin, gamma_of(Q), M)
    check(g1, r1, TOL32)
    check(g2, r2, TOL32)


@pytest.mark.parametrize("M", [0, 1, 5, 6, 7, 11, 12, 13, 16, 20])
def test_fused_apply_taylor_groups(V, M):
    """M around multiples of the group size (6 terms per group): the Horner
    accumulation across groups and the ragged last group."""
    shape = (128, 128)
    Q, u = _case(shape, 3)
    g1, g2, uin = gpu_apply_pair(V, shape, Q, u, M, V.IMPL_FUSED, V.F32)
    r1, r2 = O.seismic_operators(uin, gamma_of(Q), M)
    check(g1, r1, TOL32)
    check(g2, r2, TOL32)


def test_fused_apply_white_noise_and_nyquist(V):
    """A white field loads every frequency including both Nyquist lines."""
    shape = (256, 256)
    Q = S.q_lowpass(shape, 5)
    u = S.random_field(shape, 9)
    u[:, :] += np.cos(np.pi * np.arange(256))[None, :]  # x-Nyquist mode
    u[:, :] += 0.5 * np.cos(np.pi * np.arange(256))[:, None]  # y-Nyquist mode
    g1, g2, uin = gpu_apply_pair(V, shape, Q, u, 8, V.IMPL_FUSED, V.F32)
    r1, r2 = O.seismic_operators(uin, gamma_of(Q), 8)
    check(g1, r1, TOL32)
    check(g2, r2, TOL32)


@pytest.mark.parametrize("impl", ["fused", "plain"])
def test_radix3_grid_white_noise(V, impl):
    """768^2 (a factor 3 in every line length): a white field with both
    Nyquist lines loads every twiddle of the mixed-radix transforms."""
    shape = (768, 768)
    Q = S.q_lowpass(shape, 6)
    u = S.random_field(shape, 10)
    u += np.cos(np.pi * np.arange(768))[None, :] + 0.5 * np.cos(np.pi * np.arange(768))[:, None]
    im = V.IMPL_FUSED if impl == "fused" else V.IMPL_PLAIN
    g1, g2, uin = gpu_apply_pair(V, shape, Q, u, 12, im, V.F32)
    r1, r2 = O.seismic_operators(uin, gamma_of(Q), 12)
    check(g1, r1, TOL32)
    check(g2, r2, TOL32)


def test_fused_apply_non_square_box(V):
    """Unequal box lengths: |mu|^2 mixes 2 pi k / L_x and 2 pi k / L_y."""
    shape = (128, 256)
    lo, hi = [0.0, -1.0], [2.0, 3.0]
    Q, u = _case(shape, 11)
    g1, g2, uin = gpu_apply_pair(V, shape, Q, u, 6, V.IMPL_FUSED, V.F32, lo, hi)
    r1, r2 = O.seismic_operators(uin, gamma_of(Q), 6, lo, hi)
    check(g1, r1, TOL32)
    check(g2, r2, TOL32)


@pytest.mark.parametrize("shape", [(256,), (4096,), (128, 128), (32, 32, 32)])
def test_plain_apply_matches_oracle(V, shape):
    Q, u = _case(shape, 13)
    g1, g2, uin = gpu_apply_pair(V, shape, Q, u, 8, V.IMPL_PLAIN, V.F32)
    r1, r2 = O.seismic_operators(uin, gamma_of(Q), 8)
    check(g1, r1, TOL32)
    check(g2, r2, TOL32)
    g1, g2, uin = gpu_apply_pair(V, shape, Q, u, 8, V.IMPL_PLAIN, V.F64)
    r1, r2 = O.seismic_operators(uin, gamma_of(Q), 8)
    check(g1, r1, TOL64)
    check(g2, r2, TOL64)


def test_constant_q_single_mode_closed_form(V):
    """Uniform Q: delta = 0 and each operator is |mu|^{2 s} on a Fourier mode
    (Eq. (1.3)); checked against the closed form, not the oracle."""
    shape = (128, 256)
    Q = np.full(shape, 20.0)
    x, y = S.mesh(shape)
    kx, ky = 5, 3
    u = np.cos(kx * (x + np.pi) + ky * (y + np.pi))
    g1, g2, uin = gpu_apply_pair(V, shape, Q, u, 4, V.IMPL_FUSED, V.F32)
    gam = np.arctan(1 / 20.0) / np.pi
    m2 = kx * kx + ky * ky
    check(g1, m2 ** (1 + gam) * uin, TOL32)
    check(g2, m2 ** (0.5 + gam) * uin, TOL32)


def test_headline_size_per_apply_tolerance(V):
    """2D 1024^2, M = 16 (the headline workload's operator) on a wavefield
    of the workload's kind: a Ricker-like ring plus the low-passed field."""
    shape = (1024, 1024)
    Q = S.q_lowpass(shape, 2)
    x, y = S.mesh(shape)
    r2 = x * x + y * y
    a = (np.pi * 10.0) ** 2 * (np.sqrt(r2) - 0.4) ** 2
    u = (1 - 2 * a) * np.exp(-a) + 0.1 * S.q_lowpass(shape, 21, qmin=-1, qmax=1, sigma_k=64)
    g1, g2, uin = gpu_apply_pair(V, shape, Q, u, 16, V.IMPL_FUSED, V.F32)
    r1, r2_ = O.seismic_operators(uin, gamma_of(Q), 16)
    check(g1, r1, TOL32)
    check(g2, r2_, TOL32)
    # the plain path at the same accuracy
    p1, p2, _ = gpu_apply_pair(V, shape, Q, u, 16, V.IMPL_PLAIN, V.F32)
    check(p1, r1, TOL32)
    check(p2, r2_, TOL32)


def test_apply_single_operator_entry(V):
    import torch
    shape = (128, 128)
    Q, u = _case(shape, 17)
    with V.Solver(shape) as s:
        s.set_q(Q)
        s.set_M(5)
        ut = torch.from_numpy(u.astype(np.float32)).cuda()
        o = torch.empty_like(ut)
        s.apply(V.OP_HPG, ut, o)
        s.sync()
        r1, r2 = O.seismic_operators(u.astype(np.float32).astype(np.float64), gamma_of(Q), 5)
        check(o.cpu().numpy().astype(np.float64), r2, TOL32)
        s.apply(V.OP_1PG, ut, o)
        s.sync()
        check(o.cpu().numpy().astype(np.float64), r1, TOL32)


@pytest.mark.parametrize("impl", ["fused", "plain"])
def test_smooth_inputs_keep_fp32_accuracy(V, impl):
    """Smooth fields (a Gaussian of 5 and 8 cells, a single Fourier mode)
    concentrate the spectrum at low wavenumbers; a plain FP32 forward
    transform leaves round-off of size eps*|u| in the empty high-wavenumber
    bins, which |mu|^{2+2 gamma} amplifies past 1e-5.  Transforming the
    discrete Laplacian instead keeps both operators near FP32 round-off."""
    im = V.IMPL_FUSED if impl == "fused" else V.IMPL_PLAIN
    for shape, u in [((128, 128), S.gaussian_pulse((128, 128), 5.0)),
                     ((1024, 1024), S.gaussian_pulse((1024, 1024), 8.0)),
                     ((128, 256), np.cos(5 * (S.mesh((128, 256))[0] + np.pi)
                                         + 3 * (S.mesh((128, 256))[1] + np.pi)))]:
        Q = S.q_lowpass(shape, 2)
        g1, g2, uin = gpu_apply_pair(V, shape, Q, u, 8, im, V.F32)
        r1, r2 = O.seismic_operators(uin, gamma_of(Q), 8)
        check(g1, r1, 2e-6)
        check(g2, r2, 2e-6)


@pytest.mark.parametrize("shape,prec", [((64,), "f32"), ((256,), "f32"), ((4096,), "f32"),
                                        ((256,), "f64"), ((2048,), "f64")])
def test_fused_1d_apply_matches_oracle(V, shape, prec):
    pr = V.F32 if prec == "f32" else V.F64
    tol = TOL32 if prec == "f32" else TOL64
    for M in (0, 8, 16):
        Q, u = _case(shape, 23 + M)
        g1, g2, uin = gpu_apply_pair(V, shape, Q, u, M, V.IMPL_FUSED, pr)
        r1, r2 = O.seismic_operators(uin, gamma_of(Q), M)
        check(g1, r1, tol)
        check(g2, r2, tol)


@pytest.mark.parametrize("shape", [(64, 64, 64), (128, 128, 128), (256, 64, 128)])
def test_fused_3d_apply_matches_oracle(V, shape):
    for M in (0, 3, 8):
        Q = S.q_lowpass(shape, 31 + M)
        u = S.q_lowpass(shape, 41 + M, qmin=-1.0, qmax=1.0, sigma_k=max(shape) / 8)
        g1, g2, uin = gpu_apply_pair(V, shape, Q, u, M, V.IMPL_FUSED, V.F32)
        r1, r2 = O.seismic_operators(uin, gamma_of(Q), M)
        check(g1, r1, TOL32)
        check(g2, r2, TOL32)


def test_fused_3d_config_size_apply(V):
    """3D 256^3, M = 8, two-layer Q and a 4-cell Gaussian (the 3D workload)."""
    w = S.workload_3d_256(nsteps=1)
    g1, g2, uin = gpu_apply_pair(V, w["shape"], w["Q"], w["u0"], w["M"], V.IMPL_FUSED, V.F32)
    r1, r2 = O.seismic_operators(uin, gamma_of(w["Q"]), w["M"])
    check(g1, r1, TOL32)
    check(g2, r2, TOL32)


def test_headline_size_nyquist_column_and_top_taylor_group(V):
    """1024^2, M = 16: the x-Nyquist column (kx = nx/2, the last column of
    every half-spectrum tile and of the row transforms' packing) and the top
    Taylor group (terms 12..16, the ragged group of five) both carry weight.
    gamma swings over most of [0, 1/2), so delta ln|mu|^2 reaches ~3 and the
    top group's terms sit far above FP32 round-off: a wrong slot, tile edge
    or Nyquist handling there moves single columns or rows, which the
    pointwise bound catches."""
    shape = (1024, 1024)
    x, y = S.mesh(shape)
    gamma = 0.25 + 0.245 * np.tanh(4 * np.sin(x) * np.cos(y))
    u = (np.cos(np.pi * np.arange(1024))[None, :] * (1.0 + 0.5 * np.cos(3 * y))  # x-Nyquist column
         + np.cos(317 * x + 211 * y) + 0.5 * np.sin(5 * x - 7 * y))
    uin = u.astype(np.float32)
    import torch
    with V.Solver(shape, None, None, V.F32, V.IMPL_FUSED) as s:
        s.set_gamma(gamma)
        s.set_M(16)
        ut = torch.from_numpy(uin).cuda()
        o1, o2 = torch.empty_like(ut), torch.empty_like(ut)
        s.apply_pair(ut, o1, o2)
        s.sync()
        g1, g2 = o1.cpu().numpy().astype(np.float64), o2.cpu().numpy().astype(np.float64)
    r1, r2 = O.seismic_operators(uin.astype(np.float64), gamma, 16)
    # the top group matters: dropping terms 12..16 moves the answer past
    # the tolerance
    t1, _ = O.seismic_operators(uin.astype(np.float64), gamma, 11)
    assert rel_l2(t1, r1) > 5 * TOL32, rel_l2(t1, r1)
    check(g1, r1, TOL32)
    check(g2, r2, TOL32)
    # the general model's one operator, whose order swings far more (delta
    # up to 0.4): its terms fill both slots, so the top group lands in slot 1
    order = 1.0 - 0.4 * np.tanh(3 * np.cos(x) * np.sin(y))
    with V.Solver(shape, None, None, V.F32, V.IMPL_FUSED) as s:
        s.set_order(order)
        s.set_M(16)
        ut = torch.from_numpy(uin).cuda()
        o = torch.empty_like(ut)
        s.apply(V.OP_S, ut, o)
        s.sync()
        g = o.cpu().numpy().astype(np.float64)
    r = O.matrix_free_operator(uin.astype(np.float64), order, 16)
    t = O.matrix_free_operator(uin.astype(np.float64), order, 11)
    assert rel_l2(t, r) > 100 * TOL32, rel_l2(t, r)
    check(g, r, TOL32)


@pytest.mark.parametrize("xp,yp", [("f32", "f32"), ("f32", "f64"), ("f64", "f32"), ("f64", "f64")])
def test_rel_l2_diagnostic_matches_numpy(V, xp, yp):
    """vofl_rel_l2 (FP64 accumulation on the GPU, fixed reduction order)
    against NumPy in FP64 on the same values: the sums to round-off, the
    maxima exactly; repeated calls give the same bits."""
    import torch
    shape = (128, 256)
    rng = np.random.default_rng(7)
    dt = {"f32": torch.float32, "f64": torch.float64}
    y = torch.tensor(rng.standard_normal(shape) * 3.0, dtype=dt[yp]).cuda()
    x = (y.double() + torch.tensor(rng.standard_normal(shape) * 1e-3).cuda()).to(dt[xp])
    with V.Solver(shape) as s:
        got = s.rel_l2(x, y)
        again = s.rel_l2(x, y)
        zero = s.rel_l2(y, y)
        bad = x.clone()
        bad[77, 131] = float("nan")  # a blown-up field never reads as a match
        nan_x, nan_y = s.rel_l2(bad, y), s.rel_l2(y, bad)
    assert all(np.isnan(v) for v in nan_x[:2]) and all(np.isnan(v) for v in nan_y)
    xn, yn = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
    want = (np.linalg.norm(xn - yn) / np.linalg.norm(yn), np.max(np.abs(xn - yn)) / np.max(np.abs(yn)),
            np.linalg.norm(yn), np.max(np.abs(yn)))
    assert abs(got[0] - want[0]) <= 1e-13 * want[0] and abs(got[2] - want[2]) <= 1e-13 * want[2]
    assert got[1] == want[1] and got[3] == want[3]
    assert got == again
    assert zero[0] == 0.0 and zero[1] == 0.0
