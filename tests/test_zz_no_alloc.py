"""The allocation-free entry point vofl_apply_pair_2d_noalloc, called through
the C ABI, against the context-based vofl_apply_pair on the same input.

That entry point serves callers that may not allocate device memory when
they need the operator (an outside allocator owns the GPU memory budget,
cudaMalloc/cudaFree would synchronise the device in a latency-critical
loop, or the caller is a callback that must not enter the CUDA allocator);
its intermediates live in one fixed 6 MiB device array shared by every
call.  Consecutive calls with different shapes and Taylor powers check that
no state of one call leaks into the next.  This file is collected last so
that a run stopping at the first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_util import check

pytestmark = pytest.mark.gpu

TOL32 = 1e-5  # the per-apply tolerance used by every FP32 parity test


def _context_pair(V, shape, gamma, u, M, lo, hi):
    import torch
    with V.Solver(shape, lo, hi, V.F32, V.IMPL_FUSED) as s:
        s.set_gamma(np.ascontiguousarray(gamma))
        s.set_M(M)
        ut = torch.from_numpy(u).cuda()
        o1 = torch.empty_like(ut)
        o2 = torch.empty_like(ut)
        s.apply_pair(ut, o1, o2)
        s.sync()
        return o1.cpu().numpy().astype(np.float64), o2.cpu().numpy().astype(np.float64)


def test_noalloc_matches_context_path_on_consecutive_calls(V):
    import torch
    lib = V.lib()
    # shapes (ny, nx); M < 5 makes a group of fewer than six terms (a
    # smaller intermediate layout inside the shared array)
    cases = [((128, 128), 8, [0.0, 0.0], [2 * np.pi, 2 * np.pi], 1),
             ((256, 256), 16, [0.0, 0.0], [2 * np.pi, 2 * np.pi], 2),
             ((128, 256), 6, [0.0, -1.0], [2.0, 3.0], 3),
             ((128, 128), 8, [0.0, 0.0], [2 * np.pi, 2 * np.pi], 4),
             ((64, 64), 0, [0.0, 0.0], [2 * np.pi, 2 * np.pi], 5),
             ((256, 128), 2, [-1.0, 0.0], [3.0, 2.0], 6),
             ((256, 256), 4, [0.0, 0.0], [2 * np.pi, 2 * np.pi], 7),
             ((64, 64), 12, [0.0, 0.0], [2 * np.pi, 2 * np.pi], 8)]
    for shape, M, lo, hi, seed in cases:
        ny, nx = shape
        Q = S.q_lowpass(shape, seed)
        gamma = O.seismic_coefficients(Q, 1.0, 2 * np.pi)["gamma"]
        u = S.q_lowpass(shape, seed + 50, qmin=-1.0, qmax=1.0, sigma_k=16).astype(np.float32)
        g_dev = torch.from_numpy(np.ascontiguousarray(gamma)).cuda()
        u_dev = torch.from_numpy(u).cuda()
        o1 = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
        o2 = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        rc = lib.vofl_apply_pair_2d_noalloc(nx, ny, hi[0] - lo[0], hi[1] - lo[1], M,
                                            C.c_void_p(g_dev.data_ptr()), C.c_void_p(u_dev.data_ptr()),
                                            C.c_void_p(o1.data_ptr()), C.c_void_p(o2.data_ptr()), None)
        # 0 also says the kernels' error word (cleared by the call before
        # its kernels run) was still zero when the call ended: no bounded
        # device wait gave up, and no word left by an earlier call counts
        assert rc == 0, (shape, M, rc)
        torch.cuda.synchronize()
        assert np.isfinite(o1.cpu().numpy()).all() and np.isfinite(o2.cpu().numpy()).all()
        a1 = o1.cpu().numpy().astype(np.float64)
        a2 = o2.cpu().numpy().astype(np.float64)
        b1, b2 = _context_pair(V, shape, gamma, u, M, lo, hi)
        check(a1, b1, TOL32, (shape, M))
        check(a2, b2, TOL32, (shape, M))
        # and both agree with the FP64 oracle on the same input
        r1, r2 = O.seismic_operators(u.astype(np.float64), gamma, M, lo, hi)
        check(a1, r1, TOL32, (shape, M))
        check(a2, r2, TOL32, (shape, M))


def test_noalloc_rejects_shapes_beyond_its_limit(V):
    lib = V.lib()
    null = C.c_void_p(0)
    dummy = C.c_void_p(16)  # never dereferenced: the size check comes first
    assert lib.vofl_apply_pair_2d_noalloc(512, 512, 1.0, 1.0, 8, dummy, dummy, dummy, dummy, None) == -6
    assert lib.vofl_apply_pair_2d_noalloc(96, 96, 1.0, 1.0, 8, dummy, dummy, dummy, dummy, None) == -6
    assert lib.vofl_apply_pair_2d_noalloc(128, 128, 1.0, 1.0, 8, null, dummy, dummy, dummy, None) == -1
    assert lib.vofl_apply_pair_2d_noalloc(128, 128, 1.0, 1.0, 41, dummy, dummy, dummy, dummy, None) == -1
