"""Helpers shared by the GPU parity tests (marshalling only)."""
import numpy as np

import oracle as O


def rel_l2(a, b):
    return O.rel_l2(a, b)


def gamma_of(Q):
    return O.seismic_coefficients(Q, 1.0, 2 * np.pi)["gamma"]


def gpu_apply_pair(V, shape, Q, u, M, impl, prec, lo=None, hi=None):
    """(L1 u, L2 u) from the library, as float64 numpy arrays, plus the
    exact input the library saw (rounded to its precision)."""
    import torch
    dt = np.float32 if prec == V.F32 else np.float64
    tdt = torch.float32 if prec == V.F32 else torch.float64
    u_in = np.ascontiguousarray(u, dtype=dt)
    with V.Solver(shape, lo, hi, prec, impl) as s:
        s.set_q(np.ascontiguousarray(Q, dtype=np.float64))
        s.set_M(M)
        ut = torch.from_numpy(u_in).cuda()
        o1 = torch.empty(shape, dtype=tdt, device="cuda")
        o2 = torch.empty(shape, dtype=tdt, device="cuda")
        s.apply_pair(ut, o1, o2)
        s.sync()
        torch.cuda.synchronize()
        return o1.cpu().numpy().astype(np.float64), o2.cpu().numpy().astype(np.float64), u_in.astype(np.float64)


def gpu_run(V, shape, Q, u0, v0, M, dt, nsteps, impl, prec, src_idx=None, src=None, lo=None, hi=None,
            chunks=None):
    """Final wavefield of a library run (host arrays in, host array out)."""
    ty = np.float32 if prec == V.F32 else np.float64
    with V.Solver(shape, lo, hi, prec, impl) as s:
        s.set_q(np.ascontiguousarray(Q, dtype=np.float64))
        s.set_M(M)
        s.set_state(np.ascontiguousarray(u0, dtype=ty),
                    None if v0 is None else np.ascontiguousarray(v0, dtype=ty))
        if src is not None:
            s.set_source(src_idx, np.ascontiguousarray(src, dtype=np.float64))
        if chunks:
            for c in chunks:
                s.step(c, dt)
        else:
            s.step(nsteps, dt)
        assert s.steps_taken() == nsteps
        out = s.get_state()
        s.sync()
        return out.astype(np.float64)


# Pointwise bound beside every relative-L2 bound: max|g - r| <= PW tol max|r|.
# FP32 round-off of the transforms is spread over the grid like noise, so
# its largest entry is a few times its RMS (PW = 10 leaves room for that);
# an error confined to a few points (one tile column, the Nyquist column,
# one Taylor group's slot) can hide under a relative L2 bound but not
# under this one.
PW = 10.0


def check(g, r, tol, what=""):
    """Assert rel_l2(g, r) <= tol and max|g - r| <= PW * tol * max|r|."""
    g = np.asarray(g, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    e = rel_l2(g, r)
    assert e <= tol, (what, "rel_l2", e, tol)
    scale = float(np.max(np.abs(r)))
    pw = float(np.max(np.abs(g - r))) / scale if scale > 0 else float(np.max(np.abs(g)))
    assert pw <= PW * tol, (what, "max|g-r|/max|r|", pw, PW * tol)
