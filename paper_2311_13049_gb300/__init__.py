"""Python binding of libvofl (include/vofl.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays
(host) and torch CUDA tensors (device) to pointers and checks return codes.
There is no CPU fallback: the first call fails loudly when the library has
not been built (``python -m paper_2311_13049_gb300.build``).

Shapes are given in array order (slowest axis first, as numpy/torch); box
bounds ``lo``/``hi`` in (x, y, z) order, as in the C ABI.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libvofl.so")

_LIB = None

F32, F64 = 0, 1
OP_1PG, OP_HPG, OP_S = 0, 1, 2
IMPL_FUSED, IMPL_PLAIN = 0, 1
SCHEME_LFFP, SCHEME_TSFP2, SCHEME_CNFP = 0, 1, 2
_STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEDOUT", -5: "ESTATE",
           -6: "EUNSUPPORTED", -7: "ENOCONV"}

class Schedule(C.Structure):
    """vofl_schedule: transform schedule of the fused 2D path."""
    _fields_ = [("wide_cols", C.c_int), ("wide_rows", C.c_int), ("col_parts", C.c_int), ("group", C.c_int),
                ("fuse_forward", C.c_int), ("wide_fwd", C.c_int), ("row_split", C.c_int), ("col_pack", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_i64p = C.POINTER(C.c_int64)
_dp = C.POINTER(C.c_double)
_vp = C.c_void_p

# exported symbols and their signatures: name -> (restype, argtypes)
SIGNATURES = {
    "vofl_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _i64p, _dp, _dp, C.c_int, C.c_int, _vp]),
    "vofl_destroy": (None, [_vp]),
    "vofl_set_q": (C.c_int, [_vp, _vp, C.c_int, C.c_double, C.c_double]),
    "vofl_set_gamma": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_double, C.c_double]),
    "vofl_set_order": (C.c_int, [_vp, _vp, C.c_int, C.c_double, C.c_double, C.c_double]),
    "vofl_set_M": (C.c_int, [_vp, C.c_int]),
    "vofl_set_scheme": (C.c_int, [_vp, C.c_int]),
    "vofl_apply": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "vofl_apply_pair": (C.c_int, [_vp, _vp, _vp, _vp]),
    "vofl_set_state": (C.c_int, [_vp, _vp, _vp, C.c_int]),
    "vofl_set_source": (C.c_int, [_vp, _i64p, _vp, C.c_int64, C.c_int]),
    "vofl_step": (C.c_int, [_vp, C.c_int64, C.c_double]),
    "vofl_get_state": (C.c_int, [_vp, _vp, C.c_int]),
    "vofl_steps_taken": (C.c_int64, [_vp]),
    "vofl_suggest_dt": (C.c_int, [_vp, C.c_double, _dp]),
    "vofl_query": (C.c_int, [_vp]),
    "vofl_suggest_M": (C.c_int, [_vp, C.c_double, C.POINTER(C.c_int)]),
    "vofl_set_solver": (C.c_int, [_vp, C.c_double, C.c_int]),
    "vofl_save_state": (C.c_int, [_vp, _vp, C.POINTER(C.c_size_t)]),
    "vofl_load_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "vofl_solver_stats": (C.c_int, [_vp, _i64p, _i64p]),
    "vofl_sync": (C.c_int, [_vp]),
    "vofl_last_error": (C.c_char_p, [_vp]),
    "vofl_footprint_bytes": (C.c_size_t, [C.c_int, _i64p, C.c_int, C.c_int, C.c_int]),
    "vofl_kernel_launches": (C.c_uint64, []),
    "vofl_profile_kernels": (C.c_int, [_vp, C.c_int, C.c_char_p, C.c_size_t, _dp, _dp, C.c_int]),
    "vofl_version": (C.c_char_p, []),
    "vofl_set_schedule": (C.c_int, [_vp, C.POINTER(Schedule)]),
    "vofl_rel_l2": (C.c_int, [_vp, _vp, C.c_int, _vp, C.c_int, _dp]),
    "vofl_debug_fail_alloc": (C.c_int64, [C.c_int64]),
    "vofl_debug_canaries": (C.c_int64, [_i64p, C.c_int]),
    "vofl_get_schedule": (C.c_int, [_vp, C.POINTER(Schedule)]),
    "vofl_selftest_bounded_wait": (C.c_int, [C.POINTER(C.c_int)]),
    "vofl_apply_pair_2d_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, _vp, _vp, _vp,
                                             _vp, _vp]),
    "vofl_batch_create": (C.c_int, [C.POINTER(C.c_void_p), _vp]),
    "vofl_batch_destroy": (None, [_vp]),
    "vofl_batch_last_error": (C.c_char_p, [_vp]),
    "vofl_batch_add": (C.c_int, [_vp, _vp, C.c_double, C.POINTER(C.c_int)]),
    "vofl_batch_remove": (C.c_int, [_vp, C.c_int]),
    "vofl_batch_size": (C.c_int, [_vp]),
    "vofl_batch_step": (C.c_int, [_vp, C.c_int64]),
    "vofl_batch_kernels_per_step": (C.c_int64, [_vp]),
    "vofl_batch_query": (C.c_int, [_vp]),
    "vofl_batch_sync": (C.c_int, [_vp]),
    "vofl_batch_tune": (C.c_int, [_vp, C.c_int, _dp]),
    "vofl_batch_time": (C.c_int, [_vp, C.c_int, _dp]),
    "vofl_batch_get_schedule": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                          C.c_int]),
    "vofl_batch_set_schedule": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int]),
    "vofl_batch_tune_transform": (C.c_int, [_vp, C.c_int, _dp]),
    "vofl_batch_get_transform": (C.c_int, [_vp, C.c_int, C.POINTER(Schedule)]),
}


def lib():
    """The loaded libvofl.so (loaded on first use).  Raises if the library
    has not been built: there is no fallback implementation."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"libvofl.so not found at {LIB_PATH}; build it with "
                "`python -m paper_2311_13049_gb300.build` (needs nvcc)")
        handle = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(handle, name)
            f.restype = res
            f.argtypes = args
        _LIB = handle
    return _LIB


class VoflError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def version() -> str:
    return lib().vofl_version().decode()


def kernel_launches() -> int:
    return int(lib().vofl_kernel_launches())


def footprint_bytes(shape, prec=F32, impl=IMPL_FUSED, M=8) -> int:
    n = (C.c_int64 * 3)(*[int(v) for v in reversed(shape)])
    return int(lib().vofl_footprint_bytes(len(shape), n, prec, impl, M))


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype, what):
    """(pointer, on_device) of a numpy array (host) or torch CUDA tensor."""
    if a is None:
        return None, 0
    if _is_torch(a):
        import torch
        want = torch.float32 if dtype == np.float32 else torch.float64
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"{what}: expected a contiguous {want} tensor")
        # a CPU tensor is host memory owned by the caller
        return C.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0)
    if not isinstance(a, np.ndarray):
        raise TypeError(f"{what}: expected a numpy array or a torch tensor")
    arr = a
    if arr.dtype != dtype or not arr.flags["C_CONTIGUOUS"]:
        raise TypeError(f"{what}: expected a C-contiguous {np.dtype(dtype).name} array")
    return C.c_void_p(arr.ctypes.data), 0


class Solver:
    """One simulation context (vofl_ctx)."""

    def __init__(self, shape, lo=None, hi=None, prec=F32, impl=IMPL_FUSED, stream=None):
        self.shape = tuple(int(v) for v in shape)
        d = len(self.shape)
        lo = [-np.pi] * d if lo is None else [float(v) for v in lo]
        hi = [np.pi] * d if hi is None else [float(v) for v in hi]
        self.ndim, self.prec, self.impl = d, prec, impl
        self.dtype = np.float32 if prec == F32 else np.float64
        n = (C.c_int64 * 3)(*[v for v in reversed(self.shape)])
        lo_c = (C.c_double * 3)(*lo)
        hi_c = (C.c_double * 3)(*hi)
        h = C.c_void_p()
        s = C.c_void_p(stream) if stream else None
        rc = lib().vofl_create(C.byref(h), d, n, lo_c, hi_c, prec, impl, s)
        if rc != 0:
            raise VoflError(rc, "vofl_create failed")
        self._h = h
        self._keep = []

    # -- helpers -----------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise VoflError(rc, lib().vofl_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().vofl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- model -------------------------------------------------------------
    def set_q(self, Q, c0=1.0, omega0=2 * np.pi):
        p, dev = _ptr(Q, np.float64, "Q")
        self._check(lib().vofl_set_q(self._h, p, dev, float(c0), float(omega0)))

    def set_gamma(self, gamma, c0=1.0, omega0=2 * np.pi, c0_field=None):
        p, dev = _ptr(gamma, np.float64, "gamma")
        pc, devc = _ptr(c0_field, np.float64, "c0_field")
        if c0_field is not None and devc != dev:
            raise TypeError("gamma and c0_field must both be host or both be device arrays")
        self._check(lib().vofl_set_gamma(self._h, p, pc, dev, float(c0), float(omega0)))

    def set_order(self, s, kappa=1.0, f1=0.0, f3=0.0):
        """General model u_tt = -kappa (-Delta)^{s(x)} u + f1 u + f3 u^3."""
        p, dev = _ptr(s, np.float64, "s")
        self._check(lib().vofl_set_order(self._h, p, dev, float(kappa), float(f1), float(f3)))

    def set_scheme(self, scheme):
        """SCHEME_LFFP (default), SCHEME_TSFP2 or SCHEME_CNFP (these two:
        general model, plain path)."""
        self._check(lib().vofl_set_scheme(self._h, int(scheme)))

    def set_solver(self, tol, max_iter=5000):
        """Relative residual and CG iteration cap of the Crank-Nicolson solve."""
        self._check(lib().vofl_set_solver(self._h, float(tol), int(max_iter)))

    def save_state(self) -> bytes:
        """Checkpoint of the run (vofl_save_state)."""
        n = C.c_size_t(0)
        self._check(lib().vofl_save_state(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(lib().vofl_save_state(self._h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def load_state(self, blob: bytes):
        """Resume from a checkpoint of save_state (same grid and precision)."""
        buf = C.create_string_buffer(bytes(blob), len(blob))
        self._check(lib().vofl_load_state(self._h, buf, len(blob)))

    def solver_stats(self):
        """(CG iterations, linear solves) of the Crank-Nicolson run so far."""
        it, so = C.c_int64(), C.c_int64()
        self._check(lib().vofl_solver_stats(self._h, C.byref(it), C.byref(so)))
        return it.value, so.value

    def set_M(self, M):
        self._check(lib().vofl_set_M(self._h, int(M)))

    # -- operators (device tensors) ------------------------------------------
    def apply(self, op, u, out):
        pu, du = _ptr(u, self.dtype, "u")
        po, do = _ptr(out, self.dtype, "out")
        if not (du and do):
            raise TypeError("apply takes device tensors")
        self._check(lib().vofl_apply(self._h, int(op), pu, po))

    def apply_pair(self, u, out1, out2):
        pu, du = _ptr(u, self.dtype, "u")
        p1, _ = _ptr(out1, self.dtype, "out1")
        p2, _ = _ptr(out2, self.dtype, "out2")
        self._check(lib().vofl_apply_pair(self._h, pu, p1, p2))

    # -- time stepping -------------------------------------------------------
    def set_state(self, u0, v0=None):
        p0, d0 = _ptr(u0, self.dtype, "u0")
        p1, d1 = _ptr(v0, self.dtype, "v0")
        if v0 is not None and d1 != d0:
            raise TypeError("u0 and v0 must both be host or both be device arrays")
        self._check(lib().vofl_set_state(self._h, p0, p1, d0))

    def set_source(self, idx, samples):
        """idx in (x, y, z) order; samples r_n (float64) for n = 0.."""
        if samples is None or len(samples) == 0:
            self._check(lib().vofl_set_source(self._h, None, None, 0, 0))
            return
        i = (C.c_int64 * 3)(*[int(v) for v in idx])
        p, dev = _ptr(samples, np.float64, "samples")
        self._check(lib().vofl_set_source(self._h, i, p, len(samples), dev))

    def step(self, nsteps, dt):
        self._check(lib().vofl_step(self._h, int(nsteps), float(dt)))

    def suggest_dt(self, courant=0.25):
        """courant * 2 / omega_max of the current model (see vofl.h)."""
        dt = C.c_double()
        self._check(lib().vofl_suggest_dt(self._h, float(courant), C.byref(dt)))
        return dt.value

    def suggest_M(self, tol=1e-8):
        """Smallest Taylor power whose remainder bound is within tol (vofl.h)."""
        M = C.c_int()
        self._check(lib().vofl_suggest_M(self._h, float(tol), C.byref(M)))
        return M.value

    def steps_taken(self):
        return int(lib().vofl_steps_taken(self._h))

    def get_state(self, out=None):
        """Current u^n into `out` (torch CUDA tensor or numpy array), or a new
        numpy array."""
        if out is None:
            out = np.empty(self.shape, dtype=self.dtype)
        p, dev = _ptr(out, self.dtype, "out")
        self._check(lib().vofl_get_state(self._h, p, dev))
        return out

    def sync(self):
        self._check(lib().vofl_sync(self._h))

    def query(self):
        """True when all queued work of this context has finished (non-blocking)."""
        rc = lib().vofl_query(self._h)
        if rc < 0:
            self._check(rc)
        return rc == 1

    def set_schedule(self, wide_cols=-1, wide_rows=-1, col_parts=0, group=0, fuse_forward=-1, wide_fwd=-1,
                     row_split=0, col_pack=-1):
        """Transform schedule of the fused 2D path (-1 / 0: the size's default)."""
        sc = Schedule(int(wide_cols), int(wide_rows), int(col_parts), int(group), int(fuse_forward),
                      int(wide_fwd), int(row_split), int(col_pack))
        self._check(lib().vofl_set_schedule(self._h, C.byref(sc)))

    def schedule(self):
        sc = Schedule()
        self._check(lib().vofl_get_schedule(self._h, C.byref(sc)))
        return sc.as_dict()

    def rel_l2(self, x, y):
        """(||x - y|| / ||y||, max|x - y| / max|y|, ||y||, max|y|) of two device
        tensors of this grid (float32 or float64 each), on the GPU in FP64."""
        import torch
        prec = {torch.float32: F32, torch.float64: F64}
        for t in (x, y):
            if not (_is_torch(t) and t.is_cuda and t.dtype in prec and t.is_contiguous()):
                raise TypeError("rel_l2 takes contiguous float32/float64 CUDA tensors")
            if t.numel() != int(np.prod(self.shape)):
                raise ValueError(f"rel_l2: {t.numel()} elements, grid has {int(np.prod(self.shape))}")
        out = (C.c_double * 4)()
        self._check(lib().vofl_rel_l2(self._h, C.c_void_p(x.data_ptr()), prec[x.dtype],
                                      C.c_void_p(y.data_ptr()), prec[y.dtype], out))
        return tuple(out)

    def profile_kernels(self, reps=20):
        names = C.create_string_buffer(1024)
        ms = (C.c_double * 16)()
        units = (C.c_double * 16)()
        k = lib().vofl_profile_kernels(self._h, int(reps), names, 1024, ms, units, 16)
        if k < 0:
            self._check(k)
        nm = names.value.decode().split(";") if k > 0 else []
        return [(nm[i], ms[i], units[i]) for i in range(k)]


class Batch:
    """Many 2D simulations (Solver objects: FP32, fused, square grids)
    advanced together (vofl_batch).  While a Solver is in a batch its own
    methods raise VoflError (ESTATE); remove it (or close the batch) first."""

    def __init__(self, stream=None):
        h = C.c_void_p()
        rc = lib().vofl_batch_create(C.byref(h), C.c_void_p(stream) if stream else None)
        if rc != 0:
            raise VoflError(rc, "vofl_batch_create failed")
        self._h = h
        self._members = {}

    def _check(self, rc):
        if rc < 0:
            raise VoflError(rc, lib().vofl_batch_last_error(self._h).decode())
        return rc

    def add(self, solver, dt):
        slot = C.c_int()
        self._check(lib().vofl_batch_add(self._h, solver._h, float(dt), C.byref(slot)))
        self._members[slot.value] = solver
        return slot.value

    def remove(self, slot):
        self._check(lib().vofl_batch_remove(self._h, int(slot)))
        return self._members.pop(slot)

    def __len__(self):
        return int(lib().vofl_batch_size(self._h))

    def step(self, nsteps):
        self._check(lib().vofl_batch_step(self._h, int(nsteps)))

    def kernels_per_step(self):
        return int(self._check(lib().vofl_batch_kernels_per_step(self._h)))

    def query(self):
        """True when the batch's queued steps have finished (non-blocking)."""
        return self._check(lib().vofl_batch_query(self._h)) == 1

    def sync(self):
        self._check(lib().vofl_batch_sync(self._h))

    def tune(self, reps=2):
        ms = C.c_double()
        self._check(lib().vofl_batch_tune(self._h, int(reps), C.byref(ms)))
        return ms.value

    def tune_transform(self, reps=2):
        """Search each grid size's transform schedule, then the launch layout;
        members take the winning schedule.  Returns ms per batch step."""
        ms = C.c_double(0)
        self._check(lib().vofl_batch_tune_transform(self._h, int(reps), C.byref(ms)))
        return ms.value

    def transform(self, n):
        """The transform schedule of grid edge n (a dict, as Solver.schedule())."""
        sc = Schedule()
        self._check(lib().vofl_batch_get_transform(self._h, int(n), C.byref(sc)))
        return sc.as_dict()

    def time(self, reps=2):
        """ms per batch step of the current schedule (state left unchanged)."""
        ms = C.c_double()
        self._check(lib().vofl_batch_time(self._h, int(reps), C.byref(ms)))
        return ms.value

    def schedule(self):
        par = C.c_int()
        sizes = (C.c_int * 16)()
        chunks = (C.c_int * 16)()
        k = self._check(lib().vofl_batch_get_schedule(self._h, C.byref(par), sizes, chunks, 16))
        return bool(par.value), {sizes[i]: chunks[i] for i in range(min(k, 16))}

    def set_schedule(self, parallel, chunks):
        n = len(chunks)
        sz = (C.c_int * max(n, 1))(*[int(k) for k in chunks])
        ch = (C.c_int * max(n, 1))(*[int(v) for v in chunks.values()])
        self._check(lib().vofl_batch_set_schedule(self._h, 1 if parallel else 0, sz, ch, n))

    def close(self):
        if getattr(self, "_h", None):
            lib().vofl_batch_destroy(self._h)
            self._h = None
            self._members = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
