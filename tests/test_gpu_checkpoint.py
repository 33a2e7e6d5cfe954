"""Checkpoint / resume (vofl_save_state, vofl_load_state): a run of n1
steps, saved and loaded into a fresh context, then n2 more steps, equals
the run of n1 + n2 steps bit for bit on the same path; checkpoints of
another grid, truncated or foreign blobs are refused."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


def _seismic_2d(V, shape):
    s = V.Solver(shape)
    s.set_M(8)
    s.set_q(S.q_lowpass(shape, 11))
    s.set_state(np.zeros(shape, np.float32))
    s.set_source(S.center_index(shape), S.ricker_samples(60, 2e-3, 3.0))
    return s


def test_fused_2d_resume_is_bit_exact(V):
    shape = (128, 128)
    with _seismic_2d(V, shape) as a:
        a.step(50, 2e-3)
        ref = a.get_state()
    with _seismic_2d(V, shape) as b:
        b.step(30, 2e-3)
        blob = b.save_state()
    with V.Solver(shape) as c:  # a fresh context: model, state and source come from the blob
        c.load_state(blob)
        assert c.steps_taken() == 30
        c.step(20, 2e-3)
        got = c.get_state()
    assert np.array_equal(got, ref)


def test_fused_1d_f64_resume_is_bit_exact(V):
    w = S.workload_1d_256()

    def make():
        s = V.Solver(w["shape"], prec=V.F64)
        s.set_M(w["M"])
        s.set_q(w["Q"], w["c0"], w["omega0"])
        s.set_state(w["u0"])
        return s

    with make() as a:
        a.step(100, w["dt"])
        ref = a.get_state()
    with make() as b:
        b.step(45, w["dt"])
        blob = b.save_state()
    with V.Solver(w["shape"], prec=V.F64) as c:
        c.load_state(blob)
        c.step(55, w["dt"])
        got = c.get_state()
    assert np.array_equal(got, ref)


def test_cnfp_resume_is_bit_exact(V):
    J = 256
    x = S.axis(J, -16.0, 16.0)
    order = 1.0 + 0.3 * np.sin(np.pi * x / 8)

    def make():
        s = V.Solver((J,), [-16.0], [16.0], V.F64, V.IMPL_PLAIN)
        s.set_order(order, kappa=1.0, f3=1.0)
        s.set_M(10)
        s.set_scheme(V.SCHEME_CNFP)
        s.set_state(np.exp(-x * x))
        return s

    with make() as a:
        a.step(12, 0.05)
        ref = a.get_state()
    with make() as b:
        b.step(7, 0.05)
        blob = b.save_state()
    with V.Solver((J,), [-16.0], [16.0], V.F64, V.IMPL_PLAIN) as c:
        c.load_state(blob)
        c.step(5, 0.05)
        got = c.get_state()
    assert np.array_equal(got, ref)


def test_bad_checkpoints_are_refused(V):
    shape = (64, 64)
    with _seismic_2d(V, shape) as a:
        a.step(3, 2e-3)
        blob = a.save_state()
    with V.Solver((128, 128)) as other:  # another grid
        with pytest.raises(V.VoflError):
            other.load_state(blob)
    with V.Solver(shape) as c:
        for bad in (blob[:-8], blob + b"\0" * 8, b"not a checkpoint" * 8):
            with pytest.raises(V.VoflError):
                c.load_state(bad)
        with pytest.raises(V.VoflError):
            c.save_state()  # nothing to save yet
        c.load_state(blob)  # the context is still usable
        c.step(1, 2e-3)
        c.sync()


# byte offsets of the checkpoint header's int64 fields (after the 8-byte
# magic: ndim, n[3], prec, M, scheme, general, cur, psi_nonzero, steps,
# cn_maxit, nsrc, src_flat), then its doubles (lo[3], hi[3], dt, ...)
_HDR = {"scheme": 56, "general": 64, "cur": 72, "psi_nonzero": 80, "steps": 88, "cn_maxit": 96,
        "src_flat": 112}
_HDR_DT = 168


def test_tampered_checkpoint_headers_are_refused(V):
    """A blob of the right grid and size whose header fields are damaged
    (a state index past the two buffers, a source node off the grid, an
    unknown scheme, no solver iterations, ...) is refused with EINVAL before
    anything is copied, and the context stays usable."""
    import struct
    shape = (64, 64)
    n = shape[0] * shape[1]
    with _seismic_2d(V, shape) as a:
        a.step(3, 2e-3)
        blob = a.save_state()
    bad_values = [("cur", 2), ("cur", -1), ("src_flat", n), ("src_flat", -1), ("scheme", 7),
                  ("scheme", 1),  # TSFP2 on the seismic model
                  ("general", 2), ("psi_nonzero", 5), ("cn_maxit", 0), ("steps", -4)]
    with V.Solver(shape) as c:
        for field, val in bad_values:
            b = bytearray(blob)
            struct.pack_into("<q", b, _HDR[field], val)
            with pytest.raises(V.VoflError) as ei:
                c.load_state(bytes(b))
            assert ei.value.code == -1, (field, val, ei.value.code)
        b = bytearray(blob)
        struct.pack_into("<d", b, _HDR_DT, float("nan"))
        with pytest.raises(V.VoflError):
            c.load_state(bytes(b))
        c.load_state(blob)  # the untouched blob still loads
        c.step(1, 2e-3)
        c.sync()
