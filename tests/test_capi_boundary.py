"""The C-ABI library builds, loads and exports every symbol that
include/vofl.h declares; host-only entry points work without a GPU.  CPU
only: no compute call is made here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vofl():
    from paper_2311_13049_gb300 import build as B
    B.build()
    import paper_2311_13049_gb300 as V
    return V


def _declared():
    src = open(os.path.join(ROOT, "include", "vofl.h")).read()
    return sorted(set(re.findall(r"VOFL_API\s+[\w\s\*]*?\b(vofl_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("vofl_create", "vofl_set_q", "vofl_set_gamma", "vofl_set_M", "vofl_apply",
                 "vofl_apply_pair", "vofl_set_state", "vofl_set_source", "vofl_step",
                 "vofl_get_state", "vofl_sync", "vofl_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported_and_bound(vofl):
    lib = C.CDLL(vofl.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in vofl.SIGNATURES, f"binding lacks {name}"
    assert set(vofl.SIGNATURES) == set(_declared())


def test_host_only_entry_points(vofl):
    assert "sm_103a" in vofl.version()
    assert vofl.kernel_launches() >= 0
    f_fused = vofl.footprint_bytes((1024, 1024), vofl.F32, vofl.IMPL_FUSED, 16)
    f_plain = vofl.footprint_bytes((1024, 1024), vofl.F32, vofl.IMPL_PLAIN, 16)
    n = 1024 * 1024
    # storage does not grow with M: the fused path keeps one group of G
    # per-term column transforms (G = 17 by default, a schedule constant)
    # whatever M, the plain baseline every term's transformed field of both
    # operators (2 (M + 1) fields)
    f_fused40 = vofl.footprint_bytes((1024, 1024), vofl.F32, vofl.IMPL_FUSED, 40)
    f_plain40 = vofl.footprint_bytes((1024, 1024), vofl.F32, vofl.IMPL_PLAIN, 40)
    assert f_fused40 == f_fused
    assert 6 * 4 * n < f_fused < 60 * 4 * n
    assert f_plain > 6 * 4 * n
    assert f_plain40 > f_plain + 2 * 24 * 4 * n
    assert f_plain40 > 2 * 41 * 4 * n > f_fused
    assert vofl.footprint_bytes((256, 256, 256), vofl.F32, vofl.IMPL_PLAIN, 8) > 6 * 4 * 256 ** 3


def test_invalid_arguments_are_rejected_before_any_device_work(vofl):
    lib = vofl.lib()
    h = C.c_void_p()
    n = (C.c_int64 * 3)(15, 16, 1)  # odd size: Sec. 2 requires even J
    lo = (C.c_double * 3)(0, 0, 0)
    hi = (C.c_double * 3)(1, 1, 1)
    assert lib.vofl_create(C.byref(h), 2, n, lo, hi, 0, 1, None) == -1
    n = (C.c_int64 * 3)(16, 16, 1)
    assert lib.vofl_create(C.byref(h), 4, n, lo, hi, 0, 1, None) == -1
    bad_hi = (C.c_double * 3)(0, 1, 1)
    assert lib.vofl_create(C.byref(h), 2, n, lo, bad_hi, 0, 1, None) == -1
    # fused path only for the built shapes (16^3 is not one of them)
    n3 = (C.c_int64 * 3)(16, 16, 16)
    assert lib.vofl_create(C.byref(h), 3, n3, lo, hi, 0, 0, None) == -6
    assert lib.vofl_create(C.byref(h), 2, n, lo, hi, 1, 0, None) == -6
    assert lib.vofl_set_M(None, 3) == -1


def test_no_gpu_means_a_clean_error(vofl):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(vofl.VoflError):
        vofl.Solver((64, 64), impl=vofl.IMPL_PLAIN)


def test_schedule_struct_matches_the_header(vofl):
    """The binding's Schedule mirrors vofl_schedule field by field (all
    int, in the header's order): a field added on one side only would shift
    every later field across the C ABI."""
    src = open(os.path.join(ROOT, "include", "vofl.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\}\s*vofl_schedule;", src).group(1)
    fields = re.findall(r"\bint\s+(\w+)\s*;", body)
    assert fields and len(fields) == body.count(";")
    assert [f for f, _ in vofl.Schedule._fields_] == fields
    assert all(t is C.c_int for _, t in vofl.Schedule._fields_)
    assert C.sizeof(vofl.Schedule) == 4 * len(fields)
