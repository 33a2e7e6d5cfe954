"""Failure detection on the device without a fault: every device wait in
the kernels is bounded; when the budget runs out the kernel records an
error word, drains what it issued and returns, and the host sees the error
through the status.  The self-test waits on a barrier that nothing
completes (about 1 ms budget)."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_util import gamma_of, gpu_apply_pair, rel_l2, check

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_device_stays_usable(V):
    flag = C.c_int(0)
    assert V.lib().vofl_selftest_bounded_wait(C.byref(flag)) == 0
    assert flag.value == 1
    # the same process keeps working: a fused apply still matches the oracle
    shape = (128, 128)
    Q = S.q_lowpass(shape, 3)
    u = S.gaussian_pulse(shape, 6.0)
    g1, g2, uin = gpu_apply_pair(V, shape, Q, u, 6, V.IMPL_FUSED, V.F32)
    r1, r2 = O.seismic_operators(uin, gamma_of(Q), 6)
    check(g1, r1, 1e-5)
    check(g2, r2, 1e-5)


def test_sync_reports_ok_after_normal_work(V):
    with V.Solver((64, 64)) as s:
        s.set_q(S.q_lowpass((64, 64), 1))
        s.set_state(np.zeros((64, 64), np.float32))
        s.step(5, 1e-3)
        s.sync()  # raises on a recorded wait timeout


# ---------------------------------------------------------------------------
# Out-of-memory paths, made on the host: vofl_debug_fail_alloc(k) makes the
# k-th device allocation of the library fail as cudaMalloc does when the
# device is full.  Every allocating entry point must report ENOMEM, give
# back what it allocated in that call, and leave its context usable.
# ---------------------------------------------------------------------------
ENOMEM = -2


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _each_failure(V, call, cap=64):
    """call() once per allocation index k = 1, 2, ... with the k-th
    allocation failing, until a call makes fewer than k allocations (it then
    succeeds and the pending failure is cancelled).  Returns the number of
    allocations the call makes."""
    lib = V.lib()
    for k in range(1, cap + 1):
        lib.vofl_debug_fail_alloc(k)
        try:
            call()
        except V.VoflError as e:
            lib.vofl_debug_fail_alloc(0)
            assert e.code == ENOMEM, (k, e)
            continue
        pending = lib.vofl_debug_fail_alloc(0)
        assert pending > 0, f"allocation {k} was reached but the call succeeded"
        return k - 1
    raise AssertionError("no successful call within the cap")


@pytest.mark.parametrize("shape,prec,impl", [((128, 128), "f32", "fused"), ((1024, 1024), "f32", "fused"),
                                             ((64, 64, 64), "f32", "fused"), ((256,), "f64", "fused"),
                                             ((64, 64), "f32", "plain"), ((4096,), "f64", "plain")])
def test_create_frees_everything_on_enomem(V, shape, prec, impl):
    pr = V.F32 if prec == "f32" else V.F64
    im = V.IMPL_FUSED if impl == "fused" else V.IMPL_PLAIN
    V.Solver(shape, prec=pr, impl=im).close()  # lazy driver set-up outside the measurement
    before = _free_bytes()
    made = []

    def create():
        s = V.Solver(shape, prec=pr, impl=im)
        made.append(s)

    n = _each_failure(V, create)
    assert n >= 9  # the context's own fields, then the engine's
    for s in made:
        s.close()
    assert abs(_free_bytes() - before) <= 2 << 20


def test_context_calls_report_enomem_and_stay_usable(V):
    import torch
    shape = (256, 256)
    Q = S.q_lowpass(shape, 9)
    with V.Solver(shape) as s:
        s.set_q(Q)
        s.set_M(8)
        s.set_state(np.zeros(shape, np.float32))
        s.set_source(S.center_index(shape), S.ricker_samples(20, 1e-3, 5.0))
        s.step(3, 1e-3)
        ref = s.get_state()
        # a longer source needs a new sample buffer: on failure the old
        # source stays in place
        longer = S.ricker_samples(400, 1e-3, 5.0)
        assert _each_failure(V, lambda: s.set_source(S.center_index(shape), longer)) == 1
        # a Taylor group larger than the group buffer holds re-sizes it: on
        # failure the old schedule stays
        sched = s.schedule()
        n = _each_failure(V, lambda: s.set_schedule(-1, -1, 0, 20))
        assert n == 1 and s.schedule()["group"] == 20
        s.set_schedule()
        assert s.schedule() == sched
        # the c0 field of set_gamma is staged in a temporary buffer
        g = O.seismic_coefficients(Q, 1.0, 2 * np.pi)["gamma"]
        assert _each_failure(V, lambda: s.set_gamma(g, c0_field=np.full(shape, 1.0))) >= 1
        # still a working context: the same run again gives the same bits
        s.set_q(Q)
        s.set_state(np.zeros(shape, np.float32))
        s.set_source(S.center_index(shape), S.ricker_samples(20, 1e-3, 5.0))
        s.step(3, 1e-3)
        assert np.array_equal(s.get_state(), ref)


def test_plain_and_solver_scratch_report_enomem(V):
    """The plain path sizes its term batch at the first apply after set_M,
    and the implicit solver its scratch at its first step."""
    import torch
    J = 256
    x = S.axis(J, -16.0, 16.0)
    with V.Solver((J,), [-16.0], [16.0], V.F64, V.IMPL_PLAIN) as s:
        s.set_order(1.0 + 0.3 * np.sin(np.pi * x / 8), kappa=1.0, f3=1.0)
        s.set_M(10)
        ut = torch.from_numpy(np.exp(-x * x)).cuda()
        o = torch.empty_like(ut)
        assert _each_failure(V, lambda: s.apply(V.OP_S, ut, o)) >= 2
        s.sync()
        s.set_scheme(V.SCHEME_CNFP)
        s.set_state(np.exp(-x * x))
        assert _each_failure(V, lambda: s.step(2, 0.05)) >= 9
        s.step(2, 0.05)
        assert np.isfinite(s.get_state()).all()


def test_batch_step_reports_enomem_and_retries(V):
    shape = (128, 128)
    sols = []
    try:
        with V.Batch() as b:
            for i in range(3):
                s = V.Solver(shape)
                sols.append(s)
                s.set_q(S.q_lowpass(shape, 60 + i))
                s.set_M(6)
                s.set_state(np.zeros(shape, np.float32))
                s.set_source(S.center_index(shape), S.ricker_samples(30, 1e-3, 5.0))
                b.add(s, 1e-3)
            assert _each_failure(V, lambda: b.step(4)) >= 1
            b.step(4)
            b.sync()
    finally:
        for s in sols:
            s.close()
