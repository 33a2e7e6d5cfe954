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
