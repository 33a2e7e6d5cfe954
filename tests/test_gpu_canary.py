"""Out-of-bounds writes, checked without a memory checker: in the canary
mode (VOFL_DEBUG_CANARY=1) every device buffer of the library carries 64 KB
pads of a known byte on both sides.  A child process runs the kernel
families on small cases (fused 1D / 2D / 3D with several transform
schedules, the plain path, the implicit solver, a batch), then asks the
library whether any pad changed; a pad overwritten from the host afterwards
shows that the check sees a change."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import ctypes as C, sys
sys.path.insert(0, ROOT)
import numpy as np
import torch
import paper_2311_13049_gb300 as V
import synthetic as S

lib = V.lib()
torch.cuda.set_device(0)
keep = []

def run2d(shape, sched=None, M=12):
    s = V.Solver(shape)
    s.set_q(S.q_lowpass(shape, 3))
    s.set_M(M)
    if sched:
        s.set_schedule(*sched)
    u = torch.from_numpy(S.gaussian_pulse(shape, 4.0).astype(np.float32)).cuda()
    o1, o2 = torch.empty_like(u), torch.empty_like(u)
    s.apply_pair(u, o1, o2)
    dt = s.suggest_dt(0.25)
    s.set_state(np.zeros(shape, np.float32))
    s.set_source(S.center_index(shape), S.ricker_samples(4, dt, 10.0))
    s.step(4, dt)
    s.sync()
    keep.append(s)

for n in (64, 128, 256, 512, 768, 1024):
    run2d((n, n))
run2d((512, 512), (0, 0, 2, 5, 1, 1, 0))
run2d((1024, 1024), (1, 0, 2, 4, 1, 0, 0))
run2d((256, 256), (-1, -1, 1, 3, 0, -1, 2))
run2d((1024, 1024), (0, -1, 0, 6, 1, -1, 0, 300))
run2d((1024, 1024), (0, -1, 0, 0, 2, 0, 0, -1))
run2d((256, 256), (0, -1, 0, 0, 2, 0, 0, -1))
run2d((512, 512), (1, -1, 0, 0, -1, -1, 0, 5000))
run2d((128, 256))
run2d((256, 1024))
run2d((256, 256), M=40)
for shape in ((64, 64, 64), (256, 64, 128)):
    s = V.Solver(shape)
    s.set_q(S.q_lowpass(shape, 4))
    s.set_M(8)
    s.set_state(S.gaussian_pulse(shape, 3.0).astype(np.float32))
    s.step(3, s.suggest_dt(0.25))
    s.sync()
    keep.append(s)
for shape, prec, impl in (((256,), V.F64, V.IMPL_FUSED), ((4096,), V.F32, V.IMPL_FUSED),
                          ((4096,), V.F64, V.IMPL_PLAIN), ((128, 128), V.F32, V.IMPL_PLAIN)):
    s = V.Solver(shape, prec=prec, impl=impl)
    s.set_q(S.q_lowpass(shape, 5))
    s.set_M(8)
    s.set_state(S.gaussian_pulse(shape, 3.0).astype(s.dtype))
    s.step(3, s.suggest_dt(0.25))
    s.sync()
    keep.append(s)
for shape, M in (((256, 256), 6), ((768, 768), 0), ((1024, 1024), 3)):  # fused time splitting
    xg, yg = S.mesh(shape, [-8.0, -8.0], [8.0, 8.0])
    s = V.Solver(shape, [-8.0, -8.0], [8.0, 8.0])
    s.set_order(1.0 - 0.4 * np.cos(np.pi * xg / 4) * np.cos(np.pi * yg / 4), kappa=1.0, f3=1.0)
    s.set_M(M)
    s.set_scheme(V.SCHEME_TSFP2)
    s.set_state(np.exp(-(xg ** 2 + yg ** 2) / 2.0).astype(np.float32))
    s.step(3, 1e-3)
    s.sync()
    keep.append(s)
x = S.axis(256, -16.0, 16.0)
s = V.Solver((256,), [-16.0], [16.0], V.F64, V.IMPL_PLAIN)
s.set_order(1.0 + 0.3 * np.sin(np.pi * x / 8), kappa=1.0, f3=1.0)
s.set_M(10)
s.set_scheme(V.SCHEME_CNFP)
s.set_state(np.exp(-x * x))
s.step(3, 0.05)
s.sync()
keep.append(s)
b = V.Batch()
for n, seed in ((128, 1), (128, 2), (256, 3), (256, 4), (512, 5)):
    m = V.Solver((n, n))
    m.set_q(S.q_lowpass((n, n), seed))
    m.set_M(12)
    m.set_state(np.zeros((n, n), np.float32))
    m.set_source(S.center_index((n, n)), S.ricker_samples(6, 5e-4, 10.0))
    b.add(m, 5e-4)
    keep.append(m)
b.step(3)
b.tune_transform(reps=1)
b.step(3)
b.sync()
live = C.c_int64(0)
bad_live = lib.vofl_debug_canaries(C.byref(live), 0)
b.close()
for s in keep:
    s.close()
bad_freed = lib.vofl_debug_canaries(None, 0)
probe = V.Solver((64, 64))
bad_poked = lib.vofl_debug_canaries(None, 1)
print("CANARY", bad_live, live.value, bad_freed, bad_poked, flush=True)
'''


def test_no_kernel_writes_past_its_buffers(V):
    env = dict(os.environ, VOFL_DEBUG_CANARY="1")
    code = "ROOT = %r\n" % ROOT + CHILD
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    line = [ln for ln in p.stdout.splitlines() if ln.startswith("CANARY")][-1]
    bad_live, live, bad_freed, bad_poked = (int(v) for v in line.split()[1:])
    assert live > 100, live  # the mode was on and the buffers were padded
    assert bad_live == 0 and bad_freed == 0, (bad_live, bad_freed)
    assert bad_poked >= 1  # a changed pad is seen
