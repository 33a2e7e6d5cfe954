"""Contexts stepping at the same time on their own streams: each one's
steps include the cooperative forward launch (both forward passes with a
grid-wide barrier, every CTA resident) at 512^2 and 1024^2.  Interleaved
runs finish without a device-wait timeout and give the bits of the same
runs made one after another."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


def _make(V, n, seed, stream):
    s = V.Solver((n, n), stream=stream)
    s.set_q(S.q_lowpass((n, n), seed))
    s.set_M(12)
    s.set_state(np.zeros((n, n), np.float32))
    s.set_source(S.center_index((n, n)), S.ricker_samples(40, 5e-4, 10.0))
    assert s.schedule()["fuse_forward"] == 2
    return s


def test_concurrent_cooperative_steps_match_serial_runs(V):
    import torch
    specs = [(1024, 91), (1024, 92), (512, 93), (512, 94)]
    streams = [torch.cuda.Stream() for _ in specs]
    # one after another
    serial = []
    for (n, seed), st in zip(specs, streams):
        with _make(V, n, seed, st.cuda_stream) as s:
            s.step(30, 5e-4)
            s.sync()
            serial.append(s.get_state())
    # all at once: every context's steps queued in turn, ten at a time
    ctxs = [_make(V, n, seed, st.cuda_stream) for (n, seed), st in zip(specs, streams)]
    try:
        for _ in range(3):
            for s in ctxs:
                s.step(10, 5e-4)
        for s in ctxs:
            s.sync()  # raises on a device-wait timeout
        for s, ref in zip(ctxs, serial):
            assert np.array_equal(s.get_state(), ref)
    finally:
        for s in ctxs:
            s.close()
