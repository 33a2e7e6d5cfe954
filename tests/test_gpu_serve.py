"""Serving on the GPU: a stream of mixed requests (1D, 2D batched, 3D) through
the continuous-batching server; every answer must equal, bit for bit, the
same request run alone on a fresh context; one answer is also checked
against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from gpu_util import gamma_of, rel_l2, check

pytestmark = pytest.mark.gpu

KINDS = ((256,), (64, 64), (128, 128), (64, 64, 64))


def _source(sp, dt):
    return S.ricker_samples(sp["nsteps"], dt, sp["f0"])


@pytest.mark.parametrize("realtime,max_active", [(False, 3), (True, 16)])
def test_served_answers_equal_solo_runs(V, realtime, max_active):
    from paper_2311_13049_gb300 import serve as SV
    reqs = S.serve_requests(12, seed=7, rate=400.0, kinds=KINDS, steps=(20, 70), M=(4, 12))
    srv = SV.Server(budget_bytes=4 << 30, max_active=max_active, quantum=16, realtime=realtime)
    try:
        recs, span = srv.run(reqs, S.serve_inputs, _source)
    finally:
        srv.close()
    summ = SV.summarize(recs, span)
    assert summ["requests"] == 12 and summ["p99_s"] >= summ["p50_s"] > 0
    for r, sp in zip(recs, sorted(reqs, key=lambda d: d["arrival"])):
        Q, idx = S.serve_inputs(sp)
        want = SV.solo(sp, Q, idx, _source)
        assert np.array_equal(r["result"], want), sp


def test_served_answer_against_oracle(V):
    from paper_2311_13049_gb300 import serve as SV
    reqs = S.serve_requests(3, seed=8, kinds=((64, 64), (128,)), steps=(30, 40), M=(6, 8))
    srv = SV.Server(max_active=3, quantum=8, realtime=False)
    try:
        recs, _ = srv.run(reqs, S.serve_inputs, _source)
    finally:
        srv.close()
    for r, sp in zip(recs, sorted(reqs, key=lambda d: d["arrival"])):
        Q, idx = S.serve_inputs(sp)
        g = gamma_of(Q)
        # the oracle takes its own time step (same rule; the library's
        # agrees to ~1e-7, far inside the run tolerance)
        dt = O.suggested_dt(g, 1.0, 2 * np.pi, sp["shape"], courant=0.25)
        ref = O.seismic_lffp(g, 1.0, 2 * np.pi, np.zeros(sp["shape"]), None, dt, sp["nsteps"], sp["M"],
                             src_idx=idx, src=_source(sp, dt))
        check(r["result"].astype(np.float64), ref, 1e-4)
