"""Host logic of the continuous-batching server (paper_2311_13049_gb300.serve)
with fake library objects: admission order, slot and memory limits, the
number of steps every request receives, batch membership, context reuse
and eviction.  CPU only."""
import numpy as np
import pytest

from paper_2311_13049_gb300 import serve as SV


class FakeLib:
    def __init__(self, fp_per_point=10, finish_polls=2):
        self.fp_per_point = fp_per_point
        self.finish_polls = finish_polls
        self.created = []
        self.closed = 0
        self.max_live_bytes = 0
        lib = self

        class Solver:
            def __init__(self, shape):
                self.shape = shape
                self.steps = 0
                self.in_batch = False
                self.polls = 0
                self.closed = False
                lib.created.append(self)

            def set_q(self, Q, c0, omega0):
                assert not self.in_batch
                self.Q = Q

            def set_M(self, M):
                self.M = M

            def suggest_dt(self, courant):
                return 1e-3

            def set_state(self, u0):
                self.steps = 0

            def set_source(self, idx, samples):
                self.nsrc = len(samples)

            def step(self, n, dt):
                assert not self.in_batch
                self.steps += n
                self.polls = 0

            def query(self):
                self.polls += 1
                return not self.in_batch and self.polls >= lib.finish_polls

            def get_state(self):
                assert not self.in_batch
                return np.full(self.shape, float(self.steps), np.float32)

            def close(self):
                self.closed = True
                lib.closed += 1

        class Batch:
            def __init__(self):
                self.members = {}
                self.next = 0
                self.steps_called = []

            def add(self, s, dt):
                assert not s.in_batch
                s.in_batch = True
                self.next += 1
                self.members[self.next] = s
                return self.next

            def remove(self, slot):
                s = self.members.pop(slot)
                s.in_batch = False
                s.polls = 0

            def step(self, n):
                self.steps_called.append(n)
                for s in self.members.values():
                    s.steps += n

            def query(self):
                return True

            def close(self):
                for s in self.members.values():
                    s.in_batch = False

        self.Solver, self.Batch = Solver, Batch

    def footprint(self, shape, M):
        return int(np.prod(shape)) * self.fp_per_point


def _reqs(kinds, n, nsteps=(30, 90), arrival_gap=0.0, seed=0):
    rng = np.random.default_rng(seed)
    return [dict(id=i, arrival=i * arrival_gap, shape=kinds[i % len(kinds)], nsteps=int(rng.integers(*nsteps)),
                 M=8, c0=1.0, omega0=2 * np.pi) for i in range(n)]


def _inputs(sp):
    return np.ones(sp["shape"]), tuple(0 for _ in sp["shape"])


def _source(sp, dt):
    return np.zeros(sp["nsteps"])


def test_every_request_gets_exactly_its_steps():
    kinds = [(64,), (32, 32), (64, 64), (8, 8, 8), (48, 32)]
    reqs = _reqs(kinds, 23)
    lib = FakeLib()
    srv = SV.Server(budget_bytes=10 ** 9, max_active=5, quantum=17, realtime=False, lib=lib)
    recs, _ = srv.run(reqs, _inputs, _source)
    srv.close()
    assert len(recs) == len(reqs)
    for r, sp in zip(recs, reqs):
        assert r["id"] == sp["id"]
        assert np.all(r["result"] == sp["nsteps"])  # the fake state counts steps
        assert r["latency_s"] >= r["queue_s"] >= 0


def test_admission_is_fifo_and_respects_slots_and_budget():
    kinds = [(64, 64), (16, 16, 16), (128,)]
    reqs = _reqs(kinds, 30)
    lib = FakeLib()
    fp = {k: lib.footprint(k, 8) for k in kinds}
    budget = 3 * max(fp.values())
    srv = SV.Server(budget_bytes=budget, max_active=4, quantum=10, realtime=False, lib=lib)
    recs, _ = srv.run(reqs, _inputs, _source)
    admitted = [i for what, i in srv.events if what == "admit"]
    assert admitted == sorted(admitted) == list(range(30))
    live, live_b = set(), 0
    shapes = {sp["id"]: sp["shape"] for sp in reqs}
    for what, i in srv.events:
        if what == "admit":
            live.add(i)
            live_b += fp[shapes[i]]
        elif what == "done":
            live.discard(i)
            live_b -= fp[shapes[i]]
        assert len(live) <= 4 and live_b <= budget
    srv.close()


def test_contexts_are_reused_per_shape_and_evicted_for_memory():
    kinds = [(64, 64), (16, 16, 16)]
    reqs = _reqs(kinds, 12)
    lib = FakeLib()
    big = max(lib.footprint(k, 8) for k in kinds)
    srv = SV.Server(budget_bytes=10 ** 9, max_active=2, quantum=25, realtime=False, lib=lib)
    srv.run(reqs, _inputs, _source)
    assert len(lib.created) <= 4  # at most max_active live contexts per shape
    srv.close()
    # a budget of one context at a time: switching shape evicts the idle one
    lib2 = FakeLib()
    srv2 = SV.Server(budget_bytes=big, max_active=1, quantum=25, realtime=False, lib=lib2)
    recs, _ = srv2.run(reqs, _inputs, _source)
    assert any(what == "evict" for what, _ in srv2.events)
    assert all(np.all(r["result"] == sp["nsteps"]) for r, sp in zip(recs, reqs))
    srv2.close()


def test_batch_quanta_never_overshoot_a_member():
    reqs = _reqs([(64, 64), (128, 128)], 9, nsteps=(5, 60))
    lib = FakeLib()
    srv = SV.Server(budget_bytes=10 ** 9, max_active=9, quantum=16, realtime=False, lib=lib)
    recs, _ = srv.run(reqs, _inputs, _source)
    assert srv.batch is not None and max(srv.batch.steps_called) <= 16
    assert all(np.all(r["result"] == sp["nsteps"]) for r, sp in zip(recs, reqs))
    srv.close()


def test_realtime_waits_for_arrivals():
    reqs = _reqs([(64,)], 4, nsteps=(3, 4), arrival_gap=0.03)
    lib = FakeLib()
    srv = SV.Server(budget_bytes=10 ** 9, max_active=8, realtime=True, lib=lib)
    recs, span = srv.run(reqs, _inputs, _source)
    srv.close()
    assert span >= 0.09
    for r in recs:
        assert r["queue_s"] >= -1e-3  # never admitted before it arrived


def test_oversized_request_is_refused():
    lib = FakeLib()
    srv = SV.Server(budget_bytes=100, realtime=False, lib=lib)
    with pytest.raises(ValueError):
        srv.run(_reqs([(64, 64)], 1), _inputs, _source)


def test_prewarmed_contexts_are_used_first_and_counted():
    kinds = [(64, 64), (16, 16, 16)]
    lib = FakeLib()
    srv = SV.Server(budget_bytes=10 ** 9, max_active=4, realtime=False, lib=lib, prewarm={(64, 64): 3, (16, 16, 16): 2})
    assert len(lib.created) == 5 and srv.pooled == 3 * lib.footprint((64, 64), 16) + 2 * lib.footprint((16, 16, 16), 16)
    srv.run(_reqs(kinds, 4), _inputs, _source)
    assert len(lib.created) == 5  # no context created while serving
    srv.close()
    assert lib.closed == 5
