"""Scheduling logic of the continuous-batching loop, with a fake backend (no GPU)."""
import time

import numpy as np

from paper_2302_00414_gb300.serve import PointSet, Request, Server, latency_summary


class FakeEvent:
    def __init__(self, ticks):
        self.ticks = ticks


class FakePlan:
    def __init__(self, ps):
        self.M, self.d, self.key = ps.M, ps.d, ps.key


class FakeBackend:
    """Plans cost 100 bytes; a launched batch finishes after `latency` polls."""

    def __init__(self, latency=3, free=10 ** 9):
        self.latency, self.free = latency, free
        self.built, self.launches, self.released, self.slots = [], [], [], []

    def build_plan(self, ps, stream):
        self.built.append(ps.key)
        return FakePlan(ps)

    def plan_bytes(self, plan):
        return 100

    def estimate_bytes(self, ps):
        return 100

    def free_bytes(self):
        return self.free

    def new_stream(self, priority=0):
        return ("stream", priority)

    def launch(self, plans, fs, stream, slots):
        self.launches.append([p.key for p in plans])
        self.slots.append(list(slots))
        return [("h", p.key, f) for p, f in zip(plans, fs)], FakeEvent(self.latency)

    def done(self, ev):
        ev.ticks -= 1
        return ev.ticks <= 0

    def release(self, plan):
        self.released.append(plan.key)


def sets(n, d=2):
    return [PointSet(key=k, d=d, M=8, x=np.zeros((10, d))) for k in range(n)]


def run(server, reqs, timeout=30.0):
    for r in reqs:
        server.submit(r)
    server.drain(timeout=timeout)
    return server.completed


def test_all_complete_batched_and_overlapping():
    be = FakeBackend(latency=4)
    s = Server(be, max_batch=8, streams=3)
    for ps in sets(3):
        s.register(ps)
    reqs = [Request(rid=i, key=i % 3, f=i) for i in range(50)]
    done = run(s, reqs)
    assert sorted(r.rid for r in done) == list(range(50))
    assert all(r.out[1] == r.key and r.out[2] == r.f for r in done)
    assert s.stats["new_sets"] == 3 and sorted(be.built) == [0, 1, 2]
    assert max(len(b) for b in be.launches) > 1      # requests were batched
    assert s.stats["max_inflight"] >= 2              # batches overlapped
    assert latency_summary(done)["requests"] == 50
    s.close()


def test_requests_arriving_while_busy_join_later_batches():
    be = FakeBackend(latency=5)
    s = Server(be, max_batch=4, streams=1)
    for ps in sets(1):
        s.register(ps)
    for i in range(3):
        s.submit(Request(rid=i, key=0, f=i))
    t0 = time.perf_counter()
    while not s.inflight and time.perf_counter() - t0 < 30:   # plan built on the worker
        s.step()
    assert len(s.inflight) == 1
    for i in range(3, 9):          # arrive while the first batch runs
        s.submit(Request(rid=i, key=0, f=i))
    s.drain(timeout=30)
    assert sorted(r.rid for r in s.completed) == list(range(9))
    assert len(be.launches) >= 2
    s.close()


def test_memory_admission_evicts_idle_plans():
    be = FakeBackend(latency=1)
    s = Server(be, mem_budget=250, max_batch=4, streams=2)   # two plans fit
    for ps in sets(4):
        s.register(ps)
    done = run(s, [Request(rid=i, key=i, f=i) for i in range(4)])
    assert sorted(r.rid for r in done) == [0, 1, 2, 3]
    assert s.stats["evicted"] >= 2
    assert s.resident_bytes <= 250
    s.close()


def test_groups_by_dimension():
    be = FakeBackend(latency=2)
    s = Server(be, max_batch=16, streams=4)
    for ps in sets(2, d=2) + [PointSet(key=10, d=3, M=8, x=np.zeros((10, 3)))]:
        s.register(ps)
    run(s, [Request(rid=i, key=[0, 1, 10][i % 3], f=i) for i in range(12)])
    for batch in be.launches:
        dims = {(3 if k == 10 else 2) for k in batch}
        assert len(dims) == 1
    s.close()


def test_running_transforms_never_share_scratch():
    class Checking(FakeBackend):
        def __init__(self):
            super().__init__(latency=3)
            self.running = []          # (event, {(key, slot)})

        def launch(self, plans, fs, stream, slots):
            live = set()
            for ev, used in self.running:
                if ev.ticks > 0:
                    live |= used
            used = [(p.key, s) for p, s in zip(plans, slots)]
            assert len(set(used)) == len(used), "two jobs of a batch share a scratch set"
            assert not (set(used) & live), "a scratch set in use was given to a new batch"
            outs, ev = super().launch(plans, fs, stream, slots)
            self.running.append((ev, set(used)))
            return outs, ev

    be = Checking()
    s = Server(be, max_batch=16, streams=3, max_repeat=4)
    for ps in sets(2):
        s.register(ps)
    done = run(s, [Request(rid=i, key=0 if i % 5 else 1, f=i) for i in range(60)])
    assert sorted(r.rid for r in done) == list(range(60))
    for batch in be.launches:
        assert max(batch.count(k) for k in set(batch)) <= 4
    assert max(len(b) for b in be.launches) > 1
    assert s.stats["max_inflight"] >= 2      # the hot point set ran on several streams
    s.close()


def test_over_budget_point_set_is_an_error():
    be = FakeBackend()
    s = Server(be, mem_budget=50)
    s.register(sets(1)[0])
    try:
        s.submit(Request(rid=0, key=0, f=0))
    except MemoryError:
        pass
    else:
        raise AssertionError("expected MemoryError")
    s.close()


def test_pinned_point_sets_are_never_evicted():
    be = FakeBackend(latency=1)
    s = Server(be, mem_budget=250, max_batch=4, streams=2)
    all_sets = sets(5)
    s.register(all_sets[0], pin=True)
    for ps in all_sets[1:]:
        s.register(ps)
    for i in range(12):
        s.submit(Request(rid=i, key=i % 5, f=i))
        s.drain(timeout=30)
    assert len(s.completed) == 12
    assert 0 not in be.released and 0 in s.plans
    assert s.stats["evicted"] > 0
    s.close()


def test_reconstruction_streams_outrank_the_precompute_stream():
    s = Server(FakeBackend(), streams=3, builders=2)
    assert len(s._pstreams) == 2
    assert all(st[1] < ps[1] for st in s.streams for ps in s._pstreams)
    s.close()


def test_several_builders_build_every_set_once():
    """With three build threads every registered set is built exactly once and every request
    completes, whatever order the builds finish in."""
    be = FakeBackend(latency=1)
    s = Server(be, streams=2, builders=3)
    for k in range(9):
        s.register(PointSet(key=k, d=2, M=8, x=None, N=10))
    for i in range(27):
        s.submit(Request(rid=i, key=i % 9, f=i))
    s.drain(timeout=30)
    assert len(s.completed) == 27
    assert sorted(k for k, _ in s.build_times) == list(range(9))
    s.close()


def test_failed_builds_fail_their_requests_and_the_loop_goes_on():
    class Flaky(FakeBackend):
        def build_plan(self, ps, stream):
            if ps.key == 1:
                raise RuntimeError("INFFT_ENOMEM: injected allocation failure")
            return super().build_plan(ps, stream)

    be = Flaky(latency=2)
    s = Server(be, max_batch=8, streams=2)
    for ps in sets(3):
        s.register(ps)
    run(s, [Request(rid=i, key=i % 3, f=i) for i in range(12)])
    assert sorted(r.rid for r in s.completed) == [i for i in range(12) if i % 3 != 1]
    assert sorted(r.rid for r in s.failed) == [1, 4, 7, 10]
    assert all(isinstance(r.error, RuntimeError) for r in s.failed)
    assert s.stats["failed_sets"] == 1 and not s.reserved
    s.close()
