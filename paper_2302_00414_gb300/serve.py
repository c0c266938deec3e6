"""Continuous-batching request loop for reconstructions h = D^* F^* B^* W f (Algorithm 3.7).

Requests name a point set and carry a sample vector f.  The loop keeps plans (sorted
points, weights, tables) on the device across requests; a request for an unknown point
set is parked while a worker thread builds its plan and weights (Algorithm 3.6) on a
low-priority stream of its own; reconstructions run on high-priority streams, so that the
device schedules their blocks ahead of the precompute's.  Every iteration of ``step()``:

* retires batches whose completion event has fired and stamps their latencies;
* admits ready requests into a new batch as soon as one of the ``streams`` slots is free
  (so requests that arrive while earlier batches run are batched and overlap with them
  on the device), grouping requests by (d, precision) and launching each group as one
  batched adjoint (``infft_adjoint_batched``);
* before a new plan is built, frees least-recently-used cached plans with no queued or
  running request until the estimated device memory fits the budget (memory-based
  admission); plans being built hold their estimate meanwhile.

Transforms of one plan that overlap in time need separate scratch grids: every request
in flight is given its own scratch set of the plan (``infft_adjoint_batched_slots``), the
lowest one free, so one point set can be in several running batches and repeat within a
batch.

The compute happens in the CUDA library; this module only schedules calls.  The backend
is injectable so that the scheduling logic can be tested without a GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import queue
import threading
import time
from typing import Any, Callable, Dict, List, Optional


@dataclasses.dataclass
class Request:
    rid: int
    key: Any                 # point-set identifier
    f: Any                   # sample vector (device tensor)
    t_arrive: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    out: Any = None
    batch_size: int = 0
    error: Optional[BaseException] = None   # set when its point set could not be built


@dataclasses.dataclass
class PointSet:
    """What the loop needs to know about a point set before its plan exists."""
    key: Any
    d: int
    M: int
    x: Any                   # N x d float64 (host), or a callable returning it
    precision: str = "fp32"
    N: int = 0               # number of points (needed when x is a callable)


class Backend:
    """GPU backend over the library: plans, batched launches, completion events."""

    def __init__(self, weights_iters: int = 30, m: int = 4, sigma: float = 2.0, bopt: bool = False):
        """bopt: also optimise B (Algorithm 4.3) when a two-dimensional point set is admitted,
        and serve its reconstructions with B_opt (Algorithm 4.4) instead of the weights
        (Algorithm 3.7).  Three-dimensional sets keep the weights: with (2m+2)^3 = 1000 slots
        per point and M_sigma^3 columns their B_opt takes minutes per set on one GPU."""
        import torch

        import paper_2302_00414_gb300 as L
        self.torch, self.L = torch, L
        self.weights_iters, self.m, self.sigma, self.bopt = weights_iters, m, sigma, bopt
        self.mode = L.MODE_BOPT if bopt else L.MODE_DCF
        self._free, self._free_at = 0, -1.0
        self.phase_s = collections.Counter()     # host seconds per build phase
        self.launch_max = collections.Counter()  # longest host time of each launch phase
        self.launch_sum = collections.Counter()
        L.load()

    def build_plan(self, ps: PointSet, stream):
        t0 = time.perf_counter()
        x = ps.x() if callable(ps.x) else ps.x
        t1 = time.perf_counter()
        # pooled plan memory: building and destroying plans does not stall the launches
        p = self.L.Plan(x, ps.M, self.sigma, self.m, ps.precision, stream=stream.cuda_stream, pooled=True)
        t2 = time.perf_counter()
        p.weights(max_iter=self.weights_iters, rel_tol=1e-12, stream=stream.cuda_stream)
        t3 = time.perf_counter()
        if self.bopt and ps.d == 2:
            p.optimize_B(stream=stream.cuda_stream)
        t4 = time.perf_counter()
        self.phase_s["points"] += t1 - t0
        self.phase_s["plan"] += t2 - t1
        self.phase_s["weights"] += t3 - t2
        self.phase_s["bopt"] += t4 - t3
        return p

    def plan_bytes(self, plan) -> int:
        return plan.device_bytes

    def estimate_bytes(self, ps: PointSet) -> int:
        n = ps.N if ps.N else ps.x.shape[0]
        grid = (2 * ps.M) ** ps.d
        cg = 16 * ((4 * ps.M) ** ps.d) * 8   # float64 grids and scratch of the degree-2M solve
        extra = 0
        if self.bopt and ps.d == 2:   # float64 and plan-precision coefficients, member lists and V
            extra = n * (2 * self.m + 2) ** ps.d * (16 + 8 + 8) + 16 * n * ps.d * (2 * self.m + 2)
        return 120 * n + 40 * grid + cg + extra

    def free_bytes(self) -> int:
        # the device query can wait behind another thread's synchronising call (a plan's
        # destruction, the precompute's frees): refresh it at most every 0.5 s
        now = time.perf_counter()
        if now - self._free_at > 0.5:
            self._free = int(self.torch.cuda.mem_get_info()[0])
            self._free_at = now
        return self._free

    def new_stream(self, priority: int = 0):
        # lower number = higher priority: the device scheduler then prefers blocks of the
        # reconstruction streams over those of the precompute stream
        return self.torch.cuda.Stream(priority=priority)

    def launch(self, plans, fs, stream, slots):
        torch = self.torch
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            # outputs allocated on the launch stream; inputs marked as used by it
            outs = [torch.empty((p.M,) * p.d, dtype=f.dtype, device=f.device) for p, f in zip(plans, fs)]
            for f in fs:
                f.record_stream(stream)
            t1 = time.perf_counter()
            mode = self.mode if plans[0].d == 2 else self.L.MODE_DCF   # a batch has one d
            self.L.adjoint_batched(plans, fs, outs, mode, stream=stream.cuda_stream, slots=slots)
            t2 = time.perf_counter()
            ev = torch.cuda.Event()
            ev.record(stream)
        t3 = time.perf_counter()
        for k, dt in (("alloc", t1 - t0), ("library", t2 - t1), ("event", t3 - t2)):
            self.launch_max[k] = max(self.launch_max[k], dt)
            self.launch_sum[k] += dt
        return outs, ev

    def done(self, ev) -> bool:
        return ev.query()

    def release(self, plan):
        plan.close()


class Server:
    def __init__(self, backend, mem_budget: Optional[int] = None, max_batch: int = 64, streams: int = 3,
                 max_repeat: int = 8, clock: Callable[[], float] = time.perf_counter,
                 keep_output: Optional[Callable[[Request], bool]] = None, builders: int = 1):
        """builders: threads that build new point sets (plan, weights, B_opt), each on its own
        low-priority stream, so that the latency-bound precompute kernels of several sets
        overlap on the device."""
        self.be = backend
        # which completed requests keep their result tensor (all by default); dropping the
        # others lets the allocator reuse their memory instead of growing the heap
        self.keep_output = keep_output
        self.max_batch = max_batch
        self.max_repeat = max_repeat
        self.mem_budget = mem_budget
        self.clock = clock
        self.streams = [backend.new_stream(priority=-1) for _ in range(streams)]
        self.free_streams = list(range(streams))
        self.plans: Dict[Any, Any] = {}
        self.plan_meta: Dict[Any, PointSet] = {}
        self.plan_used: Dict[Any, float] = {}
        self.plan_size: Dict[Any, int] = {}
        self.pinned: set = set()           # point sets never evicted
        self.plan_refs: Dict[Any, int] = collections.Counter()   # requests queued or in flight
        self.resident_bytes = 0        # plans on the device
        self.reserved: Dict[Any, int] = {}   # estimates of plans being built
        self._reserved_total = 0
        self.pending: collections.deque = collections.deque()
        self.parked: Dict[Any, List[Request]] = collections.defaultdict(list)
        self._n_parked = 0
        self.inflight: List[tuple] = []
        self.completed: List[Request] = []
        self.failed: List[Request] = []       # requests whose point set failed to build
        self.stats = collections.Counter()
        self._retry: collections.deque = collections.deque()   # sets waiting for memory, FIFO
        self._deferred_keys: set = set()
        self.build_times: List[tuple] = []    # (key, seconds) of every plan built
        self.launch_times: List[float] = []   # host seconds of every batch launch
        self._lock = threading.Lock()
        self._work: queue.Queue = queue.Queue()
        self._ready: queue.Queue = queue.Queue()
        self._slots_busy: Dict[Any, set] = collections.defaultdict(set)   # scratch sets in flight
        self._workers = []
        self._pstreams = [backend.new_stream(priority=0) for _ in range(max(1, builders))]
        for st in self._pstreams:
            t = threading.Thread(target=self._precompute_loop, args=(st,), daemon=True)
            t.start()
            self._workers.append(t)
        # evicted plans are destroyed off the scheduling thread: destroying a plan waits for
        # the device, which would stall every reconstruction behind the precompute's kernels
        self._released: queue.Queue = queue.Queue()
        self._releaser = threading.Thread(target=self._release_loop, daemon=True)
        self._releaser.start()

    # ---- admission of point sets ------------------------------------------------------
    def register(self, ps: PointSet, pin: bool = False):
        self.plan_meta[ps.key] = ps
        if pin:
            self.pinned.add(ps.key)

    def _precompute_loop(self, stream):
        while True:
            ps = self._work.get()
            if ps is None:
                return
            try:
                t0 = time.perf_counter()
                plan = self.be.build_plan(ps, stream)
                self.build_times.append((ps.key, time.perf_counter() - t0))
                self._ready.put((ps.key, plan, None))
            except Exception as e:  # surfaced to the requests of this key
                self._ready.put((ps.key, None, e))

    def _release_loop(self):
        while True:
            plan = self._released.get()
            if plan is None:
                return
            self.be.release(plan)

    def _make_room(self, need: int) -> bool:
        """Evict LRU plans that are not in flight until `need` more bytes fit."""
        def fits():
            held = self.resident_bytes + self._reserved_total
            if self.mem_budget is not None and held + need > self.mem_budget:
                return False
            return self.be.free_bytes() - self._reserved_total > need
        while not fits():
            idle = [k for k in self.plans if self.plan_refs[k] == 0 and k not in self.pinned]
            if not idle:
                return False
            victim = min(idle, key=lambda k: self.plan_used[k])
            plan = self.plans.pop(victim)
            self.resident_bytes -= self.plan_size.pop(victim)
            self._released.put(plan)
            self.stats["evicted"] += 1
        return True

    def submit(self, req: Request):
        req.t_arrive = req.t_arrive or self.clock()
        if req.key in self.plans:
            self.plan_refs[req.key] += 1
            self.pending.append(req)
            return
        first = req.key not in self.parked or not self.parked[req.key]
        self.parked[req.key].append(req)
        self._n_parked += 1
        if first:
            ps = self.plan_meta[req.key]
            self.stats["new_sets"] += 1
            self._deferred_admit(ps)

    def _admit(self, ps: PointSet) -> bool:
        """Reserve memory for a new point set and queue its build; False if it does not fit."""
        need = self.be.estimate_bytes(ps)
        if self._make_room(need):
            self.reserved[ps.key] = need
            self._reserved_total += need
            self._work.put(ps)
            return True
        if not self.plans and not self.reserved:
            raise MemoryError(f"point set {ps.key!r} needs ~{need} bytes, more than the budget")
        return False

    def _deferred_admit(self, ps: PointSet):
        # sets wait in arrival order: a new set does not overtake one already waiting
        if self._retry or not self._admit(ps):
            if ps.key not in self._deferred_keys:
                self._deferred_keys.add(ps.key)
                self.stats["admit_deferred"] += 1
            self._retry.append(ps)

    # ---- the loop ------------------------------------------------------------------------
    def step(self) -> int:
        """Retire finished batches, absorb new plans, launch ready requests; returns the
        number of requests still queued or in flight."""
        now = self.clock
        t_step = time.perf_counter()
        self.stats["steps"] += 1
        # finished batches
        still = []
        for ev, reqs, sidx, outs, slots in self.inflight:
            if self.be.done(ev):
                t = now()
                for r, o, sl in zip(reqs, outs, slots):
                    r.t_done = t
                    r.out = o if self.keep_output is None or self.keep_output(r) else None
                    self.plan_refs[r.key] -= 1
                    self._slots_busy[r.key].discard(sl)
                    self.completed.append(r)
                self.free_streams.append(sidx)
            else:
                still.append((ev, reqs, sidx, outs, slots))
        self.inflight = still
        # plans built by the worker
        while True:
            try:
                key, plan, err = self._ready.get_nowait()
            except queue.Empty:
                break
            self._reserved_total -= self.reserved.pop(key, 0)
            if err is not None:   # the requests of this set fail; the loop goes on
                failed = self.parked.pop(key, [])
                self._n_parked -= len(failed)
                t = now()
                for r in failed:
                    r.error, r.t_done = err, t
                    self.failed.append(r)
                self.stats["failed_sets"] += 1
                continue
            self.plans[key] = plan
            self.plan_used[key] = now()
            self.plan_size[key] = self.be.plan_bytes(plan)
            self.resident_bytes += self.plan_size[key]
            waiting = self.parked.pop(key, [])
            self._n_parked -= len(waiting)
            self.plan_refs[key] += len(waiting)
            self.pending.extend(waiting)
        t0 = time.perf_counter()
        while self._retry and self._admit(self._retry[0]):
            self._retry.popleft()
        self.stats["admission_s"] += time.perf_counter() - t0
        # launch: one batch per (d, precision) group into free stream slots.  Every request
        # takes the lowest scratch set of its plan that no running request uses, so
        # overlapping transforms never share scratch and most plans need only set 0.
        while self.pending and self.free_streams:
            groups: Dict[tuple, List[Request]] = collections.OrderedDict()
            per_key: Dict[Any, int] = collections.Counter()
            keep = []
            n = 0
            while self.pending and n < self.max_batch:
                r = self.pending.popleft()
                if per_key[r.key] >= self.max_repeat:
                    keep.append(r)
                    continue
                ps = self.plan_meta[r.key]
                groups.setdefault((ps.d, ps.precision), []).append(r)
                per_key[r.key] += 1
                n += 1
            self.pending.extendleft(reversed(keep))
            if not groups:
                break
            for reqs in groups.values():
                if not self.free_streams:
                    self.pending.extendleft(reversed(reqs))
                    continue
                sidx = self.free_streams.pop()
                plans = [self.plans[r.key] for r in reqs]
                t = now()
                for r in reqs:
                    r.t_admit = t
                    r.batch_size = len(reqs)
                    self.plan_used[r.key] = t
                slots = []
                for r in reqs:
                    busy = self._slots_busy[r.key]
                    sl = 0
                    while sl in busy:
                        sl += 1
                    busy.add(sl)
                    slots.append(sl)
                t0 = time.perf_counter()
                outs, ev = self.be.launch(plans, [r.f for r in reqs], self.streams[sidx], slots)
                dt = time.perf_counter() - t0
                self.stats["launch_s"] += dt
                self.launch_times.append(dt)
                for k in {r.key for r in reqs}:   # repeats may have grown the plan's scratch
                    b = self.be.plan_bytes(self.plans[k])
                    self.resident_bytes += b - self.plan_size.get(k, b)
                    self.plan_size[k] = b
                self.inflight.append((ev, reqs, sidx, outs, slots))
                self.stats["batches"] += 1
                self.stats["max_inflight"] = max(self.stats["max_inflight"], len(self.inflight))
        self.stats["step_s"] += time.perf_counter() - t_step
        return len(self.pending) + self._n_parked + \
            sum(len(r) for _, r, _, _, _ in self.inflight)

    def drain(self, timeout: float = 600.0):
        t0 = time.perf_counter()
        while self.step() > 0:
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError("requests did not complete")
            time.sleep(0)

    def close(self):
        for _ in self._workers:
            self._work.put(None)
        for t in self._workers:
            t.join(timeout=5)
        self._released.put(None)
        self._releaser.join(timeout=5)

    def abort(self, timeout: float = 60.0):
        """Drop queued plan builds, wait for the one in progress and stop the worker."""
        while True:
            try:
                self._work.get_nowait()
            except queue.Empty:
                break
        for _ in self._workers:
            self._work.put(None)
        for t in self._workers:
            t.join(timeout=timeout)
        self._released.put(None)
        self._releaser.join(timeout=timeout)


def run_poisson(server: Server, requests: List[Request], rate: float, seed: int = 0,
                clock: Callable[[], float] = time.perf_counter, time_limit: Optional[float] = None,
                on_arrival: Optional[Callable[[Request], None]] = None) -> List[Request]:
    """Feed `requests` at Poisson arrival times of mean rate `rate` (per second) while
    stepping the server; returns the completed requests.  With `time_limit` (seconds)
    the run stops there: later arrivals are not submitted and unfinished requests stay
    incomplete.  `on_arrival` runs for each request just before it is submitted."""
    import random
    rng = random.Random(seed)
    t = t_start = clock()
    arrivals = []
    for r in requests:
        t += rng.expovariate(rate)
        arrivals.append((t, r))
    i = 0
    while i < len(arrivals) or server.step() > 0:
        now = clock()
        if time_limit is not None and now - t_start > time_limit:
            break
        while i < len(arrivals) and arrivals[i][0] <= now:
            arrivals[i][1].t_arrive = arrivals[i][0]
            if on_arrival is not None:
                on_arrival(arrivals[i][1])
            server.submit(arrivals[i][1])
            i += 1
        server.step()
    return server.completed


def latency_summary(reqs: List[Request]) -> dict:
    lat = sorted((r.t_done - r.t_arrive) * 1e3 for r in reqs)
    if not lat:
        return {}

    def pct(q):
        return lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
    span = max(r.t_done for r in reqs) - min(r.t_arrive for r in reqs)
    wait = sorted((r.t_admit - r.t_arrive) * 1e3 for r in reqs)
    run = sorted((r.t_done - r.t_admit) * 1e3 for r in reqs)
    return {"requests": len(lat), "p50_ms": pct(0.50), "p99_ms": pct(0.99), "max_ms": lat[-1],
            "throughput_per_s": len(lat) / span if span > 0 else None,
            "mean_batch": sum(r.batch_size for r in reqs) / len(reqs),
            "queue_p50_ms": wait[len(wait) // 2], "launch_to_done_p50_ms": run[len(run) // 2]}
