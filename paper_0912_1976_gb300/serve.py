"""Continuous-batching server of thin-domain Poisson solves.

Requests (a mesh, an aspect ratio, a boundary condition and 1-8 right-hand sides) arrive over time.
Each (mesh, aspect ratio, boundary condition) has a hierarchy and an engine (vemg_engine_*) with a
fixed number of right-hand-side slots, kept resident on the device while memory allows. A request
is admitted column by column into its engine's free slots, first come first served per engine (a
request whose columns do not all fit takes the free slots and holds back later requests of the same
engine, so wide requests are not starved by narrow ones); columns join the batch between iterations
while the other slots keep iterating. Every engine is stepped at its own pace: an idle engine with
work gets a few iterations enqueued on its own CUDA stream, and the loop polls the streams without
waiting, so small hierarchies are not held to the step time of large ones (engines of different
hierarchies overlap on the device). A column is retired as soon as it is done, freeing its slot;
a request completes when all its columns are. Hierarchies are built on first use, on a worker
thread while the engines keep stepping, if the free device memory allows (the bytes of builds in
progress counted as taken), after evicting idle ones (least recently used first).

The factories that build hierarchies and report free memory are injectable, so the scheduling
and admission logic runs on the CPU with fakes.
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import math
import time
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

# the serving workload: 8 meshes of the extruded generator (44..399 squared x 24 layers),
# aspect ratios on a log-uniform grid, Neumann / Dirichlet-top 50/50, 1-8 right-hand sides
SIZES = [44, 60, 83, 114, 156, 214, 292, 399]
NZ = 24
EPS_GRID = [1e-4, 1e-3, 1e-2, 1e-1]


@dataclasses.dataclass
class Request:
    rid: int
    mesh_id: int
    eps: float
    bc: int
    nrhs: int
    arrival: float
    seed: int
    slots: List[int] = dataclasses.field(default_factory=list)
    admitted: Optional[float] = None
    finished: Optional[float] = None
    infos: List[dict] = dataclasses.field(default_factory=list)
    x: Optional[object] = None
    pending: Optional[list] = None   # right-hand sides not yet admitted
    live: int = 0                    # columns admitted and not yet retired

    @property
    def key(self) -> Tuple[int, float, int]:
        return (self.mesh_id, self.eps, self.bc)


def make_requests(n: int = 512, rate: Optional[float] = None, seed: int = 5000, sizes=SIZES,
                  eps_grid=EPS_GRID, max_rhs: int = 8) -> List[Request]:
    """Seeded request stream: Poisson arrivals at `rate` per second (None: all at time 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, n)) if rate else np.zeros(n)
    mesh_id = rng.integers(0, len(sizes), n)
    eps = rng.integers(0, len(eps_grid), n)
    bc = rng.integers(0, 2, n)
    nrhs = rng.integers(1, max_rhs + 1, n)
    return [Request(i, int(mesh_id[i]), float(eps_grid[eps[i]]), int(bc[i]), int(nrhs[i]), float(t[i]),
                    seed + 1 + i) for i in range(n)]


@dataclasses.dataclass
class Entry:
    key: tuple
    hierarchy: object
    engine: object
    nbytes: int
    n: int
    last_used: float = 0.0
    running: int = 0   # requests holding slots


class Server:
    """build(key) -> (hierarchy, engine, nbytes, n); estimate(key) -> bytes a build will need;
    free_bytes() -> free device bytes; rhs(request, n) -> list of device right-hand sides;
    reserve: bytes never handed to hierarchies."""

    def __init__(self, build: Callable, estimate: Callable, free_bytes: Callable, rhs: Callable,
                 reserve: int = 2 << 30, iters_per_step: int = 2, keep_x: bool = False, clock=time.perf_counter,
                 new_x: Optional[Callable] = None, build_async: bool = True):
        self.build, self.estimate, self.free_bytes, self.rhs = build, estimate, free_bytes, rhs
        self.reserve, self.iters_per_step, self.keep_x, self.clock = reserve, iters_per_step, keep_x, clock
        self.new_x = new_x
        # builds run on one worker thread while the loop keeps stepping the engines (the library's
        # graph captures are thread-local); the bytes a running build will take stay reserved
        self.build_async = build_async
        self.building: Dict[tuple, tuple] = {}   # key -> (future, reserved bytes)
        self._builder: Optional[concurrent.futures.ThreadPoolExecutor] = None
        self.cache: Dict[tuple, Entry] = collections.OrderedDict()
        self.stats = dict(builds=0, build_s=0.0, evictions=0, deferred=0, peak_resident=0, hits=0)

    # ---- memory ---------------------------------------------------------------------------
    def resident_bytes(self) -> int:
        return sum(e.nbytes for e in self.cache.values())

    def _make_room(self, need: int) -> bool:
        """Evict idle entries (least recently used first) until `need` bytes fit beside the builds
        in progress."""
        while self.free_bytes() - self.reserve - sum(b for _, b in self.building.values()) < need:
            idle = [e for e in self.cache.values() if e.running == 0]
            if not idle:
                return False
            victim = min(idle, key=lambda e: e.last_used)
            self._evict(victim)
        return True

    def _evict(self, e: Entry):
        del self.cache[e.key]
        for obj in (e.engine, e.hierarchy):
            d = getattr(obj, "destroy", None)
            if d:
                d()
        self.stats["evictions"] += 1

    def _timed_build(self, key):
        t0 = time.perf_counter()
        out = self.build(key)
        return out, time.perf_counter() - t0   # mesh assembly + setup, host clock

    def _install(self, key, built, now) -> Entry:
        (h, eng, nbytes, n), dt = built
        self.stats["build_s"] += dt
        e = Entry(key, h, eng, nbytes, n, now)
        self.cache[key] = e
        self.stats["builds"] += 1
        self.stats["peak_resident"] = max(self.stats["peak_resident"], self.resident_bytes())
        return e

    def entry(self, key, now) -> Optional[Entry]:
        """The resident entry of `key`; None while its build is running or cannot start yet."""
        e = self.cache.get(key)
        if e is not None:
            self.stats["hits"] += 1
            e.last_used = now
            return e
        running = self.building.get(key)
        if running is not None:
            if not running[0].done():
                return None
            del self.building[key]
            return self._install(key, running[0].result(), now)
        need = self.estimate(key)
        if not self._make_room(need):
            self.stats["deferred"] += 1
            return None
        if self._builder is None:
            return self._install(key, self._timed_build(key), now)
        self.building[key] = (self._builder.submit(self._timed_build, key), need)
        return None

    # ---- the loop ----------------------------------------------------------------------------
    def _idle(self, e: Entry, busy: set) -> bool:
        """The engine has no enqueued work left (polled without waiting)."""
        if e.key not in busy:
            return True
        q = getattr(e.engine, "query", None)
        if q is None:
            e.engine.wait()
        elif not q():
            return False
        busy.discard(e.key)
        return True

    def run(self, requests: List[Request], rtol: float = 1e-8, max_it: int = 1000) -> List[Request]:
        if not self.build_async:
            return self._run(requests, rtol, max_it)
        self._builder = concurrent.futures.ThreadPoolExecutor(1, thread_name_prefix="vemg-build")
        try:
            return self._run(requests, rtol, max_it)
        finally:
            self._builder.shutdown(wait=True)
            self._builder = None
            for key, (fut, _) in list(self.building.items()):   # built but never used
                del self.building[key]
                if fut.exception() is None:
                    self._install(key, fut.result(), self.clock())

    def _run(self, requests: List[Request], rtol: float, max_it: int) -> List[Request]:
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting: List[Request] = []
        running: Dict[int, Request] = {}
        busy: set = set()          # keys of engines with enqueued work
        t0 = self.clock()
        done: List[Request] = []
        while pending or waiting or running:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            progressed = False
            # columns of finished solves leave their slots (engines whose stream has drained)
            for rid, req in list(running.items()):
                e = self.cache[req.key]
                if req.live == 0 or not self._idle(e, busy):
                    continue
                for i, s in enumerate(req.slots):
                    if s is None:
                        continue
                    st, info = e.engine.poll(s)
                    if st != 2:
                        continue
                    x = self.new_x(e.n) if self.new_x else None
                    e.engine.retire(s, x)
                    req.infos[i] = info            # slots are held in column order
                    if self.keep_x:
                        req.x[i] = x
                    req.slots[i] = None
                    req.live -= 1
                    progressed = True
                if req.live == 0 and not req.pending:
                    req.finished = self.clock() - t0
                    e.running -= 1
                    e.last_used = req.finished
                    del running[rid]
                    done.append(req)
            # admission, first come first served per engine, into idle engines only (the slot
            # states a poll reads are those of the engine's last completed step)
            held = set()
            for req in list(waiting):
                if req.key in held:
                    continue
                e = self.entry(req.key, now)
                if e is None or not self._idle(e, busy):
                    held.add(req.key)
                    continue
                free = e.engine.free_slots()
                if free > 0:
                    if req.pending is None:
                        req.pending = list(self.rhs(req, e.n))
                        req.infos = [None] * len(req.pending)
                        req.x = [None] * len(req.pending) if self.keep_x else None
                    take, req.pending = req.pending[:free], req.pending[free:]
                    for b in take:
                        req.slots.append(e.engine.admit(b, rtol=rtol, max_it=max_it))
                    req.live += len(take)
                    if req.admitted is None:
                        req.admitted = self.clock() - t0
                        e.running += 1
                        running[req.rid] = req
                    progressed = True
                if req.pending is None or req.pending:   # columns still to admit
                    held.add(req.key)
                else:
                    waiting.remove(req)
            # every idle engine with live columns gets its next iterations
            for e in self.cache.values():
                if e.running > 0 and e.key not in busy:
                    e.engine.launch(self.iters_per_step)
                    busy.add(e.key)
                    progressed = True
            if not progressed:
                if not running and pending and not waiting:
                    gap = pending[0].arrival - (self.clock() - t0)
                    if gap > 0:
                        time.sleep(min(gap, 0.01))
                elif busy or self.building:
                    time.sleep(0.0001)
        return done


def summarize(done: List[Request], makespan: float) -> dict:
    lat = np.array([r.finished - r.arrival for r in done])
    solves = sum(r.nrhs for r in done)
    iters = [i["iters"] for r in done for i in r.infos]
    return {"requests": len(done), "rhs_solves": solves, "makespan_s": makespan,
            "requests_per_s": len(done) / makespan, "solves_per_s": solves / makespan,
            "p50_latency_ms": 1000.0 * float(np.percentile(lat, 50)),
            "p99_latency_ms": 1000.0 * float(np.percentile(lat, 99)),
            "mean_iters": float(np.mean(iters)) if iters else 0.0,
            "all_ok": all(i["status"] == "OK" for r in done for i in r.infos),
            "columns_converged": sum(i["status"] == "OK" for r in done for i in r.infos),
            # stopped by the stagnation test at the FP64 round-off floor (relres within 10x of 1e-8)
            "columns_at_floor": sum(i["status"] == "ENOTCONV" and i["relres"] <= 1e-7 for r in done for i in r.infos),
            "columns_failed": sum(i["status"] not in ("OK", "ENOTCONV") or (i["status"] == "ENOTCONV" and
                                  i["relres"] > 1e-7) for r in done for i in r.infos),
            "not_ok": [dict(rid=r.rid, mesh=r.mesh_id, eps=r.eps, bc=r.bc, iters=i["iters"], status=i["status"],
                            relres=i["relres"]) for r in done for i in r.infos if i["status"] != "OK"][:20]}


# ---------------------------------------------------------------------------------------------
# the GPU factories

class GpuFactory:
    """Builds meshes (once per size, depth scaled per aspect ratio), hierarchies and engines."""

    def __init__(self, slots: int = 8, precision: int = 1, sizes=SIZES, nz: int = NZ, mesh_seed: int = 5000):
        import torch
        from . import inputs as I
        from . import vemg as V
        self.I, self.V = I, V
        self.device = torch.cuda.current_device()   # builds on the worker thread use the same device
        self.slots, self.precision, self.sizes, self.nz, self.mesh_seed = slots, precision, sizes, nz, mesh_seed
        self.base = {}

    def mesh(self, mesh_id: int, eps: float):
        if mesh_id not in self.base:
            nx = self.sizes[mesh_id]
            self.base[mesh_id] = self.I.make_mesh(nx, nx, self.nz, self.I.depth_sines(1.0), z_jitter=0.3,
                                                  seed=self.mesh_seed + mesh_id)
        return self.I.scale_depth(self.base[mesh_id], eps)

    def nodes(self, mesh_id: int) -> int:
        nx = self.sizes[mesh_id]
        return (nx + 1) * (nx + 1) * (self.nz + 1)

    def estimate(self, key) -> int:
        n = self.nodes(key[0])
        # hierarchy (both layouts) about 1.2 KB per node; engine work about 130 B per node and slot
        return int(n * (1200 + 130 * self.slots))

    def precision_for(self, eps: float) -> int:
        """FP32 V-cycles except at eps <= 1e-4: there the FP64 residual has reached its round-off
        floor near 1e-8 (the true residual of plain FP64 PCG stays at 2-5e-8), and the flexible-CG
        recursion with an FP32 preconditioner can stall just above the tolerance."""
        return self.V.VEMG_PREC_FP64 if eps <= 1e-4 else self.precision

    def build(self, key):
        import torch
        V = self.V
        torch.cuda.set_device(self.device)
        m = self.mesh(key[0], key[1])
        vm = V.Mesh.from_inputs(m)
        # on a stream of its own: the right-hand sides the serving loop draws on its current stream
        # do not queue behind setup kernels (setup synchronises this stream before it returns)
        with torch.cuda.stream(torch.cuda.Stream()):
            A = V.vemg_assemble(vm)
            h = V.vemg_setup(A, vm, V.vemg_default_options(bc=key[2], precision=self.precision_for(key[1])))
            A.free()
        eng = V.Engine(h, self.slots)
        return h, eng, V.vemg_hierarchy_bytes(h) + eng.bytes(), m.n

    @staticmethod
    def free_bytes() -> int:
        import torch
        return int(torch.cuda.mem_get_info()[0])

    @staticmethod
    def rhs(req: Request, n: int):
        import torch
        g = torch.Generator(device="cuda")
        g.manual_seed(req.seed)
        return [torch.randn(n, dtype=torch.float64, device="cuda", generator=g) for _ in range(req.nrhs)]

    @staticmethod
    def new_x(n: int):
        import torch
        return torch.empty(n, dtype=torch.float64, device="cuda")
