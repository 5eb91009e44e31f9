"""Host logic of the continuous-batching server with fake hierarchies and a fake free-memory
provider (no GPU): admission never oversubscribes memory, idle hierarchies are evicted least
recently used first, busy ones never, and every request completes."""
import time

import numpy as np

from paper_0912_1976_gb300 import serve as S


class FakeEngine:
    def __init__(self, slots, steps_needed):
        self.slots = [None] * slots
        self.steps_needed = steps_needed
        self.destroyed = False

    def free_slots(self):
        return sum(s is None for s in self.slots)

    def admit(self, b, rtol=1e-8, max_it=1000):
        i = self.slots.index(None)
        self.slots[i] = 0
        return i

    def launch(self, iters=1):
        for i, s in enumerate(self.slots):
            if s is not None:
                self.slots[i] = s + iters

    def wait(self):
        pass

    def poll(self, slot):
        done = self.slots[slot] >= self.steps_needed
        return (2 if done else 1), {"iters": self.slots[slot], "status": "OK"}

    def retire(self, slot, x):
        self.slots[slot] = None

    def destroy(self):
        self.destroyed = True


class Pool:
    """A fake device: `total` bytes, hierarchies take `per_node` bytes per node."""

    def __init__(self, total):
        self.total = total
        self.used = 0

    def free(self):
        return self.total - self.used


def _server(pool, sizes, slots=4, steps=3):
    def estimate(key):
        return sizes[key[0]] * 10

    def build(key):
        nbytes = estimate(key)
        assert pool.used + nbytes <= pool.total, "oversubscribed"
        pool.used += nbytes
        eng = FakeEngine(slots, steps)

        class H:
            def destroy(self_inner):
                pool.used -= nbytes
        return H(), eng, nbytes, sizes[key[0]]

    return S.Server(build, estimate, pool.free, lambda req, n: [None] * req.nrhs, reserve=0)


def test_all_requests_complete_and_memory_is_respected():
    sizes = [100, 200, 400, 800]
    pool = Pool(total=2 * 800 * 10 + 100)               # room for two of the largest at once
    srv = _server(pool, sizes)
    reqs = S.make_requests(60, rate=None, seed=3, sizes=sizes, eps_grid=[1e-3, 1e-1], max_rhs=4)
    done = srv.run(reqs)
    assert len(done) == 60
    assert all(r.finished >= r.admitted >= r.arrival for r in done)
    assert srv.stats["peak_resident"] <= pool.total
    assert srv.stats["evictions"] > 0                   # more keys than fit: idle ones were evicted
    assert pool.used == srv.resident_bytes()


def test_busy_hierarchies_are_never_evicted():
    sizes = [500]
    pool = Pool(total=500 * 10)                         # exactly one hierarchy fits
    srv = _server(pool, sizes, slots=8, steps=5)
    reqs = [S.Request(i, 0, [1e-3, 1e-2][i % 2], 0, 1, 0.0, i) for i in range(6)]
    done = srv.run(reqs)
    assert len(done) == 6
    # the two keys alternate: the second can only be built once the first is idle
    assert srv.stats["deferred"] > 0 and srv.stats["evictions"] >= 1


def test_request_stream_is_seeded_and_poisson():
    a = S.make_requests(512, rate=50.0, seed=11)
    b = S.make_requests(512, rate=50.0, seed=11)
    assert [(r.mesh_id, r.eps, r.bc, r.nrhs, r.arrival) for r in a] == [(r.mesh_id, r.eps, r.bc, r.nrhs, r.arrival) for r in b]
    gaps = np.diff([r.arrival for r in a])
    assert abs(gaps.mean() - 1 / 50.0) < 0.2 / 50.0
    assert {r.nrhs for r in a} == set(range(1, 9))
    assert abs(np.mean([r.bc for r in a]) - 0.5) < 0.1


class PacedEngine(FakeEngine):
    """An engine whose enqueued step takes `cost` polls of its stream to finish; it records the
    right-hand sides in the order they were admitted and refuses calls that need an idle stream."""

    def __init__(self, slots, steps_needed, cost):
        super().__init__(slots, steps_needed)
        self.cost, self.left, self.launches, self.admitted = cost, 0, 0, []

    def admit(self, b, rtol=1e-8, max_it=1000):
        assert self.left == 0, "admitted into a busy engine"
        self.admitted.append(b)
        return super().admit(b)

    def launch(self, iters=1):
        assert self.left == 0, "launched a busy engine"
        super().launch(iters)
        self.left, self.launches = self.cost, self.launches + 1

    def query(self):
        if self.left > 0:
            self.left -= 1
        return self.left == 0

    def wait(self):
        raise AssertionError("the server must not block on an engine")

    def poll(self, slot):
        assert self.left == 0, "polled a busy engine"
        return super().poll(slot)


def _paced_server(sizes, slots, steps, cost):
    engines = {}

    def build(key):
        eng = engines[key] = PacedEngine(slots, steps, cost[key[0]])
        return object(), eng, 0, sizes[key[0]]

    srv = S.Server(build, lambda key: 0, lambda: 1 << 40,
                   lambda req, n: [(req.rid, j) for j in range(req.nrhs)], reserve=0)
    return srv, engines


def test_engines_step_at_their_own_pace():
    # a small and a large hierarchy, both requests needing the same iterations: the small engine's
    # steps finish 50x sooner, so its request completes first instead of in the same round
    srv, engines = _paced_server([10, 1000], slots=2, steps=6, cost={0: 1, 1: 50})
    reqs = [S.Request(0, 1, 1e-3, 0, 1, 0.0, 0), S.Request(1, 0, 1e-3, 0, 1, 0.0, 1)]
    done = srv.run(reqs)
    assert [r.rid for r in done] == [1, 0]
    small, large = engines[(0, 1e-3, 0)], engines[(1, 1e-3, 0)]
    assert small.launches == large.launches == 3          # 3 steps of 2 iterations each
    assert done[0].finished < done[1].finished


def test_wide_requests_are_admitted_first_come_first_served():
    # one engine of 4 slots; a 4-column request behind a 2-column one takes the two free slots and
    # holds back the later 1-column requests until its other two columns are in
    srv, engines = _paced_server([10], slots=4, steps=3, cost={0: 2})
    reqs = [S.Request(0, 0, 1e-3, 0, 2, 0.0, 0), S.Request(1, 0, 1e-3, 0, 4, 0.0, 1)] + \
           [S.Request(i, 0, 1e-3, 0, 1, 0.0, i) for i in range(2, 8)]
    done = srv.run(reqs)
    assert len(done) == 8 and all(len(r.infos) == r.nrhs for r in done)
    log = engines[(0, 1e-3, 0)].admitted
    assert log == sorted(log)                             # columns admitted in arrival order
    wide = next(r for r in done if r.rid == 1)
    assert all(r.admitted >= wide.admitted for r in done if r.rid > 1)


def test_engines_keep_stepping_while_a_hierarchy_builds():
    # the small request runs three 30 ms steps; the large hierarchy's build, started at 0.05 s,
    # takes 0.5 s on the worker thread: the small request finishes meanwhile (a build on the loop's
    # thread would hold its last steps until 0.55 s)
    class TimedEngine(PacedEngine):
        """A step takes 30 ms of wall time."""

        def launch(self, iters=1):
            super().launch(iters)
            self.until = time.perf_counter() + 0.03

        def query(self):
            self.left = 0 if time.perf_counter() >= self.until else 1
            return self.left == 0

    engines = {}

    def build(key):
        if key[0] == 1:
            time.sleep(0.5)
        eng = engines[key] = TimedEngine(2, 6, 1)
        return object(), eng, 0, 10

    srv = S.Server(build, lambda key: 0, lambda: 1 << 40, lambda req, n: [(req.rid, j) for j in range(req.nrhs)],
                   reserve=0)
    reqs = [S.Request(0, 0, 1e-3, 0, 1, 0.0, 0), S.Request(1, 1, 1e-3, 0, 1, 0.05, 1)]
    done = {r.rid: r for r in srv.run(reqs)}
    assert done[0].finished < 0.3 < done[1].finished
    assert srv.stats["builds"] == 2 and not srv.building


def test_a_failing_build_raises_out_of_the_loop():
    # a build error (say, the device is out of memory) ends the run with that error, after the
    # worker thread has stopped
    def build(key):
        if key[0] == 1:
            raise MemoryError("no room for this hierarchy")
        return object(), PacedEngine(2, 2, 1), 0, 10

    srv = S.Server(build, lambda key: 0, lambda: 1 << 40, lambda req, n: [(req.rid, j) for j in range(req.nrhs)],
                   reserve=0)
    reqs = [S.Request(0, 0, 1e-3, 0, 1, 0.0, 0), S.Request(1, 1, 1e-3, 0, 1, 0.0, 1)]
    try:
        srv.run(reqs)
    except MemoryError:
        pass
    else:
        raise AssertionError("the build error was swallowed")
    assert srv._builder is None and not srv.building


def test_bytes_of_a_running_build_stay_reserved():
    # room for one hierarchy: while the first build runs, a second key is deferred (its bytes
    # would not fit beside the reserved ones), then built once the first is idle and evicted
    pool = Pool(total=1000)

    def build(key):
        time.sleep(0.05)
        assert pool.used + 1000 <= pool.total, "oversubscribed"
        pool.used += 1000
        eng = PacedEngine(2, 2, 1)

        class H:
            def destroy(self_inner):
                pool.used -= 1000
        return H(), eng, 1000, 10

    srv = S.Server(build, lambda key: 1000, pool.free, lambda req, n: [(req.rid, j) for j in range(req.nrhs)],
                   reserve=0)
    reqs = [S.Request(0, 0, 1e-3, 0, 1, 0.0, 0), S.Request(1, 0, 1e-2, 0, 1, 0.0, 1)]
    done = srv.run(reqs)
    assert len(done) == 2
    assert srv.stats["deferred"] > 0 and srv.stats["evictions"] >= 1 and srv.stats["builds"] == 2
