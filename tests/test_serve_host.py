"""Host logic of the continuous-batching server with fake hierarchies and a fake free-memory
provider (no GPU): admission never oversubscribes memory, idle hierarchies are evicted least
recently used first, busy ones never, and every request completes."""
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
