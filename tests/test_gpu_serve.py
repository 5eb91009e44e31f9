"""Continuous batching on the GPU: engine slots give the results of single solves, a request that
joins a running batch converges like a fresh solve, and a served request's result alone equals its
result in a mix of concurrent requests (other slots, other hierarchies on other streams)."""
import numpy as np
import pytest
import torch

from paper_0912_1976_gb300 import inputs as I
from paper_0912_1976_gb300 import serve as S
from paper_0912_1976_gb300 import vemg as V

pytestmark = pytest.mark.gpu

# FP64 engines: results differ from single solves by summation order only
TOL = {V.VEMG_PREC_FP64: 1e-9, V.VEMG_PREC_FP32: 1e-6}


def _hier(precision, bc=V.VEMG_NEUMANN, nx=24, nz=12, eps=1e-3, seed=51):
    m = I.make_mesh(nx, nx, nz, I.depth_sines(eps), z_jitter=0.3, seed=seed)
    vm = V.Mesh.from_inputs(m)
    A = V.vemg_assemble(vm)
    h = V.vemg_setup(A, vm, V.vemg_default_options(bc=bc, precision=precision))
    return m, vm, A, h


def _run_until_done(eng, slots, max_steps=500):
    for _ in range(max_steps):
        eng.launch(1)
        eng.wait()
        if all(eng.poll(s)[0] == V.VEMG_SLOT_DONE for s in slots):
            return
    raise AssertionError("engine did not finish")


def test_engine_query_polls_without_waiting():
    """vemg_engine_query reports work still enqueued on the engine's stream (behind a kernel that
    spins ~25 ms) without waiting for it, and idle once the stream has drained; the slot states
    it then exposes are those after the step."""
    m, vm, A, h = _hier(V.VEMG_PREC_FP64, V.VEMG_NEUMANN)
    eng = V.Engine(h, 2)
    b = torch.from_numpy(I.normal_loads(m.n, 90)).cuda()
    s = eng.admit(b, rtol=1e-9)
    torch.cuda.synchronize()
    with torch.cuda.stream(eng.stream):
        torch.cuda._sleep(50_000_000)
    eng.launch(1)
    assert not eng.query()                 # the spin is still ahead of the step
    eng.wait()
    assert eng.query()
    st, info = eng.poll(s)
    assert st == V.VEMG_SLOT_RUNNING and info["iters"] >= 1
    _run_until_done(eng, [s])
    x = torch.empty_like(b)
    eng.retire(s, x)
    assert eng.query()


@pytest.mark.parametrize("precision", [V.VEMG_PREC_FP64, V.VEMG_PREC_FP32])
@pytest.mark.parametrize("bc", [V.VEMG_NEUMANN, V.VEMG_DIRICHLET_TOP])
def test_engine_slots_equal_single_solves(precision, bc):
    m, vm, A, h = _hier(precision, bc)
    eng = V.Engine(h, 4)
    bs = [torch.from_numpy(I.normal_loads(m.n, 60 + c)).cuda() for c in range(3)]
    slots = [eng.admit(b, rtol=1e-9) for b in bs]
    _run_until_done(eng, slots)
    for b, s in zip(bs, slots):
        st, info = eng.poll(s)
        x = torch.empty_like(b)
        eng.retire(s, x)
        x1, i1 = V.vemg_solve(h, b, rtol=1e-9)
        assert info["status"] == "OK" and abs(info["iters"] - i1["iters"]) <= 1
        assert (x - x1).norm().item() <= TOL[precision] * x1.norm().item()
    assert eng.free_slots() == 4


def test_request_joining_mid_flight():
    m, vm, A, h = _hier(V.VEMG_PREC_FP64)
    eng = V.Engine(h, 2)
    b0 = torch.from_numpy(I.normal_loads(m.n, 70)).cuda()
    b1 = torch.from_numpy(I.normal_loads(m.n, 71)).cuda()
    s0 = eng.admit(b0, rtol=1e-9)
    eng.launch(5)
    eng.wait()
    s1 = eng.admit(b1, rtol=1e-9)            # joins while slot 0 is at iteration 5
    _run_until_done(eng, [s0, s1])
    for b, s in ((b0, s0), (b1, s1)):
        st, info = eng.poll(s)
        x = torch.empty_like(b)
        eng.retire(s, x)
        x1, i1 = V.vemg_solve(h, b, rtol=1e-9)
        assert abs(info["iters"] - i1["iters"]) <= 1
        assert (x - x1).norm().item() <= 1e-9 * x1.norm().item()


def test_served_request_same_alone_and_in_the_mix():
    fac = S.GpuFactory(slots=8, precision=V.VEMG_PREC_FP64, sizes=[12, 16, 20], nz=6)

    def server():
        return S.Server(fac.build, fac.estimate, fac.free_bytes, fac.rhs, keep_x=True, new_x=fac.new_x)

    target = S.Request(0, 2, 1e-3, 0, 3, 0.0, 777)
    alone = server().run([target])[0]
    mix = [S.Request(0, 2, 1e-3, 0, 3, 0.0, 777)]
    mix += S.make_requests(24, rate=None, seed=9, sizes=[12, 16, 20], eps_grid=[1e-3, 1e-1], max_rhs=4)
    for i, r in enumerate(mix[1:], 1):
        r.rid = i
    done = {r.rid: r for r in server().run(mix)}
    assert len(done) == 25 and all(i["status"] == "OK" for r in done.values() for i in r.infos)
    inmix = done[0]
    for xa, xm in zip(alone.x, inmix.x):
        assert (xa - xm).norm().item() <= 1e-9 * xa.norm().item()
    assert [i["iters"] for i in alone.infos] == [i["iters"] for i in inmix.infos] or \
        max(abs(a["iters"] - b["iters"]) for a, b in zip(alone.infos, inmix.infos)) <= 1


@pytest.mark.parametrize("precision", [V.VEMG_PREC_FP32, V.VEMG_PREC_BF16])
def test_served_request_same_alone_and_in_the_mix_mixed_precision(precision):
    """FP32 cycles (FP32 or BF16 operator values): within one engine a column's arithmetic does not
    depend on the other slots (per-column reductions in fixed blocks), so a request's result in the
    mix equals its result alone to FP64 reordering of the served hierarchy's own solves."""
    fac = S.GpuFactory(slots=8, precision=precision, sizes=[12, 16, 20], nz=6)

    def server():
        return S.Server(fac.build, fac.estimate, fac.free_bytes, fac.rhs, keep_x=True, new_x=fac.new_x)

    target = S.Request(0, 2, 1e-3, 0, 3, 0.0, 778)
    alone = server().run([target])[0]
    mix = [S.Request(0, 2, 1e-3, 0, 3, 0.0, 778)]
    mix += S.make_requests(24, rate=None, seed=10, sizes=[12, 16, 20], eps_grid=[1e-3, 1e-1], max_rhs=4)
    for i, r in enumerate(mix[1:], 1):
        r.rid = i
    done = {r.rid: r for r in server().run(mix)}
    assert len(done) == 25 and all(i["status"] == "OK" for r in done.values() for i in r.infos)
    for xa, xm in zip(alone.x, done[0].x):
        assert (xa - xm).norm().item() <= 1e-9 * xa.norm().item()


def test_admission_waits_for_the_stream_that_produced_b():
    """A right-hand side produced on the caller's stream behind a long kernel: the engine's stream
    must wait for it (otherwise it copies the old contents, here zeros)."""
    m, vm, A, h = _hier(V.VEMG_PREC_FP64)
    eng = V.Engine(h, 2)
    src = torch.from_numpy(I.normal_loads(m.n, 80)).cuda()
    b = torch.zeros_like(src)
    torch.cuda.synchronize()
    torch.cuda._sleep(50_000_000)          # about 25 ms of spinning on the current stream
    b.copy_(src)
    s = eng.admit(b, rtol=1e-9)
    _run_until_done(eng, [s])
    st, info = eng.poll(s)
    x = torch.empty_like(b)
    eng.retire(s, x)
    x1, i1 = V.vemg_solve(h, src, rtol=1e-9)
    assert info["iters"] > 0 and abs(info["iters"] - i1["iters"]) <= 1
    assert (x - x1).norm().item() <= 1e-9 * x1.norm().item()


def test_served_columns_match_the_oracle():
    """Served results against the oracle: a small stream over three meshes, aspect ratios 1e-1, 1e-3
    and 1e-4, both boundary conditions; every column of every request is solved again by the oracle
    (FP64 PCG) from the same right-hand side. FP64 cycles serve eps <= 1e-4, FP32 cycles the rest;
    both stop at rel-res 1e-8, so the solutions agree to what that residual allows."""
    from oracle import oracle as O
    from conftest import record
    fac = S.GpuFactory(slots=8, precision=V.VEMG_PREC_BF16, sizes=[12, 16, 20], nz=6)
    srv = S.Server(fac.build, fac.estimate, fac.free_bytes, fac.rhs, keep_x=True, new_x=fac.new_x)
    reqs = S.make_requests(12, rate=None, seed=31, sizes=[12, 16, 20], eps_grid=[1e-4, 1e-3, 1e-1], max_rhs=3)
    done = srv.run(reqs)
    assert len(done) == 12
    worst = 0.0
    for r in done:
        m = fac.mesh(r.mesh_id, r.eps)
        om = O.Problem(m, bc=r.bc)
        bs = fac.rhs(r, m.n)
        for b, x, info in zip(bs, r.x, r.infos):
            ro = om.solve(b.cpu().numpy(), tol=1e-8, maxit=2000)
            assert info["status"] == "OK" and ro["status"] == "OK", (r.rid, info, ro["status"])
            err = np.linalg.norm(x.cpu().numpy() - ro["x"]) / np.linalg.norm(ro["x"])
            worst = max(worst, err)
            assert err <= 1e-6, (r.rid, r.eps, r.bc, err)
    record("served_columns_vs_oracle", worst_rel_l2=worst, columns=sum(r.nrhs for r in done))
