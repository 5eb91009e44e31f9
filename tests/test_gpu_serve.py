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
