"""Parity at the full size of the benchmark workload (256x256x32 z-jittered mesh, 2,179,617 nodes),
in the launch configuration bench.py times, on outputs the oracle can compute one at a time:
sampled rows of the assembled matrix (bitwise: the oracle's element stiffness summed in ascending
element order), sampled column locations (the oracle's locator), and properties of the solve that
hold at any size (true residual, zero mean, the same iterations for both launch structures)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0912_1976_gb300 import inputs as I
from paper_0912_1976_gb300 import vemg as V

pytestmark = pytest.mark.gpu

_cache = {}


def _full():
    if "m" not in _cache:
        m = I.make_workload_mesh("zjit256")
        vm = V.Mesh.from_inputs(m)
        A = V.vemg_assemble(vm)
        _cache.update(m=m, vm=vm, A=A)
    return _cache["m"], _cache["vm"], _cache["A"]


def test_sampled_rows_of_A_bitwise():
    m, vm, A = _full()
    h = V.vemg_setup(A, vm, V.vemg_default_options(precision=V.VEMG_PREC_FP32))
    Ag = V.vemg_get_csr(h, "A")
    n2o = V.vemg_get_int(h, "new2old")
    o2n = np.empty_like(n2o)
    o2n[n2o] = np.arange(m.n, dtype=n2o.dtype)
    rng = np.random.default_rng(17)
    nodes = rng.choice(m.n, 200, replace=False)
    tets = m.tets
    flat = tets.ravel()
    order = np.argsort(flat, kind="stable")                # incidence: node -> elements
    start = np.searchsorted(flat[order], np.arange(m.n + 1))
    for i in nodes:
        es = np.unique(order[start[i]:start[i + 1]] // 4)    # ascending element index
        row = {}
        for e in es:
            v = tets[e]
            _, K = O.elem_stiffness(m.xyz[v])
            a = int(np.nonzero(v == i)[0][0])
            for b in range(4):
                j = int(o2n[v[b]])
                row[j] = row.get(j, 0.0) + K[a, b]
        r = int(o2n[i])
        lo, hi = Ag.indptr[r], Ag.indptr[r + 1]
        cols = Ag.indices[lo:hi]
        assert sorted(row) == list(cols)
        ref = np.array([row[j] for j in cols])
        assert np.array_equal(ref.view(np.uint64), Ag.data[lo:hi].view(np.uint64)), i


def test_sampled_extrapolation_rows():
    """E~ rows of sampled nodes: the oracle's locator gives the top triangle and its barycentric
    weights; the row is those weights on the triangle's vertices, exact zeros dropped (on an
    extruded mesh every node lies under a top vertex, so the located triangle is a tie among the
    triangles around that vertex and only the row, weight 1 on the vertex, is unique)."""
    m, vm, A = _full()
    h = V.vemg_setup(A, vm, V.vemg_default_options(precision=V.VEMG_PREC_FP32))
    E = V.vemg_get_csr(h, "E")
    n2o = V.vemg_get_int(h, "new2old")
    o2n = np.empty_like(n2o)
    o2n[n2o] = np.arange(m.n, dtype=n2o.dtype)
    rng = np.random.default_rng(18)
    r = rng.choice(m.n, 500, replace=False)
    nodes = n2o[r]
    loc, w = O.locate_points(m.top_tris, m.xyz, m.xyz[nodes, :2])
    for k, ri in enumerate(r):
        ref = {}
        for a in range(3):
            if w[k, a] != 0.0:
                j = int(o2n[m.top_tris[loc[k], a]])
                ref[j] = ref.get(j, 0.0) + w[k, a]
        lo, hi = E.indptr[ri], E.indptr[ri + 1]
        got = dict(zip(E.indices[lo:hi].tolist(), E.data[lo:hi].tolist()))
        assert sorted(ref) == sorted(got), ri
        assert all(np.float64(ref[j]).view(np.uint64) == np.float64(got[j]).view(np.uint64) for j in ref), ri


@pytest.mark.parametrize("precision,cycle", [(V.VEMG_PREC_FP32, V.VEMG_CYCLE_AUTO),
                                             (V.VEMG_PREC_FP64, V.VEMG_CYCLE_AUTO),
                                             (V.VEMG_PREC_FP64, V.VEMG_CYCLE_PERSISTENT),
                                             (V.VEMG_PREC_FP32, V.VEMG_CYCLE_HYBRID),
                                             (V.VEMG_PREC_BF16, V.VEMG_CYCLE_AUTO)])
def test_full_size_solve_properties(precision, cycle):
    m, vm, A = _full()
    h = V.vemg_setup(A, vm, V.vemg_default_options(precision=precision, cycle=cycle))
    b = torch.from_numpy(I.normal_loads(m.n, 2000)).cuda()
    x, info = V.vemg_solve(h, b, rtol=1e-8, max_it=1000)
    assert info["status"] == "OK"
    assert info["true_relres"] <= 2e-8
    assert abs(x.mean().item()) <= 1e-12 * x.abs().max().item()
    # the method's iteration count at this size (the oracle takes 27 on the same workload)
    assert 24 <= info["iters"] <= 30
