"""The coarse tail as one thread-block cluster (vemg_options.tail_cluster): every level from the
tail level down to the coarsest and back up runs in one cluster, its steps separated by the
hardware cluster barrier. Its per-row arithmetic is that of the one-kernel-per-phase cycle, so a
V-cycle, a preconditioner application and a solve must give the same bits as that cycle, and the
solve must match the oracle as the per-phase cycle does. The single-CTA tail is held to the same
bits."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0912_1976_gb300 import inputs as I
from paper_0912_1976_gb300 import vemg as V

pytestmark = pytest.mark.gpu

MESHES = {
    # A_bar chain 128,960 -> 36,537 -> 11,079 -> 4,030 (coarsening stalls there: the last level is
    # swept, not inverted), surface chain 4,030 -> 585 (dense)
    "zjit64": lambda: I.make_mesh(64, 61, 32, I.depth_sines(1e-3), z_jitter=0.3, seed=9),
    # A_bar 12,276 -> 3,634 -> 1,023 (dense), surface 1,023 (dense): a tail that is only the dense
    # coarsest level
    "clust32": lambda: I.make_mesh(32, 30, 12, I.depth_sines(1e-3), z_jitter=0.3, seed=10, cluster=0.9),
}
_cache = {}


def _pair(name, precision, bc=V.VEMG_NEUMANN, tail_rows=20000, ncta=16):
    key = (name, precision, bc, tail_rows, ncta)
    if key not in _cache:
        if name not in _cache:
            m = MESHES[name]()
            vm = V.Mesh.from_inputs(m)
            _cache[name] = (m, vm, V.vemg_assemble(vm))
        m, vm, A = _cache[name]
        ref = V.vemg_setup(A, vm, V.vemg_default_options(bc=bc, precision=precision))
        h = V.vemg_setup(A, vm, V.vemg_default_options(bc=bc, precision=precision, tail_rows=tail_rows,
                                                       tail_cluster=ncta))
        _cache[key] = (m, ref, h)
    return _cache[key]


PRECS = [V.VEMG_PREC_FP64, V.VEMG_PREC_FP32, V.VEMG_PREC_BF16]


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("ncta", [16, 8, 0])
def test_cluster_tail_cycle_is_bitwise_the_per_phase_cycle(name, precision, ncta):
    m, ref, h = _pair(name, precision, ncta=ncta)
    rng = np.random.default_rng(3)
    for c in (0, 1):
        nn = V.vemg_get_size(h, "lev.n", c, 0)
        b = torch.from_numpy(rng.standard_normal(nn)).cuda()
        x1 = V.vemg_vcycle(ref, c, b)
        x2 = V.vemg_vcycle(h, c, b)
        torch.cuda.synchronize()
        assert torch.equal(x1, x2), (c, (x1 - x2).abs().max().item())
    r = torch.from_numpy(rng.standard_normal(m.n)).cuda()
    z1 = V.vemg_precond(ref, r)
    z2 = V.vemg_precond(h, r)
    assert torch.equal(z1, z2), (z1 - z2).abs().max().item()


@pytest.mark.parametrize("precision", PRECS)
def test_cluster_tail_solve_matches_per_phase_and_oracle(precision):
    m, ref, h = _pair("zjit64", precision)
    b = I.normal_loads(m.n, 12)
    bd = torch.from_numpy(b).cuda()
    x1, i1 = V.vemg_solve(ref, bd, rtol=1e-8)
    x2, i2 = V.vemg_solve(h, bd, rtol=1e-8)
    assert i2["status"] == "OK" and i1["iters"] == i2["iters"]
    assert torch.equal(x1, x2)
    if precision == V.VEMG_PREC_FP64:
        ro = O.Problem(m).solve(b, tol=1e-8)
        assert abs(i2["iters"] - ro["iters"]) <= 1
        assert np.linalg.norm(x2.cpu().numpy() - ro["x"]) <= 1e-9 * np.linalg.norm(ro["x"])


@pytest.mark.parametrize("precision", [V.VEMG_PREC_FP64, V.VEMG_PREC_BF16])
def test_cluster_tail_dirichlet_top(precision):
    m, ref, h = _pair("zjit64", precision, bc=V.VEMG_DIRICHLET_TOP)
    b = torch.from_numpy(I.normal_loads(m.n, 13)).cuda()
    x1, i1 = V.vemg_solve(ref, b, rtol=1e-9)
    x2, i2 = V.vemg_solve(h, b, rtol=1e-9)
    assert i2["status"] == "OK" and i1["iters"] == i2["iters"] and torch.equal(x1, x2)


def test_cluster_tail_options_are_checked():
    m, vm, A = _cache.get("zjit64") or (None, None, None)
    if A is None:
        _pair("zjit64", V.VEMG_PREC_FP64)
        m, vm, A = _cache["zjit64"]
    for bad in (dict(tail_cluster=1, tail_rows=1000), dict(tail_cluster=17, tail_rows=1000),
                dict(tail_cluster=-1), dict(tail_cluster=0, tail_rows=70000)):
        with pytest.raises(V.VemgError) as e:
            V.vemg_setup(A, vm, V.vemg_default_options(**bad))
        assert e.value.code == V.VEMG_EINVAL
