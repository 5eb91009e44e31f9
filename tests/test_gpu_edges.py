"""Degenerate and limit cases of the method on the GPU, each against the oracle: a single layer of
hexes, a single column of hexes, a one-level hierarchy (the finest level is the coarsest), the
deepest hierarchy the options allow, and the empty and oversize batches."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0912_1976_gb300 import inputs as I
from paper_0912_1976_gb300 import vemg as V

pytestmark = pytest.mark.gpu


def _solve_pair(m, bc=V.VEMG_NEUMANN, **opts):
    vm = V.Mesh.from_inputs(m)
    A = V.vemg_assemble(vm)
    h = V.vemg_setup(A, vm, V.vemg_default_options(bc=bc, **opts))
    oo = {k: opts[k] for k in ("coarse_max", "max_levels") if k in opts}
    om = O.Problem(m, bc=bc, **oo)
    b = I.normal_loads(m.n, 61)
    x, info = V.vemg_solve(h, torch.from_numpy(b).cuda(), rtol=1e-9, max_it=500)
    ro = om.solve(b, tol=1e-9, maxit=500)
    return h, om, x.cpu().numpy(), info, ro


@pytest.mark.parametrize("bc", [V.VEMG_NEUMANN, V.VEMG_DIRICHLET_TOP])
@pytest.mark.parametrize("shape", [(12, 10, 1), (1, 1, 6), (2, 1, 3)])
def test_single_layer_and_single_column(shape, bc):
    nx, ny, nz = shape
    m = I.make_mesh(nx, ny, nz, I.depth_sines(1e-2), z_jitter=0.3, seed=31)
    h, om, x, info, ro = _solve_pair(m, bc)
    assert info["status"] == "OK" and ro["status"] == "OK"
    assert abs(info["iters"] - ro["iters"]) <= 1
    assert np.linalg.norm(x - ro["x"]) <= 1e-9 * np.linalg.norm(ro["x"])
    assert info["true_relres"] <= 2e-9


@pytest.mark.parametrize("opts", [dict(max_levels=1), dict(coarse_max=1), dict(coarse_max=1, max_levels=16)])
def test_one_level_and_deepest_hierarchies(opts):
    m = I.make_mesh(16, 14, 6, I.depth_sines(1e-3), z_jitter=0.3, seed=32)
    h, om, x, info, ro = _solve_pair(m, **opts)
    for c in (0, 1):
        assert V.vemg_get_size(h, "nlev", c) == om.nlev(c)
        assert V.vemg_get_size(h, "direct", c) == om.size("direct", c)
    assert info["status"] == ro["status"] == "OK"
    assert abs(info["iters"] - ro["iters"]) <= 1
    assert np.linalg.norm(x - ro["x"]) <= 1e-9 * np.linalg.norm(ro["x"])


def test_empty_and_oversize_batches():
    m = I.make_mesh(8, 8, 4, I.depth_sines(1e-2), z_jitter=0.3, seed=33)
    vm = V.Mesh.from_inputs(m)
    A = V.vemg_assemble(vm)
    h = V.vemg_setup(A, vm, V.vemg_default_options())
    B0 = torch.zeros((0, m.n), dtype=torch.float64, device="cuda")
    X, infos = V.vemg_solve_batch(h, B0, rtol=1e-8)
    assert X.shape == (0, m.n) and len(infos) == 0
    B = torch.from_numpy(np.stack([I.normal_loads(m.n, c) for c in range(129)])).cuda()
    with pytest.raises(V.VemgError):   # more columns than one batch holds (128)
        V.vemg_solve_batch(h, B, rtol=1e-8)
    X, infos = V.vemg_solve_batch(h, B[:128].contiguous(), rtol=1e-8)
    assert all(i["status"] == "OK" for i in infos)
