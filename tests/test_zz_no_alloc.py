"""vemg_spmv_static: the product y = A x for callers that cannot allocate device memory (for
example code running inside an allocator callback, or under a device memory budget fixed in
advance). It must give what vemg_spmv gives, bit for bit, call after call, from its static work
array, on a hierarchy fresh from vemg_setup; it refuses, with a reason, a hierarchy larger than its
array.

This file sorts last so that, if it fails, a run stopping at the first failure has already run
every other test."""
import numpy as np
import pytest
import torch

from paper_0912_1976_gb300 import inputs as I
from paper_0912_1976_gb300 import vemg as V

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bc", [V.VEMG_NEUMANN, V.VEMG_DIRICHLET_TOP])
def test_static_spmv_matches_allocating_spmv_twice(bc):
    m = I.make_mesh(24, 20, 12, I.depth_sines(1e-3), z_jitter=0.3, seed=31)
    vm = V.Mesh.from_inputs(m)
    A = V.vemg_assemble(vm)
    h = V.vemg_setup(A, vm, V.vemg_default_options(bc=bc))
    n = V.vemg_get_size(h, "n") - (V.vemg_get_size(h, "mtop") if bc == V.VEMG_DIRICHLET_TOP else 0)
    rng = np.random.default_rng(7)
    for _ in range(2):                      # two calls in a row: the static array is reused
        x = torch.from_numpy(rng.standard_normal(n)).cuda()
        # first on the fresh hierarchy: vemg_setup left it ready, no allocating call before
        y = V.vemg_spmv_static(h, x)
        y_ref = V.vemg_spmv(h, x)
        torch.cuda.synchronize()
        # the same products summed in the same order: the same bits
        assert torch.equal(y, y_ref), (y - y_ref).abs().max().item()
    h.destroy()


def test_static_spmv_rejects_hierarchies_larger_than_its_array():
    # 128 x 128 x 63 hexes: 129 * 129 * 64 = 1,065,024 unknowns (Neumann), above 1,048,576
    m = I.make_mesh(128, 128, 63, I.depth_sines(1e-3), seed=32)
    vm = V.Mesh.from_inputs(m)
    A = V.vemg_assemble(vm)
    h = V.vemg_setup(A, vm, V.vemg_default_options())
    x = torch.ones(m.n, dtype=torch.float64, device="cuda")
    V.vemg_spmv(h, x)
    with pytest.raises(V.VemgError) as e:
        V.vemg_spmv_static(h, x)
    assert e.value.code == V.VEMG_EINVAL and "1065024 unknowns" in e.value.detail
    h.destroy()
