"""vemg_spmv_static: the product y = A x for callers that cannot allocate device memory (for
example code running inside an allocator callback, or under a device memory budget fixed in
advance). It must give what vemg_spmv gives, call after call, from its static work array.

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
    scale = np.abs(V.vemg_get_csr(h, "A").data).max()
    rng = np.random.default_rng(7)
    for _ in range(2):                      # two calls in a row: the static array is reused
        x = torch.from_numpy(rng.standard_normal(n)).cuda()
        y_ref = V.vemg_spmv(h, x)
        y = V.vemg_spmv_static(h, x)
        torch.cuda.synchronize()
        err = (y - y_ref).abs().max().item()
        assert err <= 1e-13 * scale * x.abs().max().item(), err
    h.destroy()
