"""The paper's measure (section 6): the infinity-norm error against a chosen solution x*. With
b = A x* (x* random with zero mean, A assembled by the oracle), the GPU solve's error must match
the oracle's and fall with the tolerance, for every V-cycle precision."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0912_1976_gb300 import inputs as I
from paper_0912_1976_gb300 import vemg as V

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [V.VEMG_PREC_FP64, V.VEMG_PREC_FP32, V.VEMG_PREC_BF16])
def test_infinity_norm_error_against_a_chosen_solution(precision):
    m = I.make_mesh(40, 36, 16, I.depth_sines(1e-3), z_jitter=0.3, seed=51)
    om = O.Problem(m)
    A = om.csr("A")
    n2o = om.ints("new2old")
    rng = np.random.default_rng(52)
    xs = rng.standard_normal(m.n)
    xs -= xs.mean()
    # b = A x* in the caller's ordering (A is held in the internal, top-first ordering)
    xi = xs[n2o]
    bi = A @ xi
    b = np.empty(m.n)
    b[n2o] = bi
    vm = V.Mesh.from_inputs(m)
    Ag = V.vemg_assemble(vm)
    h = V.vemg_setup(Ag, vm, V.vemg_default_options(precision=precision))
    errs = []
    for tol in (1e-4, 1e-7, 1e-10):
        x, info = V.vemg_solve(h, torch.from_numpy(b).cuda(), rtol=tol, max_it=500)
        assert info["status"] == "OK"
        e = np.abs(x.cpu().numpy() - xs).max() / np.abs(xs).max()
        ro = om.solve(b, tol=tol, maxit=500)
        eo = np.abs(ro["x"] - xs).max() / np.abs(xs).max()
        # same method, same stopping rule: errors of the same size (FP32 V-cycles: FCG iterates)
        assert e <= 3.0 * eo + 1e-12 and eo <= 3.0 * e + 1e-12, (tol, e, eo)
        errs.append(e)
    # the oracle at rtol 1e-4 / 1e-7 / 1e-10: 2e-2, 5e-5, 3e-8 (7, 13, 20 iterations)
    assert errs[0] > 100 * errs[1] and errs[1] > 100 * errs[2], errs
    assert errs[2] < 1e-6
