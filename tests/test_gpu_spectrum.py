"""The spectrum study of section 4 on the GPU: the CG coefficients of a solve (vemg_solve_coefficients)
give the Lanczos tridiagonal of the preconditioned operator. They must equal the oracle's, plain CG
(no preconditioner) must equal the oracle's plain CG, and the condition numbers must behave as the
paper states: Cond(A) grows like eps^-2, Cond(M^-1 A) stays bounded."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0912_1976_gb300 import inputs as I
from paper_0912_1976_gb300 import vemg as V

from conftest import record

pytestmark = pytest.mark.gpu


def _pair(m, bc=V.VEMG_NEUMANN, pc=V.VEMG_PRECOND_ADDITIVE, opc=O.PC_ADDITIVE):
    vm = V.Mesh.from_inputs(m)
    A = V.vemg_assemble(vm)
    h = V.vemg_setup(A, vm, V.vemg_default_options(bc=bc, precond=pc))
    return h, O.Problem(m, bc=bc, precond=opc), A


@pytest.mark.parametrize("bc", [V.VEMG_NEUMANN, V.VEMG_DIRICHLET_TOP])
def test_pcg_coefficients_match_oracle(bc):
    m = I.make_mesh(24, 20, 12, I.depth_sines(1e-3), z_jitter=0.3, seed=7)
    h, om, A = _pair(m, bc)
    b = I.normal_loads(m.n, 41)
    x, info = V.vemg_solve(h, torch.from_numpy(b).cuda(), rtol=1e-9)
    ro = om.solve(b, tol=1e-9)
    a, bt = V.vemg_solve_coefficients(h)
    assert len(a) == info["iters"] and abs(info["iters"] - ro["iters"]) <= 1
    # the first coefficients agree to rounding; later ones drift apart as the recurrences amplify
    # the different summation orders (by ~1e-4 after 20 iterations), like any two CG runs
    k = 6
    assert np.allclose(a[:k], ro["alpha"][:k], rtol=1e-9, atol=0)
    assert bt[0] == 0.0 and np.allclose(bt[1:k], ro["beta"][1:k], rtol=1e-9, atol=0)
    # the k-step tridiagonals differ by the coefficients' rounding, and a symmetric eigenvalue
    # moves by at most the perturbation's norm: their extremes agree closely
    lo_k, hi_k = V.vemg_lanczos_extremes(a[:k], bt[:k])
    lo_ko, hi_ko = V.vemg_lanczos_extremes(ro["alpha"][:k], ro["beta"][:k])
    assert abs(lo_k - lo_ko) <= 1e-7 * lo_ko and abs(hi_k - hi_ko) <= 1e-7 * hi_ko
    # the full history's extremes move with the drifted late coefficients
    lo, hi = V.vemg_lanczos_extremes(a, bt)
    lo_o, hi_o = V.vemg_lanczos_extremes(ro["alpha"], ro["beta"])
    record("spectrum_ritz", bc=bc, k_step_lo=abs(lo_k - lo_ko) / lo_ko, k_step_hi=abs(hi_k - hi_ko) / hi_ko,
           full_lo=abs(lo - lo_o) / lo_o, full_hi=abs(hi - hi_o) / hi_o)
    assert abs(lo - lo_o) <= 1e-3 * lo_o and abs(hi - hi_o) <= 1e-3 * hi_o


@pytest.mark.parametrize("bc", [V.VEMG_NEUMANN, V.VEMG_DIRICHLET_TOP])
def test_plain_cg_matches_oracle(bc):
    m = I.make_mesh(12, 10, 6, I.depth_sines(1e-2), z_jitter=0.3, seed=3)
    h, om, A = _pair(m, bc, V.VEMG_PRECOND_NONE, O.PC_NONE)
    b = I.normal_loads(m.n, 42)
    x, info = V.vemg_solve(h, torch.from_numpy(b).cuda(), rtol=1e-8, max_it=4000)
    ro = om.solve(b, tol=1e-8, maxit=4000)
    assert info["status"] == "OK" and ro["status"] == "OK"
    # plain CG at Cond(A) ~ 1e6 takes ~2,000 iterations; rounding shifts the count by a few percent
    assert abs(info["iters"] - ro["iters"]) <= 0.05 * ro["iters"]
    xo = ro["x"]
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)
    a, bt = V.vemg_solve_coefficients(h)
    lo, hi = V.vemg_lanczos_extremes(a, bt)
    lo_o, hi_o = V.vemg_lanczos_extremes(ro["alpha"], ro["beta"])
    assert abs(lo - lo_o) <= 1e-3 * lo_o and abs(hi - hi_o) <= 1e-6 * hi_o


def test_condition_numbers_follow_section4():
    kA, kM = [], []
    for eps in (1e-2, 1e-3):
        m = I.make_mesh(16, 16, 8, I.depth_sines(eps), z_jitter=0.3, seed=4)
        b = torch.from_numpy(I.normal_loads(m.n, 43)).cuda()
        for pc, out in ((V.VEMG_PRECOND_NONE, kA), (V.VEMG_PRECOND_ADDITIVE, kM)):
            h, _, A = _pair(m, pc=pc, opc=O.PC_ADDITIVE)
            x, info = V.vemg_solve(h, b, rtol=1e-8, max_it=4096)
            # plain CG at Cond(A) ~ 1e7 does not reach 1e-8 in 4,096 iterations, but after more
            # iterations than the mesh has unknowns its extreme Ritz values have converged
            assert info["status"] == "OK" or pc == V.VEMG_PRECOND_NONE
            lo, hi = V.vemg_lanczos_extremes(*V.vemg_solve_coefficients(h))
            out.append(hi / lo)
    assert kA[1] > 30 * kA[0], kA
    assert max(kM) <= 1.5 * min(kM), kM


def test_spectrum_requests_outside_the_method_are_rejected():
    m = I.make_mesh(10, 10, 4, I.depth_sines(1e-2), z_jitter=0.3, seed=2)
    vm = V.Mesh.from_inputs(m)
    A = V.vemg_assemble(vm)
    h32 = V.vemg_setup(A, vm, V.vemg_default_options(precision=V.VEMG_PREC_FP32))
    V.vemg_solve(h32, torch.from_numpy(I.normal_loads(m.n, 1)).cuda(), rtol=1e-8)
    with pytest.raises(V.VemgError):   # flexible CG: no Lanczos recurrence
        V.vemg_solve_coefficients(h32)
    hn = V.vemg_setup(A, vm, V.vemg_default_options(precond=V.VEMG_PRECOND_NONE))
    B = torch.from_numpy(np.stack([I.normal_loads(m.n, c) for c in range(2)])).cuda()
    with pytest.raises(V.VemgError):   # batched plain CG is not offered
        V.vemg_solve_batch(hn, B, rtol=1e-8)
