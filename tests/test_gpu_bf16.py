"""BF16 operator values (VEMG_PREC_BF16) on the GPU against the oracle.

The BF16 variant rounds the off-diagonal values of every level matrix and every value of P and
P^T to BF16 (from FP32, nearest even) and runs the cycle in FP32 inside the FP64 flexible-CG
outer loop. Its cycle must equal the oracle's cycle with the same rounded operators
(Problem.round_operators_bf16) up to FP32 arithmetic, and its solves must reach the FP64
tolerance: the rounding changes the preconditioner, not the system that is solved."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0912_1976_gb300 import inputs as I
from paper_0912_1976_gb300 import vemg as V

pytestmark = pytest.mark.gpu

PCS = {"additive": (V.VEMG_PRECOND_ADDITIVE, O.PC_ADDITIVE), "vl_sor": (V.VEMG_PRECOND_VL_SOR, O.PC_VL_SOR),
       "sa": (V.VEMG_PRECOND_SA, O.PC_SA)}

CASES = {
    "zjit24": lambda: I.make_mesh(24, 20, 12, I.depth_sines(1e-3), z_jitter=0.3, seed=7),
    # several thread blocks per kernel and a ragged tail, four multigrid levels
    "zjit64": lambda: I.make_mesh(64, 61, 32, I.depth_sines(1e-3), z_jitter=0.3, seed=9),
    "clust32": lambda: I.make_mesh(32, 30, 12, I.depth_sines(1e-3), z_jitter=0.3, seed=10, cluster=0.9),
}

_cache = {}


def _setup(name, pc="additive", precision=V.VEMG_PREC_BF16, bc=V.VEMG_NEUMANN, rounded=True):
    key = (name, pc, precision, bc, rounded)
    if key not in _cache:
        m = CASES[name]()
        om = O.Problem(m, bc=bc, precond=PCS[pc][1])
        if rounded:
            om.round_operators_bf16()
        vm = V.Mesh.from_inputs(m)
        A = V.vemg_assemble(vm)
        h = V.vemg_setup(A, vm, V.vemg_default_options(bc=bc, precision=precision, precond=PCS[pc][0]))
        _cache[key] = (m, om, vm, A, h)
    return _cache[key]


def _chains(pc):
    return (0, 1) if pc == "additive" else (2,)


@pytest.mark.parametrize("name,pc", [("zjit24", "additive"), ("zjit64", "additive"), ("clust32", "additive"),
                                     ("zjit24", "vl_sor"), ("zjit24", "sa")])
def test_cycle_equals_oracle_with_rounded_operators(name, pc):
    m, om, vm, A, h = _setup(name, pc)
    _, o64, _, _, _ = _setup(name, pc, V.VEMG_PREC_FP64, rounded=False)
    rng = np.random.default_rng(4)
    for c in _chains(pc):
        nn = V.vemg_get_size(h, "lev.n", c, 0)
        b = rng.standard_normal(nn)
        v = V.vemg_vcycle(h, c, torch.from_numpy(b).cuda()).cpu().numpy()
        vo = om.vcycle(c, b)
        v64 = o64.vcycle(c, b)
        # FP32 arithmetic on the same rounded operators: ~1e-6 relative (as the FP32 cycle)
        d_round = np.linalg.norm(v - vo) / np.linalg.norm(vo)
        # the rounding itself moves the cycle by a few times BF16's unit roundoff (2^-9)
        d_fp64 = np.linalg.norm(v - v64) / np.linalg.norm(v64)
        assert d_round <= 1e-4, (c, d_round)
        if V.vemg_get_size(h, "nlev", c) > 1:
            assert d_fp64 >= 10 * d_round and d_fp64 <= 5e-2, (c, d_fp64, d_round)
        else:
            # a chain that is one dense level: its inverse keeps its precision, nothing is rounded
            assert d_fp64 <= 1e-4, (c, d_fp64)
    r = rng.standard_normal(om.n)
    z = V.vemg_precond(h, torch.from_numpy(r).cuda()).cpu().numpy()
    zo = om.precond(r)
    assert np.linalg.norm(z - zo) <= 1e-4 * np.linalg.norm(zo)


@pytest.mark.parametrize("name", list(CASES))
def test_bf16_solve_reaches_fp64_tolerance(name):
    m, om, vm, A, h = _setup(name)
    _, _, _, _, h32 = _setup(name, precision=V.VEMG_PREC_FP32, rounded=False)
    b = I.normal_loads(om.n, 21)
    x, info = V.vemg_solve(h, torch.from_numpy(b).cuda(), rtol=1e-8, max_it=500)
    x32, i32 = V.vemg_solve(h32, torch.from_numpy(b).cuda(), rtol=1e-8, max_it=500)
    assert info["status"] == "OK"
    assert info["true_relres"] <= 2e-8
    # a preconditioner perturbed by ~1e-2 costs at most a few iterations of flexible CG
    assert info["iters"] <= i32["iters"] + 3, (info["iters"], i32["iters"])
    ro = om.solve(b, tol=1e-8, maxit=500, flexible=True)   # the rounded-operator cycle in the oracle
    assert abs(info["iters"] - ro["iters"]) <= 1
    o64 = O.Problem(CASES[name]())
    rx = o64.solve(b, tol=1e-12, maxit=1000)
    err = np.linalg.norm(x.cpu().numpy() - rx["x"]) / np.linalg.norm(rx["x"])
    err32 = np.linalg.norm(x32.cpu().numpy() - rx["x"]) / np.linalg.norm(rx["x"])
    assert err <= max(10 * err32, 1e-7), (err, err32)


def test_bf16_dirichlet_top_and_persistent_request():
    m, om, vm, A, h = _setup("zjit24", bc=V.VEMG_DIRICHLET_TOP)
    b = I.normal_loads(m.n, 23)
    x, info = V.vemg_solve(h, torch.from_numpy(b).cuda(), rtol=1e-9, max_it=500)
    ro = om.solve(b, tol=1e-9, maxit=500, flexible=True)
    assert info["status"] == ro["status"] == "OK"
    assert abs(info["iters"] - ro["iters"]) <= 1
    assert info["true_relres"] <= 2e-9
    # a persistent cycle is not offered for BF16 values: the request runs the per-phase cycle
    hp = V.vemg_setup(A, vm, V.vemg_default_options(bc=V.VEMG_DIRICHLET_TOP, precision=V.VEMG_PREC_BF16,
                                                    cycle=V.VEMG_CYCLE_PERSISTENT))
    xp, ip = V.vemg_solve(hp, torch.from_numpy(b).cuda(), rtol=1e-9, max_it=500)
    assert ip["iters"] == info["iters"] and torch.equal(xp, x)


def test_bf16_batched_columns_use_the_same_rounded_operator():
    m, om, vm, A, h = _setup("zjit24")
    B = torch.from_numpy(np.stack([I.normal_loads(m.n, 500 + c) for c in range(3)])).cuda()
    X, infos = V.vemg_solve_batch(h, B, rtol=1e-9, max_it=500)
    for c in range(3):
        ro = om.solve(B[c].cpu().numpy(), tol=1e-9, maxit=500, flexible=True)
        assert infos[c]["status"] == "OK" and abs(infos[c]["iters"] - ro["iters"]) <= 1
        assert np.linalg.norm(X[c].cpu().numpy() - ro["x"]) <= 1e-7 * np.linalg.norm(ro["x"])
