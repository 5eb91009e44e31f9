"""Batched solves (vemg_solve_batch): K right-hand sides in one interleaved solve, each column
with its own Krylov scalars and convergence test. Each column must give what a single solve of
that right-hand side gives (within the FP64 reordering tolerance) and what the oracle gives."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_0912_1976_gb300 import inputs as I
from paper_0912_1976_gb300 import vemg as V

pytestmark = pytest.mark.gpu

_cache = {}


def _setup(bc=V.VEMG_NEUMANN, precision=V.VEMG_PREC_FP64):
    key = (bc, precision)
    if key not in _cache:
        m = I.make_mesh(32, 28, 16, I.depth_sines(1e-3), z_jitter=0.3, seed=41)
        vm = V.Mesh.from_inputs(m)
        A = V.vemg_assemble(vm)
        h = V.vemg_setup(A, vm, V.vemg_default_options(bc=bc, precision=precision))
        _cache[key] = (m, vm, A, h)
    return _cache[key]


def _rhs(n, k, seed):
    return torch.from_numpy(np.stack([I.normal_loads(n, seed + c) for c in range(k)])).cuda()


@pytest.mark.parametrize("k", [1, 3, 8, 33])
@pytest.mark.parametrize("precision", [V.VEMG_PREC_FP64, V.VEMG_PREC_FP32])
def test_batch_columns_equal_single_solves(k, precision):
    m, vm, A, h = _setup(precision=precision)
    B = _rhs(m.n, k, 100)
    X, infos = V.vemg_solve_batch(h, B, rtol=1e-9, max_it=300)
    for c in range(k):
        x1, i1 = V.vemg_solve(h, B[c].contiguous(), rtol=1e-9, max_it=300)
        assert infos[c]["status"] == "OK"
        assert abs(infos[c]["iters"] - i1["iters"]) <= 1
        if infos[c]["iters"] == i1["iters"]:
            err = (X[c] - x1).norm().item() / x1.norm().item()
        else:
            # the stopping test fell on different sides of rtol: compare after the same k steps
            kk = min(infos[c]["iters"], i1["iters"])
            Xk, _ = V.vemg_solve_batch(h, B[c:c + 1].contiguous(), rtol=0.0, max_it=kk)
            xk, _ = V.vemg_solve(h, B[c].contiguous(), rtol=0.0, max_it=kk)
            err = (Xk[0] - xk).norm().item() / xk.norm().item()
        assert err <= (1e-9 if precision == V.VEMG_PREC_FP64 else 1e-6), (c, err)
        assert infos[c]["true_relres"] <= 2e-9


def test_batch_matches_oracle_and_handles_zero_columns():
    m, vm, A, h = _setup()
    k = 5
    B = _rhs(m.n, k, 200)
    B[2].zero_()                                   # a zero right-hand side: x = 0, no iterations
    X, infos = V.vemg_solve_batch(h, B, rtol=1e-10, max_it=300)
    om = O.Problem(m)
    for c in range(k):
        if c == 2:
            assert infos[c]["iters"] == 0 and infos[c]["status"] == "OK"
            assert torch.all(X[c] == 0)
            continue
        ro = om.solve(B[c].cpu().numpy(), tol=1e-10)
        assert abs(infos[c]["iters"] - ro["iters"]) <= 1
        err = np.linalg.norm(X[c].cpu().numpy() - ro["x"]) / np.linalg.norm(ro["x"])
        assert err <= 1e-9, (c, err)


def test_batch_dirichlet_top():
    m, vm, A, h = _setup(bc=V.VEMG_DIRICHLET_TOP)
    B = _rhs(m.n, 4, 300)
    X, infos = V.vemg_solve_batch(h, B, rtol=1e-9, max_it=300)
    tops = torch.from_numpy((m.tags & I.TAG_TOP) != 0).cuda()
    for c in range(4):
        x1, i1 = V.vemg_solve(h, B[c].contiguous(), rtol=1e-9, max_it=300)
        assert infos[c]["status"] == "OK" and abs(infos[c]["iters"] - i1["iters"]) <= 1
        assert torch.all(X[c][tops] == 0)
        assert (X[c] - x1).norm().item() <= 1e-8 * x1.norm().item()


def test_autotuner_picks_a_launch_shape_per_kernel_class():
    m, vm, A, h = _setup()
    B = _rhs(m.n, 5, 400)                     # batch width 8
    V.vemg_solve_batch(h, B, rtol=1e-8, max_it=300)
    t = V.vemg_batch_tuning(h)
    assert t["K"] == 8
    for cls in V.BATCH_CLASSES:
        assert t[cls]["lanes_per_row"] in (4, 8) and t[cls]["warps_per_block"] in (2, 4, 8)
        assert t[cls]["us_per_launch"] > 0.0


def test_batched_results_do_not_depend_on_launch_shapes():
    """The shapes change which lanes and blocks do the work, not the arithmetic of a column: the
    same iterations and the same bits for every imposed shape."""
    m, vm, A, h = _setup(precision=V.VEMG_PREC_FP32)
    B = _rhs(m.n, 6, 500)
    out = []
    for kw, wp in ((4, 2), (8, 8), (4, 4)):
        V.vemg_batch_set_tuning(h, 8, [kw] * 3, [wp] * 3)
        X, infos = V.vemg_solve_batch(h, B, rtol=1e-9, max_it=300)
        assert V.vemg_batch_tuning(h)["sweep"]["lanes_per_row"] == kw
        out.append((X.clone(), [i["iters"] for i in infos]))
    for X, it in out[1:]:
        assert it == out[0][1]
        assert torch.equal(X, out[0][0])


def test_batched_columns_match_the_oracle_above_a_million_nodes():
    """The batched solve at scale (160x160x40, 1,062,761 nodes, four right-hand sides, FP32 cycles
    in FP64 flexible CG as in the 64-right-hand-side configuration) against the oracle's FP64 PCG
    of each column (its OpenMP build: the same bits as the plain one)."""
    from conftest import record
    m = I.make_mesh(160, 160, 40, I.depth_sines(1e-3), z_jitter=0.3, seed=43)
    vm = V.Mesh.from_inputs(m)
    A = V.vemg_assemble(vm)
    h = V.vemg_setup(A, vm, V.vemg_default_options(precision=V.VEMG_PREC_FP32))
    B = _rhs(m.n, 4, 600)
    X, infos = V.vemg_solve_batch(h, B, rtol=1e-8, max_it=300)
    om = O.Problem(m, openmp=True)
    worst = 0.0
    for c in range(4):
        ro = om.solve(B[c].cpu().numpy(), tol=1e-8)
        assert infos[c]["status"] == "OK" and ro["status"] == "OK"
        assert abs(infos[c]["iters"] - ro["iters"]) <= 2
        err = np.linalg.norm(X[c].cpu().numpy() - ro["x"]) / np.linalg.norm(ro["x"])
        worst = max(worst, err)
        assert err <= 1e-8, (c, err)
        assert infos[c]["true_relres"] <= 2e-8
    record("batched_vs_oracle_1M", n=m.n, worst_rel_l2=worst, iters=[i["iters"] for i in infos])
    h.destroy()


@pytest.mark.parametrize("precision", [V.VEMG_PREC_FP64, V.VEMG_PREC_FP32])
def test_wide_batch_results_do_not_depend_on_columns_per_pass(precision):
    """Width 64: 4 or 8 lanes per row take several columns per pass (8 with FP32 accumulators, 4
    with FP64 ones), 16 or 32 lanes one column per pass. Each column's products are added in the
    same order either way: the same iterations and the same bits."""
    m, vm, A, h = _setup(precision=precision)
    B = _rhs(m.n, 40, 700)                    # batch width 64
    out = []
    for kw, wp in ((4, 4), (8, 2), (16, 8), (32, 4)):
        V.vemg_batch_set_tuning(h, 64, [kw] * 3, [wp] * 3)
        X, infos = V.vemg_solve_batch(h, B, rtol=1e-9, max_it=300)
        assert all(i["status"] == "OK" for i in infos)
        out.append((X.clone(), [i["iters"] for i in infos]))
    for X, it in out[1:]:
        assert it == out[0][1]
        assert torch.equal(X, out[0][0])
