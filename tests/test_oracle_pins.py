"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form, an invariant, a
textbook special case or a brute-force computation written independently with numpy/scipy.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import oracle as O
from paper_0912_1976_gb300 import inputs as I

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _mesh(nx, nz, h0=0.01, zj=0.0, xyj=0.0, seed=3, flat=False):
    d = I.depth_flat(h0) if flat else I.depth_sines(h0)
    return I.make_mesh(nx, nx, nz, d, z_jitter=zj, xy_jitter=xyj, seed=seed)


def _read_golden(name):
    vals = {}
    for line in open(f"{GOLDEN}/{name}"):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = v.strip()
    return vals


# --------------------------------------------------------------------------------------------
# paper parameters (section 6)

def test_paper_parameters_golden():
    g = _read_golden("paper_parameters.txt")
    assert O.THETA == float(g["strength_threshold"])
    assert abs(O.OMEGA_P - eval(g["prolongator_omega"])) == 0.0


# --------------------------------------------------------------------------------------------
# element matrices and assembly (section 3)

def test_reference_tet_stiffness_closed_form():
    # textbook P1 stiffness of the reference tetrahedron (0,0,0),(1,0,0),(0,1,0),(0,0,1)
    det, K = O.elem_stiffness(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]]))
    ref = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    assert det == 1.0
    assert np.allclose(K, ref, rtol=0, atol=1e-15)


def test_stretched_tet_stiffness_scaling():
    # scaling z by s multiplies the z-derivative part by 1/s and the x,y part by s (section 3 A_eps)
    p = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    s = 1e-3
    q = p * np.array([1, 1, s])
    _, K = O.elem_stiffness(q)
    # gradients of the reference tet: l0 = 1-x-y-z, l1 = x, l2 = y, l3 = z (z-gradient scaled 1/s)
    G = np.array([[-1, -1, -1 / s], [1, 0, 0], [0, 1, 0], [0, 0, 1 / s]])
    ref = (s / 6.0) * G @ G.T
    assert np.allclose(K, ref, rtol=1e-13, atol=0)


def test_assembly_symmetry_nullspace_and_pattern():
    m = _mesh(6, 4, zj=0.3)
    P = O.Problem(m)
    A = P.csr("A")
    D = (A - A.T)
    assert D.count_nonzero() == 0 or abs(D).max() == 0.0           # bitwise symmetric
    assert abs(A @ np.ones(A.shape[0])).max() <= 1e-13 * abs(A).max()  # constants in the kernel
    # Freudenthal/Kuhn triangulation: an interior vertex has 14 neighbours (15 entries per row)
    n2o = P.ints("new2old")
    nz = m.nz
    k = n2o % (nz + 1)
    col = n2o // (nz + 1)
    i, j = col % (m.nx + 1), col // (m.nx + 1)
    inner = (k > 0) & (k < nz) & (i > 0) & (i < m.nx) & (j > 0) & (j < m.ny)
    rl = np.diff(A.indptr)
    assert np.all(rl[inner] == 15)


def test_neumann_spectrum_simple_zero_and_abar_spd():
    m = _mesh(6, 3, zj=0.3)
    P = O.Problem(m)
    A = P.csr("A").toarray()
    w = np.linalg.eigvalsh(A)
    assert abs(w[0]) < 1e-12 * w[-1]           # one zero eigenvalue (constants)
    assert w[1] > 1e-8 * w[-1]                 # and only one
    Abar = A[P.mtop:, P.mtop:]
    np.linalg.cholesky(Abar)                   # SPD (raises otherwise)


def test_mass_integrates_polynomials():
    # sum_i (M f)_i = integral of f for f in P1; flat box of depth h0: int 1 = h0, int z = -h0^2/2
    h0 = 0.05
    m = _mesh(5, 3, h0=h0, zj=0.3, flat=True)
    P = O.Problem(m)
    one = P.load(np.ones(m.n))
    assert abs(one.sum() - h0) < 1e-15
    z = P.load(m.xyz[:, 2])
    assert abs(z.sum() - (-h0 * h0 / 2)) < 1e-15
    x = P.load(m.xyz[:, 0])
    assert abs(x.sum() - h0 * 0.5) < 1e-15


def test_manufactured_solution_second_order():
    """O(h^2) convergence of the P1 solution of -Laplace u = f, all-Neumann, on the flat thin box
    (section 3), with u = cos(pi x) cos(pi y) cos(pi z / H)."""
    h0 = 0.01
    errs = []
    for nx, nz in [(8, 4), (16, 8), (32, 16)]:
        m = _mesh(nx, nz, h0=h0, flat=True)
        P = O.Problem(m)
        b = P.load(I.manufactured_f(m, h0))
        r = P.solve(b, tol=1e-12)
        assert r["status"] == "OK"
        u = I.manufactured_u(m, h0)
        e = r["x"] - u
        Me = P.load(e)
        e = e - Me.sum() / P.load(np.ones(m.n)).sum()        # fix the constant by the mass-weighted mean
        errs.append(math.sqrt(e @ P.load(e)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert 1.8 < rates[-1] < 2.2, (errs, rates)


# --------------------------------------------------------------------------------------------
# condition numbers (section 4)

def _cond_spd(M):
    w = np.linalg.eigvalsh(M)
    return w[-1] / w[0]


def test_condition_number_scaling_with_aspect_ratio():
    """Cond(A_eps) on the complement of constants grows like eps^-2, Cond(A_bar_eps) stays
    bounded by 2 Cond(A_bar_0) (section 4). The mesh is rescaled: same nodes, depth eps."""
    conds, condbar = [], []
    eps_list = [1e-1, 1e-2, 1e-3]
    for eps in eps_list:
        m = _mesh(6, 4, h0=eps, zj=0.3, flat=True, seed=11)
        P = O.Problem(m)
        A = P.csr("A").toarray() * eps   # rescaled operator A_eps = (H / L^2) A_phys
        w = np.linalg.eigvalsh(A)
        conds.append(w[-1] / w[1])
        condbar.append(_cond_spd(A[P.mtop:, P.mtop:]))
    r1 = conds[1] / conds[0]
    r2 = conds[2] / conds[1]
    assert 50 < r1 < 150 and 80 < r2 < 120        # x100 per decade of eps
    # A_0: the vertical part only; eps -> 0 limit of the rescaled matrix
    assert max(condbar) / min(condbar) < 2.0


# --------------------------------------------------------------------------------------------
# vertical extrapolation E~ (section 5.4) and the Galerkin surface operator

def _brute_force_locate(tris, xyz, pts):
    """argmax over ALL triangles of the smallest barycentric coordinate, ties to the lowest index"""
    a, b, c = xyz[tris[:, 0], :2], xyz[tris[:, 1], :2], xyz[tris[:, 2], :2]

    def orient(p, q, r):
        return (q[..., 0] - p[..., 0]) * (r[..., 1] - p[..., 1]) - (q[..., 1] - p[..., 1]) * (r[..., 0] - p[..., 0])

    out = np.zeros(len(pts), np.int64)
    W = np.zeros((len(pts), 3))
    for k, p in enumerate(pts):
        P = np.broadcast_to(p, a.shape)
        area = orient(a, b, c)
        la = orient(P, b, c) / area
        lb = orient(a, P, c) / area
        lc = (1.0 - la) - lb
        mn = np.minimum(np.minimum(la, lb), lc)
        t = int(np.flatnonzero(mn == mn.max())[0])
        out[k] = t
        W[k] = (la[t], lb[t], lc[t])
    return out, W


def test_location_equals_brute_force_on_jittered_surface():
    m = _mesh(7, 3, zj=0.3, xyj=0.2, seed=21)
    pts = m.xyz[:, :2]
    tri, w = O.locate_points(m.top_tris, m.xyz, pts)
    tb, wb = _brute_force_locate(m.top_tris, m.xyz, pts)
    assert np.array_equal(tri, tb)
    assert np.array_equal(w, wb)


def test_extrapolation_extruded_is_column_injection():
    m = _mesh(6, 5, zj=0.3)
    P = O.Problem(m)
    E = P.csr("E")
    assert np.all(np.diff(E.indptr) == 1) and np.all(E.data == 1.0)
    n2o = P.ints("new2old")
    col_of_node = n2o // (m.nz + 1)                        # generator column of each internal node
    top_col = col_of_node[:P.mtop]
    assert np.array_equal(top_col[E.indices], col_of_node)   # same column as its top node
    # E~^T r = column sums, exactly
    r = np.random.default_rng(0).standard_normal(P.n)
    cs = np.zeros(P.mtop)
    order = np.argsort(top_col)
    sums = np.zeros(top_col.max() + 1)
    np.add.at(sums, col_of_node, r)
    assert np.allclose(E.T @ r, sums[top_col], rtol=1e-14, atol=1e-14)


def test_extrapolation_rows_are_barycentric():
    m = _mesh(6, 4, zj=0.3, xyj=0.2, seed=5)
    P = O.Problem(m)
    E = P.csr("E")
    rs = np.asarray(E.sum(axis=1)).ravel()
    assert np.all(np.abs(rs - 1.0) <= 4e-16)
    # reproduces linear functions of (x, y): E~ x_top = x at every node
    n2o = P.ints("new2old")
    xy = m.xyz[n2o, :2]
    for c in range(2):
        assert np.allclose(E @ xy[:P.mtop, c], xy[:, c], rtol=0, atol=1e-14)


def _depth_weighted_2d_stiffness(m, mtop, old2new_top, depth_at):
    """A_c closed form on extruded meshes: sum_T area_T Hbar_T grad(l_i).grad(l_j)."""
    K = np.zeros((mtop, mtop))
    for t in m.top_tris:
        p = m.xyz[t, :2]
        area2 = (p[1, 0] - p[0, 0]) * (p[2, 1] - p[0, 1]) - (p[1, 1] - p[0, 1]) * (p[2, 0] - p[0, 0])
        G = np.array([[p[1, 1] - p[2, 1], p[2, 0] - p[1, 0]],
                      [p[2, 1] - p[0, 1], p[0, 0] - p[2, 0]],
                      [p[0, 1] - p[1, 1], p[1, 0] - p[0, 0]]]) / area2
        hbar = depth_at[t].mean()
        idx = old2new_top[t]
        K[np.ix_(idx, idx)] += 0.5 * area2 * hbar * (G @ G.T)
    return K


@pytest.mark.parametrize("zj", [0.0, 0.3])
def test_galerkin_surface_operator_closed_form(zj):
    h0 = 0.01
    m = _mesh(8, 6, h0=h0, zj=zj)
    P = O.Problem(m)
    n2o = P.ints("new2old")
    o2n = np.empty_like(n2o)
    o2n[n2o] = np.arange(P.n)
    x, y = m.xyz[:, 0], m.xyz[:, 1]
    H = I.depth_sines(h0)(x, y)
    K = _depth_weighted_2d_stiffness(m, P.mtop, o2n, H)
    Ac = P.csr("Ac").toarray()
    assert np.abs(Ac - K).max() <= 1e-10 * np.abs(K).max()
    assert np.array_equal(Ac, Ac.T)                       # exact symmetry
    assert np.abs(Ac @ np.ones(P.mtop)).max() <= 1e-10 * np.abs(K).max()


# --------------------------------------------------------------------------------------------
# the exact identity of section 5.3 (Eq. E multigrid)

def test_exact_inverse_identity():
    m = _mesh(5, 3, h0=0.01, zj=0.3, xyj=0.2, seed=2)
    P = O.Problem(m)
    A = P.csr("A").toarray()
    mt = P.mtop
    Abar = A[mt:, mt:]
    Ct = A[mt:, :mt]
    E = np.vstack([np.eye(mt), -np.linalg.solve(Abar, Ct)])
    S = E.T @ A @ E

    def pinv_on_complement(M):
        # inverse on the complement of constants: (M + s 1 1^T)^-1 projected, s > 0
        k = M.shape[0]
        Qk = np.eye(k) - np.ones((k, k)) / k
        return Qk @ np.linalg.inv(M + np.trace(M) / k ** 2) @ Qk

    Z = np.zeros((P.n, P.n - mt))
    Z[mt:] = np.eye(P.n - mt)
    Minv = E @ pinv_on_complement(S) @ E.T + Z @ np.linalg.solve(Abar, Z.T)
    Apinv = pinv_on_complement(A)
    Q = np.eye(P.n) - np.ones((P.n, P.n)) / P.n          # restrict to the complement of constants
    assert np.abs(Q @ Minv @ Q - Apinv).max() <= 1e-8 * np.abs(Apinv).max()


# --------------------------------------------------------------------------------------------
# smoothed aggregation (section 5.1, section 6)

def _lap1d(n):
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()


def test_aggregates_on_a_path_are_connected_triples_or_pairs():
    n = 30
    nagg, agg = O.sa_aggregate(_lap1d(n))
    assert sorted(set(agg.tolist())) == list(range(nagg))
    sizes = np.bincount(agg)
    assert sizes.min() >= 1 and sizes.max() <= 5
    for a in range(nagg):
        idx = np.flatnonzero(agg == a)
        assert idx.max() - idx.min() == len(idx) - 1       # contiguous on the path


def test_weak_couplings_never_aggregate():
    # two decoupled 1D chains joined by couplings below the 0.01 threshold
    n = 12
    A = sp.block_diag([_lap1d(n), _lap1d(n)]).tolil()
    for i in range(n):
        A[i, n + i] = A[n + i, i] = -0.005 * 2
    A = A.tocsr()
    nagg, agg = O.sa_aggregate(A)
    assert set(agg[:n]).isdisjoint(set(agg[n:]))


def test_isolated_nodes_unaggregated_unless_kept():
    """A node with no strong coupling gets no coarse unknown on non-singular chains (Vanek, Mandel
    and Brezina): it stays unaggregated, its prolongator row is zero. Singular chains keep it as
    a singleton so that P 1 = 1."""
    n = 10
    L = _lap1d(n).tolil()
    A = sp.block_diag([L, sp.diags([4.0, 5.0])]).tolil()
    A[0, n] = A[n, 0] = -0.001          # weak: below 0.01 sqrt(A_ii A_jj)
    A = A.tocsr()
    nagg, agg = O.sa_aggregate(A, keep_isolated=False)
    assert agg[n] == -1 and agg[n + 1] == -1 and np.all(agg[:n] >= 0)
    assert sorted(set(agg[:n].tolist())) == list(range(nagg))
    nagg1, agg1 = O.sa_aggregate(A, keep_isolated=True)
    assert nagg1 == nagg + 2 and agg1[n] != agg1[n + 1]
    assert np.sum(agg1[:n] == agg1[n]) == 0 and np.sum(agg1[:n] == agg1[n + 1]) == 0    # singletons
    same = agg[:n, None] == agg[None, :n]
    assert np.array_equal(same, agg1[:n, None] == agg1[None, :n])                       # same partition


def test_chain_drops_isolated_rows_on_a_bar_only():
    """eps = 1e-4 makes the collapsed columns of the coarse A_bar levels nearly diagonal (their
    vertical coupling to the Dirichlet top dominates), so some of their nodes have no strong
    coupling: those rows of P are empty on the A_bar chain; the singular surface chain keeps
    every node."""
    m = _mesh(48, 16, h0=1e-4, zj=0.3, seed=3)
    P = O.Problem(m)
    dropped = 0
    for l in range(P.nlev(1) - 1):
        agg = P.ints("lev.agg", 1, l)
        Pm = P.csr("lev.P", 1, l)
        rows = np.diff(Pm.indptr)
        assert np.all(rows[agg < 0] == 0) and np.all(rows[agg >= 0] > 0)
        dropped += int((agg < 0).sum())
    assert dropped > 0
    for l in range(P.nlev(0) - 1):
        assert np.all(P.ints("lev.agg", 0, l) >= 0)


def _path_with_weak_link(n, end_diag, weak=1e-3, link=(4, 7)):
    """1D Laplacian [-1, 2, -1] on a path of n nodes with end diagonals end_diag (1: Neumann ends,
    A 1 = 0; 2: Dirichlet ends, non-singular like A_bar), plus one weak symmetric coupling -weak
    between the nodes of `link`, its value lumped into their diagonals (row sums unchanged)."""
    A = _lap1d(n).tolil()
    A[0, 0] = A[n - 1, n - 1] = end_diag
    i, j = link
    A[i, j] = A[j, i] = -weak
    A[i, i] += weak
    A[j, j] += weak
    return A.tocsr()


@pytest.mark.parametrize("end_diag", [1.0, 2.0])
def test_smoothed_prolongator_closed_form_on_a_path(end_diag):
    """P = (I - omega (D^F)^-1 A^F) P_tent with omega = 2/3 (section 6) on a path with aggregates
    {0,1,2}, {3,4,5}, {6,7,8}, by hand:
      - a node inside its aggregate keeps the single entry 1 (its A row sums to 0 inside it);
      - a node at an aggregate boundary of [-1, 2, -1]: (D^-1 A P_tent) = (1/2, -1/2), so
        P = (1 - 2/3 * 1/2, 2/3 * 1/2) = (2/3, 1/3) on (own, neighbour) aggregate;
      - nodes 4 and 7 carry a weak coupling (-1e-3, below 0.01 sqrt(A_ii A_jj)): the filtered
        matrix drops it and lumps it into the diagonal (A^F_ii = A_ii - 1e-3 = 2), so their rows
        are exactly those of the plain path: 1 on their own aggregate and no entry on the other;
      - a Dirichlet end (diagonal 2, one neighbour): (D^-1 A P_tent) = 1/2 on its aggregate, so
        P = 1 - 1/3 = 2/3 (the row does not sum to 1: P 1 = 1 holds only where A 1 = 0).
    A wrong omega, a missing D^-1, the unfiltered matrix or the lumped value with the wrong sign
    each changes one of these entries."""
    A = _path_with_weak_link(9, end_diag)
    agg = np.repeat(np.arange(3), 3)
    P = O.smoothed_prolongator(A, agg, 3).toarray()
    t = 2.0 / 3.0
    e = 1.0 - t * (end_diag - 1.0) / end_diag          # 1 at a Neumann end, 2/3 at a Dirichlet end
    ref = np.array([[e, 0, 0], [1, 0, 0], [t, 1 - t, 0],
                    [1 - t, t, 0], [0, 1, 0], [0, t, 1 - t],
                    [0, 1 - t, t], [0, 0, 1], [0, 0, e]])
    assert np.abs(P - ref).max() <= 1e-15
    # the weak link leaves no stored entry on the other aggregate
    Ps = O.smoothed_prolongator(A, agg, 3)
    assert list(Ps[4].indices) == [1] and list(Ps[7].indices) == [2]


def test_smoothed_prolongator_unaggregated_and_isolated_rows():
    """An unaggregated row (agg = -1) is empty; an aggregated row with no strong coupling keeps its
    tentative row (nothing to smooth against); omega enters linearly."""
    n = 6
    A = sp.block_diag([_lap1d(n), sp.diags([4.0, 5.0])]).tolil()
    A[0, n] = A[n, 0] = -0.001
    A[0, 0] += 0.001
    A[n, n] += 0.001
    A = A.tocsr()
    agg = np.array([0, 0, 0, 1, 1, 1, 2, -1])
    P = O.smoothed_prolongator(A, agg, 3)
    assert P[7].nnz == 0
    assert list(P[6].indices) == [2] and P[6].data[0] == 1.0
    # omega = 1/3 at the boundary node 2: (1 - 1/6, 1/6)
    Pw = O.smoothed_prolongator(A, agg, 3, omega=1.0 / 3.0).toarray()
    assert np.abs(Pw[2, :2] - [5.0 / 6.0, 1.0 / 6.0]).max() <= 1e-15
    # the Dirichlet-like end 0 (diagonal 2.001 filtered back to 2, one neighbour in its aggregate)
    P2 = P.toarray()
    assert abs(P2[0, 0] - (1.0 - (2.0 / 3.0) * 0.5)) <= 1e-15


def test_chain_prolongators_are_the_smoothed_prolongator_with_omega_two_thirds():
    """Every level's P in the setup chains is the smoothed prolongator (pinned above) of that
    level's operator and aggregates with the paper's omega = 2/3 and strength 0.01: the chains
    pass the section-6 parameters through."""
    m = _mesh(10, 6, h0=1e-3, zj=0.3)
    P = O.Problem(m)
    for which in (0, 1):
        for l in range(P.nlev(which) - 1):
            A = P.csr("lev.A", which, l)
            agg = P.ints("lev.agg", which, l)
            nagg = P.size("lev.n", which, l + 1)
            ref = O.smoothed_prolongator(A, agg, nagg, omega=2.0 / 3.0, theta=0.01)
            got = P.csr("lev.P", which, l)
            assert np.array_equal(got.indptr, ref.indptr) and np.array_equal(got.indices, ref.indices)
            assert np.array_equal(got.data, ref.data)


def test_colouring_is_proper():
    m = _mesh(6, 4, zj=0.3)
    P = O.Problem(m)
    for which in (0, 1):
        for l in range(P.nlev(which)):
            A = P.csr("lev.A", which, l)
            col = P.ints("lev.colour", which, l)
            r, c = A.nonzero()
            off = r != c
            assert np.all(col[r[off]] != col[c[off]])
            assert col.max() + 1 == P.size("lev.ncolours", which, l)


def _graph(n, edges):
    r = [a for a, b in edges] + [b for a, b in edges] + list(range(n))
    c = [b for a, b in edges] + [a for a, b in edges] + list(range(n))
    return sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(n, n))


def test_smallest_last_ranks_by_brute_force():
    """Tiny random graphs: simulate the peeling round by round with Python sets (threshold k =
    max(previous k, smallest remaining degree); remove every remaining node of remaining degree
    <= k) and compare the ranks."""
    rng = np.random.default_rng(12)
    for trial in range(40):
        n = int(rng.integers(1, 30))
        p = rng.uniform(0.05, 0.5)
        edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
        A = _graph(n, edges)
        nb = {i: set() for i in range(n)}
        for a, b in edges:
            nb[a].add(b)
            nb[b].add(a)
        left, rank, t, k = set(range(n)), {}, 0, 0
        while left:
            d = {i: len(nb[i] & left) for i in left}
            k = max(k, min(d.values()))
            out = {i for i in left if d[i] <= k}
            for i in out:
                rank[i] = t
            left -= out
            t += 1
        assert O.sl_ranks(A).tolist() == [rank[i] for i in range(n)]


def test_colouring_of_paths_stars_cliques():
    # path: peeled from both ends, rank = distance to the nearer end; two colours
    n = 9
    A = _graph(n, [(i, i + 1) for i in range(n - 1)])
    assert O.sl_ranks(A).tolist() == [min(i, n - 1 - i) for i in range(n)]
    nc, col = O.colour(A)
    assert nc == 2 and col[n // 2] == 0
    # star: the leaves leave first, the centre is coloured first
    A = _graph(7, [(0, i) for i in range(1, 7)])
    assert O.sl_ranks(A).tolist() == [1] + [0] * 6
    nc, col = O.colour(A)
    assert nc == 2 and col[0] == 0 and set(col[1:].tolist()) == {1}
    # clique: one round, every node its own colour
    A = _graph(6, [(a, b) for a in range(6) for b in range(a + 1, 6)])
    assert O.sl_ranks(A).tolist() == [0] * 6
    nc, col = O.colour(A)
    assert nc == 6 and sorted(col.tolist()) == list(range(6))


def test_worklist_peeling_gives_the_same_rank_order():
    """The GPU peels on worklists: a round removes its worklist, a neighbour joins the next one
    when its degree falls from k + 1 to k, and an empty worklist raises k to the smallest remaining
    degree (its round index then goes unused). Simulated here, the rank order must equal the
    oracle's round-synchronous ranks."""
    rng = np.random.default_rng(22)
    for trial in range(30):
        n = int(rng.integers(1, 50))
        edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < rng.uniform(0.05, 0.5)]
        A = _graph(n, edges)
        nb = [set() for _ in range(n)]
        for a, b in edges:
            nb[a].add(b)
            nb[b].add(a)
        deg = [len(nb[i]) for i in range(n)]
        rank = [-1] * n
        k, t, wl, removed = 0, 0, [], 0
        while removed < n:
            if not wl:   # raise
                k = max(k, min(deg[i] for i in range(n) if rank[i] < 0))
                wl = [i for i in range(n) if rank[i] < 0 and deg[i] <= k]
                t += 1   # the empty round's index goes unused
            nxt = []
            for v in wl:
                rank[v] = t
            for v in wl:
                for j in nb[v]:
                    if rank[j] < 0:
                        deg[j] -= 1
                        if deg[j] == k:
                            nxt.append(j)
            removed += len(wl)
            wl, t = nxt, t + 1
        dense = np.unique(np.array(rank), return_inverse=True)[1]
        assert dense.tolist() == O.sl_ranks(A).tolist()


def test_jones_plassmann_rounds_equal_greedy_in_key_order():
    """The GPU colours by Jones-Plassmann rounds on fixed keys, the oracle greedily in decreasing
    key order: with distinct keys both give the same colouring (a node is coloured exactly when
    its larger-key neighbours are). Checked on random graphs with random distinct keys."""
    rng = np.random.default_rng(21)
    for trial in range(30):
        n = int(rng.integers(2, 60))
        edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < rng.uniform(0.05, 0.4)]
        nb = [set() for _ in range(n)]
        for a, b in edges:
            nb[a].add(b)
            nb[b].add(a)
        key = rng.permutation(n)

        def first_fit(i, col):
            used = {col[j] for j in nb[i] if col[j] >= 0}
            c = 0
            while c in used:
                c += 1
            return c

        greedy = [-1] * n
        for i in sorted(range(n), key=lambda i: -key[i]):
            greedy[i] = first_fit(i, greedy)
        jp = [-1] * n
        while min(jp) < 0:
            win = [i for i in range(n) if jp[i] < 0 and all(jp[j] >= 0 or key[j] < key[i] for j in nb[i])]
            new = {i: first_fit(i, jp) for i in win}
            for i, c in new.items():
                jp[i] = c
        assert jp == greedy


def test_colour_count_within_degeneracy_bound_and_clique_bound():
    """Smallest-last greedy uses at most degeneracy + 1 colours (degeneracy = the largest k with a
    non-empty k-core, from networkx); every tetrahedron is a 4-clique of the level-0 graph, so
    at least 4 colours are needed there."""
    nx = pytest.importorskip("networkx")
    m = _mesh(10, 6, zj=0.3)
    P = O.Problem(m)
    for which in (0, 1):
        for l in range(P.nlev(which) - 1):
            A = P.csr("lev.A", which, l).tocsr()
            G = nx.from_scipy_sparse_array(A)
            G.remove_edges_from(nx.selfloop_edges(G))
            degeneracy = max(nx.core_number(G).values())
            nc = P.size("lev.ncolours", which, l)
            assert nc <= degeneracy + 1, (which, l, nc, degeneracy)
    assert P.size("lev.ncolours", 1, 0) >= 4
    # the extruded Kuhn lattice is 4-colourable; smallest-last greedy needs at most twice that
    m = _mesh(8, 4, zj=0.0, flat=True)
    P = O.Problem(m)
    assert 4 <= P.size("lev.ncolours", 1, 0) <= 8


def test_hierarchy_invariants():
    m = _mesh(12, 8, h0=1e-3, zj=0.3)
    P = O.Problem(m)
    for which in (0, 1):
        for l in range(P.nlev(which) - 1):
            A = P.csr("lev.A", which, l)
            Pl = P.csr("lev.P", which, l)
            Ac = P.csr("lev.A", which, l + 1)
            agg = P.ints("lev.agg", which, l)
            assert sorted(set(agg.tolist())) == list(range(Ac.shape[0]))
            Acd = Ac.toarray()
            assert np.array_equal(Acd, Acd.T)
            ref = (Pl.T @ (A @ Pl)).toarray()
            assert np.abs(Acd - ref).max() <= 1e-12 * np.abs(ref).max()
            if which == 0:
                # singular chain: A 1 = 0 and the filtered smoothing keeps constants, P 1 = 1
                assert np.abs(Pl @ np.ones(Pl.shape[1]) - 1).max() <= 1e-9


# --------------------------------------------------------------------------------------------
# preconditioner and solver

def test_vcycle_and_preconditioner_symmetric_positive():
    m = _mesh(5, 3, h0=0.01, zj=0.3)
    P = O.Problem(m, coarse_max=40)
    n = P.n
    Mz = np.stack([P.precond(e) for e in np.eye(n)], axis=1)
    assert np.abs(Mz - Mz.T).max() <= 1e-10 * np.abs(Mz).max()
    w = np.linalg.eigvalsh(0.5 * (Mz + Mz.T))
    assert w[0] > -1e-10 * w[-1]
    assert P.nlev(1) >= 2          # a real multilevel cycle, not only the direct solve


def test_one_level_chain_cycle_is_the_exact_inverse():
    """A chain whose finest level has at most coarse_max rows is that level alone, solved by its
    dense inverse: the cycle of the non-singular A_bar chain solves A_bar exactly, and the cycle of
    the singular surface chain (constants as its nullspace) returns the zero-mean solution of a
    mean-zero right-hand side."""
    m = _mesh(8, 4, h0=1e-2, zj=0.3, seed=9)
    P = O.Problem(m)
    assert P.nlev(1) == 1 and P.nlev(0) == 1
    rng = np.random.default_rng(21)
    Ab = P.csr("lev.A", 1, 0).toarray()
    b = rng.standard_normal(Ab.shape[0])
    v = P.vcycle(1, b)
    assert np.linalg.norm(Ab @ v - b) <= 1e-12 * np.linalg.norm(b)
    Ac = P.csr("lev.A", 0, 0).toarray()
    bs = rng.standard_normal(Ac.shape[0])
    bs -= bs.mean()
    vs = P.vcycle(0, bs)
    assert abs(vs.mean()) <= 1e-12 * np.abs(vs).max()
    assert np.linalg.norm(Ac @ vs - bs) <= 1e-10 * np.linalg.norm(bs)


def test_coarsening_stops_at_the_first_level_within_coarse_max():
    """The default coarsest size (1024 rows): the A_bar chain of a 24x24x8 mesh coarsens while a
    level has more rows and ends at the first level within the limit, solved directly. With a
    512-row limit the same 625-row level is where coarsening stalls (none of its nodes has a strong
    coupling, so it has no aggregate): it stays the last level and is swept, not inverted."""
    m = _mesh(24, 8, h0=1e-3, zj=0.3, seed=9)
    P = O.Problem(m)
    sizes = P.level_sizes(1)
    assert sizes[-1] <= O.COARSE_MAX < sizes[-2] and P.size("direct", 1) == 1
    assert all(s > O.COARSE_MAX for s in sizes[:-1])
    Q = O.Problem(m, coarse_max=512)
    assert Q.level_sizes(1) == sizes and Q.size("direct", 1) == 0


def test_solve_matches_dense_bordered_system():
    for zj, xyj in [(0.3, 0.0), (0.3, 0.2)]:
        m = _mesh(8, 4, h0=1e-2, zj=zj, xyj=xyj, seed=9)
        P = O.Problem(m)
        b = I.normal_loads(P.n, 4)
        r = P.solve(b, tol=1e-11, maxit=2000)   # the xy-jittered mesh has a round-off floor near 2e-13
        assert r["status"] == "OK"
        n2o = P.ints("new2old")
        A = P.csr("A").toarray()
        bi = b[n2o] - b.mean()
        K = np.block([[A, np.ones((P.n, 1))], [np.ones((1, P.n)), np.zeros((1, 1))]])
        xs = np.linalg.solve(K, np.concatenate([bi, [0.0]]))[:P.n]
        x = r["x"][n2o]
        assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)


def test_dirichlet_top_solve_matches_dense():
    m = _mesh(8, 4, h0=1e-2, zj=0.3, seed=9)
    P = O.Problem(m, bc=O.BC_DIRICHLET_TOP)
    b = I.normal_loads(P.n, 5)
    r = P.solve(b, tol=1e-13, maxit=500)
    assert r["status"] == "OK"
    n2o = P.ints("new2old")
    A = P.csr("A").toarray()
    mt = P.mtop
    xs = np.linalg.solve(A[mt:, mt:], b[n2o][mt:])
    x = r["x"][n2o]
    assert np.all(x[:mt] == 0.0)
    assert np.linalg.norm(x[mt:] - xs) <= 1e-10 * np.linalg.norm(xs)


def test_flexible_cg_same_solution():
    m = _mesh(10, 6, h0=1e-3, zj=0.3)
    P = O.Problem(m)
    b = I.normal_loads(P.n, 1)
    a = P.solve(b, tol=1e-12)
    f = P.solve(b, tol=1e-12, flexible=True)
    assert abs(a["iters"] - f["iters"]) <= 2
    assert np.linalg.norm(a["x"] - f["x"]) <= 1e-9 * np.linalg.norm(a["x"])


def _jacobi_pcg_iters(A, b, tol, maxit=20000):
    d = A.diagonal()
    x = np.zeros_like(b)
    r = b.copy()
    z = r / d
    z -= z.mean()
    p = z.copy()
    rz = r @ z
    bn = np.linalg.norm(b)
    for k in range(maxit):
        q = A @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        if np.linalg.norm(r) <= tol * bn:
            return k + 1
        z = r / d
        z -= z.mean()
        rzn = r @ z
        p = z + (rzn / rz) * p
        rz = rzn
    return maxit


def test_iterations_independent_of_aspect_ratio():
    """Section 6.2: with vertical lumping the convergence rate no longer depends on eps, while a
    point preconditioner degrades as eps shrinks."""
    its, jac = [], []
    for eps in [1e-2, 1e-3, 1e-4]:
        m = _mesh(16, 8, h0=eps, zj=0.3, seed=4)
        P = O.Problem(m)
        b = I.normal_loads(P.n, 2)
        r = P.solve(b, tol=1e-8)
        assert r["status"] == "OK"
        its.append(r["iters"])
        bi = b[P.ints("new2old")]
        jac.append(_jacobi_pcg_iters(P.csr("A"), bi - bi.mean(), 1e-8))
    assert max(its) <= 1.25 * min(its), its
    assert jac[0] < jac[1] < jac[2] and jac[2] > 2 * jac[0], jac


# --------------------------------------------------------------------------------------------
# the two other preconditioners of section 6: vertical lumping as the first coarsening of a
# V-cycle on A with SOR smoothing (VL+SOR), and smoothed aggregation on A itself (SA)

@pytest.mark.parametrize("pc", [O.PC_VL_SOR, O.PC_SA])
def test_variant_cycles_symmetric_positive(pc):
    """Forward SOR before and backward SOR after the coarse correction, with P^T restriction, make
    the cycle a symmetric operator, positive semi-definite with the constants as kernel."""
    m = _mesh(5, 3, h0=0.01, zj=0.3)
    P = O.Problem(m, coarse_max=40, precond=pc)
    n = P.n
    Mz = np.stack([P.precond(e) for e in np.eye(n)], axis=1)
    assert np.abs(Mz - Mz.T).max() <= 1e-10 * np.abs(Mz).max()
    w = np.linalg.eigvalsh(0.5 * (Mz + Mz.T))
    assert w[0] > -1e-10 * w[-1]
    assert P.nlev(2) >= 2


def test_vl_chain_is_extrapolation_then_surface_sa():
    """VL+SOR: the finest level is A with E~ as its prolongator; the level below is the Galerkin
    product E~^T A E~ written out here with scipy, then the SA levels of that operator."""
    m = _mesh(10, 4, h0=1e-3, zj=0.3)
    P = O.Problem(m, precond=O.PC_VL_SOR)
    A, E = P.csr("A"), P.csr("E")
    assert np.array_equal(P.csr("lev.A", 2, 0).toarray(), A.toarray())
    assert np.array_equal(P.csr("lev.P", 2, 0).toarray(), E.toarray())
    Ac = P.csr("lev.A", 2, 1).toarray()
    ref = (E.T @ (A @ E)).toarray()
    assert np.abs(Ac - ref).max() <= 1e-12 * np.abs(ref).max()
    Padd = O.Problem(m)
    assert P.nlev(2) == Padd.nlev(0) + 1
    for l in range(Padd.nlev(0)):
        assert np.array_equal(P.csr("lev.A", 2, l + 1).toarray(), Padd.csr("lev.A", 0, l).toarray())
    # the finest-level colouring is a proper colouring of A's graph
    col = P.ints("lev.colour", 2, 0)
    Ac0 = A.tocoo()
    off = Ac0.row != Ac0.col
    assert not np.any(col[Ac0.row[off]] == col[Ac0.col[off]])


def test_sa_chain_galerkin_and_constants():
    m = _mesh(10, 4, h0=1e-2, zj=0.3)
    P = O.Problem(m, precond=O.PC_SA)
    assert np.array_equal(P.csr("lev.A", 2, 0).toarray(), P.csr("A").toarray())
    for l in range(P.nlev(2) - 1):
        A, Pl, Ac = P.csr("lev.A", 2, l), P.csr("lev.P", 2, l), P.csr("lev.A", 2, l + 1)
        ref = (Pl.T @ (A @ Pl)).toarray()
        assert np.abs(Ac.toarray() - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.abs(Pl @ np.ones(Pl.shape[1]) - 1).max() <= 1e-9


def test_vl_sor_rejected_with_dirichlet_top():
    m = _mesh(5, 3)
    with pytest.raises(Exception):
        O.Problem(m, bc=O.BC_DIRICHLET_TOP, precond=O.PC_VL_SOR)


def test_section6_sa_degrades_with_aspect_ratio_vl_does_not():
    """Section 6 (genuinely unstructured meshes): plain SA needs ever more iterations as the
    aspect ratio shrinks, while both forms built on vertical lumping stay nearly constant."""
    its = {pc: [] for pc in (O.PC_ADDITIVE, O.PC_VL_SOR, O.PC_SA)}
    for eps in [1e-1, 1e-2, 1e-4]:
        m = I.make_mesh(12, 12, 6, I.depth_sines(eps), z_jitter=0.3, xy_jitter=0.2, seed=8)
        for pc in its:
            P = O.Problem(m, precond=pc)
            r = P.solve(I.normal_loads(P.n, 2), tol=1e-7, maxit=2000)
            assert r["status"] == "OK"
            its[pc].append(r["iters"])
    for pc in (O.PC_ADDITIVE, O.PC_VL_SOR):
        assert max(its[pc]) <= 1.3 * min(its[pc]), its
    assert its[O.PC_SA][-1] > 5 * its[O.PC_SA][0], its
    # the multiplicative VL+SOR cycle needs fewer iterations than the additive one
    assert all(v < a for v, a in zip(its[O.PC_VL_SOR], its[O.PC_ADDITIVE])), its


# --------------------------------------------------------------------------------------------
# the clustered (multiscale) mesh of section 6

def test_cluster_map_is_identity_at_zero_and_grades_spacing():
    a = I.make_mesh(6, 5, 4, I.depth_sines(0.01), z_jitter=0.3, seed=5)
    b = I.make_mesh(6, 5, 4, I.depth_sines(0.01), z_jitter=0.3, seed=5, cluster=0.0)
    assert np.array_equal(a.xyz.view(np.uint64), b.xyz.view(np.uint64))
    c = 0.9
    m = I.make_mesh(40, 40, 12, I.depth_flat(1.0), seed=5, cluster=c)
    top = m.xyz[m.tags & I.TAG_TOP != 0]
    xs = np.unique(np.round(top[:, 0], 14))
    dx = np.diff(xs)
    # spacing (1 - c)/n at the centre, (1 + c)/n at the edges, to second order in 1/n
    assert abs(dx.min() * 40 - (1 - c)) < 0.02 and abs(dx.max() * 40 - (1 + c)) < 0.02
    assert xs[0] == 0.0 and xs[-1] == 1.0
    vol = np.linalg.det(np.stack([m.xyz[m.tets[:, k]] - m.xyz[m.tets[:, 0]] for k in (1, 2, 3)], axis=1))
    assert (vol > 0).all() and vol.max() / vol.min() > 1e3


def test_section6_clustered_mesh_sa_degrades_lumped_forms_do_not():
    """Section 6, clustered mesh: smoothed aggregation slows down as eps shrinks, while both
    vertically lumped forms reach an eps-independent rate for small eps."""
    its = {pc: [] for pc in (O.PC_ADDITIVE, O.PC_VL_SOR, O.PC_SA)}
    for eps in [1e-1, 1e-3, 1e-4]:
        m = I.make_mesh(48, 48, 12, I.depth_sines(eps), z_jitter=0.3, seed=8, cluster=0.9)
        for pc in its:
            P = O.Problem(m, precond=pc)
            r = P.solve(I.normal_loads(P.n, 2), tol=1e-8, maxit=3000)
            assert r["status"] == "OK"
            its[pc].append(r["iters"])
    assert its[O.PC_SA][1] > 2 * its[O.PC_SA][0], its
    for pc in (O.PC_ADDITIVE, O.PC_VL_SOR):
        a, b = its[pc][1], its[pc][2]
        assert abs(a - b) <= 0.2 * min(a, b), its


# --------------------------------------------------------------------------------------------
# spectrum (section 4): Lanczos tridiagonal from the CG coefficients

def _lanczos_T(alpha, beta):
    k = len(alpha)
    d = np.array([1.0 / alpha[j] + (beta[j] / alpha[j - 1] if j > 0 else 0.0) for j in range(k)])
    e = np.array([np.sqrt(beta[j + 1]) / alpha[j] for j in range(k - 1)])
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


def test_cg_coefficients_give_the_spectrum_of_A_and_of_the_preconditioned_operator():
    """Plain CG on A (Neumann, mean-zero right-hand side) is Lanczos on A restricted to the
    complement of the constants; PCG is Lanczos on M^-1 A. Their extreme Ritz values converge
    to the extreme eigenvalues computed densely."""
    m = _mesh(6, 3, h0=0.05, zj=0.3)
    b = I.normal_loads(m.xyz.shape[0], 7)
    # A on the complement of the constants
    P0 = O.Problem(m, precond=O.PC_NONE)
    A = P0.csr("A").toarray()
    n = A.shape[0]
    Q = np.linalg.qr(np.eye(n) - 1.0 / n)[0][:, : n - 1]
    w = np.linalg.eigvalsh(Q.T @ A @ Q)
    r = P0.solve(b, tol=1e-12, maxit=5000)   # converged: the extreme Ritz values have converged too
    assert r["status"] == "OK"
    lam = np.linalg.eigvalsh(_lanczos_T(r["alpha"], r["beta"]))
    assert abs(lam[-1] - w[-1]) <= 1e-8 * w[-1]
    assert abs(lam[0] - w[0]) <= 1e-6 * w[0]
    # M^-1 A for the additive preconditioner, on the same complement
    P = O.Problem(m, coarse_max=40)
    Mz = np.stack([P.precond(e) for e in np.eye(n)], axis=1)
    Mz = 0.5 * (Mz + Mz.T)
    S = Q.T @ Mz @ Q
    L = np.linalg.cholesky(S)
    wm = np.linalg.eigvalsh(L.T @ (Q.T @ A @ Q) @ L)   # similar to M^-1 A on the complement
    rp = P.solve(b, tol=1e-13, maxit=400)
    assert rp["status"] == "OK"
    lp = np.linalg.eigvalsh(_lanczos_T(rp["alpha"], rp["beta"]))
    # Ritz values lie inside the spectrum; after ~33 iterations the extreme ones have converged
    # to 1e-5 - 1e-4 (how far depends on the gaps at the ends of the spectrum of M^-1 A)
    assert lp[0] >= wm[0] * (1 - 1e-10) and lp[-1] <= wm[-1] * (1 + 1e-10)
    assert abs(lp[0] - wm[0]) <= 1e-4 * wm[0]
    assert abs(lp[-1] - wm[-1]) <= 1e-3 * wm[-1]


def test_library_lanczos_extremes_match_numpy():
    from paper_0912_1976_gb300 import vemg as V
    rng = np.random.default_rng(3)
    for k in (1, 2, 7, 40):
        alpha = rng.uniform(0.1, 2.0, k)
        beta = np.concatenate([[0.0], rng.uniform(0.01, 1.5, k - 1)])
        w = np.linalg.eigvalsh(_lanczos_T(alpha, beta))
        lo, hi = V.vemg_lanczos_extremes(alpha, beta)
        assert abs(lo - w[0]) <= 1e-12 * abs(w[-1]) and abs(hi - w[-1]) <= 1e-12 * abs(w[-1])


def test_section4_preconditioned_condition_number_independent_of_eps():
    """Section 4 / 6.2: Cond(A) grows like eps^-2, while the condition number of the preconditioned
    operator (Lanczos estimate from the PCG coefficients) stays bounded."""
    ka, km = [], []
    for eps in [1e-2, 1e-3, 1e-4]:
        m = _mesh(16, 8, h0=eps, zj=0.3, seed=4)
        b = I.normal_loads(m.xyz.shape[0], 2)
        r = O.Problem(m, precond=O.PC_NONE).solve(b, tol=1e-10, maxit=4000)
        la = np.linalg.eigvalsh(_lanczos_T(r["alpha"], r["beta"]))
        ka.append(la[-1] / la[0])
        rp = O.Problem(m).solve(b, tol=1e-8, maxit=400)   # above the eps = 1e-4 round-off floor
        lm = np.linalg.eigvalsh(_lanczos_T(rp["alpha"], rp["beta"]))
        km.append(lm[-1] / lm[0])
    assert ka[1] > 30 * ka[0] and ka[2] > 30 * ka[1], ka
    assert max(km) <= 1.5 * min(km), km


# --------------------------------------------------------------------------------------------
# BF16 operator values: rounding to bfloat16 and the cycle with rounded operators

def test_bf16_rounding_fixed_points_ties_and_overflow():
    # bfloat16 keeps 8 significant bits: near 1 its spacing is 2^-7
    assert O.round_bf16(1.0) == 1.0 and O.round_bf16(-2.5) == -2.5 and O.round_bf16(0.0) == 0.0
    assert O.round_bf16(1 + 2 ** -8) == 1.0                       # tie, 1.0 has the even significand
    assert O.round_bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6           # tie, rounds up to the even one
    assert O.round_bf16(-(1 + 3 * 2 ** -8)) == -(1 + 2 ** -6)     # sign-symmetric
    assert O.round_bf16(1 + 2 ** -8 + 2 ** -20) == 1 + 2 ** -7    # just above the tie
    big = (2 - 2 ** -7) * 2.0 ** 127                              # largest finite bfloat16
    assert O.round_bf16(big) == big
    assert math.isinf(O.round_bf16(np.finfo(np.float32).max))    # above the last midpoint: infinity
    assert math.isnan(O.round_bf16(float("nan"))) and O.round_bf16(float("inf")) == float("inf")


def test_bf16_rounding_is_nearest_of_the_two_neighbours():
    """Brute force on random binary32 numbers of every magnitude: the result is a bfloat16 (lower
    16 bits of its binary32 pattern zero), one of the two bfloat16 numbers around x, the nearer
    one, and on a tie the one with an even last significand bit."""
    rng = np.random.default_rng(11)
    x = (rng.standard_normal(4000) * np.exp2(rng.integers(-120, 120, 4000))).astype(np.float32)
    x = np.concatenate([x, (1 + np.arange(1, 200) * 2.0 ** -16).astype(np.float32)])   # many ties
    for xi in x:
        r = np.float32(O.round_bf16(float(xi)))
        rb = r.view(np.uint32)
        assert rb & 0xFFFF == 0
        lo = np.uint32(xi.view(np.uint32) & 0xFFFF0000).view(np.float32)
        hi = np.uint32((xi.view(np.uint32) & 0xFFFF0000) + 0x10000).view(np.float32)
        assert r in (lo, hi)
        other = hi if r == lo else lo
        d, do = abs(float(xi) - float(r)), abs(float(xi) - float(other))
        assert d <= do
        if d == do:
            assert (rb >> 16) & 1 == 0
    # a double is first rounded to binary32
    for v in rng.standard_normal(200):
        assert O.round_bf16(v) == O.round_bf16(float(np.float32(v)))


@pytest.mark.parametrize("pc", [O.PC_ADDITIVE, O.PC_VL_SOR, O.PC_SA])
def test_bf16_rounded_cycle_symmetric_positive_and_near_fp64(pc):
    """Rounding A (off the diagonal), P and P^T of every level elementwise keeps each level matrix
    symmetric and P^T the transpose of P, so the V-cycle stays a symmetric positive definite
    operator (on A_bar) or semi-definite (on A); it moves the cycle by a few times BF16's unit
    roundoff (2^-9 = 2e-3)."""
    m = _mesh(5, 3, h0=0.01, zj=0.3)
    P = O.Problem(m, coarse_max=40, precond=pc)
    which = 1 if pc == O.PC_ADDITIVE else 2      # the A_bar chain, or the single chain on A
    n = P.size("lev.n", which, 0)
    assert P.nlev(which) >= 2
    V64 = np.stack([P.vcycle(which, e) for e in np.eye(n)], axis=1)
    M64 = np.stack([P.precond(e) for e in np.eye(P.n)], axis=1)
    P.round_operators_bf16()
    V16 = np.stack([P.vcycle(which, e) for e in np.eye(n)], axis=1)
    M16 = np.stack([P.precond(e) for e in np.eye(P.n)], axis=1)
    for X in (V16, M16):
        assert np.abs(X - X.T).max() <= 1e-10 * np.abs(X).max()
        w = np.linalg.eigvalsh(0.5 * (X + X.T))
        assert w[0] > -1e-10 * w[-1]
    rel = np.linalg.norm(V16 - V64) / np.linalg.norm(V64)
    assert 1e-3 < rel < 2e-2, rel
    assert np.linalg.norm(M16 - M64) <= 2e-2 * np.linalg.norm(M64)


# --------------------------------------------------------------------------------------------
# smoothed aggregation with the near-nullspace {1, x, y} (surface chain of unstructured meshes)

def test_tentative_qr_orthonormal_reconstructs_and_drops_dependent_columns():
    """Local QR of an aggregate's near-nullspace rows: orthonormal Q, Q R = B, R upper triangular,
    the same column space as a textbook QR (numpy), and dependent columns dropped: one node keeps
    the constant only, two nodes keep two columns, collinear and coincident nodes lose theirs."""
    rng = np.random.default_rng(5)
    for k in (3, 5, 12, 40):
        xy = 0.5 + 0.01 * rng.standard_normal((k, 2))
        B = np.column_stack([np.ones(k), xy])
        Q, R = O.tentative_qr(B)
        assert Q.shape == (k, 3)
        assert np.abs(Q.T @ Q - np.eye(3)).max() <= 1e-12
        assert np.abs(Q @ R - B).max() <= 1e-13
        assert np.abs(np.tril(R, -1)).max() <= 1e-12 * np.abs(B).max()
        Qn, _ = np.linalg.qr(B)
        assert np.abs(Q @ Q.T - Qn @ Qn.T).max() <= 1e-10
    assert O.tentative_qr(np.array([[1.0, 0.3, 0.7]]))[0].shape == (1, 1)
    assert O.tentative_qr(np.array([[1.0, 0.3, 0.7], [1.0, 0.4, 0.2]]))[0].shape == (2, 2)
    t = np.array([0.1, 0.2, 0.35, 0.5])
    collinear = np.column_stack([np.ones(4), t, 2.0 * t + 1.0])
    assert O.tentative_qr(collinear)[0].shape == (4, 2)
    coincident = np.tile([1.0, 0.3, 0.7], (3, 1))
    assert O.tentative_qr(coincident)[0].shape == (3, 1)


def test_block_strength_is_the_frobenius_norm_of_each_block():
    """The strength of the coarse levels of the {1, x, y} chain is measured between node blocks:
    entry (I, J) is the Frobenius norm of the block A_IJ (numpy's norm of the dense block)."""
    rng = np.random.default_rng(9)
    sizes = [3, 2, 3, 1, 3]
    blk = np.repeat(np.arange(len(sizes)), sizes)
    n = blk.size
    M = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.5)
    M = M + M.T
    S = O.block_norms(sp.csr_matrix(M), blk, len(sizes)).toarray()
    for I in range(len(sizes)):
        for J in range(len(sizes)):
            blkIJ = M[np.ix_(blk == I, blk == J)]
            assert abs(S[I, J] - np.linalg.norm(blkIJ)) <= 1e-14 * max(1.0, np.linalg.norm(blkIJ))


def test_linear_prolongator_reproduces_linear_functions_on_a_path():
    """Path of 9 nodes at x_i = i h, [-1, 2, -1] with Neumann ends, aggregates of three, near-nullspace
    {1, x}: the tentative prolongator has orthonormal columns and reproduces 1 and x exactly
    (P_t B_c = B). The 1D Laplacian annihilates linear functions at interior rows, so the smoothed P
    (omega = 2/3, D^-1 of the unfiltered A) still reproduces them there; at the left end
    (A x)_0 = x_0 - x_1 = -h and D_00 = 1, so (P B_c)_0 = (1, 0 + (2/3) h) by hand."""
    n, h = 9, 0.125
    A = _lap1d(n).tolil()
    A[0, 0] = A[n - 1, n - 1] = 1.0
    A = A.tocsr()
    x = h * np.arange(n)
    B = np.column_stack([np.ones(n), x])
    agg = np.repeat(np.arange(3), 3)
    Pt, Bc = O.linear_prolongator(A, agg, 3, B, smoothed=False)
    assert Pt.shape == (n, 6) and Bc.shape == (6, 2)
    assert np.abs((Pt.T @ Pt).toarray() - np.eye(6)).max() <= 1e-14
    assert np.abs(Pt @ Bc - B).max() <= 1e-14
    P, Bc2 = O.linear_prolongator(A, agg, 3, B)
    assert np.array_equal(Bc, Bc2)
    PB = P @ Bc
    assert np.abs(PB[1:n - 1] - B[1:n - 1]).max() <= 1e-14
    assert np.abs(PB[0] - [1.0, (2.0 / 3.0) * h]).max() <= 1e-15
    assert np.abs(PB[n - 1] - [1.0, x[n - 1] - (2.0 / 3.0) * h]).max() <= 1e-15


def _xy_mesh(nx, nz, eps, seed=8):
    return I.make_mesh(nx, nx, nz, I.depth_sines(eps), z_jitter=0.3, xy_jitter=0.2, seed=seed)


def test_linear_chain_invariants():
    """On an xy-jittered mesh (surface chain of three levels or more): every coarse level has at most three
    unknowns per aggregate; its near-nullspace rows are reproduced by the smoothed prolongator as
    (I - omega D^-1 A) applied to the fine ones; the coarse constant (first near-nullspace column)
    is prolonged to the fine constant and spans the kernel of every coarse operator; the coarse
    operators are exactly symmetric Galerkin products."""
    m = _xy_mesh(32, 12, 1e-4)
    P = O.Problem(m, surf_ns=3, coarse_max=40)
    assert P.size("nsd", 0) == 3 and P.nlev(0) >= 3
    for l in range(P.nlev(0) - 1):
        A = P.csr("lev.A", 0, l)
        Pl = P.csr("lev.P", 0, l)
        Ac = P.csr("lev.A", 0, l + 1).toarray()
        Bf, Bc = P.nullspace(0, l), P.nullspace(0, l + 1)
        nagg = len(set(P.ints("lev.agg", 0, l).tolist()))
        assert nagg <= Bc.shape[0] <= 3 * nagg
        D = A.diagonal()
        ref = Bf - (2.0 / 3.0) * (A @ Bf) / D[:, None]
        assert np.abs(Pl @ Bc - ref).max() <= 1e-10 * np.abs(Bf).max()
        # (A B_f[:, 0] vanishes only to rounding, amplified by D^-1 of these eps = 1e-4 levels)
        assert np.abs(Pl @ Bc[:, 0] - Bf[:, 0]).max() <= 1e-9 * np.abs(Bf[:, 0]).max()
        assert np.array_equal(Ac, Ac.T)
        refA = (Pl.T @ (A @ Pl)).toarray()
        assert np.abs(Ac - refA).max() <= 1e-12 * np.abs(refA).max()
        assert np.abs(Ac @ Bc[:, 0]).max() <= 1e-10 * np.abs(Ac).max() * np.abs(Bc[:, 0]).max()
    # level 0 holds {1, x, y} of the top nodes in the internal order
    n2o = P.ints("new2old")
    B0 = P.nullspace(0, 0)
    assert np.array_equal(B0[:, 1:], m.xyz[n2o[:P.mtop], :2]) and np.all(B0[:, 0] == 1.0)


def test_linear_chain_preconditioner_symmetric_positive_and_solves():
    m = _xy_mesh(9, 4, 1e-3, seed=4)
    P = O.Problem(m, surf_ns=3, coarse_max=20)
    assert P.nlev(0) >= 2
    n = P.n
    Mz = np.stack([P.precond(e) for e in np.eye(n)], axis=1)
    assert np.abs(Mz - Mz.T).max() <= 1e-10 * np.abs(Mz).max()
    w = np.linalg.eigvalsh(0.5 * (Mz + Mz.T))
    assert w[0] > -1e-10 * w[-1]
    b = I.normal_loads(n, 4)
    r = P.solve(b, tol=1e-11, maxit=2000)
    assert r["status"] == "OK"
    n2o = P.ints("new2old")
    A = P.csr("A").toarray()
    bi = b[n2o] - b.mean()
    K = np.block([[A, np.ones((n, 1))], [np.ones((1, n)), np.zeros((1, 1))]])
    xs = np.linalg.solve(K, np.concatenate([bi, [0.0]]))[:n]
    assert np.linalg.norm(r["x"][n2o] - xs) <= 1e-8 * np.linalg.norm(xs)


def test_section62_linear_nullspace_gives_eps_independent_rate_on_unstructured_mesh():
    """Section 6.2: on unstructured meshes the vertically lumped preconditioner converges at a rate
    independent of eps for small eps. On a 24x24x24 xy-jittered mesh (surface chain of three levels)
    the constants-only surface chain does not (iterations x1.8 from eps = 1e-2 to 1e-4); with
    {1, x, y} the counts stay within 10% over eps in {1e-2, 1e-3, 1e-4}."""
    it = {1: [], 3: []}
    for eps in (1e-2, 1e-3, 1e-4):
        m = _xy_mesh(24, 24, eps)
        for ns in (1, 3):
            # coarse_max 512: the 625-node surface operator is coarsened, not solved directly
            P = O.Problem(m, surf_ns=ns, coarse_max=512)
            r = P.solve(I.normal_loads(P.n, 12), tol=1e-8, maxit=3000)
            assert r["status"] == "OK"
            it[ns].append(r["iters"])
    assert max(it[3]) <= 1.1 * min(it[3]), it
    assert it[1][-1] >= 1.8 * it[1][0], it
    assert it[3][-1] * 3 <= it[1][-1], it


def test_openmp_timing_build_gives_the_same_bits():
    """The OpenMP build of the oracle (its timing build on all host cores) runs the solve's row loops
    in parallel and sums vectors in fixed blocks, so x, the iteration count and every residual are
    the same bits as the single-threaded build's, whatever the number of threads."""
    m = _mesh(20, 8, h0=1e-3, zj=0.3)
    b = I.normal_loads(m.n, 31)
    r1 = O.Problem(m).solve(b, tol=1e-9)
    Lo = O.lib(openmp=True)
    for t in (1, 3, 4):
        Lo.or_set_threads(t)
        assert Lo.or_threads() == t
        r = O.Problem(m, openmp=True).solve(b, tol=1e-9)
        assert r["iters"] == r1["iters"] and r["relres"] == r1["relres"]
        assert np.array_equal(r["x"].view(np.uint64), r1["x"].view(np.uint64))
