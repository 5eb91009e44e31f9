"""ctypes wrapper of the plain FP64 CPU oracle (vemg_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the benchmark's
CPU-baseline leg. The product path never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vemg_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")   # the OpenMP timing build

BC_NEUMANN = 0
BC_DIRICHLET_TOP = 1
# the three preconditioners of section 6
PC_ADDITIVE, PC_VL_SOR, PC_SA, PC_NONE = 0, 1, 2, 3
STATUS = {0: "OK", 1: "EINVAL", 2: "EMESH", 3: "ENOMEM", 4: "ENOTCONV", 5: "EBREAKDOWN"}

# the paper's smoothed-aggregation parameters (section 6)
THETA = 0.01
OMEGA_P = 2.0 / 3.0
# the size of a directly solved coarsest level and the level cap: the paper states neither
COARSE_MAX = 1024
MAX_LEVELS = 10


def build_oracle(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle (plain, single-threaded) or its OpenMP timing build (the same source with
    -fopenmp: row loops on all cores, sums in fixed blocks, the same bits)."""
    out = LIB_OMP if openmp else LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11"] +
                              (["-fopenmp"] if openmp else []) + ["-shared", "-fPIC", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, out)
    return out


_libs = {}


def lib(openmp: bool = False):
    if openmp not in _libs:
        path = build_oracle(openmp=True) if openmp else (build_oracle(), LIB)[1]
        L = C.CDLL(path)
        dp, ip, u8p = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_uint8)
        L.or_setup.restype = C.c_void_p
        L.or_setup.argtypes = [C.c_int, dp, C.c_int, ip, u8p, C.c_int, ip, C.c_int, C.c_double,
                               C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, ip]
        L.or_tentative_qr.argtypes = [C.c_int, C.c_int, dp, dp, dp]
        L.or_linear_prolongator.argtypes = [C.c_int, ip, ip, dp, ip, C.c_int, dp, C.c_int, C.c_double, C.c_int,
                                            ip, ip, dp, dp, C.c_int]
        L.or_get_nullspace.argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
        L.or_block_norms.argtypes = [C.c_int, ip, ip, dp, ip, C.c_int, ip, ip, dp, C.c_int]
        L.or_free.argtypes = [C.c_void_p]
        L.or_size.restype = C.c_long
        L.or_size.argtypes = [C.c_void_p, C.c_char_p, C.c_int, C.c_int]
        L.or_get_csr.argtypes = [C.c_void_p, C.c_char_p, C.c_int, C.c_int, ip, ip, dp]
        L.or_get_int.argtypes = [C.c_void_p, C.c_char_p, C.c_int, C.c_int, ip]
        L.or_solve.argtypes = [C.c_void_p, dp, dp, C.c_double, C.c_int, C.c_int, ip, dp, dp, dp, C.c_int, dp,
                               C.c_int]
        L.or_precond.argtypes = [C.c_void_p, dp, dp]
        L.or_spmv.argtypes = [C.c_void_p, dp, dp]
        L.or_load.argtypes = [C.c_void_p, dp, dp]
        L.or_vcycle.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.or_sa_aggregate.argtypes = [C.c_int, ip, ip, dp, C.c_double, C.c_int, ip]
        L.or_colour.argtypes = [C.c_int, ip, ip, ip]
        L.or_smoothed_prolongator.argtypes = [C.c_int, ip, ip, dp, ip, C.c_int, C.c_double, C.c_double, ip, ip,
                                              dp, C.c_int]
        L.or_sl_ranks.argtypes = [C.c_int, ip, ip, ip]
        L.or_locate_points.argtypes = [C.c_int, ip, dp, C.c_int, dp, ip, dp]
        L.or_elem_stiffness.restype = C.c_double
        L.or_elem_stiffness.argtypes = [dp, dp]
        L.or_round_bf16.argtypes = [C.c_double]
        L.or_round_bf16.restype = C.c_double
        L.or_round_operators_bf16.argtypes = [C.c_void_p]
        L.or_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        _libs[openmp] = L
    return _libs[openmp]


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


class Problem:
    """Oracle setup of one mesh: ordering, A, E~, E~^T A E~, and the two SA chains."""

    def __init__(self, mesh, bc: int = BC_NEUMANN, theta=THETA, omega_p=OMEGA_P, coarse_max=COARSE_MAX,
                 max_levels=MAX_LEVELS, natural_order=False, precond=PC_ADDITIVE, surf_ns=1, openmp=False):
        L = self.L = lib(openmp)
        self._keep = (_f64(mesh.xyz), _i32(mesh.tets), np.ascontiguousarray(mesh.tags, dtype=np.uint8),
                      _i32(mesh.top_tris))
        xyz, tets, tags, tris = self._keep
        st = C.c_int(0)
        self.h = L.or_setup(xyz.shape[0], _p(xyz, C.c_double), tets.shape[0], _p(tets, C.c_int),
                            _p(tags, C.c_uint8), tris.shape[0], _p(tris, C.c_int), bc, theta, omega_p,
                            coarse_max, max_levels, int(natural_order), precond, surf_ns, C.byref(st))
        if not self.h:
            raise OracleError(f"or_setup failed: {STATUS.get(st.value, st.value)}")
        self.bc = bc
        self.n = self.size("n")
        self.mtop = self.size("mtop")

    def __del__(self):
        if getattr(self, "h", None):
            self.L.or_free(self.h)
            self.h = None

    def size(self, key, which=1, level=0) -> int:
        return int(self.L.or_size(self.h, key.encode(), which, level))

    def csr(self, name, which=1, level=0) -> sp.csr_matrix:
        shapes = {"A": (self.n, self.n), "E": (self.n, self.mtop), "ET": (self.mtop, self.n),
                  "Ac": (self.mtop, self.mtop)}
        if name in shapes:
            nrow, ncol = shapes[name]
        else:
            nrow = self.size("lev.n", which, level)
            ncol = nrow if name == "lev.A" else self.size("lev.n", which, level + 1)
        nnz_key = {"A": "nnzA", "E": "nnzE", "ET": "nnzE", "Ac": "nnzAc", "lev.A": "lev.nnz",
                   "lev.P": "lev.nnzP"}[name]
        nnz = self.size(nnz_key, which, level)
        rp = np.zeros(nrow + 1, np.int32)
        ci = np.zeros(max(nnz, 1), np.int32)
        v = np.zeros(max(nnz, 1), np.float64)
        rc = self.L.or_get_csr(self.h, name.encode(), which, level, _p(rp, C.c_int), _p(ci, C.c_int),
                              _p(v, C.c_double))
        if rc:
            raise OracleError(f"no matrix {name}")
        return sp.csr_matrix((v[:nnz], ci[:nnz], rp), shape=(nrow, ncol))

    def ints(self, name, which=1, level=0) -> np.ndarray:
        cnt = self.n if name in ("new2old", "tri_of") else self.size("lev.n", which, level)
        out = np.zeros(cnt, np.int32)
        rc = self.L.or_get_int(self.h, name.encode(), which, level, _p(out, C.c_int))
        if rc:
            raise OracleError(f"no int array {name}")
        return out

    def nullspace(self, which=0, level=0) -> np.ndarray:
        """Near-nullspace rows (lev.n x nsd) of a level of a {1, x, y} chain."""
        nsd = self.size("nsd", which)
        out = np.zeros((self.size("lev.n", which, level), nsd))
        rc = self.L.or_get_nullspace(self.h, which, level, _p(out, C.c_double))
        if rc:
            raise OracleError("no near-nullspace rows")
        return out

    def nlev(self, which):
        return self.size("nlev", which)

    def level_sizes(self, which):
        return [self.size("lev.n", which, l) for l in range(self.nlev(which))]

    def load(self, f):
        f = _f64(f)
        b = np.zeros(self.n)
        self.L.or_load(self.h, _p(f, C.c_double), _p(b, C.c_double))
        return b

    def solve(self, b, tol=1e-8, maxit=1000, flexible=False, hist_len=1000):
        b = _f64(b)
        x = np.zeros(self.n)
        it = C.c_int(0)
        rr, tr = C.c_double(0), C.c_double(0)
        hist = np.zeros(hist_len)
        coef = np.zeros(2 * maxit + 2)
        st = self.L.or_solve(self.h, _p(b, C.c_double), _p(x, C.c_double), tol, maxit, int(flexible),
                            C.byref(it), C.byref(rr), C.byref(tr), _p(hist, C.c_double), hist_len,
                            _p(coef, C.c_double), len(coef))
        k = it.value
        # alpha_0..alpha_{k-1}; beta_0 = 0 and beta_1..beta_{k-1} (the last beta is never used)
        alpha = coef[0:2 * k:2].copy()
        beta = np.concatenate([[0.0], coef[1:2 * k - 1:2]]) if k > 0 else np.zeros(0)
        return dict(x=x, iters=k, relres=rr.value, true_relres=tr.value, status=STATUS[st],
                    hist=hist[:min(k, hist_len)], alpha=alpha, beta=beta)

    def nunk(self):
        return self.n if self.bc == BC_NEUMANN else self.n - self.mtop

    def precond(self, r):
        r = _f64(r)
        z = np.zeros(self.nunk())
        self.L.or_precond(self.h, _p(r, C.c_double), _p(z, C.c_double))
        return z

    def spmv(self, x):
        x = _f64(x)
        y = np.zeros(self.nunk())
        self.L.or_spmv(self.h, _p(x, C.c_double), _p(y, C.c_double))
        return y

    def vcycle(self, which, b):
        b = _f64(b)
        x = np.zeros_like(b)
        self.L.or_vcycle(self.h, which, _p(b, C.c_double), _p(x, C.c_double))
        return x

    def round_operators_bf16(self):
        """Round the stored cycle operators to BF16 (off-diagonals of every level matrix, P and
        P^T), in place: the operator the BF16 variant of the cycle applies."""
        self.L.or_round_operators_bf16(self.h)


def round_bf16(a: float) -> float:
    """a rounded to binary32, then to bfloat16 (nearest, ties to even)."""
    return lib().or_round_bf16(float(a))


def sa_aggregate(A: sp.csr_matrix, theta=THETA, keep_isolated=True):
    """Aggregates of the rows of A (-1: an isolated row left unaggregated, keep_isolated False)."""
    A = A.tocsr()
    A.sort_indices()
    rp, ci, v = _i32(A.indptr), _i32(A.indices), _f64(A.data)
    agg = np.zeros(A.shape[0], np.int32)
    nagg = lib().or_sa_aggregate(A.shape[0], _p(rp, C.c_int), _p(ci, C.c_int), _p(v, C.c_double), theta,
                                 int(keep_isolated), _p(agg, C.c_int))
    return nagg, agg


def smoothed_prolongator(A: sp.csr_matrix, agg, nagg, omega=OMEGA_P, theta=THETA):
    """The smoothed prolongator of the given aggregates (agg[i] = -1: unaggregated row)."""
    A = A.tocsr()
    A.sort_indices()
    n = A.shape[0]
    rp, ci, v, ag = _i32(A.indptr), _i32(A.indices), _f64(A.data), _i32(agg)
    cap = max(int(A.nnz) + n, 1)
    prp = np.zeros(n + 1, np.int32)
    pci = np.zeros(cap, np.int32)
    pv = np.zeros(cap)
    nnz = lib().or_smoothed_prolongator(n, _p(rp, C.c_int), _p(ci, C.c_int), _p(v, C.c_double), _p(ag, C.c_int),
                                        int(nagg), omega, theta, _p(prp, C.c_int), _p(pci, C.c_int),
                                        _p(pv, C.c_double), cap)
    if nnz < 0:
        raise OracleError("prolongator capacity")
    return sp.csr_matrix((pv[:nnz], pci[:nnz], prp), shape=(n, int(nagg)))


def block_norms(A: sp.csr_matrix, blk, nblk):
    """Block strength matrix: (I, J) = Frobenius norm of A's block (I, J) (blocks: consecutive rows)."""
    A = A.tocsr()
    A.sort_indices()
    rp, ci, v, bk = _i32(A.indptr), _i32(A.indices), _f64(A.data), _i32(blk)
    cap = A.nnz + 1
    srp = np.zeros(nblk + 1, np.int32)
    sci = np.zeros(cap, np.int32)
    sv = np.zeros(cap)
    nnz = lib().or_block_norms(A.shape[0], _p(rp, C.c_int), _p(ci, C.c_int), _p(v, C.c_double), _p(bk, C.c_int),
                               int(nblk), _p(srp, C.c_int), _p(sci, C.c_int), _p(sv, C.c_double), cap)
    return sp.csr_matrix((sv[:nnz], sci[:nnz], srp), shape=(nblk, nblk))


def tentative_qr(Bj):
    """Local QR of one aggregate's near-nullspace rows (k x d): (Q k x kept, R kept x d)."""
    Bj = _f64(Bj)
    k, d = Bj.shape
    Q = np.zeros((k, d))
    R = np.zeros((d, d))
    kept = lib().or_tentative_qr(k, d, _p(Bj, C.c_double), _p(Q, C.c_double), _p(R, C.c_double))
    return Q[:, :kept].copy(), R[:kept].copy()


def linear_prolongator(A: sp.csr_matrix, agg, nagg, B, omega=OMEGA_P, smoothed=True):
    """Tentative (smoothed=False) or smoothed prolongator of the {1, x, y} chain for the given
    aggregates and near-nullspace rows B (n x d); returns (P, coarse near-nullspace rows)."""
    A = A.tocsr()
    A.sort_indices()
    n = A.shape[0]
    B = _f64(B)
    d = B.shape[1]
    rp, ci, v, ag = _i32(A.indptr), _i32(A.indices), _f64(A.data), _i32(agg)
    cap = (A.nnz + n) * d * 4 + 16
    prp = np.zeros(n + 1, np.int32)
    pci = np.zeros(cap, np.int32)
    pv = np.zeros(cap)
    Bc = np.zeros((int(nagg) * d, d))
    nc = lib().or_linear_prolongator(n, _p(rp, C.c_int), _p(ci, C.c_int), _p(v, C.c_double), _p(ag, C.c_int),
                                     int(nagg), _p(B, C.c_double), d, omega, int(smoothed), _p(prp, C.c_int),
                                     _p(pci, C.c_int), _p(pv, C.c_double), _p(Bc, C.c_double), cap)
    if nc < 0:
        raise OracleError("prolongator capacity")
    nnz = int(prp[n])
    return sp.csr_matrix((pv[:nnz], pci[:nnz], prp), shape=(n, nc)), Bc[:nc].copy()


def colour(A: sp.csr_matrix):
    A = A.tocsr()
    A.sort_indices()
    rp, ci = _i32(A.indptr), _i32(A.indices)
    col = np.zeros(A.shape[0], np.int32)
    nc = lib().or_colour(A.shape[0], _p(rp, C.c_int), _p(ci, C.c_int), _p(col, C.c_int))
    return nc, col


def sl_ranks(A: sp.csr_matrix):
    """Round of removal of each node in the round-synchronous smallest-last peeling."""
    A = A.tocsr()
    A.sort_indices()
    rp, ci = _i32(A.indptr), _i32(A.indices)
    rank = np.zeros(A.shape[0], np.int32)
    lib().or_sl_ranks(A.shape[0], _p(rp, C.c_int), _p(ci, C.c_int), _p(rank, C.c_int))
    return rank


def locate_points(tris, xyz, pts_xy):
    tris, xyz, pts = _i32(tris), _f64(xyz), _f64(pts_xy)
    out = np.zeros(pts.shape[0], np.int32)
    w = np.zeros((pts.shape[0], 3))
    lib().or_locate_points(tris.shape[0], _p(tris, C.c_int), _p(xyz, C.c_double), pts.shape[0],
                           _p(pts, C.c_double), _p(out, C.c_int), _p(w, C.c_double))
    return out, w


def elem_stiffness(p4x3):
    p = _f64(p4x3).reshape(4, 3)
    K = np.zeros(16)
    det = lib().or_elem_stiffness(_p(p, C.c_double), _p(K, C.c_double))
    return det, K.reshape(4, 4)
