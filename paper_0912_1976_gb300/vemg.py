"""Python binding of libvemg (include/vemg.h): argument marshalling only.

Every entry point keeps the C name. Device arrays are torch CUDA tensors; the mesh is given as
host numpy arrays. There is no CPU fallback: if libvemg.so is missing or CUDA is unavailable,
the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

VEMG_OK, VEMG_EINVAL, VEMG_EMESH, VEMG_ENOMEM, VEMG_ENOTCONV, VEMG_EBREAKDOWN, VEMG_ETIMEOUT, VEMG_ECUDA, \
    VEMG_EINTERNAL = range(9)
VEMG_NEUMANN, VEMG_DIRICHLET_TOP = 0, 1
VEMG_PREC_FP64, VEMG_PREC_FP32, VEMG_PREC_BF16 = 0, 1, 2
VEMG_PRECOND_ADDITIVE, VEMG_PRECOND_VL_SOR, VEMG_PRECOND_SA, VEMG_PRECOND_NONE = 0, 1, 2, 3
VEMG_CYCLE_PERSISTENT, VEMG_CYCLE_LAUNCHES, VEMG_CYCLE_AUTO, VEMG_CYCLE_HYBRID = 0, 1, 2, 3
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "EMESH", 3: "ENOMEM", 4: "ENOTCONV", 5: "EBREAKDOWN",
                6: "ETIMEOUT", 7: "ECUDA", 8: "EINTERNAL"}


class vemg_mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("xyz", C.POINTER(C.c_double)), ("n_tets", C.c_int64),
                ("tets", C.POINTER(C.c_int32)), ("tags", C.POINTER(C.c_uint8)), ("n_top_tris", C.c_int64),
                ("top_tris", C.POINTER(C.c_int32))]


class vemg_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


class vemg_options(C.Structure):
    _fields_ = [("bc", C.c_int), ("precision", C.c_int), ("strength", C.c_double), ("omega_p", C.c_double),
                ("coarse_max", C.c_int), ("max_levels", C.c_int), ("precond", C.c_int), ("cycle", C.c_int), ("tail_rows", C.c_int),
                ("surf_nullspace", C.c_int), ("tail_cluster", C.c_int)]


class vemg_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("relres", C.c_double), ("true_relres", C.c_double),
                ("b_mean", C.c_double)]

    def as_dict(self):
        return dict(iters=self.iters, status=STATUS_NAMES.get(self.status, self.status), relres=self.relres,
                    true_relres=self.true_relres, b_mean=self.b_mean)


class VemgError(RuntimeError):
    def __init__(self, code, what):
        msg = f"{what}: {STATUS_NAMES.get(code, code)}"
        if code == VEMG_ECUDA and _lib is not None:
            msg += f" ({(_lib.vemg_last_error() or b'').decode(errors='replace')})"
        super().__init__(msg)
        self.code = code


_lib = None

# the exported symbols and their prototypes, as declared in include/vemg.h
_VP, _DP, _I64 = C.c_void_p, C.c_void_p, C.c_int64
PROTOTYPES = {
    "vemg_default_options": (None, [C.POINTER(vemg_options)]),
    "vemg_last_error": (C.c_char_p, []),
    "vemg_selftest_barrier": (C.c_int, [C.c_int, C.c_int, _VP]),
    "vemg_solve_coefficients": (C.c_int, [_VP, C.c_int, _DP, _DP, C.POINTER(C.c_int)]),
    "vemg_lanczos_extremes": (C.c_int, [_DP, _DP, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "vemg_assemble": (C.c_int, [C.POINTER(vemg_mesh), C.POINTER(vemg_csr), _VP]),
    "vemg_load": (C.c_int, [C.POINTER(vemg_mesh), _DP, _DP, _VP]),
    "vemg_csr_free": (None, [C.POINTER(vemg_csr)]),
    "vemg_setup": (C.c_int, [C.POINTER(vemg_csr), C.POINTER(vemg_mesh), C.POINTER(vemg_options), _VP,
                             C.POINTER(C.c_void_p)]),
    "vemg_destroy": (None, [_VP]),
    "vemg_solve": (C.c_int, [_VP, _DP, _DP, C.c_double, C.c_int, C.POINTER(vemg_info), _VP]),
    "vemg_solve_host": (C.c_int, [_VP, _DP, _DP, C.c_double, C.c_int, C.POINTER(vemg_info), _VP]),
    "vemg_solve_batch": (C.c_int, [_VP, C.c_int, _DP, _I64, _DP, _I64, C.c_double, C.c_int,
                                   C.POINTER(vemg_info), _VP]),
    "vemg_hierarchy_bytes": (C.c_int, [_VP, C.POINTER(C.c_size_t)]),
    "vemg_set_allocator": (C.c_int, [_VP, _VP, _VP]),
    "vemg_strerror": (C.c_char_p, [C.c_int]),
    "vemg_get_size": (C.c_int, [_VP, C.c_char_p, C.c_int, C.c_int, C.POINTER(C.c_int64)]),
    "vemg_get_csr": (C.c_int, [_VP, C.c_char_p, C.c_int, C.c_int, _VP, _VP, _VP]),
    "vemg_get_int": (C.c_int, [_VP, C.c_char_p, C.c_int, C.c_int, _VP]),
    "vemg_get_nullspace": (C.c_int, [_VP, C.c_int, C.c_int, _VP]),
    "vemg_batch_tuning": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                    C.POINTER(C.c_float)]),
    "vemg_batch_set_tuning": (C.c_int, [_VP, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _VP]),
    "vemg_spmv": (C.c_int, [_VP, _DP, _DP, _VP]),
    "vemg_precond": (C.c_int, [_VP, _DP, _DP, _VP]),
    "vemg_vcycle": (C.c_int, [_VP, C.c_int, _DP, _DP, _VP]),
    "vemg_spmv_static": (C.c_int, [_VP, _DP, _DP, _VP]),
    "vemg_engine_create": (C.c_int, [_VP, C.c_int, _VP, C.POINTER(C.c_void_p)]),
    "vemg_engine_destroy": (None, [_VP]),
    "vemg_engine_admit": (C.c_int, [_VP, _DP, C.c_double, C.c_int, C.POINTER(C.c_int)]),
    "vemg_engine_launch": (C.c_int, [_VP, C.c_int]),
    "vemg_engine_wait": (C.c_int, [_VP]),
    "vemg_engine_query": (C.c_int, [_VP, C.POINTER(C.c_int)]),
    "vemg_engine_poll": (C.c_int, [_VP, C.c_int, C.POINTER(vemg_info), C.POINTER(C.c_int)]),
    "vemg_engine_retire": (C.c_int, [_VP, C.c_int, _DP]),
    "vemg_engine_slots": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "vemg_engine_bytes": (C.c_int, [_VP, C.POINTER(C.c_size_t)]),
    "vemg_probe": (C.c_int, [_VP, C.c_int]),
    "vemg_kernel_launches": (C.c_int, [_VP, C.POINTER(C.c_int64)]),
    "vemg_probe_read": (C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "vemg_probe_phases": (C.c_int, [_VP, C.c_int, C.POINTER(C.c_int), _VP, _VP, _VP, _VP]),
}
(VEMG_PROBE_NONE, VEMG_PROBE_SPMV_A, VEMG_PROBE_SOR_COARSE, VEMG_PROBE_RESIDUAL, VEMG_PROBE_SOR_FINE, VEMG_PROBE_VCYCLE,
 VEMG_PROBE_TRANSFER, VEMG_PROBE_VECTOR, VEMG_PROBE_DENSE, VEMG_PROBE_TAIL) = range(10)
VEMG_PROBE_SOR = VEMG_PROBE_SOR_COARSE


def lib_path() -> str:
    return _build.LIB


def lib() -> C.CDLL:
    """Load libvemg.so (building it first if its sources are newer). Raises if it cannot."""
    global _lib
    if _lib is None:
        if _build.needs_build():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libvemg.so is not built; run __graft_entry__.build()")
        L = C.CDLL(_build.LIB)
        for name, (res, args) in PROTOTYPES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, what):
    if rc != VEMG_OK:
        raise VemgError(rc, what)


def _stream(stream):
    if stream is None:
        if not torch.cuda.is_available():
            raise RuntimeError("libvemg needs a CUDA device")
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype=torch.float64):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"expected a contiguous CUDA {dtype} tensor")
    return C.c_void_p(t.data_ptr())


class _CudaArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape), "typestr": typestr,
                                         "version": 3, "strides": None}


def _view(ptr, shape, typestr) -> torch.Tensor:
    return torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")


class Mesh:
    """Host-side mesh arrays held alive for the duration of the calls that use them."""

    def __init__(self, xyz, tets, tags, top_tris):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)
        self.tags = np.ascontiguousarray(tags, dtype=np.uint8)
        self.top_tris = np.ascontiguousarray(top_tris, dtype=np.int32)
        self.c = vemg_mesh(self.xyz.shape[0], self.xyz.ctypes.data_as(C.POINTER(C.c_double)), self.tets.shape[0],
                           self.tets.ctypes.data_as(C.POINTER(C.c_int32)), self.tags.shape[0] and
                           self.tags.ctypes.data_as(C.POINTER(C.c_uint8)), self.top_tris.shape[0],
                           self.top_tris.ctypes.data_as(C.POINTER(C.c_int32)))

    @property
    def n(self):
        return self.xyz.shape[0]

    @classmethod
    def from_inputs(cls, m):
        return cls(m.xyz, m.tets, m.tags, m.top_tris)


class Csr:
    """A matrix returned by vemg_assemble (device arrays owned by the library)."""

    def __init__(self, c: vemg_csr):
        self.c = c

    @property
    def n(self):
        return self.c.n

    @property
    def nnz(self):
        return self.c.nnz

    def tensors(self):
        """Zero-copy torch views (rowptr, col, val) of the device arrays."""
        n, nnz = int(self.c.n), int(self.c.nnz)
        return (_view(self.c.rowptr, (n + 1,), "<i4"), _view(self.c.col, (nnz,), "<i4"),
                _view(self.c.val, (nnz,), "<f8"))

    def to_host(self):
        import scipy.sparse as sp
        rp, ci, v = (t.cpu().numpy() for t in self.tensors())
        return sp.csr_matrix((v, ci, rp), shape=(self.n, self.n))

    def free(self):
        if self.c.rowptr:
            lib().vemg_csr_free(C.byref(self.c))

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def vemg_default_options(**over) -> vemg_options:
    o = vemg_options()
    lib().vemg_default_options(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def vemg_assemble(mesh: Mesh, stream=None) -> Csr:
    c = vemg_csr()
    _check(lib().vemg_assemble(C.byref(mesh.c), C.byref(c), _stream(stream)), "vemg_assemble")
    return Csr(c)


def vemg_load(mesh: Mesh, f_dev: torch.Tensor, b_dev: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if b_dev is None:
        b_dev = torch.empty_like(f_dev)
    _check(lib().vemg_load(C.byref(mesh.c), _dev(f_dev), _dev(b_dev), _stream(stream)), "vemg_load")
    return b_dev


class Hierarchy:
    def __init__(self, handle, n, mesh, A):
        self.h = C.c_void_p(handle)
        self.n = n
        self._mesh, self._A = mesh, A

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            lib().vemg_destroy(self.h)
            self.h = C.c_void_p(None)

    def destroy(self):
        self.__del__()


def vemg_setup(A: Csr, mesh: Mesh, opts: vemg_options | None = None, stream=None) -> Hierarchy:
    out = C.c_void_p()
    _check(lib().vemg_setup(C.byref(A.c), C.byref(mesh.c), C.byref(opts) if opts is not None else None,
                            _stream(stream), C.byref(out)), "vemg_setup")
    return Hierarchy(out.value, int(A.n), mesh, A)


def vemg_destroy(h: Hierarchy):
    h.destroy()


def vemg_solve(h: Hierarchy, b_dev: torch.Tensor, x_dev: torch.Tensor | None = None, rtol=1e-8, max_it=1000,
               stream=None, check=False):
    if x_dev is None:
        x_dev = torch.empty_like(b_dev)
    info = vemg_info()
    rc = lib().vemg_solve(h.h, _dev(b_dev), _dev(x_dev), rtol, max_it, C.byref(info), _stream(stream))
    if rc not in (VEMG_OK, VEMG_ENOTCONV, VEMG_EBREAKDOWN) or (check and rc != VEMG_OK):
        raise VemgError(rc, "vemg_solve")
    return x_dev, info.as_dict()


def vemg_solve_host(h: Hierarchy, b_host: np.ndarray, x_host: np.ndarray | None = None, rtol=1e-8, max_it=1000,
                    stream=None):
    b_host = np.ascontiguousarray(b_host, dtype=np.float64)
    if x_host is None:
        x_host = np.empty_like(b_host)
    info = vemg_info()
    rc = lib().vemg_solve_host(h.h, C.c_void_p(b_host.ctypes.data), C.c_void_p(x_host.ctypes.data), rtol, max_it,
                               C.byref(info), _stream(stream))
    if rc not in (VEMG_OK, VEMG_ENOTCONV, VEMG_EBREAKDOWN):
        raise VemgError(rc, "vemg_solve_host")
    return x_host, info.as_dict()


def vemg_solve_batch(h: Hierarchy, B_dev: torch.Tensor, X_dev: torch.Tensor | None = None, rtol=1e-8, max_it=1000,
                     stream=None):
    """B_dev: (k, ld) with ld >= n; right-hand side c is row c (column c of the column-major block)."""
    if X_dev is None:
        X_dev = torch.empty_like(B_dev)
    k = B_dev.shape[0]
    infos = (vemg_info * max(k, 1))()
    rc = lib().vemg_solve_batch(h.h, k, _dev(B_dev), B_dev.stride(0), _dev(X_dev), X_dev.stride(0), rtol, max_it,
                                infos, _stream(stream))
    if rc not in (VEMG_OK, VEMG_ENOTCONV, VEMG_EBREAKDOWN):
        raise VemgError(rc, "vemg_solve_batch")
    return X_dev, [infos[i].as_dict() for i in range(k)]


def vemg_hierarchy_bytes(h: Hierarchy) -> int:
    v = C.c_size_t()
    _check(lib().vemg_hierarchy_bytes(h.h, C.byref(v)), "vemg_hierarchy_bytes")
    return int(v.value)


def vemg_selftest_barrier(claimed_blocks: int, launched_blocks: int, stream=None) -> int:
    """Status of one bounded grid-barrier wait: VEMG_OK or VEMG_ETIMEOUT (returned, not raised)."""
    return lib().vemg_selftest_barrier(claimed_blocks, launched_blocks, _stream(stream))


def vemg_solve_coefficients(h: Hierarchy):
    """(alpha, beta) numpy arrays of the last vemg_solve on h (FP64 V-cycles)."""
    cnt = C.c_int(0)
    lib().vemg_solve_coefficients(h.h, 0, None, None, C.byref(cnt))
    n = cnt.value
    a, b = np.zeros(max(n, 1)), np.zeros(max(n, 1))
    _check(lib().vemg_solve_coefficients(h.h, n, C.c_void_p(a.ctypes.data), C.c_void_p(b.ctypes.data),
                                         C.byref(cnt)), "vemg_solve_coefficients")
    return a[:n], b[:n]


def vemg_lanczos_extremes(alpha, beta):
    """(lambda_min, lambda_max) of the Lanczos tridiagonal of CG coefficients."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    lo, hi = C.c_double(), C.c_double()
    _check(lib().vemg_lanczos_extremes(C.c_void_p(a.ctypes.data), C.c_void_p(b.ctypes.data), len(a), C.byref(lo),
                                       C.byref(hi)), "vemg_lanczos_extremes")
    return lo.value, hi.value


def vemg_strerror(code: int) -> str:
    return lib().vemg_strerror(code).decode()


def vemg_get_size(h: Hierarchy, key: str, chain=1, level=0) -> int:
    v = C.c_int64()
    _check(lib().vemg_get_size(h.h, key.encode(), chain, level, C.byref(v)), "vemg_get_size")
    return int(v.value)


def vemg_get_csr(h: Hierarchy, name: str, chain=1, level=0):
    import scipy.sparse as sp
    n_, m_ = {"A": ("n", "n"), "E": ("n", "mtop"), "Ac": ("mtop", "mtop")}.get(name, (None, None))
    if n_:
        nrow, ncol = vemg_get_size(h, n_), vemg_get_size(h, m_)
    else:
        nrow = vemg_get_size(h, "lev.n", chain, level)
        ncol = nrow if name == "lev.A" else vemg_get_size(h, "lev.n", chain, level + 1)
    nnz = vemg_get_size(h, {"A": "nnzA", "E": "nnzE", "Ac": "nnzAc", "lev.A": "lev.nnz", "lev.P": "lev.nnzP"}[name],
                        chain, level)
    rp = np.zeros(nrow + 1, np.int32)
    ci = np.zeros(max(nnz, 1), np.int32)
    v = np.zeros(max(nnz, 1), np.float64)
    _check(lib().vemg_get_csr(h.h, name.encode(), chain, level, C.c_void_p(rp.ctypes.data),
                              C.c_void_p(ci.ctypes.data), C.c_void_p(v.ctypes.data)), f"vemg_get_csr({name})")
    return sp.csr_matrix((v[:nnz], ci[:nnz], rp), shape=(nrow, ncol))


def vemg_get_int(h: Hierarchy, name: str, chain=1, level=0) -> np.ndarray:
    cnt = vemg_get_size(h, "n") if name in ("new2old", "tri_of") else vemg_get_size(h, "lev.n", chain, level)
    out = np.zeros(max(cnt, 1), np.int32)
    _check(lib().vemg_get_int(h.h, name.encode(), chain, level, C.c_void_p(out.ctypes.data)),
           f"vemg_get_int({name})")
    return out[:cnt]


def vemg_get_nullspace(h: Hierarchy, chain=0, level=0) -> np.ndarray:
    """Near-nullspace rows (lev.n x 3) of a level of a chain built with surf_nullspace = 3."""
    cnt = vemg_get_size(h, "lev.n", chain, level)
    out = np.zeros((max(cnt, 1), 3))
    _check(lib().vemg_get_nullspace(h.h, chain, level, C.c_void_p(out.ctypes.data)), "vemg_get_nullspace")
    return out[:cnt]


BATCH_CLASSES = ("sweep", "cycle", "outer")


def vemg_batch_tuning(h: Hierarchy) -> dict:
    """Launch shapes the batched solves of this hierarchy use (after its first batched solve)."""
    K = C.c_int()
    kw, wp, us = (C.c_int * 3)(), (C.c_int * 3)(), (C.c_float * 3)()
    _check(lib().vemg_batch_tuning(h.h, C.byref(K), kw, wp, us), "vemg_batch_tuning")
    return {"K": K.value, **{c: {"lanes_per_row": kw[i], "warps_per_block": wp[i], "us_per_launch": us[i]}
                             for i, c in enumerate(BATCH_CLASSES)}}


def vemg_batch_set_tuning(h: Hierarchy, K: int, kw, warps, stream=None):
    a, b = (C.c_int * 3)(*kw), (C.c_int * 3)(*warps)
    _check(lib().vemg_batch_set_tuning(h.h, K, a, b, _stream(stream)), "vemg_batch_set_tuning")


def vemg_spmv(h: Hierarchy, x_dev, y_dev=None, stream=None):
    if y_dev is None:
        y_dev = torch.empty_like(x_dev)
    _check(lib().vemg_spmv(h.h, _dev(x_dev), _dev(y_dev), _stream(stream)), "vemg_spmv")
    return y_dev


def vemg_precond(h: Hierarchy, r_dev, z_dev=None, stream=None):
    if z_dev is None:
        z_dev = torch.empty_like(r_dev)
    _check(lib().vemg_precond(h.h, _dev(r_dev), _dev(z_dev), _stream(stream)), "vemg_precond")
    return z_dev


def vemg_vcycle(h: Hierarchy, chain: int, b_dev, x_dev=None, stream=None):
    if x_dev is None:
        x_dev = torch.empty_like(b_dev)
    _check(lib().vemg_vcycle(h.h, chain, _dev(b_dev), _dev(x_dev), _stream(stream)), "vemg_vcycle")
    return x_dev


# ------------------------------------------------------------------------------------------
# optional: route the library's device allocations through torch's caching allocator

_ALLOC_T = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_T = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


@_ALLOC_T
def _torch_alloc(nbytes, ctx):
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device())
    except Exception:
        return None


@_FREE_T
def _torch_free(ptr, ctx):
    torch.cuda.caching_allocator_delete(ptr)


def vemg_set_allocator(use_torch: bool = True):
    if use_torch:
        _check(lib().vemg_set_allocator(C.cast(_torch_alloc, C.c_void_p), C.cast(_torch_free, C.c_void_p), None),
               "vemg_set_allocator")
    else:
        _check(lib().vemg_set_allocator(None, None, None), "vemg_set_allocator")


def vemg_probe(h: Hierarchy, kind: int):
    _check(lib().vemg_probe(h.h, kind), "vemg_probe")


def vemg_probe_read(h: Hierarchy):
    ms, n, b = C.c_double(), C.c_int64(), C.c_double()
    _check(lib().vemg_probe_read(h.h, C.byref(ms), C.byref(n), C.byref(b)), "vemg_probe_read")
    return dict(ms=ms.value, launches=n.value, bytes=b.value)


PHASE_OPS = {0: "sor", 1: "residual", 2: "transfer", 3: "prolong_add", 4: "surface_restrict", 5: "dense"}


def vemg_probe_phases(h: Hierarchy):
    """Per-phase cycles of the persistent preconditioner since vemg_probe(h, VEMG_PROBE_VCYCLE):
    a list of dicts (op, level, group, cycles)."""
    cnt = C.c_int(0)
    lib().vemg_probe_phases(h.h, 0, C.byref(cnt), None, None, None, None)
    n = cnt.value
    if n == 0:
        return []
    op, lev, grp = (np.zeros(n, np.int32) for _ in range(3))
    cyc = np.zeros(n, np.float64)
    _check(lib().vemg_probe_phases(h.h, n, C.byref(cnt), C.c_void_p(op.ctypes.data), C.c_void_p(lev.ctypes.data),
                                   C.c_void_p(grp.ctypes.data), C.c_void_p(cyc.ctypes.data)), "vemg_probe_phases")
    return [dict(op=PHASE_OPS.get(int(op[k]), int(op[k])), level=int(lev[k]), group=int(grp[k]), cycles=float(cyc[k]))
            for k in range(n)]


def vemg_kernel_launches(h: Hierarchy) -> int:
    v = C.c_int64()
    _check(lib().vemg_kernel_launches(h.h, C.byref(v)), "vemg_kernel_launches")
    return int(v.value)


def vemg_spmv_static(h: Hierarchy, x_dev, y_dev=None, stream=None):
    """y = A x with no device allocation (work buffers in the library's static device array)."""
    if y_dev is None:
        y_dev = torch.empty_like(x_dev)
    rc = lib().vemg_spmv_static(h.h, _dev(x_dev), _dev(y_dev), _stream(stream))
    if rc != VEMG_OK:
        err = VemgError(rc, "vemg_spmv_static")
        err.detail = (lib().vemg_last_error() or b"").decode(errors="replace")
        raise err
    return y_dev


# ------------------------------------------------------------------------------------------
# continuous batching engine

VEMG_SLOT_FREE, VEMG_SLOT_RUNNING, VEMG_SLOT_DONE = 0, 1, 2


class Engine:
    """K right-hand-side slots of one hierarchy; requests join and leave between iterations."""

    def __init__(self, h: Hierarchy, slots: int, stream=None):
        self.hier = h
        self.stream = stream if stream is not None else torch.cuda.Stream()
        out = C.c_void_p()
        _check(lib().vemg_engine_create(h.h, slots, C.c_void_p(self.stream.cuda_stream), C.byref(out)),
               "vemg_engine_create")
        self.e = out
        n, f = C.c_int(), C.c_int()
        lib().vemg_engine_slots(self.e, C.byref(n), C.byref(f))
        self.slots = n.value

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "e", None) and self.e.value:
            lib().vemg_engine_destroy(self.e)
            self.e = C.c_void_p(None)

    def admit(self, b_dev: torch.Tensor, rtol=1e-8, max_it=1000) -> int:
        """The engine's stream reads b_dev: it first waits for the caller's current stream (where b
        was produced), and the caching allocator keeps b's memory until the engine's stream has
        passed the copy."""
        cur = torch.cuda.current_stream(b_dev.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)
            b_dev.record_stream(self.stream)
        slot = C.c_int()
        _check(lib().vemg_engine_admit(self.e, _dev(b_dev), rtol, max_it, C.byref(slot)), "vemg_engine_admit")
        return slot.value

    def launch(self, iters=1):
        _check(lib().vemg_engine_launch(self.e, iters), "vemg_engine_launch")

    def wait(self):
        _check(lib().vemg_engine_wait(self.e), "vemg_engine_wait")

    def query(self) -> bool:
        """True when the engine's stream has completed its enqueued work (no waiting)."""
        busy = C.c_int()
        _check(lib().vemg_engine_query(self.e, C.byref(busy)), "vemg_engine_query")
        return busy.value == 0

    def poll(self, slot):
        info, st = vemg_info(), C.c_int()
        _check(lib().vemg_engine_poll(self.e, slot, C.byref(info), C.byref(st)), "vemg_engine_poll")
        return st.value, info.as_dict()

    def retire(self, slot, x_dev: torch.Tensor):
        """x_dev is written on the engine's stream, which the call synchronises; it first waits for
        the caller's stream, where x_dev was allocated."""
        cur = torch.cuda.current_stream(x_dev.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)
        _check(lib().vemg_engine_retire(self.e, slot, _dev(x_dev)), "vemg_engine_retire")

    def free_slots(self) -> int:
        n, f = C.c_int(), C.c_int()
        _check(lib().vemg_engine_slots(self.e, C.byref(n), C.byref(f)), "vemg_engine_slots")
        return f.value

    def bytes(self) -> int:
        v = C.c_size_t()
        _check(lib().vemg_engine_bytes(self.e, C.byref(v)), "vemg_engine_bytes")
        return int(v.value)
