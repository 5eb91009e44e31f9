"""Seeded synthetic inputs: thin extruded tetrahedral meshes and right-hand sides.

This module is the only code shared by the CUDA path and the CPU oracle. It
builds geometry and random loads; it holds none of the solver's arithmetic
(no element matrices, no operators, no preconditioner).

The paper's own meshes (a Delaunay mesh of 57,453 points and a clustered
mesh of 99,017 points in the unit cube, rescaled to various aspect ratios,
section 6) are not available; these generators stand in for them with
structured hex meshes split into tetrahedra and jittered so that the layers
are not aligned (z-jitter) or the mesh is unstructured in the horizontal
as well (xy-jitter).

Geometry (section 2.1): z points up, the top surface is z = 0, the floor is
z = -H(x, y), the coasts are the vertical walls x in {0, 1}, y in {0, 1}.

Node numbering is column-major: node id = col * (nz + 1) + k with
col = j * (nx + 1) + i, and k = 0 on the top surface, k = nz on the floor.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TAG_TOP = 1
TAG_FLOOR = 2
TAG_COAST = 4


@dataclasses.dataclass
class Mesh:
    xyz: np.ndarray        # (n, 3) float64
    tets: np.ndarray       # (ne, 4) int32, positive orientation
    tags: np.ndarray       # (n,) uint8 bitmask TOP=1 FLOOR=2 COAST=4
    top_tris: np.ndarray   # (nt, 3) int32 node ids of top nodes, counter-clockwise in (x, y)
    nx: int
    ny: int
    nz: int
    redraw_passes: int = 0

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_top(self) -> int:
        return int(np.count_nonzero(self.tags & TAG_TOP))


def _uniform_pm1(rng: np.random.Generator, size: int) -> np.ndarray:
    """Uniform draws in [-1, 1) built from raw 64-bit outputs with exact arithmetic only,
    so that the values are bit-identical on every platform."""
    raw = rng.bit_generator.random_raw(size)
    u = (raw >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)  # [0, 1), exact
    return u * 2.0 - 1.0                                                        # exact


def depth_flat(h0: float):
    return lambda x, y: np.full_like(x, h0)


def depth_sines(h0: float):
    """H(x, y) = h0 * (1 + 0.5 sin(2 pi x) sin(2 pi y))."""
    return lambda x, y: h0 * (1.0 + 0.5 * np.sin(2.0 * np.pi * x) * np.sin(2.0 * np.pi * y))


def _kuhn_tets():
    """The 6 Kuhn tetrahedra of the unit hex as corner offsets (a, b, c) along (i, j, k):
    (v0, v0 + e_s1, v0 + e_s1 + e_s2, v7) for each permutation s of the three axes."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        c = [np.zeros(3, dtype=np.int64)]
        for ax in perm:
            nxt = c[-1].copy()
            nxt[ax] += 1
            c.append(nxt)
        out.append(c)
    return out


def _tet_volumes6(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Six times the signed volume of each tetrahedron (validity check of the generator)."""
    p0 = xyz[tets[:, 0]]
    d1 = xyz[tets[:, 1]] - p0
    d2 = xyz[tets[:, 2]] - p0
    d3 = xyz[tets[:, 3]] - p0
    return np.einsum("ij,ij->i", d1, np.cross(d2, d3))


def _cluster_map(t: np.ndarray, c: float):
    """Monotone map of [0, 1] onto itself (for 0 <= c < 1) whose slope is 1 - c at t = 1/2 and
    1 + c at the ends: grid points crowd towards the centre. Returns (map, slope)."""
    w = 2.0 * np.pi * t
    return t + c * np.sin(w) / (2.0 * np.pi), 1.0 + c * np.cos(w)


def make_mesh(nx: int, ny: int, nz: int, depth, *, z_jitter: float = 0.0,
              xy_jitter: float = 0.0, seed: int = 0, max_passes: int = 100, cluster: float = 0.0) -> Mesh:
    """Extruded hex mesh of the unit square x [-H(x,y), 0], each hex split into 6 Kuhn tets.

    cluster: 0 <= c < 1. The grid coordinates i/nx, j/ny and the layer fraction k/nz pass through
      a monotone map whose spacing shrinks by a factor (1 - c)/(1 + c) from the edges to the
      centre: a multiscale mesh with small elements at the centre of the domain (the clustered
      mesh of section 6). Jitter amplitudes below are scaled by the local spacing.

    z_jitter: nodes strictly between top and floor move vertically by
      U(-z_jitter, z_jitter) times the local layer thickness H(x, y) / nz.
    xy_jitter: nodes off the coast (0 < i < nx, 0 < j < ny), on every layer,
      move horizontally by U(-xy_jitter, xy_jitter) times the grid spacing,
      each node independently. Depths are evaluated at the moved position.
    Tets of non-positive volume have the jitter of their non-coast vertices
      redrawn, pass by pass, from a fresh stream seeded (seed, pass).
    """
    ncol = (nx + 1) * (ny + 1)
    n = ncol * (nz + 1)
    nid = np.arange(n, dtype=np.int64)
    k = nid % (nz + 1)
    col = nid // (nz + 1)
    i = col % (nx + 1)
    j = col // (nx + 1)
    if not (0.0 <= cluster < 1.0):
        raise ValueError("cluster must lie in [0, 1)")
    x0, sx = _cluster_map(i.astype(np.float64) / nx, cluster)
    y0, sy = _cluster_map(j.astype(np.float64) / ny, cluster)
    zeta, sz = _cluster_map(k.astype(np.float64) / nz, cluster)

    tags = np.zeros(n, dtype=np.uint8)
    tags[k == 0] |= TAG_TOP
    tags[k == nz] |= TAG_FLOOR
    coast = (i == 0) | (i == nx) | (j == 0) | (j == ny)
    tags[coast] |= TAG_COAST

    movable_xy = (~coast) if xy_jitter > 0.0 else np.zeros(n, dtype=bool)
    movable_z = ((k > 0) & (k < nz)) if z_jitter > 0.0 else np.zeros(n, dtype=bool)

    rng = np.random.Generator(np.random.PCG64(seed))
    jx = _uniform_pm1(rng, n)
    jy = _uniform_pm1(rng, n)
    jz = _uniform_pm1(rng, n)

    def coords(jx, jy, jz):
        x = np.where(movable_xy, x0 + xy_jitter * jx * (sx / nx), x0)
        y = np.where(movable_xy, y0 + xy_jitter * jy * (sy / ny), y0)
        h = depth(x, y)
        z = -h * zeta
        z = np.where(movable_z, z + z_jitter * jz * (h * sz / nz), z)
        z = np.where(k == 0, 0.0, z)
        return np.stack([x, y, z], axis=1)

    # tets: hex (i, j, k) has corners (i + a, j + b, k + c)
    kt = _kuhn_tets()
    hi, hj, hk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()
    # order hexes column-major like the nodes: (j, i) column, then k downwards
    order = np.lexsort((hk, hi, hj))
    hi, hj, hk = hi[order], hj[order], hk[order]
    tet_list = []
    for corners in kt:
        verts = [((hj + c[1]) * (nx + 1) + (hi + c[0])) * (nz + 1) + (hk + c[2]) for c in corners]
        tet_list.append(np.stack(verts, axis=1))
    tets = np.stack(tet_list, axis=1).reshape(-1, 4)
    # orient on the unjittered geometry (k grows downwards)
    ref = np.stack([x0, y0, -(k.astype(np.float64) / nz)], axis=1)
    neg = _tet_volumes6(ref, tets) < 0.0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    tets = tets.astype(np.int32)

    xyz = coords(jx, jy, jz)
    passes = 0
    while True:
        bad = _tet_volumes6(xyz, tets) <= 0.0
        if not bad.any():
            break
        passes += 1
        if passes > max_passes:
            raise RuntimeError("mesh generator: tets with non-positive volume remain after redraw passes")
        redo = np.zeros(n, dtype=bool)
        redo[tets[bad].ravel()] = True
        redo &= ~coast
        r2 = np.random.Generator(np.random.PCG64([seed, passes]))
        jx = np.where(redo, _uniform_pm1(r2, n), jx)
        jy = np.where(redo, _uniform_pm1(r2, n), jy)
        jz = np.where(redo, _uniform_pm1(r2, n), jz)
        xyz = coords(jx, jy, jz)

    # top triangulation: each top quad split along its (0,0)-(1,1) diagonal, counter-clockwise
    qi, qj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    qi, qj = qi.T.ravel(), qj.T.ravel()   # quad q = j * nx + i
    def top(ii, jj):
        return (jj * (nx + 1) + ii) * (nz + 1)
    v00, v10, v11, v01 = top(qi, qj), top(qi + 1, qj), top(qi + 1, qj + 1), top(qi, qj + 1)
    tris = np.stack([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 1).reshape(-1, 3)
    return Mesh(xyz=np.ascontiguousarray(xyz), tets=np.ascontiguousarray(tets), tags=tags,
                top_tris=np.ascontiguousarray(tris.astype(np.int32)), nx=nx, ny=ny, nz=nz,
                redraw_passes=passes)


# ---------------------------------------------------------------------------
# right-hand sides

def manufactured_f(mesh: Mesh, h0: float) -> np.ndarray:
    """Nodal values of f = -Laplace(u) for u = cos(pi x) cos(pi y) cos(pi z / h0) on a flat box of
    depth h0: f = pi^2 (2 + 1/h0^2) u. u satisfies the homogeneous Neumann condition on every face."""
    x, y, z = mesh.xyz[:, 0], mesh.xyz[:, 1], mesh.xyz[:, 2]
    return (math.pi ** 2) * (2.0 + 1.0 / h0 ** 2) * manufactured_u(mesh, h0)


def manufactured_u(mesh: Mesh, h0: float) -> np.ndarray:
    x, y, z = mesh.xyz[:, 0], mesh.xyz[:, 1], mesh.xyz[:, 2]
    return np.cos(math.pi * x) * np.cos(math.pi * y) * np.cos(math.pi * z / h0)


def normal_loads(n: int, seed: int, k: int = 1) -> np.ndarray:
    """i.i.d. N(0, 1) nodal loads, shape (n,) for k == 1 else (k, n) (one row per right-hand side)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    b = rng.standard_normal((k, n))
    return b[0] if k == 1 else b


# ---------------------------------------------------------------------------
# named workloads (sizes and value distributions of the thin-domain configurations)

WORKLOADS = {
    # 16x16x8, flat depth 0.01 (aspect ratio 1e-2), manufactured right-hand side, rtol 1e-10
    "box16": dict(nx=16, ny=16, nz=8, depth=("flat", 0.01), z_jitter=0.0, xy_jitter=0.0,
                  seed=1000, rhs="manufactured", rtol=1e-10),
    # 256x256x32, H = 1e-3 (1 + 0.5 sin sin), z-jitter 0.3, N(0,1) loads, rtol 1e-8
    "zjit256": dict(nx=256, ny=256, nz=32, depth=("sines", 1e-3), z_jitter=0.3, xy_jitter=0.0,
                    seed=2000, rhs="normal", rtol=1e-8),
    # 192x192x48, H = 1e-4 (1 + 0.5 sin sin), z-jitter 0.3 and xy-jitter 0.2, rtol 1e-8
    "xyjit192": dict(nx=192, ny=192, nz=48, depth=("sines", 1e-4), z_jitter=0.3, xy_jitter=0.2,
                     seed=3000, rhs="normal", rtol=1e-8),
    # 384x384x24, H = 1e-3 (1 + 0.5 sin sin), z-jitter 0.3, 64 right-hand sides
    "zjit384x64": dict(nx=384, ny=384, nz=24, depth=("sines", 1e-3), z_jitter=0.3, xy_jitter=0.0,
                       seed=4000, rhs="normal", nrhs=64, rtol=1e-8),
    # multiscale stand-in for the clustered mesh of section 6: 128x128x24 with spacing 19x finer at
    # the centre than at the edges (horizontally and vertically), z-jitter 0.3, H = 1e-3 (...)
    "cluster128": dict(nx=128, ny=128, nz=24, depth=("sines", 1e-3), z_jitter=0.3, xy_jitter=0.0,
                       cluster=0.9, seed=6000, rhs="normal", rtol=1e-8),
}


def depth_fn(spec):
    kind, h0 = spec
    return depth_flat(h0) if kind == "flat" else depth_sines(h0)


def make_workload_mesh(name: str, **over) -> Mesh:
    w = dict(WORKLOADS[name])
    w.update(over)
    return make_mesh(w["nx"], w["ny"], w["nz"], depth_fn(w["depth"]), z_jitter=w["z_jitter"],
                     xy_jitter=w["xy_jitter"], seed=w["seed"], cluster=w.get("cluster", 0.0))


def scale_depth(mesh: Mesh, factor: float) -> Mesh:
    """The same mesh with every depth multiplied by `factor`. The generator's z coordinates (layers
    and z-jitter) are all proportional to the depth scale, so a mesh generated with depth scale 1
    and scaled by eps is the mesh generated with depth scale eps."""
    xyz = mesh.xyz.copy()
    xyz[:, 2] *= factor
    return Mesh(xyz=xyz, tets=mesh.tets, tags=mesh.tags, top_tris=mesh.top_tris, nx=mesh.nx, ny=mesh.ny,
                nz=mesh.nz, redraw_passes=mesh.redraw_passes)
