"""Seeded synthetic triangle meshes for 2-D Smart Laplacian smoothing.

This module only *generates inputs*: coordinates, triangles, boundary flags and
node numberings.  It holds none of the smoothing arithmetic, so the oracle and
the CUDA library can both consume its output without sharing any of the
method's code.

The paper measures on Delaunay triangulations of uniformly random points
(Section 4), made with a generator and Triangle that are not available here.
``delaunay_random`` rebuilds that family with Qhull; structured jittered grids
of the same kind (planar, valence about 6, interior nodes free, the outer ring
fixed) serve for the large workloads:

* an ``nx x ny`` vertex grid with spacing ``h = 1/(ny-1)``;
* every quad split along one of its two diagonals (a seeded coin per quad, or
  the same diagonal everywhere);
* interior nodes displaced by ``U(-J*h, J*h)`` independently in x and y;
* optionally a fraction of interior nodes pulled towards the nearest of a set
  of seeded centres (clustered, skewed and sometimes inverted triangles);
* node numbering natural (row-major), Morton (Z-order of the grid indices) or
  a seeded random permutation.  Triangles keep their vertex order under
  renumbering.

``fast_grid`` makes grids of the same construction in C (``fastgrid.c``,
built by ``build()``) with a counter-based generator, for request streams too
large to generate with numpy ahead of time; its meshes are of the same kind
as ``jittered_grid``'s, not the same meshes.
"""
from __future__ import annotations

import ctypes as _C
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_FAST_SRC = os.path.join(_HERE, "fastgrid.c")
_FAST_LIB = os.path.join(_HERE, "_build", "libfastgrid.so")
_fast = None
_fast_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compiles fastgrid.c into _build/libfastgrid.so (portable C, no
    machine-specific flags)."""
    os.makedirs(os.path.dirname(_FAST_LIB), exist_ok=True)
    if force or not os.path.exists(_FAST_LIB) or os.path.getmtime(_FAST_LIB) < os.path.getmtime(_FAST_SRC):
        tmp = _FAST_LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _FAST_SRC, "-o", tmp], check=True)
        os.replace(tmp, _FAST_LIB)
    return _FAST_LIB


def _fastlib():
    global _fast
    with _fast_lock:
        if _fast is None:
            build()
            L = _C.CDLL(_FAST_LIB)
            L.fastgrid.restype = _C.c_int
            L.fastgrid.argtypes = [_C.c_int64, _C.c_int64, _C.c_double, _C.c_double, _C.c_uint64, _C.c_int,
                                   _C.c_void_p, _C.c_void_p, _C.c_void_p]
            _fast = L
        return _fast

BASE_SEED = 150200355


@dataclass
class Mesh:
    xy: np.ndarray          # (n, 2) float64, node coordinates
    tri: np.ndarray         # (m, 3) int32, vertex ids in stored (CCW before jitter) order
    boundary: np.ndarray    # (n,) uint8, 1 = fixed node
    nx: int = 0
    ny: int = 0
    perm: np.ndarray | None = None   # natural grid id -> node id
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xy.shape[0])

    @property
    def m(self) -> int:
        return int(self.tri.shape[0])


def _part1by1(v: np.ndarray) -> np.ndarray:
    v = v.astype(np.uint64) & np.uint64(0xFFFFFFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x0000FFFF0000FFFF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF00FF00FF)
    v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F0F0F0F0F)
    v = (v | (v << np.uint64(2))) & np.uint64(0x3333333333333333)
    v = (v | (v << np.uint64(1))) & np.uint64(0x5555555555555555)
    return v


def morton_order(i: np.ndarray, j: np.ndarray) -> np.ndarray:
    """Return node ids such that ids sorted ascending follow the Z-order curve of (i, j)."""
    code = _part1by1(i) | (_part1by1(j) << np.uint64(1))
    order = np.argsort(code, kind="stable")
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size, dtype=order.dtype)
    return rank


def grid_triangles(nx: int, ny: int, diag: np.ndarray) -> np.ndarray:
    """Two triangles per quad; ``diag[q]`` picks the diagonal of quad q (row-major over quads)."""
    qi, qj = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), indexing="xy")
    qi = qi.ravel().astype(np.int64)
    qj = qj.ravel().astype(np.int64)
    v00 = qj * nx + qi
    v10 = v00 + 1
    v01 = v00 + nx
    v11 = v01 + 1
    d = diag.astype(bool)
    t0 = np.where(d[:, None], np.stack([v00, v10, v01], 1), np.stack([v00, v10, v11], 1))
    t1 = np.where(d[:, None], np.stack([v10, v11, v01], 1), np.stack([v00, v11, v01], 1))
    tri = np.empty((2 * qi.size, 3), dtype=np.int64)
    tri[0::2] = t0
    tri[1::2] = t1
    return tri


def jittered_grid(nx: int, ny: int, jitter: float, seed: int, *, h: float | None = None,
                  diagonals: str = "random", numbering: str = "morton",
                  pull_fraction: float = 0.0, pull_centres: int = 1024,
                  perm_seed: int | None = None) -> Mesh:
    """Jittered structured triangulation.

    ``h`` defaults to ``1/(ny-1)``; a dyadic ``h`` (e.g. 1.0 or 2**-k) with
    ``jitter=0`` gives coordinates that are exact binary fractions.
    ``diagonals``: "random" (seeded coin per quad) or "uniform" (all quads split
    v00-v11).  ``numbering``: "natural", "morton" or "random".
    """
    if nx < 2 or ny < 2:
        raise ValueError("grid needs at least 2x2 vertices")
    rng = np.random.Generator(np.random.PCG64(seed))
    if h is None:
        h = 1.0 / (ny - 1)
    gi, gj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    gi = gi.ravel()
    gj = gj.ravel()
    n = nx * ny
    x = gi.astype(np.float64) * h
    y = gj.astype(np.float64) * h
    bnd = ((gi == 0) | (gi == nx - 1) | (gj == 0) | (gj == ny - 1)).astype(np.uint8)
    nq = (nx - 1) * (ny - 1)
    if diagonals == "random":
        diag = rng.integers(0, 2, size=nq)
    elif diagonals == "uniform":
        diag = np.zeros(nq, dtype=np.int64)
    else:
        raise ValueError(diagonals)
    if jitter > 0.0:
        jx = rng.uniform(-jitter * h, jitter * h, size=n)
        jy = rng.uniform(-jitter * h, jitter * h, size=n)
        free = bnd == 0
        x = np.where(free, x + jx, x)
        y = np.where(free, y + jy, y)
    if pull_fraction > 0.0:
        interior = np.flatnonzero(bnd == 0)
        k = int(round(pull_fraction * interior.size))
        chosen = rng.choice(interior, size=k, replace=False)
        cx = rng.uniform(0.0, (nx - 1) * h, size=pull_centres)
        cy = rng.uniform(0.0, (ny - 1) * h, size=pull_centres)
        lam = rng.uniform(0.25, 0.75, size=k)
        px = x[chosen]
        py = y[chosen]
        best = np.full(k, np.inf)
        bx = np.zeros(k)
        by = np.zeros(k)
        for c0 in range(0, pull_centres, 64):
            dx = cx[None, c0:c0 + 64] - px[:, None]
            dy = cy[None, c0:c0 + 64] - py[:, None]
            d2 = dx * dx + dy * dy
            a = np.argmin(d2, axis=1)
            v = d2[np.arange(k), a]
            better = v < best
            best = np.where(better, v, best)
            bx = np.where(better, cx[c0 + a], bx)
            by = np.where(better, cy[c0 + a], by)
        sx = lam * (bx - px)
        sy = lam * (by - py)
        step = np.sqrt(sx * sx + sy * sy)
        cap = 2.0 * h
        scale = np.where(step > cap, cap / np.maximum(step, 1e-300), 1.0)
        x[chosen] = px + sx * scale
        y[chosen] = py + sy * scale
    tri_nat = grid_triangles(nx, ny, diag)
    if numbering == "natural":
        perm = np.arange(n, dtype=np.int64)
    elif numbering == "morton":
        perm = morton_order(gi, gj).astype(np.int64)
    elif numbering == "random":
        prng = np.random.Generator(np.random.PCG64(seed + 7919 if perm_seed is None else perm_seed))
        perm = prng.permutation(n).astype(np.int64)
    else:
        raise ValueError(numbering)
    xy = np.empty((n, 2), dtype=np.float64)
    xy[perm, 0] = x
    xy[perm, 1] = y
    boundary = np.empty(n, dtype=np.uint8)
    boundary[perm] = bnd
    tri = perm[tri_nat].astype(np.int32)
    return Mesh(xy=xy, tri=tri, boundary=boundary, nx=nx, ny=ny, perm=perm,
                meta=dict(nx=nx, ny=ny, h=h, jitter=jitter, seed=seed, diagonals=diagonals,
                          numbering=numbering, pull_fraction=pull_fraction))


def delaunay_random(n: int, seed: int, *, numbering: str = "morton", perm_seed: int | None = None) -> Mesh:
    """Delaunay triangulation of ``n`` seeded uniform random points in the unit
    square: the paper's mesh family (Section 4), made with Qhull through
    ``scipy.spatial.Delaunay`` in place of the paper's generator and Triangle.

    Triangles are stored counter-clockwise; the convex-hull vertices are the
    fixed nodes (points Qhull leaves out of every triangle, if any, are fixed
    too).  Interior valence ranges from 3 to about 12.  ``numbering``: "natural"
    (generation order), "morton" (Z-order of the points on a 2^16 grid) or
    "random"; ``perm`` maps generation order to node id.
    """
    from scipy.spatial import Delaunay

    if n < 3:
        raise ValueError("need at least 3 points")
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.uniform(0.0, 1.0, size=(n, 2))
    dt = Delaunay(pts)
    tri_nat = dt.simplices.astype(np.int64)
    a, b, c = pts[tri_nat[:, 0]], pts[tri_nat[:, 1]], pts[tri_nat[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    cw = cross < 0
    tri_nat[cw, 1], tri_nat[cw, 2] = tri_nat[cw, 2].copy(), tri_nat[cw, 1].copy()
    bnd = np.ones(n, dtype=np.uint8)
    bnd[np.unique(tri_nat)] = 0
    bnd[np.unique(dt.convex_hull)] = 1
    if numbering == "natural":
        perm = np.arange(n, dtype=np.int64)
    elif numbering == "morton":
        q = np.minimum((pts * 65536.0).astype(np.int64), 65535)
        perm = morton_order(q[:, 0], q[:, 1]).astype(np.int64)
    elif numbering == "random":
        prng = np.random.Generator(np.random.PCG64(seed + 7919 if perm_seed is None else perm_seed))
        perm = prng.permutation(n).astype(np.int64)
    else:
        raise ValueError(numbering)
    xy = np.empty((n, 2), dtype=np.float64)
    xy[perm] = pts
    boundary = np.empty(n, dtype=np.uint8)
    boundary[perm] = bnd
    tri = perm[tri_nat].astype(np.int32)
    return Mesh(xy=xy, tri=tri, boundary=boundary, perm=perm,
                meta=dict(kind="delaunay", n=n, seed=seed, numbering=numbering))


def fast_grid(nx: int, ny: int, jitter: float, seed: int, *, numbering: str = "morton",
              h: float | None = None) -> Mesh:
    """Jittered grid made by fastgrid.c: the construction of ``jittered_grid``
    (random diagonals, interior jitter U(-J h, J h), outer ring fixed, Morton
    or natural numbering) with counter-based random numbers.  Releases the GIL
    while it works, so threads can make several meshes at once."""
    if numbering not in ("morton", "natural"):
        raise ValueError(numbering)
    if h is None:
        h = 1.0 / (ny - 1)
    n, m = nx * ny, 2 * (nx - 1) * (ny - 1)
    xy = np.empty((n, 2), np.float64)
    tri = np.empty((m, 3), np.int32)
    boundary = np.empty(n, np.uint8)
    rc = _fastlib().fastgrid(nx, ny, float(jitter), float(h), seed & 0xFFFFFFFFFFFFFFFF,
                             1 if numbering == "morton" else 0, xy.ctypes.data, tri.ctypes.data,
                             boundary.ctypes.data)
    if rc != 0:
        raise ValueError(f"fastgrid failed for {nx}x{ny}")
    return Mesh(xy=xy, tri=tri, boundary=boundary, nx=nx, ny=ny,
                meta=dict(kind="fast_grid", nx=nx, ny=ny, h=h, jitter=jitter, seed=seed, numbering=numbering))


def unpermute(xy: np.ndarray, mesh: Mesh) -> np.ndarray:
    """Coordinates back in natural (row-major grid) order."""
    return xy[mesh.perm]


# --- the workloads ---------------------------------------------------------

def small_grid() -> Mesh:
    """64x64 vertices (4,096 nodes, 7,938 triangles), jitter 0.3h, Morton numbering."""
    return jittered_grid(64, 64, 0.3, BASE_SEED + 1, numbering="morton")


def medium_grid(numbering: str = "morton") -> Mesh:
    """1024x1024 vertices (1,048,576 nodes, 2,093,058 triangles), jitter 0.35h."""
    return jittered_grid(1024, 1024, 0.35, BASE_SEED + 2, numbering=numbering)


def large_grid(nx: int = 4096, ny: int = 4096) -> Mesh:
    """4096x4096 vertices (16,777,216 nodes, 33,538,050 triangles), jitter 0.35h,
    5% of interior nodes pulled towards the nearest of 1,024 seeded centres."""
    return jittered_grid(nx, ny, 0.35, BASE_SEED + 3, numbering="morton", pull_fraction=0.05)


def delaunay_mesh(n: int = 100_000) -> Mesh:
    """The paper's largest workload: a Delaunay mesh of 100,000 uniform random
    points, Morton numbering."""
    return delaunay_random(n, BASE_SEED + 4, numbering="morton")


def batch_specs(k: int = 2048, lo: int = 1024, hi: int = 262144, seed: int = BASE_SEED + 1000):
    """Per-mesh (nx, ny, iterations, seed) for the batched workload: node counts
    log-uniform in [lo, hi], aspect ratio uniform in [1, 4], iterations uniform in [10, 100]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for r in range(k):
        nk = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        a = rng.uniform(1.0, 4.0)
        ny = max(2, int(round(math.sqrt(nk / a))))
        nx = max(2, int(round(nk / ny)))
        iters = int(rng.integers(10, 101))
        out.append((nx, ny, iters, seed + r))
    return out


def batch_mesh(spec) -> Mesh:
    nx, ny, _iters, s = spec
    return jittered_grid(nx, ny, 0.3, s, numbering="morton")


def serve_requests(count: int = 10000, rate: float = 2000.0, lo: int = 1024, hi: int = 4 * 1024 * 1024,
                   seed: int = BASE_SEED + 5):
    """Poisson arrivals: per request (arrival_s, nx, ny, cap, mesh_seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for r in range(count):
        nk = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        side = max(2, int(round(math.sqrt(nk))))
        cap = int(rng.integers(10, 201))
        out.append((float(t[r]), side, side, cap, BASE_SEED + 10000 + r))
    return out


def edge_case_meshes() -> list[Mesh]:
    """Small meshes at the edges of the method, for parity tests: a single
    triangle (every node on the boundary; flags left to be derived), a grid
    with free nodes moved exactly onto a neighbour or onto the midpoint of
    the opposite edge (zero-length edges, triangles collapsed to a point or a
    segment, inverted triangles), a free node in 40 triangles, and an ordinary
    grid (twice)."""
    one = Mesh(xy=np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), tri=np.array([[0, 1, 2]], np.int32),
               boundary=None)
    deg = jittered_grid(25, 19, 0.3, BASE_SEED + 20, numbering="morton")
    xy = deg.xy.copy()
    free = deg.boundary == 0
    rng = np.random.default_rng(BASE_SEED + 21)
    for k, t in enumerate(rng.choice(deg.m, 40, replace=False)):
        a, b, c = deg.tri[t]
        if not free[a]:
            continue
        if k % 3 == 0:
            xy[a] = xy[b]
        elif k % 3 == 1:
            xy[a] = 0.5 * (xy[b] + xy[c])
        else:
            xy[a] = xy[b]
            if free[c]:
                xy[c] = xy[b]
    deg.xy = xy
    k = 40
    ang = np.linspace(0.0, 2.0 * np.pi, k, endpoint=False)
    ring = np.c_[np.cos(ang) * (1.0 + 0.3 * np.sin(5.0 * ang)), np.sin(ang)]
    fan = Mesh(xy=np.vstack([ring, [[0.05, -0.02]]]),
               tri=np.array([[k, j, (j + 1) % k] for j in range(k)], dtype=np.int32),
               boundary=(np.arange(k + 1) < k).astype(np.uint8))
    grid = jittered_grid(31, 17, 0.35, BASE_SEED + 22, numbering="random")
    return [one, deg, fan, grid, grid]
