"""The device adjacency build of sls_mesh_create against the host build.

Both builds must give the same mesh (free-node count, bounding-box diagonal)
and, since the summation order and the triangle codes decide every bit of a
pass, bit-identical smoothing results.  Bad meshes must be rejected with the
same status and message either way.
"""
import ctypes as C

import numpy as np
import pytest

import meshgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1502_00355_gb300 as mod
    mod.build()
    mod.lib()
    return mod


def _smooth(sls, mesh, host_build, iters=12, bnd="given", **opts):
    b = mesh.boundary if bnd == "given" else None
    with sls.Mesh(mesh.xy, mesh.tri, b, host_build=host_build, record_accept=True, **opts) as g:
        stats = (g.n, g.m, g.n_free, g.diag)
        info = g.smooth(iters)
        return stats, g.coords(), g.accept_mask(), info


def _meshes():
    yield "small", meshgen.small_grid()
    yield "random-numbering", meshgen.jittered_grid(97, 61, 0.4, 5, numbering="random", perm_seed=9)
    yield "uniform-diagonals", meshgen.jittered_grid(40, 33, 0.3, 6, diagonals="uniform")
    # negative and mixed-sign coordinates, and a -0.0 on the bounding box
    m = meshgen.jittered_grid(50, 50, 0.3, 7)
    xy = m.xy * np.array([3.0, -0.5]) - np.array([1.5, 0.0])
    xy[0] = [-1.5, -0.0]
    yield "signed", meshgen.Mesh(xy=xy, tri=m.tri, boundary=m.boundary)
    # an isolated node (no triangle) and a node in 40 triangles (host fallback)
    k = 40
    ang = np.linspace(0, 2 * np.pi, k, endpoint=False)
    fxy = np.vstack([np.c_[np.cos(ang), np.sin(ang)], [[0.05, -0.02]], [[5.0, 5.0]]])
    ftri = np.array([[k, j, (j + 1) % k] for j in range(k)], dtype=np.int32)
    yield "fan-40+isolated", meshgen.Mesh(xy=fxy, tri=ftri, boundary=None)


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("bnd", ["given", "derived"])
def test_device_build_matches_host_build(sls, layout, bnd):
    for name, mesh in _meshes():
        if mesh.boundary is None and bnd == "given":
            continue
        d = _smooth(sls, mesh, False, bnd=bnd, layout=layout)
        h = _smooth(sls, mesh, True, bnd=bnd, layout=layout)
        assert d[0] == h[0], name
        assert np.array_equal(d[1], h[1]), name
        assert np.array_equal(d[2], h[2]), name
        assert d[3] == h[3], name


def test_device_build_matches_oracle_on_medium_grid(sls):
    mesh = meshgen.medium_grid(numbering="random")
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary, openmp=True)
    ref_xy, ref_info, _ = om.smooth(mesh.xy, 6)
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary) as g:
        info = g.smooth(6)
        assert np.array_equal(g.coords(), ref_xy)
    assert info["accepted_last"] == ref_info["accepted_last"]
    assert info["maxd2_last"] == ref_info["maxd2_last"]


def _create(L, sls, xy, tri, host_build):
    xy = np.ascontiguousarray(xy, np.float64)
    tri = np.ascontiguousarray(tri, np.int32)
    h = C.c_void_p()
    opt = sls.make_options(host_build=host_build)
    st = L.sls_mesh_create(xy.ctypes.data_as(C.c_void_p), xy.shape[0], tri.ctypes.data_as(C.c_void_p),
                           tri.shape[0], None, C.byref(opt), C.byref(h))
    if st == 0:
        L.sls_mesh_destroy(h)
    return st, L.sls_last_error().decode()


def test_device_build_rejects_like_host_build(sls):
    L = sls.lib()
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0], [0.5, -1.0]])
    nan = xy.copy()
    nan[3, 1] = np.nan
    inf = xy.copy()
    inf[1, 0] = -np.inf
    cases = [
        (xy, [[0, 1, 2], [1, 3, 2], [0, 1, 5]]),          # id out of range
        (xy, [[0, 1, 2], [0, -1, 2]]),                    # negative id
        (xy, [[0, 1, 2], [1, 3, 3], [4, 9, 4]]),          # repeat before a range error
        (xy, [[4, 9, 4], [1, 3, 3]]),                     # both errors in one triangle
        (nan, [[0, 1, 2]]),
        (inf, [[0, 1, 7]]),                               # coordinates are checked first
        (xy, [[0, 1, 2], [1, 0, 3], [0, 1, 4]]),          # non-manifold edge
        (xy, [[0, 1, 2], [1, 3, 2]]),                     # valid
    ]
    for xyc, tri in cases:
        got = _create(L, sls, xyc, tri, False)
        want = _create(L, sls, xyc, tri, True)
        assert got[0] == want[0], (tri, got, want)
        if want[0] != 0:
            assert got[1] == want[1], (tri, got, want)
