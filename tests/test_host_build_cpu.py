"""The library's host adjacency build (csrc/mesh_build.cpp, Sections 3.3.2 and
3.3.3), compiled on its own with g++ and checked word by word against the
oracle's neighbour sets, summation order and constraints.  No GPU: the
library's own entry points upload right after building, so this test calls
the build function directly through a small C shim.

Per node the stream holds a meta word (fixed bit, triangle count, degree);
for a free node, then, its neighbours in summation order and one code per
incident triangle (ascending triangle ids): the node's slot in the stored
triangle and the positions, in the neighbour list, of the other two vertices
in stored order."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import meshgen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1502_00355_gb300", "csrc")

SHIM = r"""
#include <cstring>
#include <string>
#include "internal.h"
namespace sls {
void set_error(const std::string &) {}
sls_status fail(sls_status code, const std::string &) { return code; }
}
extern "C" int hb_build(const double *xy, long long n, const int *tri, long long m, const unsigned char *bnd,
                        unsigned *node_off, unsigned *adj, long long cap, unsigned char *fixed,
                        long long *n_free, double *diag, long long *words) {
    sls::HostMesh hm;
    sls_status st = sls::build_host_mesh(xy, n, tri, m, bnd, hm, 2);
    if (st != SLS_OK) return (int)st;
    *words = (long long)hm.adj.size();
    if (*words > cap) return -1;
    std::memcpy(node_off, hm.node_off.data(), sizeof(unsigned) * (n + 1));
    std::memcpy(adj, hm.adj.data(), sizeof(unsigned) * hm.adj.size());
    std::memcpy(fixed, hm.fixed.data(), (size_t)n);
    *n_free = hm.n_free;
    *diag = hm.diag;
    return 0;
}
"""


@pytest.fixture(scope="module")
def hb(tmp_path_factory):
    d = tmp_path_factory.mktemp("hostbuild")
    shim = d / "shim.cpp"
    shim.write_text(SHIM)
    so = d / "libhb.so"
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-ffp-contract=off",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, str(shim), os.path.join(CSRC, "mesh_build.cpp"),
           "-o", str(so)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        pytest.fail("g++ failed:\n" + r.stderr)
    L = C.CDLL(str(so))
    L.hb_build.restype = C.c_int
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _build(hb, xy, tri, boundary):
    n, m = len(xy), len(tri)
    xy = np.ascontiguousarray(xy, np.float64)
    tri = np.ascontiguousarray(tri, np.int32)
    bnd = None if boundary is None else np.ascontiguousarray(boundary, np.uint8)
    cap = n + 9 * m
    node_off = np.zeros(n + 1, np.uint32)
    adj = np.zeros(cap, np.uint32)
    fixed = np.zeros(n, np.uint8)
    n_free, diag, words = C.c_longlong(0), C.c_double(0.0), C.c_longlong(0)
    st = hb.hb_build(_p(xy), C.c_longlong(n), _p(tri), C.c_longlong(m), _p(bnd), _p(node_off), _p(adj),
                     C.c_longlong(cap), _p(fixed), C.byref(n_free), C.byref(diag), C.byref(words))
    return st, node_off, adj[: words.value], fixed, n_free.value, diag.value


def _check_against_oracle(hb, mesh, boundary):
    st, node_off, adj, fixed, n_free, diag = _build(hb, mesh.xy, mesh.tri, boundary)
    assert st == 0
    nbr_ptr, nbr, tri_ptr, tri_of, ofixed = oracle.OracleMesh(mesh.xy, mesh.tri, boundary).adjacency()
    assert np.array_equal(fixed, ofixed)
    assert n_free == int((ofixed == 0).sum())
    wx = mesh.xy[:, 0].max() - mesh.xy[:, 0].min()
    wy = mesh.xy[:, 1].max() - mesh.xy[:, 1].min()
    assert diag == np.sqrt(wx * wx + wy * wy)
    assert node_off[-1] == len(adj)
    for i in range(mesh.n):
        w = adj[node_off[i]:node_off[i + 1]]
        meta = int(w[0])
        if ofixed[i]:
            assert len(w) == 1 and meta == 0x80000000, i
            continue
        deg, ntri = meta & 0xFFFF, (meta >> 16) & 0x7FFF
        ref_nb = nbr[nbr_ptr[i]:nbr_ptr[i + 1]]
        ref_t = tri_of[tri_ptr[i]:tri_ptr[i + 1]]
        assert meta >> 31 == 0 and deg == len(ref_nb) and ntri == len(ref_t), i
        assert len(w) == 1 + deg + ntri, i
        nb = w[1:1 + deg].astype(np.int64)
        assert np.array_equal(nb, ref_nb), i                      # summation order (R1)
        for code, t in zip(w[1 + deg:], ref_t):                   # ascending triangle ids
            code = int(code)
            slot, pa, pb = code >> 30, (code >> 15) & 0x7FFF, code & 0x7FFF
            v = mesh.tri[t]
            assert v[slot] == i, (i, t)
            others = [v[s] for s in range(3) if s != slot]       # stored order
            assert [nb[pa], nb[pb]] == others, (i, t)


def _fan(k, centre=(0.05, -0.02)):
    ang = np.linspace(0, 2 * np.pi, k, endpoint=False)
    xy = np.vstack([np.c_[np.cos(ang) * (1 + 0.3 * np.sin(5 * ang)), np.sin(ang)], [centre]])
    tri = np.array([[k, j, (j + 1) % k] if j % 2 else [(j + 1) % k, k, j] for j in range(k)], dtype=np.int32)
    return meshgen.Mesh(xy=xy, tri=tri, boundary=(np.arange(k + 1) < k).astype(np.uint8))


@pytest.mark.parametrize("case", ["small", "random", "natural_derived", "delaunay", "delaunay_derived",
                                  "coincident", "fan30", "fan40_derived"])
def test_host_build_matches_oracle(hb, case):
    if case == "small":
        mesh, bnd = meshgen.small_grid(), "given"
    elif case == "random":
        mesh, bnd = meshgen.jittered_grid(37, 29, 0.35, 7, numbering="random"), "given"
    elif case == "natural_derived":
        mesh, bnd = meshgen.jittered_grid(23, 41, 0.3, 8, numbering="natural"), None
    elif case == "delaunay":
        mesh, bnd = meshgen.delaunay_random(3000, 21, numbering="morton"), "given"
    elif case == "delaunay_derived":
        mesh, bnd = meshgen.delaunay_random(1500, 22, numbering="random"), None
    elif case == "coincident":
        # many equal coordinates: the summation order falls back to node ids
        mesh = meshgen.jittered_grid(30, 30, 0.3, 9, numbering="morton")
        mesh.xy = np.round(mesh.xy * 4) / 4
        bnd = "given"
    elif case == "fan30":
        mesh, bnd = _fan(30), "given"        # a free node in 30 triangles, mixed orientations
    else:
        mesh, bnd = _fan(40), None
    _check_against_oracle(hb, mesh, mesh.boundary if bnd == "given" else None)


def test_host_build_rejects_like_the_oracle(hb):
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0], [0.5, -1.0]])
    # an edge (0, 1) shared by three triangles
    st = _build(hb, xy, np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]]), None)[0]
    assert st == 2
    assert _build(hb, xy, np.array([[0, 1, 5]]), None)[0] == 1         # vertex id out of range
    assert _build(hb, xy, np.array([[0, 1, 1]]), None)[0] == 1         # repeated vertex
    bad = xy.copy()
    bad[3, 1] = np.inf
    assert _build(hb, bad, np.array([[0, 1, 2]]), None)[0] == 1        # non-finite coordinate


def test_roofline_word_count_matches_the_build(hb):
    # bench.py's algorithmic bytes use a closed-form count of the adjacency
    # stream (one meta word per node, degree + triangle count per free node,
    # degree = triangle count for a free node of a closed fan); it must equal
    # the words the build writes on the benchmark's kinds of mesh
    import bench
    meshes = [meshgen.small_grid(), meshgen.large_grid(96, 80),
              meshgen.batch_mesh(meshgen.batch_specs(4)[1]), meshgen.delaunay_random(2000, 5)]
    for mesh in meshes:
        st, node_off, adj, fixed, n_free, _ = _build(hb, mesh.xy, mesh.tri, mesh.boundary)
        assert st == 0
        assert len(adj) == bench.adjacency_words(mesh)
        assert n_free == int((mesh.boundary == 0).sum())
