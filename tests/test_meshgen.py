"""The synthetic input generator: shapes, seeds and structure the workloads rely on."""
import numpy as np
import pytest

import meshgen


def test_counts_and_boundary():
    m = meshgen.jittered_grid(64, 64, 0.3, 1)
    assert m.n == 4096 and m.m == 7938
    assert int(m.boundary.sum()) == 4 * 63
    big = meshgen.jittered_grid(1024, 1024, 0.35, 2)
    assert big.n == 1048576 and big.m == 2093058


def test_triangles_ccw_before_jitter_and_jitter_bounded():
    m = meshgen.jittered_grid(20, 17, 0.0, 3, numbering="random")
    a, b, c = (m.xy[m.tri[:, k]] for k in range(3))
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert (cross > 0).all()
    j = meshgen.jittered_grid(20, 17, 0.3, 3, numbering="natural")
    g = meshgen.jittered_grid(20, 17, 0.0, 3, numbering="natural")
    h = g.meta["h"]
    d = np.abs(j.xy - g.xy)
    assert d.max() <= 0.3 * h + 1e-15
    assert np.array_equal(d[j.boundary == 1], np.zeros_like(d[j.boundary == 1]))


def test_seeded_and_numberings_are_permutations():
    a = meshgen.jittered_grid(30, 40, 0.3, 7, numbering="morton")
    b = meshgen.jittered_grid(30, 40, 0.3, 7, numbering="morton")
    assert np.array_equal(a.xy, b.xy) and np.array_equal(a.tri, b.tri)
    r = meshgen.jittered_grid(30, 40, 0.3, 7, numbering="random")
    assert np.array_equal(np.sort(a.perm), np.arange(a.n)) and np.array_equal(np.sort(r.perm), np.arange(r.n))
    assert np.array_equal(meshgen.unpermute(a.xy, a), meshgen.unpermute(r.xy, r))


def test_morton_order_is_z_curve():
    i = np.array([0, 1, 0, 1, 2, 3, 2, 3])
    j = np.array([0, 0, 1, 1, 0, 0, 1, 1])
    assert meshgen.morton_order(i, j).tolist() == [0, 1, 2, 3, 4, 5, 6, 7]


def test_pull_moves_five_percent_and_caps_step():
    base = meshgen.jittered_grid(200, 200, 0.35, 11, numbering="natural")
    pulled = meshgen.jittered_grid(200, 200, 0.35, 11, numbering="natural", pull_fraction=0.05)
    moved = (pulled.xy != base.xy).any(1)
    interior = int((base.boundary == 0).sum())
    assert abs(int(moved.sum()) - round(0.05 * interior)) <= 1
    step = np.sqrt(((pulled.xy - base.xy) ** 2).sum(1))
    assert step.max() <= 2 * base.meta["h"] * (1 + 1e-12)


def test_batch_and_serve_specs():
    specs = meshgen.batch_specs(64)
    assert len(specs) == 64
    for nx, ny, it, _ in specs:
        assert 10 <= it <= 100 and nx >= 2 and ny >= 2
        assert 700 <= nx * ny <= 300000
    reqs = meshgen.serve_requests(50)
    t = [r[0] for r in reqs]
    assert t == sorted(t) and all(10 <= r[3] <= 200 for r in reqs)


def test_delaunay_random_is_a_ccw_delaunay_triangulation():
    pytest.importorskip("scipy")
    m = meshgen.delaunay_random(300, 21, numbering="random")
    p = m.xy
    a, b, c = p[m.tri[:, 0]], p[m.tri[:, 1]], p[m.tri[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert (cross > 0).all()
    # Euler: a triangulated convex polygon with h hull vertices has 2n - h - 2 triangles
    h = int(m.boundary.sum())
    assert m.m == 2 * m.n - h - 2
    # every hull edge lies in one triangle, every other edge in two; the fixed
    # nodes are exactly the ends of one-triangle edges
    e = np.sort(np.concatenate([m.tri[:, [0, 1]], m.tri[:, [1, 2]], m.tri[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    assert set(cnt.tolist()) == {1, 2}
    ends = np.unique(np.unique(e, axis=0)[cnt == 1])
    assert np.array_equal(np.flatnonzero(m.boundary), ends)
    # empty circumcircles (brute force): the in-circle determinant of every
    # other point against every CCW triangle is not positive
    def rows(V):
        d = V[None, :] - p
        return np.stack([d[:, 0], d[:, 1], d[:, 0] ** 2 + d[:, 1] ** 2], 1)
    for t in range(m.m):
        incircle = np.linalg.det(np.stack([rows(a[t]), rows(b[t]), rows(c[t])], 1))
        others = np.ones(m.n, bool)
        others[m.tri[t]] = False
        assert (incircle[others] < 1e-12).all(), t


def test_delaunay_numberings_are_permutations_of_one_mesh():
    pytest.importorskip("scipy")
    a = meshgen.delaunay_random(2000, 5, numbering="morton")
    r = meshgen.delaunay_random(2000, 5, numbering="random")
    assert np.array_equal(meshgen.unpermute(a.xy, a), meshgen.unpermute(r.xy, r))
    ta = np.sort(np.sort(a.perm.argsort()[a.tri], axis=1), axis=0)
    tr = np.sort(np.sort(r.perm.argsort()[r.tri], axis=1), axis=0)
    assert np.array_equal(np.unique(ta, axis=0), np.unique(tr, axis=0))


def test_fast_grid_construction():
    """fastgrid.c against the numpy construction: the Morton numbering equals
    morton_order, the triangles are grid_triangles of the diagonals it drew,
    the outer ring is fixed and exact, the interior jitter stays within J h,
    and the same arguments give the same mesh."""
    for nx, ny in [(2, 2), (5, 3), (17, 33), (64, 64), (100, 37)]:
        m = meshgen.fast_grid(nx, ny, 0.3, 12345 + nx)
        h = 1.0 / (ny - 1)
        gi, gj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
        gi, gj = gi.ravel(), gj.ravel()
        perm = meshgen.morton_order(gi, gj)
        nat = m.xy[perm]
        ring = (gi == 0) | (gj == 0) | (gi == nx - 1) | (gj == ny - 1)
        assert np.array_equal(m.boundary[perm], ring.astype(np.uint8))
        assert np.array_equal(nat[ring, 0], gi[ring] * h) and np.array_equal(nat[ring, 1], gj[ring] * h)
        assert np.all(np.abs(nat[:, 0] - gi * h) <= 0.3 * h * (1 + 1e-12))
        assert np.all(np.abs(nat[:, 1] - gj * h) <= 0.3 * h * (1 + 1e-12))
        if (~ring).any():
            assert np.any(nat[~ring, 0] != gi[~ring] * h)
        # recover the diagonals from the first triangle of each quad
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        t_nat = inv[m.tri]
        nq = (nx - 1) * (ny - 1)
        diag = (t_nat[0::2, 2] != t_nat[0::2, 1] + nx).astype(np.int64)
        assert np.array_equal(t_nat, meshgen.grid_triangles(nx, ny, diag))
        if nq >= 64:
            assert 0.3 < diag.mean() < 0.7
        again = meshgen.fast_grid(nx, ny, 0.3, 12345 + nx)
        assert np.array_equal(again.xy, m.xy) and np.array_equal(again.tri, m.tri)
    nat = meshgen.fast_grid(9, 7, 0.3, 1, numbering="natural")
    mor = meshgen.fast_grid(9, 7, 0.3, 1, numbering="morton")
    gi, gj = np.meshgrid(np.arange(9), np.arange(7), indexing="xy")
    perm = meshgen.morton_order(gi.ravel(), gj.ravel())
    assert np.array_equal(mor.xy[perm], nat.xy)
