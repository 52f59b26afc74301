"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

None of these retype the oracle's formulas: alpha is checked against Heron's
formula and closed-form triangles, decisions against exact rational
arithmetic, whole runs against closed-form fixed points, the hand-worked
hexagon, invariants (boundary, permutation, resume) and brute force.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import meshgen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQ3_2 = math.sqrt(3.0) / 2.0


# ---- alpha (Section 3.3.1; Lee and Lo's measure) --------------------------

def test_alpha_equilateral_is_one():
    for (ax, ay, sc) in [(0.0, 0.0, 1.0), (3.5, -2.25, 0.01), (-1e3, 7.0, 250.0)]:
        q = oracle.alpha(ax, ay, ax + sc, ay, ax + 0.5 * sc, ay + SQ3_2 * sc)
        assert abs(q - 1.0) < 1e-14, q


def test_alpha_right_isosceles_and_degenerate():
    # cross = 1, sum of squared edges = 1 + 1 + 2: alpha = 2*sqrt(3)/4 = sqrt(3)/2
    assert oracle.alpha(0.0, 0.0, 1.0, 0.0, 0.0, 1.0) == SQ3_2
    # collinear: zero area
    assert oracle.alpha(0.0, 0.0, 1.0, 1.0, 2.0, 2.0) == 0.0
    # all three points equal: no edge length, defined as 0
    assert oracle.alpha(0.5, 0.5, 0.5, 0.5, 0.5, 0.5) == 0.0


def test_alpha_orientation_flips_sign_exactly():
    rng = np.random.default_rng(1)
    for _ in range(200):
        p = rng.uniform(-1, 1, 6)
        q1 = oracle.alpha(*p)
        q2 = oracle.alpha(p[0], p[1], p[4], p[5], p[2], p[3])
        assert q1 == -q2


def _heron_alpha(p):
    ax, ay, bx, by, cx, cy = (float(v) for v in p)
    a = math.hypot(bx - cx, by - cy)
    b = math.hypot(ax - cx, ay - cy)
    c = math.hypot(ax - bx, ay - by)
    s = 0.5 * (a + b + c)
    area = math.sqrt(max(s * (s - a) * (s - b) * (s - c), 0.0))
    sign = 1.0 if (bx - ax) * (cy - ay) - (by - ay) * (cx - ax) >= 0 else -1.0
    return sign * 4.0 * math.sqrt(3.0) * area / (a * a + b * b + c * c)


def test_alpha_matches_heron_formula():
    rng = np.random.default_rng(2)
    checked = 0
    for _ in range(2000):
        p = rng.uniform(-1, 1, 6)
        ref = _heron_alpha(p)
        if abs(ref) < 1e-3:  # Heron loses digits on slivers; skip them
            continue
        q = oracle.alpha(*p)
        assert abs(q - ref) < 1e-11, (p, q, ref)
        checked += 1
    assert checked > 1500


def test_alpha_exact_rational():
    # alpha in exact rationals up to the constant K = 2*sqrt(3): cross/sum
    rng = np.random.default_rng(3)
    K = Fraction(3.4641016151377544)
    for _ in range(300):
        p = [Fraction(float(v)) for v in rng.uniform(-1, 1, 6)]
        ax, ay, bx, by, cx, cy = p
        cr = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
        s = (bx - ax) ** 2 + (by - ay) ** 2 + (cx - ax) ** 2 + (cy - ay) ** 2 + (cx - bx) ** 2 + (cy - by) ** 2
        exact = K * cr / s
        q = oracle.alpha(*(float(v) for v in p))
        assert abs(Fraction(q) - exact) <= Fraction(1, 10 ** 12) * (abs(K * cr) / s + Fraction(1, 10 ** 4))


# ---- the hand-worked hexagon (Section 2.1) ---------------------------------

def _load_hexagon():
    rows = []
    with open(os.path.join(GOLDEN, "hexagon.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(v) for v in line.split()])
    rows = np.array(rows)
    xy = rows[:, :2].copy()
    fixed = rows[:, 2].astype(np.uint8)
    tri = np.array([[6, k, (k + 1) % 6] for k in range(6)], dtype=np.int32)
    return xy, tri, fixed


@pytest.mark.parametrize("strict", [False, True])
@pytest.mark.parametrize("flags", ["given", "derived"])
def test_hexagon_centre_moves_exactly_to_origin(strict, flags):
    xy, tri, fixed = _load_hexagon()
    om = oracle.OracleMesh(xy, tri, fixed if flags == "given" else None)
    _, _, _, _, fx = om.adjacency()
    assert fx.tolist() == [1, 1, 1, 1, 1, 1, 0]
    nxt, acc, maxd2, nacc = om.sweep(xy, strict=strict)
    assert nxt[6, 0] == 0.0 and nxt[6, 1] == 0.0
    assert acc.tolist() == [0, 0, 0, 0, 0, 0, 1] and nacc == 1
    assert maxd2 == 0.125 ** 2 + 0.0625 ** 2
    assert np.array_equal(nxt[:6], xy[:6])
    # and then it stays: the centre of a regular ring is its own centroid
    nxt2, acc2, maxd2b, _ = om.sweep(nxt, strict=strict)
    assert np.array_equal(nxt2, nxt) and maxd2b == 0.0
    assert acc2[6] == (0 if strict else 1)


def test_smart_test_rejects_an_inverting_move():
    # A dart-shaped ring: the centroid of the ring lies outside the region
    # from which the whole ring is visible, so moving there inverts a triangle
    # (Section 2.1: the smart test exists to stop exactly this).
    xy = np.array([[4.0, 0.0], [-1.0, 1.0], [2.0, 0.0], [-1.0, -1.0], [2.5, 0.0]])
    tri = np.array([[4, 0, 1], [4, 1, 2], [4, 2, 3], [4, 3, 0]], dtype=np.int32)
    om = oracle.OracleMesh(xy, tri)
    assert om.adjacency()[4].tolist() == [1, 1, 1, 1, 0]
    out, acc, d2, qo, qn, cand = om.update_nodes(xy, [4])
    assert cand[0].tolist() == [1.0, 0.0]          # plain Laplacian would go here
    assert qo[0] > 0.0 and qn[0] < 0.0             # ... and invert (O', B, C)
    assert acc[0] == 0 and out[0].tolist() == [2.5, 0.0] and d2[0] == 0.0


# ---- closed form: a symmetric dyadic grid is a fixed point (Eq. 2) ---------

@pytest.mark.parametrize("nx,ny,h", [(8, 8, 1.0), (16, 9, 2.0 ** -6), (5, 12, 0.125)])
def test_uniform_dyadic_grid_is_fixed_point(nx, ny, h):
    mesh = meshgen.jittered_grid(nx, ny, 0.0, 5, h=h, diagonals="uniform", numbering="morton")
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    nf = int((mesh.boundary == 0).sum())
    xy, info, acc = om.smooth(mesh.xy, 6)
    assert np.array_equal(xy, mesh.xy)
    assert info["maxd2_last"] == 0.0 and info["accepted_last"] == nf
    xy, info, acc = om.smooth(mesh.xy, 6, strict=True)
    assert np.array_equal(xy, mesh.xy) and info["accepted_last"] == 0
    # with a tolerance the run stops after the first pass
    xy, info, _ = om.smooth(mesh.xy, 50, tol=1e-12)
    assert info["iterations"] == 1 and info["converged"] == 1


def test_random_diagonal_grid_centres_are_off_node():
    # With mixed diagonals the one-rings are not centrally symmetric, so plain
    # Laplacian smoothing would move nodes; the fixed-point case above is not
    # vacuous.  Every move off the regular grid lowers the worst angle of some
    # right-isosceles triangle, so the smart test keeps such nodes in place.
    mesh = meshgen.jittered_grid(8, 8, 0.0, 5, h=1.0, diagonals="random", numbering="natural")
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    free = np.flatnonzero(mesh.boundary == 0)
    out, acc, d2, qo, qn, cand = om.update_nodes(mesh.xy, free)
    moved = (cand != mesh.xy[free]).any(1)
    assert moved.sum() > len(free) // 4
    assert (qn[moved] < qo[moved]).all() and not acc[moved].any()


# ---- constraints (Section 3.3.3) -------------------------------------------

@pytest.mark.parametrize("nx,ny,diag", [(7, 5, "random"), (12, 12, "uniform"), (2, 9, "random")])
def test_derived_boundary_is_the_outer_ring(nx, ny, diag):
    mesh = meshgen.jittered_grid(nx, ny, 0.2, 11, diagonals=diag, numbering="random")
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    assert np.array_equal(om.adjacency()[4], mesh.boundary)


def test_boundary_nodes_never_move():
    mesh = meshgen.small_grid()
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    xy, info, acc = om.smooth(mesh.xy, 10)
    b = mesh.boundary == 1
    assert np.array_equal(xy[b], mesh.xy[b])
    assert not acc[b].any()
    assert not np.array_equal(xy[~b], mesh.xy[~b])


def test_neighbour_sets_and_canonical_order():
    mesh = meshgen.jittered_grid(9, 7, 0.3, 21, numbering="random")
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    nbr_ptr, nbr, tri_ptr, tri_of, _ = om.adjacency()
    for i in range(mesh.n):
        ts = [t for t in range(mesh.m) if i in mesh.tri[t]]
        assert sorted(tri_of[tri_ptr[i]:tri_ptr[i + 1]].tolist()) == ts
        want = {int(v) for t in ts for v in mesh.tri[t] if v != i}
        got = nbr[nbr_ptr[i]:nbr_ptr[i + 1]].tolist()
        assert set(got) == want and len(got) == len(want)
        keys = [(mesh.xy[j, 0], mesh.xy[j, 1], j) for j in got]
        assert keys == sorted(keys)


def test_invalid_meshes_are_rejected():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    good = np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32)
    oracle.OracleMesh(xy, good)
    for bad in ([[0, 1, 4]], [[0, 1, -1]], [[0, 1, 1]]):
        with pytest.raises(oracle.OracleError) as e:
            oracle.OracleMesh(xy, np.array(bad, dtype=np.int32))
        assert e.value.code == 1
    xy_nan = xy.copy()
    xy_nan[2, 1] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.OracleMesh(xy_nan, good)
    assert e.value.code == 1
    # three triangles on edge (0, 1): non-manifold
    xy5 = np.vstack([xy, [[0.5, -1.0]]])
    nm = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]], dtype=np.int32)
    with pytest.raises(oracle.OracleError) as e:
        oracle.OracleMesh(xy5, nm)
    assert e.value.code == 2


# ---- exact-rational brute force of the accept decisions (Sections 2.1, 3.3.4)

def _exact_alpha_ratio(p):
    (ax, ay), (bx, by), (cx, cy) = p
    cr = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    s = (bx - ax) ** 2 + (by - ay) ** 2 + (cx - ax) ** 2 + (cy - ay) ** 2 + (cx - bx) ** 2 + (cy - by) ** 2
    return cr / s if s > 0 else Fraction(0)


def _check_decisions_exact(mesh, strict):
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    free = np.flatnonzero(mesh.boundary == 0)
    out, acc, d2, qo, qn, cand = om.update_nodes(mesh.xy, free, strict=strict)
    X = [(Fraction(float(a)), Fraction(float(b))) for a, b in mesh.xy]
    near = 0
    for r, i in enumerate(free):
        ts = [t for t in range(mesh.m) if i in mesh.tri[t]]
        nb = sorted({int(v) for t in ts for v in mesh.tri[t] if v != i})
        # the centre in exact arithmetic; the FP64 one is within a few ulps
        ex = sum(X[j][0] for j in nb) / len(nb)
        ey = sum(X[j][1] for j in nb) / len(nb)
        bound = Fraction(len(nb) + 1, 2 ** 52) * max(abs(X[j][0]) + abs(X[j][1]) for j in nb)
        assert abs(Fraction(float(cand[r, 0])) - ex) <= bound
        assert abs(Fraction(float(cand[r, 1])) - ey) <= bound
        c = (Fraction(float(cand[r, 0])), Fraction(float(cand[r, 1])))
        before = min(_exact_alpha_ratio([X[v] for v in mesh.tri[t]]) for t in ts)
        after = min(_exact_alpha_ratio([c if v == i else X[v] for v in mesh.tri[t]]) for t in ts)
        K = Fraction(3.4641016151377544)
        assert abs(Fraction(float(qo[r])) - K * before) < Fraction(1, 10 ** 13)
        assert abs(Fraction(float(qn[r])) - K * after) < Fraction(1, 10 ** 13)
        diff = after - before
        if abs(diff) < Fraction(1, 10 ** 12) and diff != 0:
            near += 1
            continue
        exact_ok = diff > 0 if strict else diff >= 0
        assert bool(acc[r]) == exact_ok, (i, float(diff))
        if acc[r]:
            assert tuple(out[r]) == (float(cand[r, 0]), float(cand[r, 1]))
        else:
            assert tuple(out[r]) == tuple(mesh.xy[i]) and d2[r] == 0.0
    return near


@pytest.mark.parametrize("strict", [False, True])
def test_accept_decisions_match_exact_arithmetic_3x3(strict):
    near = 0
    pats = 0
    for pattern in range(16):
        for s in range(12):
            rng = np.random.default_rng(1000 * pattern + s)
            mesh = meshgen.jittered_grid(3, 3, 0.0, 0, h=1.0, diagonals="uniform", numbering="natural")
            # set the diagonal of each quad from the pattern bits
            diag = np.array([(pattern >> q) & 1 for q in range(4)])
            mesh.tri = meshgen.grid_triangles(3, 3, diag).astype(np.int32)
            # jitter the single interior node and (within 0.3) the edge midpoints stay fixed
            mesh.xy[4] += rng.uniform(-0.45, 0.45, 2)
            near += _check_decisions_exact(mesh, strict)
            pats += 1
    assert pats == 192 and near == 0


def test_accept_decisions_match_exact_arithmetic_4x4():
    near = 0
    for pattern in range(0, 512, 3):
        rng = np.random.default_rng(pattern)
        mesh = meshgen.jittered_grid(4, 4, 0.0, 0, h=1.0, diagonals="uniform", numbering="natural")
        diag = np.array([(pattern >> q) & 1 for q in range(9)])
        mesh.tri = meshgen.grid_triangles(4, 4, diag).astype(np.int32)
        free = mesh.boundary == 0
        mesh.xy[free] += rng.uniform(-0.35, 0.35, (int(free.sum()), 2))
        near += _check_decisions_exact(mesh, strict=bool(pattern & 1))
    assert near == 0


# ---- invariants of Form A (Eq. 2) ------------------------------------------

def test_permutation_invariance():
    runs = []
    for numbering in ("natural", "morton", "random"):
        mesh = meshgen.jittered_grid(48, 40, 0.35, 77, numbering=numbering)
        om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
        xy, info, acc = om.smooth(mesh.xy, 25)
        runs.append((meshgen.unpermute(xy, mesh), info, acc[mesh.perm]))
    for xy, info, acc in runs[1:]:
        assert np.array_equal(xy, runs[0][0])
        assert info == runs[0][1]
        assert np.array_equal(acc, runs[0][2])


def test_resume_equals_one_run():
    mesh = meshgen.jittered_grid(30, 20, 0.3, 3)
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    a, _, _ = om.smooth(mesh.xy, 12)
    b, _, _ = om.smooth(mesh.xy, 7)
    b, _, _ = om.smooth(b, 5)
    assert np.array_equal(a, b)


def test_openmp_build_is_bit_identical():
    mesh = meshgen.jittered_grid(200, 150, 0.35, 9)
    a = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    b = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary, openmp=True)
    xa, ia, aa = a.smooth(mesh.xy, 15)
    xb, ib, ab = b.smooth(mesh.xy, 15)
    assert np.array_equal(xa, xb) and ia == ib and np.array_equal(aa, ab)


def test_stop_rule_stops_at_first_pass_below_tolerance():
    mesh = meshgen.jittered_grid(20, 20, 0.3, 4)
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    tol = 1e-4
    thr = (tol * om.diag) ** 2
    xy, info, _ = om.smooth(mesh.xy, 10000, tol=tol)
    k = info["iterations"]
    assert info["converged"] == 1 and 1 < k < 10000
    assert info["maxd2_last"] < thr
    _, prev, _ = om.smooth(mesh.xy, k - 1)
    assert prev["maxd2_last"] >= thr
    # max d2 is the largest squared move of the pass, recomputed independently
    before, _, _ = om.smooth(mesh.xy, k - 1)
    d = xy - before
    assert info["maxd2_last"] == pytest.approx(float((d * d).sum(1).max()), rel=1e-12)
    # accepted moves include zero-length ones, so they are at least the nodes that moved
    assert info["accepted_last"] >= int(((d != 0).any(1)).sum())


def test_diag_is_bbox_diagonal():
    mesh = meshgen.jittered_grid(10, 30, 0.3, 8)
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    lo = mesh.xy.min(0)
    hi = mesh.xy.max(0)
    assert om.diag == pytest.approx(math.hypot(*(hi - lo)), rel=1e-15)


# ---- histogram -------------------------------------------------------------

def test_histogram_against_independent_alpha():
    mesh = meshgen.jittered_grid(30, 30, 0.45, 12)
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    nb = 16
    counts, qmin, qmean = om.histogram(mesh.xy, nb, -1.0, 1.0)
    ref = np.array([_heron_alpha(mesh.xy[t].ravel()) for t in mesh.tri])
    assert counts.sum() == mesh.m
    edges = np.linspace(-1.0, 1.0, nb + 1)
    assert np.min(np.abs(ref[:, None] - edges[None, :])) > 1e-9  # no value on an edge
    want = np.clip(np.floor((ref + 1.0) / 2.0 * nb), 0, nb - 1).astype(int)
    assert np.array_equal(counts, np.bincount(want, minlength=nb))
    assert qmin == pytest.approx(ref.min(), abs=1e-11)
    assert qmean == pytest.approx(ref.mean(), abs=1e-11)


@pytest.mark.parametrize("strict", [False, True])
def test_accept_rule_holds_over_sweeps_of_a_clustered_grid(strict):
    # Sections 2.1 and 3.3.4 on the benchmark's kind of mesh (clustered,
    # skewed, partly inverted triangles): in every pass each free node's
    # decision is q_new >= q_old (q_new > q_old when strict), both minima
    # taken on the coordinates before the pass (Eq. 2, Jacobi); the sweep
    # applies exactly those decisions; spot checks recompute both minima in
    # exact rational arithmetic at the FP64 centre
    mesh = meshgen.jittered_grid(40, 36, 0.45, 31, numbering="morton", pull_fraction=0.15)
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    free = np.flatnonzero(mesh.boundary == 0)
    tris_of = [[] for _ in range(mesh.n)]
    for t, v in enumerate(mesh.tri):
        for i in v:
            tris_of[int(i)].append(t)
    rng = np.random.default_rng(3)
    xy = mesh.xy.copy()
    inverted = 0
    for q in range(6):
        P = xy[mesh.tri]
        inverted += int((((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                          - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0])) < 0).sum())
        out, acc, d2, qo, qn, cand = om.update_nodes(xy, free, strict=strict)
        assert np.array_equal(acc.astype(bool), qn > qo if strict else qn >= qo)
        assert np.array_equal(out[acc == 1], cand[acc == 1])
        assert np.array_equal(out[acc == 0], xy[free][acc == 0])
        nxt, sacc, maxd2, nacc = om.sweep(xy, strict=strict)
        assert np.array_equal(nxt[free], out) and np.array_equal(sacc[free], acc)
        assert np.array_equal(nxt[mesh.boundary == 1], mesh.xy[mesh.boundary == 1])
        assert nacc == int(acc.sum()) and maxd2 == d2.max()
        for r in rng.choice(free.size, 20, replace=False):
            i = int(free[r])
            X = {int(v): (Fraction(float(xy[v, 0])), Fraction(float(xy[v, 1])))
                 for t in tris_of[i] for v in mesh.tri[t]}
            c = (Fraction(float(cand[r, 0])), Fraction(float(cand[r, 1])))
            before = min(_exact_alpha_ratio([X[int(v)] for v in mesh.tri[t]]) for t in tris_of[i])
            after = min(_exact_alpha_ratio([c if v == i else X[int(v)] for v in mesh.tri[t]]) for t in tris_of[i])
            if abs(after - before) > Fraction(1, 10 ** 12):
                assert bool(acc[r]) == (after > before), (q, i)
        xy = nxt
    assert inverted > 0  # the rule was exercised on inverted elements
