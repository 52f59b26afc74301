"""Pins of the oracle's Form B (Eq. 3) made deterministic as multicolour
Gauss-Seidel: the Jones-Plassmann colouring against a separate brute-force
statement of it, the colour classes read the coordinates their neighbours
got earlier in the same sweep (checked step by step, decisions in exact
rational arithmetic), Form B equals Form A when the free nodes are pairwise
apart, the symmetric dyadic grid stays a fixed point, boundary nodes never
move.  CPU only."""
from fractions import Fraction

import numpy as np
import pytest

import meshgen
import oracle

M64 = (1 << 64) - 1


def _splitmix64(x):
    # Steele, Lea and Flood (2014), the published finaliser
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _neighbours(mesh):
    nb = [set() for _ in range(mesh.n)]
    for a, b, c in mesh.tri:
        for u, v in ((a, b), (b, c), (c, a)):
            nb[u].add(int(v))
            nb[v].add(int(u))
    return nb


def _brute_force_jp(mesh, fixed, seed):
    """Jones-Plassmann rounds written out directly."""
    nb = _neighbours(mesh)
    prio = [_splitmix64(seed + i) for i in range(mesh.n)]
    colour = [-1] * mesh.n
    left = {i for i in range(mesh.n) if not fixed[i]}
    rounds = 0
    while left:
        winners = [i for i in sorted(left)
                   if all((prio[i], i) > (prio[j], j) for j in nb[i] if j in left)]
        for i in winners:
            taken = {colour[j] for j in nb[i] if colour[j] >= 0}
            c = 0
            while c in taken:
                c += 1
            colour[i] = c
        left -= set(winners)
        rounds += 1
    return colour, rounds


@pytest.mark.parametrize("which", ["grid", "delaunay", "random-numbering"])
def test_colouring_is_proper_and_matches_brute_force(which):
    if which == "grid":
        mesh = meshgen.jittered_grid(12, 9, 0.3, 4)
    elif which == "delaunay":
        pytest.importorskip("scipy")
        mesh = meshgen.delaunay_random(400, 9)
    else:
        mesh = meshgen.jittered_grid(10, 11, 0.3, 5, numbering="random")
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    col, nc, rounds = om.colouring()
    fixed = om.adjacency()[4]
    assert ((col < 0) == (fixed == 1)).all()
    nb = _neighbours(mesh)
    for i in range(mesh.n):
        if col[i] >= 0:
            assert all(col[j] != col[i] for j in nb[i] if col[j] >= 0)
    assert nc == col.max() + 1
    ref, ref_rounds = _brute_force_jp(mesh, fixed, oracle.COLOUR_SEED)
    assert col.tolist() == ref and rounds == ref_rounds


def _exact_alpha_ratio(p):
    (ax, ay), (bx, by), (cx, cy) = p
    cr = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    s = (bx - ax) ** 2 + (by - ay) ** 2 + (cx - ax) ** 2 + (cy - ay) ** 2 + (cx - bx) ** 2 + (cy - by) ** 2
    return cr / s if s > 0 else Fraction(0)


def test_colour_classes_read_the_moves_of_earlier_classes():
    mesh = meshgen.jittered_grid(6, 6, 0.35, 77, numbering="random")
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    col, nc, _ = om.colouring()
    swept, acc_b, maxd2, nacc = om.sweep_coloured(mesh.xy, col, nc)
    jacobi = om.update_nodes(mesh.xy, np.flatnonzero(col >= 0))[0]
    state = mesh.xy.copy()
    nb = _neighbours(mesh)
    differs = 0
    for c in range(nc):
        idx = np.flatnonzero(col == c)
        out, acc, d2, qo, qn, cand = om.update_nodes(state, idx)
        assert np.array_equal(swept[idx], out)
        assert np.array_equal(acc_b[idx], acc)
        X = [(Fraction(float(a)), Fraction(float(b))) for a, b in state]
        for r, i in enumerate(idx):
            ts = [t for t in range(mesh.m) if i in mesh.tri[t]]
            ex = sum(X[j][0] for j in nb[i]) / len(nb[i])
            bound = Fraction(len(nb[i]) + 1, 2 ** 52) * max(abs(X[j][0]) + abs(X[j][1]) for j in nb[i])
            assert abs(Fraction(float(cand[r, 0])) - ex) <= bound
            cpos = (Fraction(float(cand[r, 0])), Fraction(float(cand[r, 1])))
            before = min(_exact_alpha_ratio([X[v] for v in mesh.tri[t]]) for t in ts)
            after = min(_exact_alpha_ratio([cpos if v == i else X[v] for v in mesh.tri[t]]) for t in ts)
            if abs(after - before) > Fraction(1, 10 ** 12):
                assert bool(acc[r]) == (after >= before)
        state[idx] = out
    assert np.array_equal(state, swept)
    # the sweep is not the Jacobi pass: later classes saw moved neighbours
    free = np.flatnonzero(col >= 0)
    differs = int((swept[free] != jacobi).any(1).sum())
    assert differs > 0
    assert nacc == int(acc_b.sum())


def test_form_b_equals_form_a_on_pairwise_separated_free_nodes():
    mesh = meshgen.jittered_grid(11, 11, 0.3, 3, numbering="natural")
    gi, gj = np.meshgrid(np.arange(11), np.arange(11), indexing="xy")
    keep = ((gi % 2 == 0) & (gj % 2 == 0)).ravel() & (mesh.boundary == 0)
    bnd = (~keep).astype(np.uint8)
    om = oracle.OracleMesh(mesh.xy, mesh.tri, bnd)
    col, nc, rounds = om.colouring()
    assert nc == 1 and rounds == 1
    a = om.smooth(mesh.xy, 7)
    b = om.smooth(mesh.xy, 7, form="B")
    assert np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[2], b[2])


def test_form_b_fixed_point_boundary_and_faster_convergence():
    grid = meshgen.jittered_grid(9, 7, 0.0, 0, h=0.25, diagonals="uniform", numbering="natural")
    om = oracle.OracleMesh(grid.xy, grid.tri, grid.boundary)
    xy, info, _ = om.smooth(grid.xy, 5, form="B")
    assert np.array_equal(xy, grid.xy) and info["iterations"] == 5
    mesh = meshgen.small_grid()
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    xa, ia, _ = om.smooth(mesh.xy, 200, tol=1e-9)
    xb, ib, _ = om.smooth(mesh.xy, 200, tol=1e-9, form="B")
    fixed = mesh.boundary == 1
    assert np.array_equal(xb[fixed], mesh.xy[fixed])
    # Form B needs fewer sweeps than Form A (the paper's observation)
    assert ia["converged"] and ib["converged"] and ib["iterations"] < ia["iterations"]
