"""Pins of the oracle's binary32 variant (reading R11: the paper's precision,
every operation one binary32 round-to-nearest operation in the order of the
FP64 definition).  Closed forms of alpha in binary32, the hexagon worked
case, the dyadic fixed point, exact-rational brute force of the accept
decisions at binary32 positions, closeness to the FP64 oracle and the count
of decisions that flip against it, numbering invariance.  CPU only."""
from fractions import Fraction

import numpy as np
import pytest

import meshgen
import oracle

K32 = np.float32(3.4641016151377544)


def test_alpha32_closed_forms():
    # right isosceles: cross 1, edge sum (1 + 1) + 2 = 4, all exact: K32 / 4
    assert oracle.alpha32(0, 0, 1, 0, 0, 1) == K32 / np.float32(4)
    assert oracle.alpha32(0, 0, 0, 1, 1, 0) == -(K32 / np.float32(4))
    # equilateral: 1 within the float rounding of its six operations
    s = np.float32(np.sqrt(3) / 2)
    assert abs(float(oracle.alpha32(0, 0, 1, 0, 0.5, s)) - 1.0) < 4e-7
    assert oracle.alpha32(0, 0, 1, 1, 2, 2) == 0.0  # degenerate


def test_alpha32_tracks_alpha64():
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(3000):
        p = rng.uniform(-1, 1, 6).astype(np.float32).astype(np.float64)
        a64 = oracle.alpha(*p)
        if abs(a64) < 0.05:
            continue  # nearly degenerate: large relative condition
        worst = max(worst, abs(float(oracle.alpha32(*p)) - a64))
    assert worst < 2e-5


def _hexagon(dtype):
    s = 0.8660254037844386
    xy = np.array([[1.0, 0.0], [0.5, s], [-0.5, s], [-1.0, 0.0], [-0.5, -s], [0.5, -s], [0.125, -0.0625]])
    tri = np.array([[6, k, (k + 1) % 6] for k in range(6)], dtype=np.int32)
    return xy, tri


def test_hexagon_centre_is_exactly_the_origin_in_binary32():
    xy, tri = _hexagon(np.float32)
    om = oracle.OracleMesh(xy, tri)
    out, info, acc = om.smooth(xy, 1, precision=32)
    assert out[6, 0] == 0.0 and out[6, 1] == 0.0 and acc[6] == 1 and info["accepted_last"] == 1


def test_dyadic_grid_is_a_binary32_fixed_point():
    grid = meshgen.jittered_grid(9, 7, 0.0, 0, h=0.25, diagonals="uniform", numbering="natural")
    om = oracle.OracleMesh(grid.xy, grid.tri, grid.boundary)
    for form in ("A", "B"):
        out, info, _ = om.smooth(grid.xy, 4, precision=32, form=form)
        assert np.array_equal(out, grid.xy) and info["iterations"] == 4


def _exact_alpha_ratio(p):
    (ax, ay), (bx, by), (cx, cy) = p
    cr = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    s = (bx - ax) ** 2 + (by - ay) ** 2 + (cx - ax) ** 2 + (cy - ay) ** 2 + (cx - bx) ** 2 + (cy - by) ** 2
    return cr / s if s > 0 else Fraction(0)


def test_binary32_decisions_match_exact_arithmetic():
    near = checked = 0
    for pattern in range(16):
        for seed in range(8):
            rng = np.random.default_rng(77 * pattern + seed)
            mesh = meshgen.jittered_grid(3, 3, 0.0, 0, h=1.0, diagonals="uniform", numbering="natural")
            mesh.tri = meshgen.grid_triangles(3, 3, np.array([(pattern >> q) & 1 for q in range(4)])).astype(np.int32)
            mesh.xy[4] += rng.uniform(-0.45, 0.45, 2)
            x32 = mesh.xy.astype(np.float32).astype(np.float64)
            om = oracle.OracleMesh(x32, mesh.tri, mesh.boundary)
            out, info, acc = om.smooth(x32, 1, precision=32)
            X = [(Fraction(float(a)), Fraction(float(b))) for a, b in x32]
            nb = sorted({int(v) for t in mesh.tri if 4 in t for v in t if v != 4})
            # the binary32 centre is within a few float units of the exact one
            cx32 = np.float32(0)
            cy32 = np.float32(0)
            for k, j in enumerate(sorted(nb, key=lambda j: (x32[j, 0], x32[j, 1], j))):
                cx32 = np.float32(x32[j, 0]) if k == 0 else np.float32(cx32 + np.float32(x32[j, 0]))
                cy32 = np.float32(x32[j, 1]) if k == 0 else np.float32(cy32 + np.float32(x32[j, 1]))
            c = (Fraction(float(np.float32(cx32 / np.float32(len(nb))))),
                 Fraction(float(np.float32(cy32 / np.float32(len(nb))))))
            ex = sum(X[j][0] for j in nb) / len(nb)
            assert abs(c[0] - ex) <= Fraction(len(nb) + 1, 2 ** 22)
            ts = [t for t in mesh.tri if 4 in t]
            before = min(_exact_alpha_ratio([X[v] for v in t]) for t in ts)
            after = min(_exact_alpha_ratio([c if v == 4 else X[v] for v in t]) for t in ts)
            if abs(after - before) < Fraction(1, 10 ** 5):
                near += 1
                continue
            checked += 1
            assert bool(acc[4]) == (after >= before), (pattern, seed)
            if acc[4]:
                assert (Fraction(float(out[4, 0])), Fraction(float(out[4, 1]))) == c
    assert checked > 100 and near < 8


def test_binary32_stays_close_to_fp64_and_counts_flips():
    mesh = meshgen.small_grid()
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    a64 = om.sweep(mesh.xy)
    out32, info, acc32 = om.smooth(mesh.xy, 1, precision=32)
    flips = int((a64[1] != acc32).sum())
    free = mesh.boundary == 0
    assert flips <= 0.02 * free.sum()
    same = (a64[1] == acc32) & free
    assert np.abs(out32[same] - a64[0][same]).max() < 1e-6


def test_binary32_results_do_not_depend_on_numbering():
    a = meshgen.jittered_grid(30, 40, 0.3, 7, numbering="morton")
    r = meshgen.jittered_grid(30, 40, 0.3, 7, numbering="random")
    oa = oracle.OracleMesh(a.xy, a.tri, a.boundary).smooth(a.xy, 6, precision=32)[0]
    orr = oracle.OracleMesh(r.xy, r.tri, r.boundary).smooth(r.xy, 6, precision=32)[0]
    assert np.array_equal(meshgen.unpermute(oa, a), meshgen.unpermute(orr, r))
