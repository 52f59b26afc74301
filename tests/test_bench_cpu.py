"""Host-side figures of bench.py, checked on the CPU: the edge count and the
survey's algorithmic bytes per pass, and that figures taken from an ncu
capture are withheld once the kernel's sources change."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import meshgen  # noqa: E402


def _edges_brute(mesh):
    s = set()
    for a, b, c in mesh.tri.tolist():
        for u, v in ((a, b), (b, c), (c, a)):
            s.add((min(u, v), max(u, v)))
    return len(s)


def test_edge_count_matches_brute_force_and_euler():
    for mesh in (meshgen.jittered_grid(9, 7, 0.3, 5), meshgen.delaunay_random(300, 11),
                 meshgen.jittered_grid(12, 12, 0.3, 6, numbering="random")):
        e = bench.edge_count(mesh)
        assert e == _edges_brute(mesh)
        # a triangulated disk: V - E + F = 1
        assert mesh.n - e + mesh.m == 1


def test_survey_bytes_of_the_benchmark_mesh():
    """16n + 16n_free + 8(n+1) + 4nnz + 12m + 12m + n for the 4096x4096 grid
    (nnz = 2E, E = n + m - 1 for a disk), from the counts alone."""
    n, m = 4096 * 4096, 2 * 4095 * 4095
    n_free = 4094 * 4094
    e = n + m - 1
    expect = 16 * n + 16 * n_free + 8 * (n + 1) + 4 * 2 * e + 12 * m + 12 * m + n
    assert expect == 1_895_039_104

    small = meshgen.jittered_grid(30, 20, 0.3, 3)
    got = bench.survey_bytes_per_pass(small, int(np.count_nonzero(small.boundary == 0)))
    e = _edges_brute(small)
    assert got == (16 * small.n + 16 * 28 * 18 + 8 * (small.n + 1) + 8 * e + 24 * small.m + small.n)


def test_profile_figures_are_withheld_for_changed_sources(monkeypatch):
    fig = dict(bench.PROFILE_FIGURES["pass_screened"])
    fig["sha256"] = bench.sources_sha256(fig["files"])
    monkeypatch.setitem(bench.PROFILE_FIGURES, "pass_screened", fig)
    assert bench.profile_figures("pass_screened") is fig
    stale = dict(fig, sha256="0" * 64)
    monkeypatch.setitem(bench.PROFILE_FIGURES, "pass_screened", stale)
    assert bench.profile_figures("pass_screened") is None


def test_both_arms_print_the_same_config():
    class A:
        kernel, layout, copy_back, form, precision = "auto", "aos", False, "A", 64
        skip_unchanged = l2_window = False
    mesh = meshgen.small_grid()
    c1 = bench.large_config(A, mesh, "w", 1)
    c2 = bench.large_config(A, mesh, "w", 1)
    assert c1 == c2 and c1["n_free"] == int(np.count_nonzero(mesh.boundary == 0))
