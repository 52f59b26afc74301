"""Skipping of unchanged tiles (sls_options.skip_unchanged): a tile of 32
consecutive nodes whose nodes and neighbours all kept their coordinates in
the previous pass has that pass's inputs, so Form A (Eq. 2) gives it that
pass's results again.  With the option on, every run must stay bit-identical
to the FP64 oracle and to the run without it (coordinates, accept decisions,
iteration counts, accepted counts, largest squared move), and tiles must
actually be skipped once the mesh settles."""
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


def _same(a, b, what):
    if not np.array_equal(a, b):
        bad = np.flatnonzero((a != b).any(1))
        raise AssertionError(f"{what}: {bad.size} nodes differ, first {bad[0]}")


def _check(sls, mesh, iters, tol=0.0, strict=False, omp=False, boundary="given", **opts):
    bnd = mesh.boundary if boundary == "given" else None
    om = oracle.OracleMesh(mesh.xy, mesh.tri, bnd, openmp=omp)
    rxy, rinfo, racc = om.smooth(mesh.xy, iters, tol=tol, strict=strict)
    with sls.Mesh(mesh.xy, mesh.tri, bnd, strict=strict, record_accept=True, skip_unchanged=True, **opts) as g:
        info = g.smooth(iters, tol)
        xy = g.coords()
        acc = g.accept_mask()
    what = f"n={mesh.n} iters={iters} tol={tol} strict={strict} {opts}"
    _same(xy, rxy, what)
    for k in ("iterations", "converged", "accepted_last", "maxd2_last"):
        assert info[k] == rinfo[k], (what, k, info[k], rinfo[k])
    if rinfo["iterations"] > 0:
        assert np.array_equal(acc, racc), what
    return info


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("copy_back", [False, True])
@pytest.mark.parametrize("strict", [False, True])
def test_small_grid_to_tolerance(sls, layout, copy_back, strict):
    mesh = meshgen.small_grid()
    info = _check(sls, mesh, 300, tol=1e-9, strict=strict, layout=layout, copy_back=copy_back)
    assert info["converged"] == 1
    assert info["nodes_skipped"] > 0


def test_ragged_tail_and_derived_boundary(sls):
    # 61 x 47 = 2,867 nodes: the last tile is partial
    mesh = meshgen.jittered_grid(61, 47, 0.35, 11)
    _check(sls, mesh, 150, tol=1e-10, boundary="derived")
    _check(sls, mesh, 40, block_size=64)


def test_medium_grid_to_tolerance_both_numberings(sls):
    # Morton numbering: tiles are compact, most settle and are skipped.
    # Random numbering: a tile's neighbours fall in more tiles than its list
    # holds, so such tiles are always computed; results still identical.
    for numbering in ("morton", "random"):
        mesh = meshgen.medium_grid(numbering)
        info = _check(sls, mesh, 200, tol=1e-9, omp=True)
        if numbering == "morton":
            assert info["nodes_skipped"] > 0.1 * mesh.n * info["iterations"]


def test_delaunay_to_tolerance(sls):
    # the paper's mesh family, 100,000 points, some nodes past the screened
    # kernel's degree limit (finished by the exact path)
    mesh = meshgen.delaunay_mesh()
    info = _check(sls, mesh, 300, tol=1e-9, omp=True)
    assert info["converged"] == 1 and info["nodes_skipped"] > 0


def test_resume_and_set_coords(sls):
    # every sls_smooth call recomputes its first pass, so a call boundary or
    # new coordinates never reuse stale tile state
    mesh = meshgen.jittered_grid(70, 50, 0.35, 9)
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    ref60, _, _ = om.smooth(mesh.xy, 60)
    ref25, _, _ = om.smooth(mesh.xy, 25)
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, skip_unchanged=True) as g:
        for k in (20, 1, 19, 20):
            g.smooth(k)
        _same(g.coords(), ref60, "20 + 1 + 19 + 20 passes")
        g.set_coords(mesh.xy)
        g.smooth(25)
        _same(g.coords(), ref25, "after set_coords")
        g.set_coords(ref25)
        g.smooth(35)
        _same(g.coords(), ref60, "25 then 35 from the set coordinates")


def test_same_as_without_skipping_and_batch_unaffected(sls):
    mesh = meshgen.jittered_grid(200, 130, 0.35, 21)
    outs = []
    for skip in (False, True):
        with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, skip_unchanged=skip, record_accept=True) as g:
            info = g.smooth(400, 1e-10)
            outs.append((g.coords(), g.accept_mask(), info))
    _same(outs[0][0], outs[1][0], "skip on/off")
    assert np.array_equal(outs[0][1], outs[1][1])
    for k in ("iterations", "converged", "accepted_last", "maxd2_last"):
        assert outs[0][2][k] == outs[1][2][k]
    assert outs[0][2]["nodes_skipped"] == 0 and outs[1][2]["nodes_skipped"] > 0
    # the batched form computes every tile of a mesh that has the option on
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, skip_unchanged=True) as h:
        b = sls.Batch([h], [400], [1e-10], block_size=128)
        try:
            b.smooth()
            _same(b.coords(0), outs[0][0], "batched")
        finally:
            b.close()


def test_rejected_where_unsupported(sls):
    mesh = meshgen.jittered_grid(20, 20, 0.3, 1)
    for opts in (dict(kernel="fp64"), dict(form="B"), dict(precision=32)):
        with pytest.raises(sls.SlsError) as e:
            sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, skip_unchanged=True, **opts)
        assert e.value.code == 1
    with pytest.raises(sls.SlsError) as e:
        sls.Server(skip_unchanged=True)
    assert e.value.code == 1


@pytest.mark.parametrize("transform", ["shift_negative", "mixed_binades"])
def test_domain_edges_and_random_numbering(sls, transform):
    # signs and binades that send nodes through the screen's fallbacks, a
    # random numbering that overflows the tile lists: still identical
    mesh = meshgen.jittered_grid(70, 55, 0.35, 41, numbering="random")
    xy = mesh.xy.copy()
    xy = xy - 0.5 if transform == "shift_negative" else xy * 3.0 - 1.0
    mesh.xy = xy
    for strict in (False, True):
        _check(sls, mesh, 200, tol=1e-10, strict=strict)
    m2 = meshgen.jittered_grid(70, 55, 0.35, 41, numbering="morton")
    m2.xy = m2.xy - 0.5 if transform == "shift_negative" else m2.xy * 3.0 - 1.0
    info = _check(sls, m2, 200, tol=1e-10)
    assert info["nodes_skipped"] > 0
