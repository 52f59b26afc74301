"""GPU parity of the binary32 variant (the paper's precision) against the
oracle's binary32 definition, bit for bit: coordinates (floats, widened
exactly), accept decisions, pass counts, the last pass's accepted count and
largest squared move, for both forms, both layouts and the copy-back form."""
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


def _run_both(sls, mesh, iters, tol=0.0, strict=False, form="A", boundary="given", **opts):
    bnd = mesh.boundary if boundary == "given" else None
    ref = oracle.OracleMesh(mesh.xy, mesh.tri, bnd).smooth(mesh.xy, iters, tol=tol, strict=strict, form=form,
                                                           precision=32)
    with sls.Mesh(mesh.xy, mesh.tri, bnd, strict=strict, record_accept=True, form=form, precision=32, **opts) as g:
        info = g.smooth(iters, tol)
        got = (g.coords(), info, g.accept_mask())
    return got, ref


def _check(got, ref, what):
    (xy, info, acc), (rxy, rinfo, racc) = got, ref
    if not np.array_equal(xy, rxy):
        bad = np.flatnonzero((xy != rxy).any(1))
        raise AssertionError(f"{what}: {bad.size} nodes differ, first {bad[0]}: {xy[bad[0]]} vs {rxy[bad[0]]}")
    for k in ("iterations", "converged", "accepted_last", "maxd2_last"):
        assert info[k] == rinfo[k], (what, k, info[k], rinfo[k])
    assert np.array_equal(acc, racc), what


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("copy_back", [False, True])
def test_small_grid_binary32(sls, layout, copy_back):
    got, ref = _run_both(sls, meshgen.small_grid(), 10, layout=layout, copy_back=copy_back)
    _check(got, ref, f"small {layout} copy_back={copy_back}")


@pytest.mark.parametrize("form", ["A", "B"])
def test_binary32_strict_derived_and_tolerance(sls, form):
    mesh = meshgen.jittered_grid(70, 45, 0.35, 12, numbering="random")
    got, ref = _run_both(sls, mesh, 8, strict=True, boundary="derived", form=form)
    _check(got, ref, f"strict derived {form}")
    got, ref = _run_both(sls, meshgen.small_grid(), 200, tol=1e-9, form=form)
    _check(got, ref, f"tolerance {form}")
    assert got[1]["converged"] == 1


@pytest.mark.parametrize("form", ["A", "B"])
def test_binary32_medium_and_delaunay(sls, form):
    got, ref = _run_both(sls, meshgen.medium_grid("random"), 12, form=form)
    _check(got, ref, f"medium {form}")
    got, ref = _run_both(sls, meshgen.delaunay_mesh(), 300, tol=1e-9, form=form)
    _check(got, ref, f"delaunay {form}")


def test_binary32_coordinate_round_trip_and_rejections(sls):
    import torch
    mesh = meshgen.small_grid()
    x32 = mesh.xy.astype(np.float32).astype(np.float64)
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, precision=32) as g:
        assert np.array_equal(g.coords(), x32)                 # rounded to nearest, widened exactly
        assert np.array_equal(g.coords_device().cpu().numpy(), x32)
        g.set_coords(torch.from_numpy(mesh.xy + 1e-3).cuda())
        assert np.array_equal(g.coords(), (mesh.xy + 1e-3).astype(np.float32).astype(np.float64))
        counts, qmin, qmean = g.histogram(10)
        assert counts.sum() == mesh.m
        with pytest.raises(sls.SlsError):
            sls.Batch([g], [3])
        t = torch.from_numpy(mesh.xy).cuda()
        with pytest.raises(sls.SlsError):
            g.smooth_noalloc(t, torch.empty_like(t), 3)
    with pytest.raises(sls.SlsError):
        sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, precision=16)
