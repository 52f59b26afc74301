"""GPU parity of Form B (Eq. 3) as multicolour Gauss-Seidel: the device
colouring and the colour-by-colour in-place sweeps against the oracle, bit
for bit (coordinates, accept decisions, sweep counts, the last sweep's
accepted count and largest squared move)."""
import numpy as np
import pytest

import meshgen
import oracle

pytestmark = pytest.mark.gpu

KERNELS = ["fp64", "filtered"]


@pytest.fixture(scope="module")
def sls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1502_00355_gb300 as mod
    mod.build()
    mod.lib()
    return mod


def _run_both(sls, mesh, iters, tol=0.0, strict=False, boundary="given", omp=False, **opts):
    bnd = mesh.boundary if boundary == "given" else None
    om = oracle.OracleMesh(mesh.xy, mesh.tri, bnd, openmp=omp)
    ref = om.smooth(mesh.xy, iters, tol=tol, strict=strict, form="B")
    with sls.Mesh(mesh.xy, mesh.tri, bnd, strict=strict, record_accept=True, form="B", **opts) as g:
        info = g.smooth(iters, tol)
        got = (g.coords(), info, g.accept_mask())
    return got, ref


def _check(got, ref, what):
    (xy, info, acc), (rxy, rinfo, racc) = got, ref
    if not np.array_equal(xy, rxy):
        bad = np.flatnonzero((xy != rxy).any(1))
        raise AssertionError(f"{what}: {bad.size} nodes differ, first {bad[0]}")
    for k in ("iterations", "converged", "accepted_last", "maxd2_last"):
        assert info[k] == rinfo[k], (what, k, info[k], rinfo[k])
    assert np.array_equal(acc, racc), what


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_small_grid_form_b(sls, kernel, layout):
    got, ref = _run_both(sls, meshgen.small_grid(), 10, kernel=kernel, layout=layout)
    _check(got, ref, f"small {kernel} {layout}")


@pytest.mark.parametrize("kernel", KERNELS)
def test_form_b_strict_derived_boundary_and_tolerance(sls, kernel):
    mesh = meshgen.jittered_grid(70, 45, 0.35, 12, numbering="random")
    got, ref = _run_both(sls, mesh, 8, strict=True, boundary="derived", kernel=kernel)
    _check(got, ref, "strict derived")
    got, ref = _run_both(sls, meshgen.small_grid(), 200, tol=1e-9, kernel=kernel)
    _check(got, ref, "tolerance")
    assert got[1]["converged"] == 1


@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_form_b_class_windows_grouped(sls, layout):
    # numbering = 2: each colour class's windows of 128 ids listed by loop
    # length inside the library (a Delaunay mesh of degrees 3 to about 12)
    mesh = meshgen.delaunay_random(6000, 11, numbering="random")
    got, ref = _run_both(sls, mesh, 30, tol=1e-9, numbering="grouped", layout=layout)
    _check(got, ref, f"grouped classes {layout}")
    got, ref = _run_both(sls, meshgen.jittered_grid(70, 45, 0.35, 12, numbering="random"), 8, strict=True,
                         boundary="derived", numbering="grouped")
    _check(got, ref, "grouped classes strict derived")


@pytest.mark.parametrize("numbering", ["morton", "random"])
def test_medium_grid_form_b(sls, numbering):
    mesh = meshgen.medium_grid(numbering)
    got, ref = _run_both(sls, mesh, 20, omp=True)
    _check(got, ref, f"medium {numbering}")


def test_delaunay_form_b_to_tolerance(sls):
    mesh = meshgen.delaunay_mesh()
    got, ref = _run_both(sls, mesh, 300, tol=1e-9)
    _check(got, ref, "delaunay-100k")
    assert got[1]["converged"] == 1


def test_form_b_needs_fewer_sweeps_and_is_rejected_where_unsupported(sls):
    import torch
    mesh = meshgen.small_grid()
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary) as a, sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, form="B") as b:
        ia = a.smooth(200, 1e-9)
        ib = b.smooth(200, 1e-9)
        assert ib["converged"] and ib["iterations"] < ia["iterations"]
        with pytest.raises(sls.SlsError):
            sls.Batch([b], [5])
        t_in = torch.from_numpy(mesh.xy).cuda()
        with pytest.raises(sls.SlsError):
            b.smooth_noalloc(t_in, torch.empty_like(t_in), 3)
