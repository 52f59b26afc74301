"""The library's internal numbering of Form-A meshes (nodes grouped by
incident-triangle count inside windows of 128 ids: numbering = 2, and by
default for meshes of 2^20 nodes or more) against the caller's numbering
(numbering = 1) and the oracle:
coordinates, decisions, statistics, the histogram and every entry point that
takes node ids or coordinates in the caller's numbering must be unchanged."""
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


MESHES = {
    # ragged last window (n not a multiple of 128), random diagonals: degrees 4-8
    "grid_ragged": lambda: meshgen.jittered_grid(97, 61, 0.35, 21, pull_fraction=0.05, pull_centres=32),
    # the paper's family: degrees 3 to about 12, random numbering
    "delaunay_random": lambda: meshgen.delaunay_random(5000, 4, numbering="random"),
    # fewer nodes than one window
    "tiny": lambda: meshgen.jittered_grid(9, 7, 0.3, 2),
}


def _run(sls, mesh, iters, tol, **opts):
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, record_accept=True, **opts) as g:
        info = g.smooth(iters, tol)
        return g.coords(), info, g.accept_mask(), g.histogram(16)


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("opts", [dict(), dict(layout="soa"), dict(copy_back=True), dict(kernel="fp64"),
                                  dict(strict=True), dict(host_build=True)],
                         ids=["aos", "soa", "copy_back", "fp64", "strict", "host_build"])
def test_grouped_equals_given_and_oracle(sls, name, opts):
    mesh = MESHES[name]()
    xy, info, acc, hist = _run(sls, mesh, 40, 1e-9, numbering="grouped", **opts)
    kxy, kinfo, kacc, khist = _run(sls, mesh, 40, 1e-9, numbering="given", **opts)
    assert np.array_equal(xy, kxy)
    assert np.array_equal(acc, kacc)
    for key in ("iterations", "converged", "accepted_last", "maxd2_last", "fp64_fallbacks"):
        assert info[key] == kinfo[key], key
    # counts and minimum exact; the mean is a sum of atomic additions, whose
    # order varies from run to run
    assert np.array_equal(hist[0], khist[0]) and hist[1] == khist[1]
    assert abs(hist[2] - khist[2]) <= 1e-12 * abs(khist[2])
    rxy, rinfo, racc = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary).smooth(
        mesh.xy, 40, tol=1e-9, strict=opts.get("strict", False))
    assert np.array_equal(xy, rxy)
    assert info["iterations"] == rinfo["iterations"]
    assert np.array_equal(acc, racc)


def test_binary32_grouped(sls):
    # binary32 meshes keep the caller's numbering even when asked: equal runs
    mesh = MESHES["grid_ragged"]()
    a = _run(sls, mesh, 25, 0.0, precision=32, numbering="grouped")
    b = _run(sls, mesh, 25, 0.0, precision=32, numbering="given")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])


def test_set_coords_and_device_transfers(sls):
    import torch
    mesh = MESHES["delaunay_random"]()
    rng = np.random.default_rng(5)
    start = mesh.xy + np.where(mesh.boundary[:, None] == 0, rng.uniform(-1e-3, 1e-3, mesh.xy.shape), 0.0)
    outs = []
    for numbering in ("grouped", "given"):
        with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, numbering=numbering) as g:
            g.set_coords(start)
            assert np.array_equal(g.coords(), start)
            g.smooth(7)
            dev = g.coords_device()
            g.set_coords(dev * 1.0)                      # device round trip in the caller's numbering
            g.smooth(5)
            idx = torch.tensor([0, 17, mesh.n - 1, 4321], dtype=torch.int32, device="cuda")
            got = torch.empty((4, 2), dtype=torch.float64, device="cuda")
            g.gather(idx, got)
            assert np.array_equal(got.cpu().numpy(), g.coords()[[0, 17, mesh.n - 1, 4321]])
            g.scatter(idx[:2], got[:2] + 0.25)
            xy = g.coords()
            assert np.array_equal(xy[[0, 17]], got[:2].cpu().numpy() + 0.25)
            outs.append(xy)
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_and_batch_on_grouped_meshes(sls):
    import torch
    mesh = MESHES["grid_ragged"]()
    ref_xy, ref_info, _ = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary).smooth(mesh.xy, 31, tol=1e-12)
    for passes in (30, 31):  # the result ends in either buffer
        with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, numbering="grouped") as g:
            xin = torch.from_numpy(mesh.xy.copy()).cuda()
            xout = torch.empty_like(xin)
            info = g.smooth_noalloc(xin, xout, passes)
            want, _, _ = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary).smooth(mesh.xy, passes)
            assert info["iterations"] == passes
            assert np.array_equal(xout.cpu().numpy(), want)
    meshes = [sls.Mesh(m.xy, m.tri, m.boundary, numbering="grouped") for m in (mesh, MESHES["delaunay_random"](), MESHES["tiny"]())]
    try:
        with sls.Batch(meshes, [31, 12, 9], [1e-12, 0.0, 0.0]) as b:
            b.smooth()
            assert np.array_equal(b.coords(0), ref_xy)
            m1 = MESHES["delaunay_random"]()
            want, _, _ = oracle.OracleMesh(m1.xy, m1.tri, m1.boundary).smooth(m1.xy, 12)
            assert np.array_equal(b.coords(1), want)
    finally:
        for g in meshes:
            g.close()


def test_skip_unchanged_keeps_the_callers_numbering(sls):
    # grouping is not applied with skip_unchanged (even when asked for);
    # results equal either way
    mesh = MESHES["grid_ragged"]()
    a = _run(sls, mesh, 60, 1e-9, skip_unchanged=True, numbering="grouped")
    b = _run(sls, mesh, 60, 1e-9, numbering="grouped")
    assert np.array_equal(a[0], b[0]) and a[1]["iterations"] == b[1]["iterations"]


def test_numbering_option_checked(sls):
    mesh = MESHES["tiny"]()
    with pytest.raises(sls.SlsError) as e:
        sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, numbering=3)
    assert e.value.code == 1


@pytest.mark.parametrize("kernel", ["auto", "fp64"])
def test_grouped_edge_meshes(sls, kernel):
    # a node of degree 40 (past the fast path's 16 and the device build's 32
    # triangles: host build, exact path), the dart whose centre inverts a
    # triangle, and a lone triangle with nothing free
    k = 40
    ang = np.linspace(0, 2 * np.pi, k, endpoint=False)
    fan = meshgen.Mesh(xy=np.vstack([np.c_[np.cos(ang) * (1 + 0.3 * np.sin(5 * ang)), np.sin(ang)], [[0.05, -0.02]]]),
                       tri=np.array([[k, j, (j + 1) % k] for j in range(k)], dtype=np.int32),
                       boundary=(np.arange(k + 1) < k).astype(np.uint8))
    dart = meshgen.Mesh(xy=np.array([[4.0, 0.0], [-1.0, 1.0], [2.0, 0.0], [-1.0, -1.0], [2.5, 0.0]]),
                        tri=np.array([[4, 0, 1], [4, 1, 2], [4, 2, 3], [4, 3, 0]], dtype=np.int32),
                        boundary=np.array([1, 1, 1, 1, 0], np.uint8))
    one = meshgen.Mesh(xy=np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), tri=np.array([[0, 1, 2]], np.int32),
                       boundary=np.ones(3, np.uint8))
    for name, mesh, iters in (("fan-40", fan, 3), ("dart", dart, 2), ("one", one, 4)):
        xy, info, acc, _ = _run(sls, mesh, iters, 0.0, numbering="grouped", kernel=kernel)
        rxy, rinfo, racc = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary).smooth(mesh.xy, iters)
        assert np.array_equal(xy, rxy), name
        assert np.array_equal(acc, racc), name
        assert info["accepted_last"] == rinfo["accepted_last"] and info["maxd2_last"] == rinfo["maxd2_last"], name
