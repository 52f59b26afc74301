"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

The bar is bit-exactness: coordinates, accept decisions, iteration counts,
accepted counts and the largest squared move must be identical.
"""
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


def _assert_same(xy_gpu, xy_ref, what=""):
    if not np.array_equal(xy_gpu, xy_ref):
        bad = np.flatnonzero((xy_gpu != xy_ref).any(1))
        i = bad[0]
        raise AssertionError(f"{what}: {bad.size} nodes differ; first {i}: gpu {xy_gpu[i].tolist()} "
                             f"oracle {xy_ref[i].tolist()}")


def _run_both(sls, mesh, iters, tol=0.0, strict=False, omp=False, boundary="given", **opts):
    bnd = mesh.boundary if boundary == "given" else None
    om = oracle.OracleMesh(mesh.xy, mesh.tri, bnd, openmp=omp)
    ref_xy, ref_info, ref_acc = om.smooth(mesh.xy, iters, tol=tol, strict=strict)
    with sls.Mesh(mesh.xy, mesh.tri, bnd, strict=strict, record_accept=True, **opts) as g:
        info = g.smooth(iters, tol)
        xy = g.coords()
        acc = g.accept_mask()
    return (xy, info, acc), (ref_xy, ref_info, ref_acc)


def _check(got, ref, what):
    (xy, info, acc), (rxy, rinfo, racc) = got, ref
    _assert_same(xy, rxy, what)
    assert info["iterations"] == rinfo["iterations"], what
    assert info["converged"] == rinfo["converged"], what
    assert info["accepted_last"] == rinfo["accepted_last"], what
    assert info["maxd2_last"] == rinfo["maxd2_last"], what
    if rinfo["iterations"] > 0:
        assert np.array_equal(acc, racc), what


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("copy_back", [False, True])
def test_small_grid_bit_exact(sls, kernel, layout, copy_back):
    # 64x64 vertices, 10 passes (the small workload)
    mesh = meshgen.small_grid()
    got, ref = _run_both(sls, mesh, 10, kernel=kernel, layout=layout, copy_back=copy_back)
    _check(got, ref, f"{kernel}/{layout}/cb={copy_back}")


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("strict", [False, True])
def test_strict_mode_and_derived_boundary(sls, kernel, strict):
    mesh = meshgen.jittered_grid(37, 23, 0.4, 5, numbering="random")
    got, ref = _run_both(sls, mesh, 17, strict=strict, boundary="derived", kernel=kernel)
    _check(got, ref, f"strict={strict}")


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("block", [32, 64, 128, 512, 1024])
def test_ragged_sizes_and_block_sizes(sls, kernel, block):
    # node counts that are not multiples of the block or the warp
    for nx, ny in [(3, 3), (5, 7), (33, 31), (129, 67)]:
        mesh = meshgen.jittered_grid(nx, ny, 0.3, nx * 1000 + ny, numbering="morton")
        got, ref = _run_both(sls, mesh, 6, kernel=kernel, block_size=block)
        _check(got, ref, f"{nx}x{ny} block={block}")


@pytest.mark.parametrize("kernel", KERNELS)
def test_tolerance_stop_matches(sls, kernel):
    mesh = meshgen.jittered_grid(40, 40, 0.3, 8)
    for tol, chunk in [(1e-4, 16), (1e-4, 1), (1e-4, 5), (1e-6, 3), (10.0, 16)]:
        got, ref = _run_both(sls, mesh, 500, tol=tol, kernel=kernel, passes_per_check=chunk)
        _check(got, ref, f"tol={tol} chunk={chunk}")
    assert ref[1]["converged"] == 1


@pytest.mark.parametrize("kernel", KERNELS)
def test_resume_zero_passes_and_set_coords(sls, kernel):
    mesh = meshgen.jittered_grid(30, 50, 0.35, 3)
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    ref, _, _ = om.smooth(mesh.xy, 12)
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, kernel=kernel) as g:
        info = g.smooth(0)
        assert info["iterations"] == 0
        _assert_same(g.coords(), mesh.xy, "zero passes")
        g.smooth(7)
        g.smooth(5)
        _assert_same(g.coords(), ref, "7 + 5 passes")
        g.set_coords(mesh.xy)
        g.smooth(12)
        _assert_same(g.coords(), ref, "after set_coords")


@pytest.mark.parametrize("kernel", KERNELS)
def test_hexagon_and_fan_cases(sls, kernel):
    # the hand-worked hexagon: the centre lands exactly on (0, 0)
    s = 0.8660254037844386
    xy = np.array([[1.0, 0.0], [0.5, s], [-0.5, s], [-1.0, 0.0], [-0.5, -s], [0.5, -s], [0.125, -0.0625]])
    tri = np.array([[6, k, (k + 1) % 6] for k in range(6)], dtype=np.int32)
    with sls.Mesh(xy, tri, kernel=kernel) as g:
        info = g.smooth(1)
        out = g.coords()
    assert out[6, 0] == 0.0 and out[6, 1] == 0.0 and info["accepted_last"] == 1
    # a node of degree 40 (long loops) and the dart whose centre inverts a triangle
    k = 40
    ang = np.linspace(0, 2 * np.pi, k, endpoint=False)
    xy = np.vstack([np.c_[np.cos(ang) * (1 + 0.3 * np.sin(5 * ang)), np.sin(ang)], [[0.05, -0.02]]])
    tri = np.array([[k, j, (j + 1) % k] for j in range(k)], dtype=np.int32)
    mesh = meshgen.Mesh(xy=xy, tri=tri, boundary=(np.arange(k + 1) < k).astype(np.uint8))
    got, ref = _run_both(sls, mesh, 3, kernel=kernel)
    _check(got, ref, "fan-40")
    dart = meshgen.Mesh(xy=np.array([[4.0, 0.0], [-1.0, 1.0], [2.0, 0.0], [-1.0, -1.0], [2.5, 0.0]]),
                        tri=np.array([[4, 0, 1], [4, 1, 2], [4, 2, 3], [4, 3, 0]], dtype=np.int32),
                        boundary=np.array([1, 1, 1, 1, 0], np.uint8))
    got, ref = _run_both(sls, dart, 2, kernel=kernel)
    _check(got, ref, "dart")
    assert got[2][4] == 0


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("boundary", ["given", "derived"])
def test_delaunay_random_points(sls, kernel, boundary):
    # the paper's mesh family: valence 3 to 12 and more, hull nodes fixed,
    # some nodes past the screened kernel's degree limit
    mesh = meshgen.delaunay_random(20000, 17, numbering="random")
    got, ref = _run_both(sls, mesh, 40, boundary=boundary, kernel=kernel)
    _check(got, ref, f"delaunay-20k-{boundary}")


def test_delaunay_paper_size_to_tolerance(sls):
    # 100,000 points (the paper's largest mesh), smoothed to the tolerance
    mesh = meshgen.delaunay_mesh()
    got, ref = _run_both(sls, mesh, 300, tol=1e-9, omp=True)
    _check(got, ref, "delaunay-100k")
    assert got[1]["converged"] == 1


@pytest.mark.parametrize("kernel", KERNELS)
def test_histogram_matches_oracle(sls, kernel):
    mesh = meshgen.jittered_grid(100, 80, 0.45, 31)
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    xy, _, _ = om.smooth(mesh.xy, 5)
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, kernel=kernel) as g:
        for layout_xy in (mesh.xy, xy):
            g.set_coords(layout_xy)
            for nb, lo, hi in [(20, -1.0, 1.0), (7, 0.2, 0.9), (1, -1.0, 1.0)]:
                c, qmin, qmean = g.histogram(nb, lo, hi)
                rc, rqmin, rqmean = om.histogram(layout_xy, nb, lo, hi)
                assert np.array_equal(c, rc)
                assert qmin == rqmin
                assert qmean == pytest.approx(rqmean, rel=1e-12)


@pytest.mark.parametrize("kernel", KERNELS)
def test_medium_grid_all_forms(sls, kernel):
    # 1024x1024 vertices, 100 passes, {ping-pong, copy-back} x {AoS, SoA} x
    # {Morton, random numbering}; every run bit-identical to the oracle, and
    # the two numberings identical to each other after un-permuting.
    results = {}
    for numbering in ("morton", "random"):
        mesh = meshgen.medium_grid(numbering)
        om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary, openmp=True)
        rxy, rinfo, racc = om.smooth(mesh.xy, 100)
        for layout in ("aos", "soa"):
            for cb in (False, True):
                with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, kernel=kernel, layout=layout,
                              copy_back=cb, record_accept=True) as g:
                    info = g.smooth(100)
                    xy = g.coords()
                    acc = g.accept_mask()
                _check((xy, info, acc), (rxy, rinfo, racc), f"{numbering}/{layout}/cb={cb}")
        results[numbering] = meshgen.unpermute(rxy, mesh)
    assert np.array_equal(results["morton"], results["random"])


def test_large_grid_sampled_passes(sls):
    # 4096x4096 vertices with clustered pulls: the timed configuration.
    # Sampled nodes of passes 1, 2, 50 and 200 recomputed one by one by the
    # oracle from the GPU's previous pass; the GPU stays in the timed launch
    # configuration (default kernel, AoS, ping-pong).
    mesh = meshgen.large_grid()
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(mesh.n, 20000, replace=False))
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, record_accept=True) as g:
        done = 0
        for target in (1, 2, 50, 200):
            if target - 1 > done:
                g.smooth(target - 1 - done)
                done = target - 1
            prev = g.coords()
            info = g.smooth(1)
            done += 1
            cur = g.coords()
            acc = g.accept_mask()
            out, racc, d2, _, _, _ = om.update_nodes(prev, sample)
            _assert_same(cur[sample], out, f"pass {target}")
            assert np.array_equal(acc[sample], racc), f"pass {target}"
            # property at full size: every node moved by at most the reported max
            d = cur - prev
            dd = (d * d).sum(1)
            assert dd.max() == pytest.approx(info["maxd2_last"], rel=1e-12)
            assert info["accepted_last"] >= int((dd > 0).sum())
            assert np.array_equal(cur[mesh.boundary == 1], mesh.xy[mesh.boundary == 1])


def test_large_grid_full_run_bit_exact(sls):
    # The whole timed configuration: 4096x4096 vertices with clustered pulls,
    # smoothed to the tolerance in the launch configuration the benchmark
    # times (default kernel, AoS, ping-pong, no accept mask), every coordinate
    # against the OpenMP oracle; a second run records the last pass's
    # decisions
    mesh = meshgen.large_grid()
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary, openmp=True)
    rxy, rinfo, racc = om.smooth(mesh.xy, 200, tol=1e-9)
    assert rinfo["iterations"] == 77 and rinfo["converged"] == 1
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary) as g:
        info = g.smooth(200, 1e-9)
        xy = g.coords()
    _assert_same(xy, rxy, "4096x4096 to tolerance")
    for key in ("iterations", "converged", "accepted_last", "maxd2_last"):
        assert info[key] == rinfo[key], key
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, record_accept=True) as g:
        g.smooth(200, 1e-9)
        assert np.array_equal(g.accept_mask(), racc)


@pytest.mark.parametrize("transform", ["shift_negative", "tiny", "huge", "far_offset", "signed_zeros",
                                       "denormal_scale", "mixed_binades"])
def test_screened_kernel_domain_edges(sls, transform):
    # the screened kernel's fast path has limits (exponent window, sign,
    # zeros); every case must stay bit-identical through its fallbacks
    mesh = meshgen.jittered_grid(45, 38, 0.35, 99, numbering="random")
    xy = mesh.xy.copy()
    if transform == "shift_negative":
        xy -= 0.5
    elif transform == "tiny":
        xy *= 1e-9
    elif transform == "huge":
        xy *= 1e12
    elif transform == "far_offset":
        xy += np.array([1e6, -3e5])
    elif transform == "signed_zeros":
        xy -= 0.5
        xy[np.abs(xy) < 0.05] = -0.0
    elif transform == "denormal_scale":
        xy *= 2.0 ** -1040
    elif transform == "mixed_binades":
        xy = xy * 3.0 - 1.0
    mesh.xy = xy
    for strict in (False, True):
        got, ref = _run_both(sls, mesh, 12, strict=strict, kernel="filtered")
        _check(got, ref, f"{transform} strict={strict}")


def test_screened_matches_fp64_on_many_meshes(sls):
    rng = np.random.default_rng(12345)
    for r in range(25):
        nx, ny = int(rng.integers(3, 60)), int(rng.integers(3, 60))
        mesh = meshgen.jittered_grid(nx, ny, float(rng.uniform(0.0, 0.49)), 500 + r,
                                     numbering=["natural", "morton", "random"][r % 3],
                                     pull_fraction=0.1 if r % 4 == 0 else 0.0)
        outs = []
        for kernel in ("fp64", "filtered"):
            # long enough to reach the near-converged regime, where decisions
            # hinge on differences down to the FP64 rounding level
            with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, kernel=kernel, record_accept=True) as g:
                info = g.smooth(150)
                outs.append((g.coords(), g.accept_mask(), info))
        _assert_same(outs[1][0], outs[0][0], f"mesh {r}")
        assert np.array_equal(outs[1][1], outs[0][1])
        for key in ("iterations", "accepted_last", "maxd2_last"):
            assert outs[1][2][key] == outs[0][2][key]


def test_l2_window_same_results(sls):
    # the persisting-L2 option changes caching only
    for mesh, iters in ((meshgen.small_grid(), 30), (meshgen.jittered_grid(300, 200, 0.35, 4), 60)):
        got, ref = _run_both(sls, mesh, iters, tol=1e-10, l2_window=True)
        _check(got, ref, f"l2 window n={mesh.n}")
        got, ref = _run_both(sls, mesh, iters, l2_window=True, layout="soa", copy_back=True)
        _check(got, ref, f"l2 window soa/copy-back n={mesh.n}")


def _degenerate_mesh():
    """A jittered grid with free nodes moved exactly onto a neighbour
    (zero-length edges; triangles whose three vertices coincide have edge sum
    0 and alpha 0), onto the midpoint of the opposite edge (zero or
    rounding-level area), plus the inverted triangles this leaves."""
    mesh = meshgen.jittered_grid(40, 33, 0.3, 77, numbering="morton")
    xy = mesh.xy.copy()
    free = mesh.boundary == 0
    rng = np.random.default_rng(5)
    for k, t in enumerate(rng.choice(mesh.m, 60, replace=False)):
        a, b, c = mesh.tri[t]
        if not free[a]:
            continue
        if k % 3 == 0:
            xy[a] = xy[b]
        elif k % 3 == 1:
            xy[a] = 0.5 * (xy[b] + xy[c])
        else:
            xy[a] = xy[b]
            if free[c]:
                xy[c] = xy[b]
    mesh.xy = xy
    return mesh


@pytest.mark.parametrize("variant", [{"kernel": "fp64"}, {"kernel": "filtered"}, {"form": "B"},
                                     {"precision": 32}, {"precision": 32, "form": "B"}])
def test_degenerate_triangles_and_no_free_node(sls, variant):
    form, precision = variant.get("form", "A"), variant.get("precision", 64)
    deg = _degenerate_mesh()
    P = deg.xy[deg.tri]
    e = [P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 2] - P[:, 1]]
    assert (sum((v * v).sum(1) for v in e) == 0.0).any()  # some triangle collapsed to a point
    # a single triangle: every node is on the boundary, nothing may move, and
    # every pass still counts (the tolerance stops after the first)
    one = meshgen.Mesh(xy=np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), tri=np.array([[0, 1, 2]], np.int32),
                       boundary=np.ones(3, np.uint8))
    for mesh, bnd, what in [(deg, deg.boundary, "degenerate"), (one, None, "single triangle")]:
        for strict in (False, True):
            for tol in (0.0, 1e-3):
                om = oracle.OracleMesh(mesh.xy, mesh.tri, bnd)
                ref = om.smooth(mesh.xy, 8, tol=tol, strict=strict, form=form, precision=precision)
                with sls.Mesh(mesh.xy, mesh.tri, bnd, strict=strict, record_accept=True, **variant) as g:
                    info = g.smooth(8, tol)
                    got = (g.coords(), info, g.accept_mask())
                _check(got, ref, f"{what} {variant} strict={strict} tol={tol}")
    assert ref[1]["iterations"] == 1 and ref[1]["converged"] == 1
