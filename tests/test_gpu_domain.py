"""Domain decomposition on the GPU: subdomains of one mesh, each an sls_mesh
driven by domain.LibraryBackend, with the ghost exchange through
sls_gather_coords / sls_scatter_coords.  The ranks are emulated in one
process on one GPU, one after another (no kernel waits on another): every
subdomain runs its pass, then the exchange lists move device to device.
The assembled result must equal the whole mesh smoothed by sls_smooth and
the oracle, bit for bit."""
import numpy as np
import pytest

import meshgen
import oracle
from paper_1502_00355_gb300 import domain

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


def _run_split(mesh, world, iters, tol, **options):
    subs = [domain.partition(mesh.n, mesh.tri, mesh.boundary, world, r) for r in range(world)]
    bes = [domain.LibraryBackend(s, mesh.xy[s.nodes], **options) for s in subs]
    lo, hi = mesh.xy.min(axis=0), mesh.xy.max(axis=0)
    diag = domain.bbox_diagonal(lo[0], hi[0], lo[1], hi[1])
    thr = (tol * diag) * (tol * diag) if tol > 0 else None
    it, conv, d2, nacc = 0, 0, 0.0, 0
    for _ in range(iters):
        res = [be.step() for be in bes]
        msgs = {}
        for r, s in enumerate(subs):
            for p, v in s.send.items():
                buf = bes[r].buffer(v.size)
                bes[r].gather(p, buf)
                msgs[(r, p)] = buf
        for r, s in enumerate(subs):
            for p in s.recv:
                bes[r].scatter(p, msgs[(p, r)])
        d2 = max(x[0] for x in res)
        nacc = sum(x[1] for x in res)
        it += 1
        if thr is not None and d2 < thr:
            conv = 1
            break
    xy = np.concatenate([be.coords()[s.owned] for be, s in zip(bes, subs)])
    for be in bes:
        be.close()
    return xy, dict(iterations=it, converged=conv, accepted_last=nacc, maxd2_last=d2)


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("numbering", ["given", "grouped"])
def test_subdomains_equal_the_whole_mesh(sls, world, layout, numbering):
    # with numbering = grouped every subdomain is renumbered inside the
    # library, and the exchange lists (caller's ids) go through its maps
    mesh = meshgen.jittered_grid(300, 200, 0.35, 5, numbering="morton", pull_fraction=0.05, pull_centres=64)
    xy, info = _run_split(mesh, world, 60, 1e-9, layout=layout, numbering=numbering)
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, layout=layout) as g:
        ref = g.smooth(60, 1e-9)
        ref_xy = g.coords()
    assert np.array_equal(xy, ref_xy)
    for key in ("iterations", "converged", "accepted_last", "maxd2_last"):
        assert info[key] == ref[key], key


def test_subdomains_equal_the_oracle_random_numbering(sls):
    mesh = meshgen.jittered_grid(90, 70, 0.35, 8, numbering="random")
    xy, info = _run_split(mesh, 3, 15, 0.0)
    rxy, rinfo, _ = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary).smooth(mesh.xy, 15)
    assert np.array_equal(xy, rxy)
    assert info["accepted_last"] == rinfo["accepted_last"] and info["maxd2_last"] == rinfo["maxd2_last"]


def test_gather_scatter_checks_ids(sls):
    import torch
    mesh = meshgen.jittered_grid(20, 20, 0.3, 3)
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary) as g:
        idx = torch.tensor([0, 5, 399], dtype=torch.int32, device="cuda")
        out = torch.empty((3, 2), dtype=torch.float64, device="cuda")
        g.gather(idx, out)
        assert np.array_equal(out.cpu().numpy(), mesh.xy[[0, 5, 399]])
        g.scatter(idx, out * 0.5)
        got = g.coords()
        assert np.array_equal(got[[0, 5, 399]], mesh.xy[[0, 5, 399]] * 0.5)
        bad = torch.tensor([1, 400], dtype=torch.int32, device="cuda")
        with pytest.raises(sls.SlsError) as e:
            g.gather(bad, out[:2])
        assert e.value.code == 1
        with pytest.raises(sls.SlsError) as e:
            g.scatter(torch.tensor([-1], dtype=torch.int32, device="cuda"), out[:1])
        assert e.value.code == 1
        empty = torch.empty(0, dtype=torch.int32, device="cuda")
        g.gather(empty, out[:0])


def test_distributed_driver_at_one_rank(sls):
    """domain.DistributedMesh with the library backend and no process group
    (the path bench.py --decompose runs per rank): the stop rule with D from
    the owned coordinates gives the whole mesh's run."""
    mesh = meshgen.jittered_grid(120, 90, 0.35, 12, numbering="morton")
    sub = domain.partition(mesh.n, mesh.tri, mesh.boundary, 1, 0)
    be = domain.LibraryBackend(sub, mesh.xy[sub.nodes])
    dm = domain.DistributedMesh(sub, be, mesh.xy[sub.lo:sub.hi], device="cuda")
    info = dm.smooth(200, 1e-9)
    xy = dm.owned_coords()
    be.close()
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary) as g:
        ref = g.smooth(200, 1e-9)
        assert np.array_equal(xy, g.coords())
    for key in ("iterations", "converged", "accepted_last", "maxd2_last"):
        assert info[key] == ref[key], key
    assert dm.diag == g.diag
