"""Domain decomposition of one mesh (paper_1502_00355_gb300/domain.py), on the
CPU: the partition and its exchange plan, and the whole distributed pass loop
run as gloo ranks (world size 2 and 3) with the oracle doing each rank's
subdomain passes.  The assembled coordinates, the iteration count, the last
pass's accepted count and largest squared move must equal a single oracle
run on the whole mesh, bit for bit (Form A reads only the previous pass, so
the split changes nothing)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import meshgen  # noqa: E402
import oracle  # noqa: E402
from paper_1502_00355_gb300 import domain  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _meshes():
    return {
        "small": meshgen.small_grid(),
        "random": meshgen.jittered_grid(41, 29, 0.35, 17, numbering="random"),
        "pulled": meshgen.jittered_grid(48, 40, 0.35, 23, numbering="morton", pull_fraction=0.05,
                                        pull_centres=16),
        "delaunay": meshgen.delaunay_random(1500, 5),
    }


@pytest.mark.parametrize("name", ["small", "random", "pulled", "delaunay"])
@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_partition_covers_the_mesh_and_each_owned_ring(name, world):
    mesh = _meshes()[name]
    nbr_ptr, nbr, tri_ptr, tri_of, fixed = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary).adjacency()
    subs = [domain.partition(mesh.n, mesh.tri, mesh.boundary, world, r) for r in range(world)]
    owned = np.concatenate([s.nodes[s.owned] for s in subs])
    assert np.array_equal(owned, np.arange(mesh.n))
    for s in subs:
        assert np.all(np.diff(s.nodes) > 0)
        local = set(s.nodes.tolist())
        ghosts = np.setdiff1d(np.arange(s.n_local), s.owned)
        # ghosts are fixed, owned nodes keep their flags
        assert np.all(s.boundary[ghosts] == 1)
        assert np.array_equal(s.boundary[s.owned], mesh.boundary[s.lo:s.hi])
        # every owned node: all neighbours and all incident triangles are local,
        # the triangles with their stored vertex order
        tri_local_g = s.nodes[s.tri]
        tset = {tuple(t) for t in tri_local_g.tolist()}
        for i in range(s.lo, s.hi):
            assert set(nbr[nbr_ptr[i]:nbr_ptr[i + 1]].tolist()) <= local
            for t in tri_of[tri_ptr[i]:tri_ptr[i + 1]]:
                assert tuple(mesh.tri[t].tolist()) in tset
        # the ghosts are exactly what the peers send
        recv_all = np.concatenate([v for v in s.recv.values()]) if s.recv else np.zeros(0, np.int32)
        assert np.array_equal(np.sort(recv_all), ghosts)
        for p, v in s.recv.items():
            peer = subs[p]
            assert np.array_equal(s.nodes[v], peer.nodes[peer.send[s.rank]])
            assert np.all((s.nodes[v] >= peer.lo) & (s.nodes[v] < peer.hi))


class OracleBackend:
    """Test stand-in for the library: the oracle runs the subdomain's passes."""

    def __init__(self, sub, xy_local):
        self.sub = sub
        self.om = oracle.OracleMesh(xy_local, sub.tri, sub.boundary)
        self.xy = np.ascontiguousarray(xy_local, dtype=np.float64).copy()

    def step(self):
        nxt, _acc, maxd2, nacc = self.om.sweep(self.xy)
        self.xy = nxt
        return maxd2, nacc

    def buffer(self, k):
        return torch.empty((k, 2), dtype=torch.float64)

    def gather(self, peer, out):
        out.copy_(torch.from_numpy(self.xy[self.sub.send[peer]]))

    def scatter(self, peer, values):
        self.xy[self.sub.recv[peer]] = values.numpy()

    def coords(self):
        return self.xy


def _worker(rank, world, port, name, iters, tol, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.build()
    mesh = _meshes()[name]
    sub = domain.partition(mesh.n, mesh.tri, mesh.boundary, world, rank)
    be = OracleBackend(sub, mesh.xy[sub.nodes])
    dm = domain.DistributedMesh(sub, be, mesh.xy[sub.lo:sub.hi])
    info = dm.smooth(iters, tol)
    parts = [None] * world
    dist.all_gather_object(parts, (sub.lo, dm.owned_coords()))
    out[rank] = (info, parts, dm.diag)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name,world,iters,tol", [("small", 2, 10, 0.0), ("random", 2, 25, 1e-6),
                                                   ("pulled", 3, 30, 0.0), ("delaunay", 2, 200, 1e-9)])
def test_decomposed_passes_equal_one_rank(name, world, iters, tol):
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, name, iters, tol, out), nprocs=world, join=True)
    mesh = _meshes()[name]
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary)
    ref_xy, ref_info, _ = om.smooth(mesh.xy, iters, tol=tol)
    info, parts, diag = out[0]
    got = np.concatenate([xy for _lo, xy in sorted(parts, key=lambda p: p[0])])
    assert np.array_equal(got, ref_xy)
    for key in ("iterations", "converged", "accepted_last", "maxd2_last"):
        assert info[key] == ref_info[key], key
    for r in range(1, world):
        assert out[r][0] == info
    # D of the whole mesh, with the library's formula
    lo, hi = mesh.xy.min(axis=0), mesh.xy.max(axis=0)
    assert diag == domain.bbox_diagonal(lo[0], hi[0], lo[1], hi[1])
