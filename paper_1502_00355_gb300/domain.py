"""One mesh smoothed by several GPUs: domain decomposition of the Form-A pass.

Form A computes pass q+1 from the coordinates of pass q alone (Eq. 2), and a
node's update reads only its one-ring: its neighbours and its incident
triangles (Sections 2.1 and 3.3.4).  So the nodes are split into contiguous
id ranges, one per rank (with a Morton numbering these are compact pieces of
the domain), and each rank holds a subdomain mesh: every triangle with a
vertex in its range, and the vertices of those triangles.  Vertices owned by
other ranks are ghosts, fixed in the subdomain's mesh.  A pass on the
subdomain then updates every owned node exactly as a pass on the whole mesh
does, because

* an owned node has all its incident triangles, hence all its neighbours,
  in the subdomain, with the same stored vertex order;
* local ids ascend with the global ids, so the summation order (ascending
  creation coordinates, then id) is the same;
* ghosts hold their owners' coordinates of pass q: after every pass each
  rank sends the coordinates of its nodes that are ghosts elsewhere and
  writes what it receives into its ghosts (the exchange step);
* the largest squared move of a pass is the maximum over ranks (one
  all-reduce), compared with (tol D)^2, D the bounding-box diagonal of the
  whole mesh's creation coordinates (reduced once at set-up).

The results are therefore bit-identical to one GPU.  This module holds the
host logic: the partition, the exchange plan and the pass loop over
torch.distributed point-to-point messages (NCCL between GPUs, gloo on the
CPU).  The pass itself and the ghost gather/scatter run in the library's
kernels (``LibraryBackend``); the stop rule is the same as the library's.
Form A in FP64 only (a Form-B colouring depends on the numbering, so a
subdomain would colour differently).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Subdomain:
    rank: int
    world: int
    lo: int                      # owned global ids: [lo, hi)
    hi: int
    nodes: np.ndarray            # global ids of the subdomain's nodes, ascending (int64)
    tri: np.ndarray              # (m_local, 3) int32 local ids, stored vertex order kept
    boundary: np.ndarray         # (n_local,) uint8: owned nodes keep their flags, ghosts are fixed
    owned: np.ndarray            # local ids of the owned nodes (int32, ascending)
    send: dict = field(default_factory=dict)  # peer -> local ids of owned nodes the peer holds as ghosts
    recv: dict = field(default_factory=dict)  # peer -> local ids of ghosts the peer owns

    @property
    def n_local(self) -> int:
        return int(self.nodes.size)


def ranges(n: int, world: int) -> np.ndarray:
    """Bounds of the contiguous owned ranges: rank r owns [b[r], b[r+1])."""
    return np.array([(r * n) // world for r in range(world + 1)], dtype=np.int64)


def partition(n: int, tri: np.ndarray, boundary: np.ndarray, world: int, rank: int) -> Subdomain:
    """The subdomain of `rank` out of `world` for a mesh of n nodes (every
    rank must own at least one node: world <= n)."""
    if boundary is None:
        raise ValueError("the decomposed path needs the boundary flags of the whole mesh")
    if not 1 <= world <= n or not 0 <= rank < world:
        raise ValueError("need 1 <= world <= n and 0 <= rank < world")
    tri = np.ascontiguousarray(tri, dtype=np.int64).reshape(-1, 3)
    b = ranges(n, world)
    lo, hi = int(b[rank]), int(b[rank + 1])
    owner = np.searchsorted(b, tri, side="right") - 1          # (m, 3) rank of each vertex
    mine = (owner == rank).any(axis=1)
    local_tri_g = tri[mine]
    nodes = np.union1d(np.arange(lo, hi, dtype=np.int64), np.unique(local_tri_g))
    loc = np.searchsorted(nodes, local_tri_g).astype(np.int32)
    bnd = np.ones(nodes.size, dtype=np.uint8)
    owned = np.searchsorted(nodes, np.arange(lo, hi, dtype=np.int64)).astype(np.int32)
    bnd[owned] = np.asarray(boundary, dtype=np.uint8)[lo:hi]
    sub = Subdomain(rank=rank, world=world, lo=lo, hi=hi, nodes=nodes, tri=loc, boundary=bnd, owned=owned)
    # a triangle with vertices of ranks r and p makes r's vertices ghosts of p
    # and p's vertices ghosts of r
    own_t = owner[mine]
    for p in range(world):
        if p == rank:
            continue
        with_p = (own_t == p).any(axis=1)
        if not with_p.any():
            continue
        tp = local_tri_g[with_p]
        op = own_t[with_p]
        send_g = np.unique(tp[op == rank])
        recv_g = np.unique(tp[op == p])
        sub.send[p] = np.searchsorted(nodes, send_g).astype(np.int32)
        sub.recv[p] = np.searchsorted(nodes, recv_g).astype(np.int32)
    return sub


def bbox_diagonal(xmin: float, xmax: float, ymin: float, ymax: float) -> float:
    """D of the stop rule, with the library's rounding: sqrt(wx*wx + wy*wy)."""
    wx, wy = xmax - xmin, ymax - ymin
    return math.sqrt(wx * wx + wy * wy)


class LibraryBackend:
    """The subdomain's passes and ghost transfers in the library's kernels
    (one sls_mesh on this rank's GPU)."""

    def __init__(self, sub: Subdomain, xy_local: np.ndarray, **options):
        import torch

        import paper_1502_00355_gb300 as sls
        self.torch = torch
        self.mesh = sls.Mesh(xy_local, sub.tri, sub.boundary, **options)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.idx = {("s", p): torch.from_numpy(v).to(dev) for p, v in sub.send.items()}
        self.idx.update({("r", p): torch.from_numpy(v).to(dev) for p, v in sub.recv.items()})
        self.device = dev

    def step(self):
        info = self.mesh.smooth(1, 0.0)
        return info["maxd2_last"], info["accepted_last"]

    def buffer(self, k: int):
        return self.torch.empty((k, 2), dtype=self.torch.float64, device=self.device)

    def gather(self, peer: int, out):
        self.mesh.gather(self.idx[("s", peer)], out)

    def scatter(self, peer: int, values):
        self.mesh.scatter(self.idx[("r", peer)], values)

    def coords(self) -> np.ndarray:
        return self.mesh.coords()

    def close(self):
        self.mesh.close()


class DistributedMesh:
    """This rank's part of one mesh smoothed by `world` ranks.

    backend: step() -> (largest squared move, accepted count) of one pass on
    the subdomain; buffer(k) -> a (k, 2) float64 tensor the process group can
    send; gather(peer, out) / scatter(peer, values) move the exchange lists'
    coordinates; coords() -> the subdomain's coordinates."""

    def __init__(self, sub: Subdomain, backend, xy_owned_initial: np.ndarray, group=None, device="cpu"):
        import torch
        import torch.distributed as dist
        self.sub, self.backend, self.group, self.dev = sub, backend, group, device
        self.torch, self.dist = torch, dist
        # D of the whole mesh from each rank's owned creation coordinates
        if xy_owned_initial.size:
            ext = [float(xy_owned_initial[:, 0].min()), float(xy_owned_initial[:, 1].min()),
                   -float(xy_owned_initial[:, 0].max()), -float(xy_owned_initial[:, 1].max())]
        else:
            ext = [math.inf] * 4
        t = torch.tensor(ext, dtype=torch.float64, device=device)
        self._reduce(t, dist.ReduceOp.MIN)
        xmin, ymin, xmax, ymax = float(t[0]), float(t[1]), -float(t[2]), -float(t[3])
        self.diag = bbox_diagonal(xmin, xmax, ymin, ymax)
        self.sendbuf = {p: backend.buffer(v.size) for p, v in sub.send.items()}
        self.recvbuf = {p: backend.buffer(v.size) for p, v in sub.recv.items()}

    def _reduce(self, t, op):
        if self.dist.is_initialized() and self.dist.get_world_size(self.group) > 1:
            self.dist.all_reduce(t, op=op, group=self.group)

    def exchange(self):
        """Every ghost takes its owner's current coordinates."""
        for p, buf in self.sendbuf.items():
            self.backend.gather(p, buf)
        reqs = []
        for p in sorted(set(self.sendbuf) | set(self.recvbuf)):
            if p in self.recvbuf:
                reqs.append(self.dist.irecv(self.recvbuf[p], src=p, group=self.group))
            if p in self.sendbuf:
                reqs.append(self.dist.isend(self.sendbuf[p], dst=p, group=self.group))
        for r in reqs:
            r.wait()
        if reqs and str(self.dev).startswith("cuda"):
            # with NCCL, wait() orders only the current CUDA stream after the
            # transfer; the scatter runs on the mesh's own stream, so wait here
            torch = self.torch
            torch.cuda.synchronize()
        for p, buf in self.recvbuf.items():
            self.backend.scatter(p, buf)

    def smooth(self, max_iter: int, tol: float = 0.0) -> dict:
        """Up to max_iter passes, or until the first pass whose largest squared
        move is below (tol D)^2: the library's stop rule on the whole mesh."""
        torch, dist = self.torch, self.dist
        thr = (tol * self.diag) * (tol * self.diag) if tol > 0.0 else None
        it, conv, d2, nacc = 0, 0, 0.0, 0
        for _ in range(max_iter):
            d2, nacc = self.backend.step()
            self.exchange()
            t = torch.tensor([d2], dtype=torch.float64, device=self.dev)
            c = torch.tensor([nacc], dtype=torch.int64, device=self.dev)
            self._reduce(t, dist.ReduceOp.MAX)
            self._reduce(c, dist.ReduceOp.SUM)
            d2, nacc = float(t.item()), int(c.item())
            it += 1
            if thr is not None and d2 < thr:
                conv = 1
                break
        return dict(iterations=it, converged=conv, accepted_last=nacc, maxd2_last=d2)

    def owned_coords(self) -> np.ndarray:
        """Coordinates of the owned nodes, global ids lo .. hi-1."""
        return self.backend.coords()[self.sub.owned]
