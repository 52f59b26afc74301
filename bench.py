"""Benchmark: Smart Laplacian smoothing of the 4096x4096-vertex jittered grid.

One step = reset the coordinates to the initial mesh (device-to-device copy)
and smooth until 200 Jacobi passes or until the largest move of a pass is
below 1e-9 x the bounding-box diagonal.  The metric is node-updates per
second: nodes x passes executed / GPU time.  The mesh (16,777,216 nodes,
33,538,050 triangles, 5% of interior nodes pulled towards seeded centres,
Morton numbering) is synthetic and seeded; its coordinates (2 x 268 MB) and
adjacency (~1 GB) are larger than L2, so no L2 flush is needed between steps.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (a bounded number of passes per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import meshgen  # noqa: E402

WORKLOAD = "grid4096x4096_jitter0.35_pull5pct_morton"
MAX_PASSES = 200
TOL = 1e-9
METRIC = "node-updates/s"
CSRC = os.path.join(ROOT, "paper_1502_00355_gb300", "csrc")

# Figures that only an ncu capture gives (DRAM bytes, FP64 instruction mix),
# per kernel, from the capture named in `source` (its summary under
# profiles/ gives the command).  Each entry holds the SHA-256 of the sources
# the kernel was built from at capture time; once any of them changes the
# figures no longer describe the kernel and the bench line reports null.
PROFILE_FIGURES = {
    "pass_screened": {
        "files": ["pass_screened.cu", "screen.cuh", "node_exact.cuh", "div_small.cuh", "device.cuh",
                  "numbering.cu"],
        "sha256": "db9df0c964a12160525e9538431b1f0be20dcc278b1dfac8ff092a618a9895ef",
        "dram_bytes_per_node": (309215744 + 54800128) / (2048 * 2048),
        "fp64_warp_inst_per_32_nodes": (2132648 + 795086 + 157073) / (2048 * 2048 / 32),
        "source": "profiles/pass_screened_grid2048.md (2048x2048 capture, per node)",
    },
    "batch_pass": {
        "files": ["pass_screened.cu", "screen.cuh", "node_exact.cuh", "div_small.cuh", "device.cuh", "batch.cu",
                  "numbering.cu"],
        "sha256": "716f3492b8a2cc0ea034315c6b2a5adf884f3866f6fbc7a78722a5074c3f14d3",
        "dram_per_alg_byte": (1008215808 + 171628032) / 994046024,
        "source": "profiles/batch_pass_batch256.md (round 0 of a 256-mesh batch, scaled by algorithmic bytes)",
    },
}


def sources_sha256(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


def profile_figures(kernel: str):
    """The ncu figures of `kernel` if they were taken on its current sources, else None."""
    fig = PROFILE_FIGURES[kernel]
    if fig["sha256"] is None or sources_sha256(fig["files"]) != fig["sha256"]:
        return None
    return fig


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons.  Started before the
    warm-up (its start-up takes driver time that must not fall in the timed
    region); mark_start()/mark_end() bracket the timed region, and summary()
    uses the samples taken inside it (all samples if none arrived there)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[tuple[float, str]] = []
        self.reader = None
        self.t0 = self.t1 = None

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_end(self):
        self.t1 = time.perf_counter()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.reader.join(timeout=2)

    def summary(self) -> dict:
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if self.t0 is not None and self.t1 is not None:
            # a sample arrives up to one 200 ms period after it was taken
            inside = [(t, l) for t, l in lines if self.t0 <= t <= self.t1 + 0.2]
            lines = inside or lines
        for _, line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def edge_count(mesh) -> int:
    """Distinct edges of the triangle mesh."""
    tri = mesh.tri.astype(np.int64)
    a = tri.ravel()
    b = tri[:, [1, 2, 0]].ravel()
    key = np.minimum(a, b) * mesh.n + np.maximum(a, b)
    key.sort()
    return 1 + int(np.count_nonzero(key[1:] != key[:-1])) if key.size else 0


def survey_bytes_per_pass(mesh, n_free: int, coord_bytes: int = 16) -> int:
    """Algorithmic bytes of one pass in the survey's accounting (each array read
    once at ideal reuse): coordinates read for every node and written for every
    free node, int32 CSR neighbour lists (offsets n+1, 2 per edge) and incident
    triangle lists (offsets n+1, 3 per triangle), the triangles' int32 vertex
    ids and one boundary flag per node:
    16n + 16n_free + 8(n+1) + 4 nnz + 4*3m + 12m + n (coordinates 8 B in binary32)."""
    n, m = mesh.n, mesh.m
    nnz = 2 * edge_count(mesh)
    return coord_bytes * n + coord_bytes * n_free + 8 * (n + 1) + 4 * nnz + 12 * m + 12 * m + n


def fp64_pipe_peak(device="cuda") -> float:
    """FP64 lane operations per second the GPU sustains: cuBLAS DGEMM (n^3
    fused multiply-adds for an n x n product), best of three, CUDA events."""
    import torch
    n = 4096
    a = torch.rand((n, n), dtype=torch.float64, device=device)
    b = torch.rand((n, n), dtype=torch.float64, device=device)
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    del a, b
    return n ** 3 / best


def algorithmic_bytes_per_pass(n, n_free, adj_words, coord_bytes=16):
    """Bytes one pass must move at ideal reuse: every node's coordinates read
    once (16 B in FP64, 8 B in binary32), every free node's new coordinates
    written, the node offsets (4 B per node + 1) and the adjacency words (4 B
    each)."""
    return coord_bytes * n + coord_bytes * n_free + 4 * (n + 1) + 4 * adj_words


def adjacency_words(mesh):
    """Words of the library's adjacency stream: 1 meta word per node plus,
    per free node, its neighbours and incident triangles."""
    free = mesh.boundary == 0
    deg_plus_tri = np.zeros(mesh.n, np.int64)
    # incident triangles per node
    np.add.at(deg_plus_tri, mesh.tri.ravel(), 1)
    # interior node of a closed fan: degree == incident triangles
    return int(mesh.n + 2 * deg_plus_tri[free].sum())


def reduce_over_ranks(ms: float, updates: float, device="cpu"):
    """Max of the per-rank timed milliseconds and sum of node-updates over all
    ranks (replicas), so value = total updates / slowest rank's time."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([updates], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def rank_env():
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank: int, world: int):
    """The items of one rank: every world-th one from position `rank` on.
    The batched and served workloads are independent meshes, so ranks share
    no data; with a list of world x k items each rank gets k of them."""
    return list(items)[rank::world]


def reduce_flag(ok: bool, device="cpu") -> bool:
    """Logical AND of a flag over all ranks."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([1 if ok else 0], dtype=torch.int32, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return bool(t.item())


def init_ranks():
    """One process per GPU: select the local GPU and join the NCCL group."""
    import torch
    import torch.distributed as dist
    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    return world, rank


def cpu_oracle_rate(mesh, passes: int, precision: int = 64, form: str = "A", openmp: bool = True):
    """Times `passes` passes of the oracle: Form A FP64 on all host cores
    (OpenMP build) when `openmp`; otherwise, and for binary32 or Form B, on
    one core (the oracle's sequential loops)."""
    import oracle
    omp = openmp and precision == 64 and form == "A"
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.boundary, openmp=omp)
    t0 = time.perf_counter()
    if omp:
        xy = mesh.xy.copy()
        for _ in range(passes):
            xy, _, _, _ = om.sweep(xy)
    else:
        om.smooth(mesh.xy, passes, form=form, precision=precision)
    dt = time.perf_counter() - t0
    return mesh.n * passes / dt, dt, (os.cpu_count() if omp else 1)


def large_config(args, mesh, workload: str, world: int) -> dict:
    """The single-mesh workload as both arms print it."""
    return {"workload": workload, "n": mesh.n, "m": mesh.m,
            "n_free": int(np.count_nonzero(mesh.boundary == 0)),
            "max_passes": MAX_PASSES, "tol_rel": TOL, "kernel": args.kernel,
            "layout": args.layout, "copy_back": bool(args.copy_back),
            "form": "A (Jacobi)" if args.form == "A" else "B (coloured Gauss-Seidel, in place)",
            "precision": args.precision,
            "l2": "inputs larger than L2 (no flush)" if mesh.n >= 4 * 1024 * 1024
            else "inputs fit L2 (no flush; see l2_hit_rate)",
            "parallelism": "replicas" if world > 1 else "single",
            "skip_unchanged": bool(args.skip_unchanged), "l2_window": bool(args.l2_window),
            "library_numbering": getattr(args, "lib_numbering", "auto")}


def run_reference(args, mesh, workload):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    passes = args.ref_passes
    for _ in range(args.warmup):
        cpu_oracle_rate(mesh, 1)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt, cores = cpu_oracle_rate(mesh, passes)
        rates.append(r)
        times.append(dt)
    value = mesh.n * passes * len(times) / sum(times)
    sample = f"{passes} passes of the {workload} mesh per step (OpenMP oracle build)"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "node-updates/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": large_config(args, mesh, workload, args.gpus),
           "cpu_baseline": {"value": value, "unit": "node-updates/s", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "node-updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batch(args):
    """Batched form: many meshes of uneven size in one graph launch, against
    smoothing the same meshes one request at a time (same kernels)."""
    import torch
    import torch.distributed as dist
    import paper_1502_00355_gb300 as sls
    world, rank = init_ranks()
    sls.lib()
    # weak scaling: every rank smooths its own batch of batch_meshes meshes
    specs = shard(meshgen.batch_specs(args.batch_meshes * world, lo=args.batch_min_n, hi=args.batch_max_n), rank, world)
    meshes = [meshgen.batch_mesh(sp) for sp in specs]
    iters = [sp[2] for sp in specs]
    total_nodes = sum(m.n for m in meshes)
    # the meshes are created once and smoothed at every step: the grouped
    # internal numbering (paid at creation) is what a repeated batch wants
    handles = [sls.Mesh(m.xy, m.tri, m.boundary, numbering=args.batch_numbering) for m in meshes]
    stream = torch.cuda.Stream()
    batch = sls.Batch(handles, iters, stream=stream.cuda_stream)  # autotunes its block size
    for _ in range(args.warmup):
        batch.reset()
        batch.smooth()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    times, dev_ms = [], []
    for _ in range(args.steps):
        batch.reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        infos = batch.smooth()                       # one cudaGraphLaunch, returns when done
        times.append(time.perf_counter() - t0)
        e1.record(stream)
        torch.cuda.synchronize()
        dev_ms.append(e0.elapsed_time(e1))
    updates = sum(m.n * inf["iterations"] for m, inf in zip(meshes, infos))
    # algorithmic bytes of one smooth: each mesh's per-pass bytes times its
    # executed passes; the graph replay runs one batch-pass launch per round
    step_bytes = sum(algorithmic_bytes_per_pass(m.n, int((m.boundary == 0).sum()), adjacency_words(m))
                     * inf["iterations"] for m, inf in zip(meshes, infos))
    rounds = max(iters) if iters else 0
    if world > 1:
        dist.barrier()
    ms_max, all_updates = reduce_over_ranks(1e3 * sum(times) / len(times), float(updates), device="cuda")
    batched = all_updates / (ms_max * 1e-3)
    got = [batch.coords(j) for j in range(len(meshes))]
    # one request at a time: the same meshes, each smoothed by its own calls
    batch.reset()
    t0 = time.perf_counter()
    for h, it in zip(handles, iters):
        h.smooth(it)
    per_req_s = time.perf_counter() - t0
    per_ms_max, _ = reduce_over_ranks(1e3 * per_req_s, float(updates), device="cuda")
    per_request = all_updates / (per_ms_max * 1e-3)
    same = reduce_flag(all(np.array_equal(h.coords(), g) for h, g in zip(handles, got)), device="cuda")
    if rank != 0:
        return
    peak, peak_kind = _peaks()
    dev_mean = sum(dev_ms) / len(dev_ms)
    achieved = step_bytes / (dev_mean * 1e-3) / 1e9
    # DRAM bytes per algorithmic byte of the batch-pass kernel (ncu), scaled
    # to the step; None once the kernel's sources changed since the capture
    bfig = profile_figures("batch_pass")
    traffic = bfig["dram_per_alg_byte"] * step_bytes if bfig else None
    out = {"metric": "node-updates/s (batched)", "value": batched, "unit": "node-updates/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": (f"batch{len(meshes) * world}_logu1K-256K_aspect1-4_iters10-100"
                                   if (args.batch_min_n, args.batch_max_n) == (1024, 262144) else
                                   f"batch{len(meshes) * world}_logu{args.batch_min_n}-{args.batch_max_n}_aspect1-4_iters10-100"),
                      "meshes_per_gpu": len(meshes), "meshes": len(meshes) * world,
                      "nodes_rank0": total_nodes, "launch_shape": {"block": batch.shape[0], "chunk": batch.shape[1]},
                      "library_numbering": args.batch_numbering,
                      "parallelism": f"{world} ranks, independent meshes (no collective)" if world > 1 else "single"},
           "per_request": {"value": per_request, "unit": "node-updates/s", "seconds": per_req_s},
           "speedup_vs_per_request": batched / per_request, "identical_results": bool(same),
           "gpu_launches": rounds * args.steps,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                        "traffic_source": bfig["source"] if bfig else "no capture of the current kernel sources",
                        "bytes_per_step": step_bytes, "device_ms_per_step": dev_mean,
                        "timed": "CUDA events on the batch stream around each graph replay (job table upload, "
                                 "statistics clear, the round launches, statistics read-back)"}}
    print(json.dumps(out), flush=True)


class ResultPrint:
    """A 64-bit fingerprint of a coordinate array: the wrapping sum of its
    words times fixed odd random weights.  Two results with the same print
    are taken as identical (an accidental collision has probability 2^-64)."""

    def __init__(self, max_words: int, seed: int = 7):
        rng = np.random.Generator(np.random.PCG64(seed))
        self.w = rng.integers(0, 2 ** 63, size=max_words, dtype=np.uint64) * np.uint64(2) + np.uint64(1)

    def __call__(self, xy: np.ndarray) -> int:
        v = np.ascontiguousarray(xy).view(np.uint64).ravel()
        return int(np.dot(v, self.w[:v.size]))  # one pass, wrapping uint64 arithmetic


def serve_stream(args, world: int, rank: int):
    """This rank's requests (arrival_s, nx, ny, cap, seed) of the served workload."""
    return shard(meshgen.serve_requests(args.serve_requests * world, rate=args.serve_rate * world,
                                        hi=args.serve_max_n), rank, world)


class Prefetch:
    """Makes the requests' meshes ahead of their turn on a few threads
    (meshgen.fast_grid releases the GIL), at most `depth` ahead of the
    consumer, so the stream never has to exist in memory at once."""

    def __init__(self, reqs, threads: int, depth: int):
        from concurrent.futures import ThreadPoolExecutor
        self.reqs = reqs
        self.ex = ThreadPoolExecutor(max_workers=threads)
        self.depth = depth
        self.fut = {}
        self.next = 0

    def _fill(self, k):
        while self.next < len(self.reqs) and self.next < k + self.depth:
            _, nx, ny, _, seed = self.reqs[self.next]
            self.fut[self.next] = self.ex.submit(meshgen.fast_grid, nx, ny, 0.3, seed)
            self.next += 1

    def get(self, k):
        self._fill(k)
        m = self.fut.pop(k).result()
        self._fill(k + 1)
        return m

    def close(self):
        self.ex.shutdown(wait=True, cancel_futures=True)


def run_serve(args):
    """Served form: a Poisson stream of smoothing requests through the
    continuous-batching server, against one request at a time (FIFO, one
    sls_mesh_create + sls_smooth + sls_get_coords per request).  Latency runs
    from a request's scheduled arrival to its result on the host, so it
    includes any wait for the client to get the request in (the server's
    queue holds at most --serve-queue jobs; a client that finds it full waits
    and retries)."""
    import threading
    import torch
    import torch.distributed as dist
    import paper_1502_00355_gb300 as sls
    world, rank = init_ranks()
    sls.lib()
    meshgen.build()
    reqs = serve_stream(args, world, rank)
    arrivals = [r[0] for r in reqs]
    caps = [r[3] for r in reqs]
    sizes = [r[1] * r[2] for r in reqs]
    fp = ResultPrint(2 * max(sizes))
    # warm-up: a few requests through a server
    srv = sls.Server()
    for k in range(min(4, len(reqs))):
        m = meshgen.fast_grid(64, 64, 0.3, 1 + k)
        srv.wait(srv.submit(m.xy, m.tri, m.boundary, max_iter=10, tol=TOL))
    srv.close()

    # ---- served: continuous batching ----
    # several clients: request k is submitted by client k % clients at its
    # arrival time (each client makes its own meshes ahead of their turn), and
    # two pollers collect the results (request k by poller k % 2)
    srv = sls.Server(max_queue=args.serve_queue, numbering=args.lib_numbering)
    clients, pollers = max(1, args.serve_clients), 2
    pres = [Prefetch([reqs[k] for k in range(c, len(reqs), clients)], max(1, args.gen_threads // clients),
                     args.gen_depth) for c in range(clients)]
    done_t = [None] * len(reqs)
    prints = [None] * len(reqs)
    iters = [0] * len(reqs)
    pending = [dict() for _ in range(pollers)]  # job id -> (request index, output buffer)
    locks = [threading.Lock() for _ in range(pollers)]
    left = [clients]
    left_lock = threading.Lock()
    busy_retries = [0] * clients
    host_s = {"submit": [0.0] * clients, "get_mesh": [0.0] * clients, "try_wait": [0.0] * pollers,
              "fingerprint": [0.0] * pollers}
    if world > 1:
        dist.barrier()
    t_start = time.perf_counter()

    def submitter(c):
        for local, k in enumerate(range(c, len(reqs), clients)):
            t0 = time.perf_counter()
            m = pres[c].get(local)
            host_s["get_mesh"][c] += time.perf_counter() - t0
            delay = arrivals[k] - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            while True:
                try:
                    t0 = time.perf_counter()
                    jid = srv.submit(m.xy, m.tri, m.boundary, max_iter=caps[k], tol=TOL)
                    host_s["submit"][c] += time.perf_counter() - t0
                    break
                except sls.SlsError as e:
                    if e.code != 6:  # SLS_ERR_BUSY: the queue is full, try again shortly
                        raise
                    busy_retries[c] += 1
                    time.sleep(0.0005)
            p = k % pollers
            with locks[p]:
                pending[p][jid] = k
        with left_lock:
            left[0] -= 1

    # each poller receives its results into one scratch buffer of the largest
    # size (touched once here, so no result pays for fresh pages): the results
    # are only fingerprinted, not kept
    scratch = [np.zeros((max(sizes), 2), np.float64) for _ in range(pollers)]

    def poller(p):
        while True:
            with locks[p]:
                items = list(pending[p].items())
            if not items:
                with left_lock:
                    finished = left[0] == 0
                if finished:
                    with locks[p]:
                        if not pending[p]:
                            return
            for jid, k in items:
                buf = scratch[p][:sizes[k]]
                t0 = time.perf_counter()
                info = srv.try_wait(jid, buf)
                host_s["try_wait"][p] += time.perf_counter() - t0
                if info is None:
                    continue
                done_t[k] = time.perf_counter() - t_start
                t0 = time.perf_counter()
                prints[k] = fp(buf)
                host_s["fingerprint"][p] += time.perf_counter() - t0
                iters[k] = info["iterations"]
                with locks[p]:
                    del pending[p][jid]
            time.sleep(0.0005)

    ths = [threading.Thread(target=submitter, args=(c,)) for c in range(clients)] + \
          [threading.Thread(target=poller, args=(p,)) for p in range(pollers)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    wall = time.perf_counter() - t_start
    for pr in pres:
        pr.close()
    st = srv.stats()
    srv.close()
    lat = [1e3 * (d - a) for d, a in zip(done_t, arrivals)]
    updates = float(sum(n * it for n, it in zip(sizes, iters)))
    busy_retries = [sum(busy_retries)]

    # ---- FIFO: one request at a time, same arrivals, same kernels ----
    pre = Prefetch(reqs, args.gen_threads, args.gen_depth)
    if world > 1:
        dist.barrier()
    fifo_lat, busy, same = [], 0.0, True
    out = scratch[0]  # the results land in a buffer touched before, as the served ones do
    t_start = time.perf_counter()
    for k in range(len(reqs)):
        m = pre.get(k)
        now = time.perf_counter() - t_start
        if now < arrivals[k]:
            time.sleep(arrivals[k] - now)
        t0 = time.perf_counter()
        with sls.Mesh(m.xy, m.tri, m.boundary, numbering=args.lib_numbering) as g:
            inf = g.smooth(caps[k], TOL)
            xy = g.coords(out=out[:sizes[k]])
        busy += time.perf_counter() - t0
        fifo_lat.append(1e3 * (time.perf_counter() - t_start - arrivals[k]))
        same = same and fp(xy) == prints[k] and inf["iterations"] == iters[k]
    fifo_wall = time.perf_counter() - t_start
    pre.close()

    # over ranks: slowest wall times, summed work, worst percentiles
    wall_ms, all_updates = reduce_over_ranks(1e3 * wall, updates, device="cuda")
    fifo_ms, _ = reduce_over_ranks(1e3 * fifo_wall, 0.0, device="cuda")
    busy_ms, _ = reduce_over_ranks(1e3 * busy, 0.0, device="cuda")
    p50, _ = reduce_over_ranks(float(np.percentile(lat, 50)), 0.0, device="cuda")
    p99, _ = reduce_over_ranks(float(np.percentile(lat, 99)), 0.0, device="cuda")
    f50, _ = reduce_over_ranks(float(np.percentile(fifo_lat, 50)), 0.0, device="cuda")
    f99, _ = reduce_over_ranks(float(np.percentile(fifo_lat, 99)), 0.0, device="cuda")
    same = reduce_flag(same, device="cuda")
    if rank != 0:
        return
    served = all_updates / (wall_ms * 1e-3)
    fifo = all_updates / (fifo_ms * 1e-3)
    fifo_busy = all_updates / (busy_ms * 1e-3)
    out = {"metric": "node-updates/s (served)", "value": served, "unit": "node-updates/s", "n_gpus": world,
           "steps": 1, "warmup": 1, "ms_per_step": wall_ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"serve{len(reqs) * world}_poisson{args.serve_rate:g}_logu1K-"
                                  f"{'4M' if args.serve_max_n == 4 * 1024 * 1024 else args.serve_max_n}"
                                  "_cap10-200_tol1e-9",
                      "requests_per_gpu": len(reqs), "requests": len(reqs) * world,
                      "offered_req_per_s_per_gpu": args.serve_rate, "nodes_rank0": int(sum(sizes)),
                      "mesh_generator": "meshgen.fast_grid (jittered grid, J = 0.3, Morton)",
                      "server_queue_limit": args.serve_queue, "clients": args.serve_clients,
                      "library_numbering": args.lib_numbering,
                      "parallelism": f"{world} ranks, one server each (no collective)" if world > 1 else "single"},
           "served": {"p50_ms": p50, "p99_ms": p99, "wall_s": wall_ms * 1e-3,
                      "req_per_s": len(reqs) * world / (wall_ms * 1e-3),
                      "node_updates_per_s_busy_rank0": st["node_updates_per_s"],
                      "server_p50_ms_from_submit": st["p50_ms"], "server_p99_ms_from_submit": st["p99_ms"],
                      "busy_retries_rank0": busy_retries[0],
                      "host_thread_s_rank0": {k: round(sum(v), 3) for k, v in host_s.items()}},
           "fifo": {"p50_ms": f50, "p99_ms": f99, "node_updates_per_s": fifo, "wall_s": fifo_ms * 1e-3,
                    "node_updates_per_s_busy": fifo_busy, "busy_s": busy_ms * 1e-3},
           "speedup_vs_fifo": served / fifo,
           "speedup_vs_fifo_busy": served / fifo_busy,
           # work rate against work rate: the server's node-updates over the
           # device time of its rounds, FIFO's over the time its calls took
           "speedup_busy_vs_busy": st["node_updates_per_s"] / fifo_busy if world == 1 else None,
           "identical_results": bool(same),
           "latency": "scheduled arrival to result on the host"}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="large", choices=["large", "batch", "serve"])
    ap.add_argument("--batch-meshes", type=int, default=2048)
    ap.add_argument("--batch-min-n", type=int, default=1024)
    ap.add_argument("--batch-max-n", type=int, default=262144)
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-max-n", type=int, default=4 * 1024 * 1024)
    ap.add_argument("--serve-queue", type=int, default=64,
                    help="jobs the server queues before a client must wait (host memory of queued inputs)")
    ap.add_argument("--serve-clients", type=int, default=4,
                    help="client threads submitting the stream (request k by client k %% clients)")
    ap.add_argument("--gen-threads", type=int, default=8)
    ap.add_argument("--gen-depth", type=int, default=24)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lib-numbering", default="auto", choices=["auto", "given", "grouped"],
                    help="node numbering inside the library (single mesh, served jobs and their FIFO baseline)")
    ap.add_argument("--batch-numbering", default="grouped", choices=["auto", "given", "grouped"],
                    help="node numbering of the batch's meshes (created once, smoothed every step)")
    ap.add_argument("--kernel", default="auto")
    ap.add_argument("--config", default="large", choices=["large", "small", "medium"],
                    help="single-mesh workload: large 4096^2 (the headline), small 64^2, medium 1024^2")
    ap.add_argument("--numbering", default="morton", choices=["morton", "random"],
                    help="node numbering of the medium mesh")
    ap.add_argument("--layout", default="aos", choices=["aos", "soa"])
    ap.add_argument("--copy-back", action="store_true",
                    help="copy each pass back over the old coordinates (the paper's swap form)")
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--ny", type=int, default=4096)
    ap.add_argument("--ref-passes", type=int, default=3)
    ap.add_argument("--cpu-passes", type=int, default=80)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", type=int, default=64, choices=[64, 32],
                    help="64: FP64 (the headline); 32: binary32, the paper's precision")
    ap.add_argument("--form", default="A", choices=["A", "B"],
                    help="A: Jacobi (the headline); B: multicolour Gauss-Seidel")
    ap.add_argument("--skip-unchanged", action="store_true",
                    help="leave unchanged tiles as they are (identical results; not the headline)")
    ap.add_argument("--decompose", action="store_true",
                    help="split the single mesh over the ranks (domain decomposition) instead of replicas")
    ap.add_argument("--l2-window", action="store_true",
                    help="persisting L2 window over the gathered coordinates (identical results)")
    args = ap.parse_args()
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)

    return run_single(args)


def single_workload(args):
    """(mesh, workload name, max passes, tolerance) of the single-mesh workloads:
    large (the headline, 4096x4096 with the clustered pull, to the tolerance),
    small (64x64, 10 passes) and medium (1024x1024, 100 passes, Morton or
    random numbering)."""
    if args.config == "small":
        return meshgen.small_grid(), "grid64x64_jitter0.3_morton_10passes", 10, 0.0
    if args.config == "medium":
        return (meshgen.medium_grid(args.numbering), f"grid1024x1024_jitter0.35_{args.numbering}_100passes",
                100, 0.0)
    mesh = meshgen.large_grid(args.nx, args.ny)
    workload = WORKLOAD if (args.nx, args.ny) == (4096, 4096) else f"grid{args.nx}x{args.ny}_jitter0.35_pull5pct_morton"
    return mesh, workload, MAX_PASSES, TOL


def run_decomposed(args, mesh, workload, max_passes, tol):
    """The single mesh split over the ranks by domain decomposition (one
    subdomain per GPU, a ghost exchange and a max all-reduce per pass;
    paper_1502_00355_gb300/domain.py).  Strong scaling: the whole mesh's
    node-updates over the slowest rank's time."""
    import torch
    import torch.distributed as dist
    import paper_1502_00355_gb300 as sls
    from paper_1502_00355_gb300 import domain
    world, rank = init_ranks()
    sls.lib()
    sub = domain.partition(mesh.n, mesh.tri, mesh.boundary, world, rank)
    stream = torch.cuda.Stream()
    be = domain.LibraryBackend(sub, mesh.xy[sub.nodes], stream=stream.cuda_stream)
    dm = domain.DistributedMesh(sub, be, mesh.xy[sub.lo:sub.hi], device="cuda")
    xy0 = torch.from_numpy(np.ascontiguousarray(mesh.xy[sub.nodes])).cuda()

    def step():
        be.mesh.set_coords(xy0)
        return dm.smooth(max_passes, tol)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        clk.mark_start()
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
    if world > 1:
        dist.barrier()
    passes = sum(i["iterations"] for i in infos)
    ms_max, _ = reduce_over_ranks(e0.elapsed_time(e1), 0.0, device="cuda")
    value = mesh.n * passes / (ms_max * 1e-3)
    be.close()
    if rank == 0:
        cfg = large_config(args, mesh, workload, world)
        cfg["parallelism"] = f"domain decomposition over {world} ranks (ghost exchange + max all-reduce per pass)"
        out = {"metric": METRIC, "value": value, "unit": "node-updates/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
               "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": cfg,
               "run": {"passes_per_step": passes / args.steps, "owned_nodes_rank0": sub.hi - sub.lo,
                       "local_nodes_rank0": sub.n_local},
               "gpu_launches": passes * (1 + 2 * len(sub.send)),
               "timed": "CUDA events on rank 0's library stream around the steps (every pass ends in a host "
                        "synchronisation for the exchange)",
               "clocks": clk.summary()}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_single(args):
    mesh, workload, max_passes, tol = single_workload(args)
    if args.impl == "reference":
        run_reference(args, mesh, workload)
        return
    if args.decompose:
        return run_decomposed(args, mesh, workload, max_passes, tol)

    import torch
    import torch.distributed as dist
    import paper_1502_00355_gb300 as sls

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    sls.lib()

    stream = torch.cuda.Stream()
    variant = dict(kernel=args.kernel, precision=args.precision, form=args.form, layout=args.layout,
                   numbering=args.lib_numbering,
                   copy_back=args.copy_back, skip_unchanged=args.skip_unchanged, l2_window=args.l2_window)
    g = sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, stream=stream.cuda_stream, **variant)
    xy0 = torch.from_numpy(mesh.xy).to("cuda")
    torch.cuda.synchronize()

    def step():
        g.set_coords(xy0)
        return g.smooth(max_passes, tol)

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk.mark_start()
        ev0.record(stream)
        for _ in range(args.steps):
            infos.append(step())
        ev1.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
    ms = ev0.elapsed_time(ev1)
    passes = sum(i["iterations"] for i in infos)
    # kernel-only view: per-pass time, events around the passes alone (for the
    # copy-back form this includes its copy kernel)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pass_ms = float("inf")
    for _ in range(2):
        g.set_coords(xy0)
        torch.cuda.synchronize()
        e0.record(stream)
        info_k = g.smooth(max_passes, tol)
        e1.record(stream)
        torch.cuda.synchronize()
        pass_ms = min(pass_ms, e0.elapsed_time(e1) / max(1, info_k["iterations"]))

    ms_max, total_updates = reduce_over_ranks(ms, float(mesh.n * passes), device="cuda")
    value = total_updates / (ms_max * 1e-3)

    # end to end through the public API with host buffers: create (H2D of the
    # inputs, adjacency build), smooth, read the coordinates back (D2H)
    e2e_times = []
    pinned = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    xy_h, tri_h, bnd_h = pinned(mesh.xy), pinned(mesh.tri), pinned(mesh.boundary)
    out_host = torch.empty(mesh.xy.shape, dtype=torch.float64).pin_memory().numpy()
    e2e_passes = 0
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with sls.Mesh(xy_h, tri_h, bnd_h, **variant) as h:
            inf = h.smooth(max_passes, tol)
            h.coords(out=out_host)
        e2e_times.append(time.perf_counter() - t0)
        e2e_passes += inf["iterations"]
    e2e_value = mesh.n * e2e_passes * world / sum(e2e_times) if e2e_times else None

    peak, peak_kind = _peaks()
    headline = (args.kernel == "auto" and args.precision == 64 and args.form == "A" and not args.skip_unchanged
                and not args.l2_window and args.layout == "aos" and not args.copy_back)
    coord_bytes = 16 if args.precision == 64 else 8
    bytes_pass = survey_bytes_per_pass(mesh, g.n_free, coord_bytes)
    bytes_ours = algorithmic_bytes_per_pass(mesh.n, g.n_free, adjacency_words(mesh), coord_bytes)
    achieved = bytes_pass / (pass_ms * 1e-3) / 1e9
    fig = profile_figures("pass_screened") if headline else None
    traffic = fig["dram_bytes_per_node"] * mesh.n if fig else None
    hbm = {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
           "peak_kind": peak_kind,
           "traffic_source": fig["source"] if fig else "no capture of the current kernel sources",
           "bytes_per_pass": bytes_pass, "bytes_source": "16n + 16n_free + 8(n+1) + 4nnz + 12m + 12m + n",
           "bytes_per_pass_library_encoding": bytes_ours}
    roofline = {"bound": "hbm", **hbm, "pass_ms": pass_ms}
    if args.precision == 64 and args.form == "A":
        # The FP64 pipe: every FP64 warp instruction occupies it for all 32
        # lanes.  Peak from the unit count and clock: 2 FP64 lane operations
        # per clock per SM (the FMA pipe's sustained peak) x SMs x max SM clock.
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        clk_max = clk.summary().get("sm_max_mhz") or 2070.0
        fp64_peak = 2.0 * sms * clk_max * 1e6
        fp64_dgemm = fp64_pipe_peak()
        # algorithmic FP64 operations of a pass: what the exact result cannot
        # avoid, per free node 2(deg-1) additions for the neighbour sums, 2
        # multiplications for the divisions, 2 subtractions for the move and
        # 3 operations for its square (degree = incident triangles on these
        # meshes: words = n + sum over free nodes of (deg + ntri))
        sum_deg_free = (adjacency_words(mesh) - mesh.n) // 2
        fp64_alg = 2 * sum_deg_free + 5 * g.n_free
        t = pass_ms * 1e-3
        fp64 = {"achieved": fp64_alg / t / 1e12, "peak": fp64_peak / 1e12, "unit": "T FP64 op/s",
                "frac": fp64_alg / t / fp64_peak, "ops_per_pass": fp64_alg,
                "ops_source": "per free node 2(deg-1) + 2 + 2 + 3",
                "peak_source": f"2 FP64 lane operations per clock per SM x {sms} SMs x {clk_max:.0f} MHz",
                "measured_dgemm": fp64_dgemm / 1e12}
        if fig:
            # issued FP64 lane slots from the capture: warp instructions x 32 lanes / 32 nodes
            fp64_issued = fig["fp64_warp_inst_per_32_nodes"] * mesh.n
            fp64.update({"pipe_occupancy": fp64_issued / t / fp64_peak,
                         "issued_lane_slots_per_pass": fp64_issued, "issued_source": fig["source"]})
        roofline["hbm"] = dict(hbm)
        roofline["fp64"] = fp64
        if fp64["frac"] > hbm["frac"]:
            # the binding unit is the FP64 pipe: the line's roofline describes it
            roofline = {"bound": "alu", "achieved": fp64["achieved"], "peak": fp64["peak"], "unit": fp64["unit"],
                        "frac": fp64["frac"], "traffic": traffic, "peak_kind": "derived (unit count x clock)",
                        "pass_ms": pass_ms, "hbm": dict(hbm), "fp64": fp64}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        omp = args.config == "large"
        cpu_passes = args.cpu_passes if args.config == "large" else max_passes
        rate, dt, cores = cpu_oracle_rate(mesh, cpu_passes, args.precision, args.form, openmp=omp)
        cpu = {"value": rate, "unit": "node-updates/s", "cores": cores, "kind": "oracle",
               "sample": f"{cpu_passes} Form-{args.form} passes ({'FP64' if args.precision == 64 else 'binary32'}) "
                         f"of the same mesh from its initial coordinates ({dt:.1f} s, "
                         f"{'OpenMP oracle build on all host cores' if cores > 1 else 'sequential oracle, one core'})"}

    if rank == 0:
        cfg = large_config(args, mesh, workload, world)
        cfg["n_free"] = g.n_free
        out = {"metric": METRIC, "value": value, "unit": "node-updates/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f64" if args.precision == 64 else "f32",
               "data": "synthetic",
               "config": cfg,
               "run": {"passes_per_step": passes / args.steps,
                       "nodes_skipped_frac": sum(i["nodes_skipped"] for i in infos) / (mesh.n * max(1, passes)),
                       "fp64_fallbacks_per_pass": sum(i["fp64_fallbacks"] for i in infos) / max(1, passes)},
               "e2e": {"value": e2e_value, "unit": "node-updates/s",
                       "h2d_bytes_per_step": int(mesh.xy.nbytes + mesh.tri.nbytes + mesh.boundary.nbytes),
                       "d2h_bytes_per_step": int(mesh.xy.nbytes)},
               "gpu_launches": sum(i["launches"] for i in infos),
               "roofline": roofline if not args.skip_unchanged else None,
               "cpu_baseline": cpu,
               "clocks": clk.summary()}
        print(json.dumps(out), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
