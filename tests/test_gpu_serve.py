"""GPU parity of the served form (continuous batching): every job's result
must be bit-identical to the oracle and to smoothing it alone, whatever else
shares the GPU rounds with it."""
import threading

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


def _jobs(k, seed):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(k):
        n = int(round(np.exp(rng.uniform(np.log(100), np.log(30000)))))
        side = max(3, int(round(np.sqrt(n))))
        cap = int(rng.integers(1, 60))
        tol = 1e-6 if r % 2 else 0.0
        out.append((meshgen.jittered_grid(side, side + r % 3, 0.3, 9000 + r, numbering="morton"), cap, tol))
    return out


def test_served_jobs_equal_oracle_in_the_mix(sls):
    jobs = _jobs(30, 1)
    srv = sls.Server()
    ids = [srv.submit(m.xy, m.tri, m.boundary, max_iter=cap, tol=tol) for m, cap, tol in jobs]
    for (m, cap, tol), jid in zip(jobs, ids):
        xy, info = srv.wait(jid, timeout=120.0)
        om = oracle.OracleMesh(m.xy, m.tri, m.boundary)
        rxy, rinfo, _ = om.smooth(m.xy, cap, tol=tol)
        assert np.array_equal(xy, rxy)
        for key in ("iterations", "converged", "accepted_last", "maxd2_last"):
            assert info[key] == rinfo[key], key
    st = srv.stats()
    assert st["completed"] == len(jobs) and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_served_jobs_in_the_callers_numbering(sls):
    # jobs built without the internal grouped numbering give the same bits
    jobs = _jobs(12, 7)
    out = []
    for numbering in ("grouped", "given"):
        srv = sls.Server(numbering=numbering)
        ids = [srv.submit(m.xy, m.tri, m.boundary, max_iter=cap, tol=tol) for m, cap, tol in jobs]
        out.append([srv.wait(jid, timeout=120.0) for jid in ids])
        srv.close()
    for (xa, ia), (xb, ib) in zip(*out):
        assert np.array_equal(xa, xb)
        assert ia["iterations"] == ib["iterations"] and ia["maxd2_last"] == ib["maxd2_last"]


def test_served_concurrent_clients_and_budget(sls):
    # a small memory budget forces jobs to wait for each other; four client
    # threads submit and wait concurrently
    jobs = _jobs(24, 2)
    srv = sls.Server(hbm_budget=64 * 1024 * 1024)
    results = {}

    def client(part):
        for idx in part:
            m, cap, tol = jobs[idx]
            jid = srv.submit(m.xy, m.tri, m.boundary, max_iter=cap, tol=tol)
            results[idx] = srv.wait(jid, timeout=300.0)

    threads = [threading.Thread(target=client, args=(list(range(c, len(jobs), 4)),)) for c in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert len(results) == len(jobs)
    for idx, (m, cap, tol) in enumerate(jobs):
        with sls.Mesh(m.xy, m.tri, m.boundary) as g:
            info = g.smooth(cap, tol)
            alone = g.coords()
        xy, sinfo = results[idx]
        assert np.array_equal(xy, alone)
        assert sinfo["iterations"] == info["iterations"]
    srv.close()


def test_server_rejects_and_times_out(sls):
    srv = sls.Server(hbm_budget=1024 * 1024)
    big = meshgen.jittered_grid(300, 300, 0.3, 5)
    with pytest.raises(sls.SlsError) as e:
        srv.submit(big.xy, big.tri, big.boundary, max_iter=5)
    assert e.value.code == 7
    bad = np.array([[0, 1, 99]], dtype=np.int32)
    jid = srv.submit(big.xy[:10], bad, None, max_iter=5)
    with pytest.raises(sls.SlsError) as e:
        srv.wait(jid, timeout=30.0)
    assert e.value.code == 1
    small = meshgen.jittered_grid(20, 20, 0.3, 6)
    jid = srv.submit(small.xy, small.tri, small.boundary, max_iter=0)
    xy, info = srv.wait(jid, timeout=30.0)
    assert info["iterations"] == 0 and np.array_equal(xy, small.xy)
    with pytest.raises(sls.SlsError) as e:
        srv.wait(123456789, timeout=0.1)
    assert e.value.code == 8
    srv.close()


def test_server_destroyed_with_jobs_in_flight(sls):
    # closing a server while jobs are building, queued, uploading and running
    # cancels them and returns promptly (the uploader and builders stop first)
    jobs = _jobs(40, 9)
    srv = sls.Server(hbm_budget=48 * 1024 * 1024)
    for m, cap, tol in jobs:
        srv.submit(m.xy, m.tri, m.boundary, max_iter=200, tol=0.0)
    done = threading.Event()

    def closer():
        srv.close()
        done.set()

    t = threading.Thread(target=closer)
    t.start()
    t.join(timeout=120.0)
    assert done.is_set(), "sls_server_destroy did not return"
    # the device is still usable afterwards
    m = meshgen.jittered_grid(30, 30, 0.3, 3)
    with sls.Mesh(m.xy, m.tri, m.boundary) as g:
        assert g.smooth(3)["iterations"] == 3


def test_served_edge_meshes(sls):
    # a single triangle (nothing moves, every pass counts), degenerate
    # triangles, a node in 40 triangles, a zero-pass job, in one mix
    meshes = meshgen.edge_case_meshes()
    caps = [5, 9, 4, 0, 13]
    tols = [0.0, 1e-4, 0.0, 0.0, 1e-6]
    srv = sls.Server()
    ids = [srv.submit(m.xy, m.tri, m.boundary, max_iter=c, tol=t) for m, c, t in zip(meshes, caps, tols)]
    for m, c, t, jid in zip(meshes, caps, tols, ids):
        xy, info = srv.wait(jid, timeout=120.0)
        rxy, rinfo, _ = oracle.OracleMesh(m.xy, m.tri, m.boundary).smooth(m.xy, c, tol=t)
        assert np.array_equal(xy, rxy)
        for key in ("iterations", "converged", "accepted_last", "maxd2_last"):
            assert info[key] == rinfo[key], key
    srv.close()


def test_served_million_node_job_in_a_mix(sls):
    """A 1024x1024 (1,048,576-node) job submitted between small ones, built
    on the device by the server's builders, equals the oracle bit for bit;
    so does a job from meshgen.fast_grid, the served benchmark's generator."""
    big = meshgen.jittered_grid(1024, 1024, 0.3, 777, numbering="morton")
    fast = meshgen.fast_grid(300, 280, 0.3, 4242)
    small = _jobs(12, 5)
    srv = sls.Server()
    ids = [srv.submit(m.xy, m.tri, m.boundary, max_iter=cap, tol=tol) for m, cap, tol in small[:6]]
    jb = srv.submit(big.xy, big.tri, big.boundary, max_iter=12, tol=1e-9)
    jf = srv.submit(fast.xy, fast.tri, fast.boundary, max_iter=40, tol=1e-9)
    ids += [srv.submit(m.xy, m.tri, m.boundary, max_iter=cap, tol=tol) for m, cap, tol in small[6:]]
    xy_b, info_b = srv.wait(jb, timeout=300.0)
    xy_f, info_f = srv.wait(jf, timeout=300.0)
    for (m, cap, tol), jid in zip(small, ids):
        xy, info = srv.wait(jid, timeout=300.0)
        rxy, rinfo, _ = oracle.OracleMesh(m.xy, m.tri, m.boundary).smooth(m.xy, cap, tol=tol)
        assert np.array_equal(xy, rxy)
    srv.close()
    rxy, rinfo, _ = oracle.OracleMesh(big.xy, big.tri, big.boundary, openmp=True).smooth(big.xy, 12, tol=1e-9)
    assert np.array_equal(xy_b, rxy)
    for key in ("iterations", "converged", "accepted_last", "maxd2_last"):
        assert info_b[key] == rinfo[key], key
    rxy, rinfo, _ = oracle.OracleMesh(fast.xy, fast.tri, fast.boundary).smooth(fast.xy, 40, tol=1e-9)
    assert np.array_equal(xy_f, rxy)
    assert info_f["iterations"] == rinfo["iterations"]


def test_server_rejects_the_soa_layout(sls):
    with pytest.raises(sls.SlsError) as e:
        sls.Server(layout="soa")
    assert e.value.code == 1
