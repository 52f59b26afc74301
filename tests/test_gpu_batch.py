"""GPU parity of the batched form: every mesh of a batch must come out
bit-identical to the oracle (and to smoothing it alone), whatever its size,
iteration count, tolerance or accept mode."""
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


def _specs(k, seed, lo=60, hi=4000):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(k):
        n = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        a = rng.uniform(1.0, 4.0)
        ny = max(2, int(round(np.sqrt(n / a))))
        nx = max(2, int(round(n / ny)))
        out.append((nx, ny, int(rng.integers(1, 40)), 777 + r))
    return out


@pytest.mark.parametrize("block", [0, 64, 128])
def test_batch_matches_oracle_per_mesh(sls, block):
    specs = _specs(24, 3 + block)
    meshes = [meshgen.jittered_grid(nx, ny, 0.3, s, numbering="morton") for nx, ny, _, s in specs]
    iters = [it for _, _, it, _ in specs]
    tols = [1e-5 if r % 3 == 0 else 0.0 for r in range(len(specs))]
    strict = [r % 5 == 1 for r in range(len(specs))]
    handles = [sls.Mesh(m.xy, m.tri, m.boundary, strict=st, record_accept=True) for m, st in zip(meshes, strict)]
    batch = sls.Batch(handles, iters, tols, block_size=block)
    infos = batch.smooth()
    for j, m in enumerate(meshes):
        om = oracle.OracleMesh(m.xy, m.tri, m.boundary)
        rxy, rinfo, racc = om.smooth(m.xy, iters[j], tol=tols[j], strict=strict[j])
        got = batch.coords(j)
        assert np.array_equal(got, rxy), f"mesh {j} ({m.n} nodes, {iters[j]} passes)"
        for key in ("iterations", "converged", "accepted_last", "maxd2_last"):
            assert infos[j][key] == rinfo[key], (j, key)
        if rinfo["iterations"] > 0:
            assert np.array_equal(handles[j].accept_mask(), racc)
    # reset and run again: identical
    batch.reset()
    infos2 = batch.smooth()
    assert infos2 == infos
    for j, m in enumerate(meshes):
        om = oracle.OracleMesh(m.xy, m.tri, m.boundary)
        rxy, _, _ = om.smooth(m.xy, iters[j], tol=tols[j], strict=strict[j])
        assert np.array_equal(batch.coords(j), rxy)
    batch.close()
    for h in handles:
        h.close()


def test_batch_equals_alone_and_continues(sls):
    specs = _specs(10, 42, lo=500, hi=20000)
    meshes = [meshgen.jittered_grid(nx, ny, 0.35, s, numbering="random") for nx, ny, _, s in specs]
    iters = [it for _, _, it, _ in specs]
    alone = []
    for m, it in zip(meshes, iters):
        with sls.Mesh(m.xy, m.tri, m.boundary) as g:
            g.smooth(it)
            g.smooth(it)
            alone.append(g.coords())
    handles = [sls.Mesh(m.xy, m.tri, m.boundary) for m in meshes]
    batch = sls.Batch(handles, iters)
    batch.smooth()
    batch.smooth()  # continues from where the first call stopped
    for j in range(len(meshes)):
        assert np.array_equal(handles[j].coords(), alone[j])
    batch.close()


def test_batch_rejects_bad_input(sls):
    m = meshgen.jittered_grid(10, 10, 0.3, 1)
    h = sls.Mesh(m.xy, m.tri, m.boundary)
    with pytest.raises(sls.SlsError):
        sls.Batch([h, h], [3, 3])
    with pytest.raises(sls.SlsError):
        sls.Batch([h], [-1])
    h2 = sls.Mesh(m.xy, m.tri, m.boundary, layout="soa")
    with pytest.raises(sls.SlsError):
        sls.Batch([h, h2], [3, 3])
    b = sls.Batch([h], [0])
    assert b.smooth()[0]["iterations"] == 0
    assert np.array_equal(h.coords(), m.xy)
    with pytest.raises(sls.SlsError) as e:  # the kernel is built for blocks of at most 128
        sls.Batch([h], [3], block_size=256)
    assert e.value.code == 1


def test_batch_edge_meshes(sls):
    # a single triangle (nothing moves, every pass counts), degenerate
    # triangles, a node in 40 triangles (the exact path), a zero-pass mesh
    meshes = meshgen.edge_case_meshes()
    iters = [5, 9, 4, 0, 13]
    tols = [0.0, 1e-4, 0.0, 0.0, 1e-6]
    handles = [sls.Mesh(m.xy, m.tri, m.boundary) for m in meshes]
    batch = sls.Batch(handles, iters, tols)
    infos = batch.smooth()
    for j, m in enumerate(meshes):
        rxy, rinfo, _ = oracle.OracleMesh(m.xy, m.tri, m.boundary).smooth(m.xy, iters[j], tol=tols[j])
        assert np.array_equal(batch.coords(j), rxy), j
        for key in ("iterations", "converged", "accepted_last", "maxd2_last"):
            assert infos[j][key] == rinfo[key], (j, key)
    assert infos[0]["iterations"] == 5 and infos[3]["iterations"] == 0
    batch.close()
    for h in handles:
        h.close()


def test_every_launch_shape_gives_the_same_results(sls):
    """The warp chunk and block size change only who computes what: every
    shape (contiguous shares, grid-stride chunks, counter-claimed chunks)
    gives results identical to smoothing each mesh alone."""
    meshes = [meshgen.jittered_grid(nx, ny, 0.3, 600 + k, numbering="morton")
              for k, (nx, ny) in enumerate([(40, 30), (7, 5), (120, 64), (33, 97), (3, 3), (64, 64)])]
    iters = [12, 3, 25, 7, 1, 18]
    alone = []
    for m, it in zip(meshes, iters):
        with sls.Mesh(m.xy, m.tri, m.boundary) as g:
            g.smooth(it)
            alone.append(g.coords())
    handles = [sls.Mesh(m.xy, m.tri, m.boundary) for m in meshes]
    b = sls.Batch(handles, iters)
    assert b.shape[0] in (64, 128)
    for block, chunk in [(128, 0), (64, 1), (128, 4), (96, 16), (128, -1), (64, -8), (32, -3)]:
        b.set_shape(block, chunk)
        assert b.shape == (block, chunk)
        b.reset()
        b.smooth()
        for j, ref in enumerate(alone):
            assert np.array_equal(b.coords(j), ref), (block, chunk, j)
    with pytest.raises(sls.SlsError):
        b.set_shape(100, 0)
    b.close()
    for h in handles:
        h.close()
