"""The library's device memory pool: destroyed handles return their memory
to the pool, a later handle of the same size reuses it, and sls_trim_memory
hands it back to the driver."""
import numpy as np
import pytest

import meshgen

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


def test_pool_keeps_and_trims(sls):
    import torch
    mesh = meshgen.jittered_grid(1024, 1024, 0.3, 3)   # about 150 MB on the device
    sls.trim_memory(0)
    free0 = torch.cuda.mem_get_info()[0]
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary) as g:
        a = g.smooth(3)
        xa = g.coords()
    torch.cuda.synchronize()
    kept = free0 - torch.cuda.mem_get_info()[0]
    assert kept > 100 * 2**20                           # the pool kept the mesh's memory
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary) as g:  # reuses it
        b = g.smooth(3)
        assert np.array_equal(g.coords(), xa) and a["maxd2_last"] == b["maxd2_last"]
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] <= kept + 64 * 2**20
    sls.trim_memory(0)
    assert torch.cuda.mem_get_info()[0] >= free0 - 32 * 2**20


def test_many_meshes_alive_and_destroyed_out_of_order(sls):
    meshes = [meshgen.jittered_grid(40 + 7 * k, 30 + 5 * k, 0.3, 50 + k) for k in range(12)]
    handles = [sls.Mesh(m.xy, m.tri, m.boundary, numbering="grouped" if k % 2 else "given")
               for k, m in enumerate(meshes)]
    outs = {}
    for k in (5, 0, 11, 3, 7, 1, 9, 2, 10, 4, 8, 6):
        handles[k].smooth(8)
        outs[k] = handles[k].coords()
        handles[k].close()
    for k, m in enumerate(meshes):
        with sls.Mesh(m.xy, m.tri, m.boundary) as g:
            g.smooth(8)
            assert np.array_equal(g.coords(), outs[k])
