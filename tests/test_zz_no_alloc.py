"""sls_smooth_noalloc: the entry point for callers that cannot allocate device
memory while they smooth (in a loop that must not synchronise the device
through cudaMalloc/cudaFree, under a host application that owns the whole
memory budget, or in a service whose memory is fixed at start-up).  It must give the same
coordinates and statistics as sls_smooth, bit for bit, call after call,
although every call reuses the same fixed scratch array.

This file is collected last so that a failure here stops a -x run only after
every other test has run; it also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1502_00355_gb300 as sls
    sls.build()
    sls.lib()
    return sls, torch


def _reference(sls, mesh, kernel, max_iter, tol):
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, kernel=kernel) as g:
        info = g.smooth(max_iter, tol)
        return g.coords(), info


@pytest.mark.parametrize("kernel", ["auto", "fp64"])
def test_noalloc_matches_smooth_on_consecutive_calls(env, kernel):
    sls, torch = env
    L = sls.lib()
    mesh = meshgen.jittered_grid(300, 200, 0.35, 2024, numbering="morton")
    g = sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, kernel=kernel)
    # two calls in a row with different lengths: the second must not see the
    # first call's statistics (the array is cleared per call)
    for max_iter, tol in [(40, 1e-6), (17, 0.0), (300, 1e-7)]:
        ref_xy, ref_info = _reference(sls, mesh, kernel, max_iter, tol)
        xy_in = torch.from_numpy(mesh.xy.copy()).cuda()
        xy_out = torch.empty_like(xy_in)
        info = sls.Info()
        st = L.sls_smooth_noalloc(g.handle, C.c_void_p(xy_in.data_ptr()), C.c_void_p(xy_out.data_ptr()),
                                  max_iter, tol, None, C.byref(info))
        assert st == 0, L.sls_last_error()
        torch.cuda.synchronize()
        got = xy_out.cpu().numpy()
        assert np.array_equal(got, ref_xy)
        d = info.as_dict()
        for key in ("iterations", "converged", "accepted_last", "maxd2_last"):
            assert d[key] == ref_info[key], key
    g.close()


def test_noalloc_rejects_what_it_cannot_do(env):
    sls, torch = env
    L = sls.lib()
    mesh = meshgen.jittered_grid(20, 20, 0.3, 7)
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary) as g:
        a = torch.from_numpy(mesh.xy.copy()).cuda()
        b = torch.empty_like(a)
        info = sls.Info()
        st = L.sls_smooth_noalloc(g.handle, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()),
                                  4097, 0.0, None, C.byref(info))
        assert st == 1 and b"SLS_NOALLOC_MAX_PASSES" in L.sls_last_error()
        st = L.sls_smooth_noalloc(g.handle, C.c_void_p(a.data_ptr()), C.c_void_p(a.data_ptr()),
                                  5, 0.0, None, C.byref(info))
        assert st == 1
        # zero passes: the output is the input
        st = L.sls_smooth_noalloc(g.handle, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()),
                                  0, 0.0, None, C.byref(info))
        assert st == 0 and info.iterations == 0
        torch.cuda.synchronize()
        assert torch.equal(a, b)
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, layout="soa") as g:
        st = L.sls_smooth_noalloc(g.handle, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()),
                                  5, 0.0, None, C.byref(info))
        assert st == 1


def _noalloc(L, sls, g, xy_in, xy_out, max_iter, tol, stream=None):
    info = sls.Info()
    st = L.sls_smooth_noalloc(g.handle, C.c_void_p(xy_in.data_ptr()), C.c_void_p(xy_out.data_ptr()),
                              max_iter, tol, None if stream is None else C.c_void_p(stream), C.byref(info))
    assert st == 0, L.sls_last_error()
    return info.as_dict()


def test_noalloc_leaves_free_device_memory_unchanged(env):
    """The reason the entry point exists: a caller whose memory budget is
    fully spoken for can smooth without the library taking any of it.  The
    device's free memory is the same before and after a call (the scratch
    array was placed on the device when the mesh was created)."""
    sls, torch = env
    L = sls.lib()
    mesh = meshgen.jittered_grid(128, 96, 0.35, 4242, numbering="morton")
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary) as g:
        a = torch.from_numpy(mesh.xy.copy()).cuda()
        b = torch.empty_like(a)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        _noalloc(L, sls, g, a, b, 25, 1e-9)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        a.copy_(torch.from_numpy(mesh.xy))
        free2, _ = torch.cuda.mem_get_info()
        _noalloc(L, sls, g, a, b, 25, 1e-9)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free2


@pytest.mark.parametrize("options", [dict(skip_unchanged=True), dict(copy_back=True)])
def test_noalloc_on_a_side_stream_at_the_pass_limit(env, options):
    """A call on a caller's own (non-default) stream, at the largest pass count
    with the tolerance on, on meshes created with options the entry point does
    not apply: the results equal sls_smooth's, bit for bit, twice in a row."""
    sls, torch = env
    L = sls.lib()
    mesh = meshgen.jittered_grid(40, 30, 0.3, 99, numbering="morton")
    ref_xy, ref_info = None, None
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, **options) as r:
        ref_info = r.smooth(4096, 1e-13)
        ref_xy = r.coords()
    side = torch.cuda.Stream()
    with sls.Mesh(mesh.xy, mesh.tri, mesh.boundary, **options) as g:
        for _ in range(2):
            with torch.cuda.stream(side):
                a = torch.from_numpy(mesh.xy.copy()).to("cuda", non_blocking=False)
                b = torch.empty_like(a)
            side.synchronize()
            info = _noalloc(L, sls, g, a, b, 4096, 1e-13, stream=side.cuda_stream)
            got = b.cpu().numpy()
            assert np.array_equal(got, ref_xy)
            for key in ("iterations", "converged", "accepted_last", "maxd2_last"):
                assert info[key] == ref_info[key], key
