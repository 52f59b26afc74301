"""C-ABI library checks that need no GPU: it loads, exports every symbol the
header declares, and rejects bad meshes on the host before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1502_00355_gb300 as sls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    sls.build()
    return sls.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "slsmooth.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sls_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("sls_mesh_create", "sls_smooth", "sls_get_coords", "sls_quality_histogram",
              "sls_batch_create", "sls_batch_smooth", "sls_server_create", "sls_submit", "sls_wait"):
        assert s in syms


def test_library_exports_every_declared_symbol(L):
    for s in declared_symbols():
        assert hasattr(L, s), s


def _create(L, xy, tri, bnd=None, host_build=True):
    """Host validation runs before any device call when the host build is
    selected, so these checks need no GPU."""
    xy = np.ascontiguousarray(xy, np.float64)
    tri = np.ascontiguousarray(tri, np.int32)
    h = C.c_void_p()
    bp = None if bnd is None else np.ascontiguousarray(bnd, np.uint8).ctypes.data_as(C.c_void_p)
    opt = sls.make_options(host_build=host_build)
    st = L.sls_mesh_create(xy.ctypes.data_as(C.c_void_p), xy.shape[0], tri.ctypes.data_as(C.c_void_p),
                           tri.shape[0], bp, C.byref(opt), C.byref(h))
    if st == 0:
        L.sls_mesh_destroy(h)
    return st, L.sls_last_error().decode()


def test_host_validation_rejects_bad_meshes(L):
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0], [0.5, -1.0]])
    assert _create(L, xy, [[0, 1, 5]])[0] == 1
    assert _create(L, xy, [[0, -1, 2]])[0] == 1
    assert _create(L, xy, [[0, 2, 2]])[0] == 1
    assert _create(L, xy[:2], [[0, 1, 0]])[0] == 1
    bad = xy.copy()
    bad[1, 0] = np.inf
    st, msg = _create(L, bad, [[0, 1, 2]])
    assert st == 1 and "finite" in msg
    st, msg = _create(L, xy, [[0, 1, 2], [1, 0, 3], [0, 1, 4]])
    assert st == 2 and "more than two" in msg
    assert L.sls_status_str(2) == b"non-manifold edge"


def test_null_arguments(L):
    assert L.sls_smooth(None, 1, 0.0, None) == 1
    assert L.sls_get_coords(None, None, 0) == 1
    assert L.sls_mesh_destroy(None) == 0


def test_fails_loudly_without_a_gpu(L):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    for host_build in (True, False):
        st, msg = _create(L, xy, [[0, 1, 2]], host_build=host_build)
        assert st == 4 and msg  # SLS_ERR_CUDA with a message: no silent CPU path


def _c_layout(struct: str, fields) -> dict:
    """sizeof and field offsets of a header struct, from a C program built
    against the header with the system compiler."""
    import subprocess
    import tempfile
    body = "\n".join(f'    printf("{f} %zu\\n", offsetof({struct}, {f}));' for f in fields)
    src = f"""#include <stddef.h>
#include <stdio.h>
#include "slsmooth.h"
int main(void) {{
    printf("sizeof %zu\\n", sizeof({struct}));
{body}
    return 0;
}}
"""
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.parametrize("pystruct, cname", [(sls.Options, "sls_options"), (sls.Info, "sls_info")])
def test_binding_structs_match_the_header(pystruct, cname):
    fields = [f for f, _ in pystruct._fields_]
    lay = _c_layout(cname, fields)
    assert lay["sizeof"] == C.sizeof(pystruct)
    for f in fields:
        assert lay[f] == getattr(pystruct, f).offset, f
