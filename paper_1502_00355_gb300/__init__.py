"""GB300-native Smart Laplacian mesh smoothing (Zhao, Mei, Xu, Zhang).

Thin ctypes binding over the C ABI in ``include/slsmooth.h``: argument
marshalling only.  Every step of the smoothing runs in the library's CUDA
kernels (``csrc/``); there is no CPU fallback, and loading fails loudly when
the library has not been built (``build()`` or ``__graft_entry__.build()``).

PyTorch is used only as plumbing: ``Mesh.coords_device`` copies into a torch
CUDA tensor, and a torch stream can be handed to the library.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import LIB as _LIB_PATH
from .build import build

__all__ = ["build", "lib", "Mesh", "Batch", "Server", "SlsError", "Options", "Info",
           "KERNEL_AUTO", "KERNEL_FP64", "KERNEL_FILTERED"]

KERNEL_AUTO, KERNEL_FP64, KERNEL_FILTERED = 0, 1, 2
_KERNELS = {"auto": KERNEL_AUTO, "fp64": KERNEL_FP64, "filtered": KERNEL_FILTERED}

SLS_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid", 2: "nonmanifold", 3: "oom", 4: "cuda", 5: "timeout",
                6: "busy", 7: "rejected", 8: "not_found"}


class Options(C.Structure):
    _fields_ = [("accept_strict", C.c_int32), ("copy_back", C.c_int32), ("layout", C.c_int32),
                ("kernel", C.c_int32), ("record_accept", C.c_int32), ("block_size", C.c_int32),
                ("l2_window", C.c_int32), ("passes_per_check", C.c_int32), ("host_build", C.c_int32),
                ("form", C.c_int32), ("precision", C.c_int32), ("skip_unchanged", C.c_int32),
                ("numbering", C.c_int32), ("stream", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("accepted_last", C.c_int64),
                ("max_d2_last", C.c_double), ("fp64_fallbacks", C.c_int64), ("launches", C.c_int64),
                ("nodes_skipped", C.c_int64)]

    def as_dict(self) -> dict:
        return dict(iterations=self.iterations, converged=self.converged,
                    accepted_last=self.accepted_last, maxd2_last=self.max_d2_last,
                    fp64_fallbacks=self.fp64_fallbacks, launches=self.launches,
                    nodes_skipped=self.nodes_skipped)


class SlsError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def lib() -> C.CDLL:
    """The loaded libslsmooth.so.  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"{_LIB_PATH} is missing: the CUDA library has not been built "
                                   "(call paper_1502_00355_gb300.build())")
            L = C.CDLL(_LIB_PATH)
            P, I32, I64, D, S = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_int
            PP = C.POINTER(C.c_void_p)
            sigs = {
                "sls_default_options": (None, [P]),
                "sls_mesh_create": (S, [P, I64, P, I64, P, P, PP]),
                "sls_smooth": (S, [P, I32, D, P]),
                "sls_get_coords": (S, [P, P, I32]),
                "sls_set_coords": (S, [P, P, I32]),
                "sls_get_accept": (S, [P, P]),
                "sls_gather_coords": (S, [P, P, I64, P]),
                "sls_scatter_coords": (S, [P, P, I64, P]),
                "sls_quality_histogram": (S, [P, I32, D, D, P, P, P]),
                "sls_mesh_stats": (S, [P, P, P, P, P]),
                "sls_mesh_destroy": (S, [P]),
                "sls_batch_create": (S, [P, I32, P, P, P, PP]),
                "sls_batch_smooth": (S, [P, P]),
                "sls_batch_get_coords": (S, [P, I32, P]),
                "sls_batch_reset": (S, [P]),
                "sls_batch_shape": (S, [P, P, P]),
                "sls_batch_set_shape": (S, [P, I32, I64]),
                "sls_batch_destroy": (S, [P]),
                "sls_server_create": (S, [C.c_size_t, I32, P, PP]),
                "sls_submit": (S, [P, P, I64, P, I64, P, I32, D, C.POINTER(C.c_uint64)]),
                "sls_wait": (S, [P, C.c_uint64, D, P, P]),
                "sls_server_stats": (S, [P, P, P, P, P]),
                "sls_server_destroy": (S, [P]),
                "sls_smooth_noalloc": (S, [P, P, P, I32, D, P, P]),
                "sls_trim_memory": (S, [C.c_size_t]),
                "sls_status_str": (C.c_char_p, [S]),
                "sls_last_error": (C.c_char_p, []),
            }
            for name, (res, args) in sigs.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def trim_memory(keep_bytes: int = 0):
    """Hand the library pool's unused device memory (current device) back to
    the driver, keeping at most keep_bytes (``sls_trim_memory``)."""
    _check(lib().sls_trim_memory(int(keep_bytes)), "sls_trim_memory")


def _check(code: int, where: str):
    if code != SLS_OK:
        msg = lib().sls_last_error().decode(errors="replace")
        raise SlsError(code, where, msg)


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_options(*, strict=False, copy_back=False, layout="aos", kernel="auto", record_accept=False,
                 block_size=0, l2_window=False, passes_per_check=0, host_build=False, form="A",
                 precision=64, skip_unchanged=False, numbering="auto", stream=None) -> Options:
    o = Options()
    lib().sls_default_options(C.byref(o))
    o.accept_strict = int(bool(strict))
    o.copy_back = int(bool(copy_back))
    o.layout = {"aos": 0, "soa": 1}[layout] if isinstance(layout, str) else int(layout)
    o.kernel = _KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    o.record_accept = int(bool(record_accept))
    o.block_size = int(block_size)
    o.l2_window = int(bool(l2_window))
    o.passes_per_check = int(passes_per_check)
    o.host_build = int(bool(host_build))
    o.form = {"A": 0, "B": 1}[form]
    o.precision = int(precision)
    o.skip_unchanged = int(bool(skip_unchanged))
    o.numbering = {"auto": 0, "given": 1, "grouped": 2}[numbering] if isinstance(numbering, str) else int(numbering)
    o.stream = None if stream is None else C.c_void_p(int(stream))
    return o


class Mesh:
    """A mesh resident on the current CUDA device (``sls_mesh``)."""

    def __init__(self, xy, tri, boundary=None, **options):
        L = lib()
        self._xy_shape = None
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
        bnd = None if boundary is None else np.ascontiguousarray(boundary, dtype=np.uint8)
        if bnd is not None and bnd.shape != (xy.shape[0],):
            raise ValueError("boundary must have one flag per node")
        self.options = make_options(**options)
        h = C.c_void_p()
        _check(L.sls_mesh_create(_p(xy), xy.shape[0], _p(tri), tri.shape[0], _p(bnd),
                                 C.byref(self.options), C.byref(h)), "sls_mesh_create")
        self._h = h
        n, m, nf, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_double()
        _check(L.sls_mesh_stats(h, C.byref(n), C.byref(m), C.byref(nf), C.byref(d)), "sls_mesh_stats")
        self.n, self.m, self.n_free, self.diag = n.value, m.value, nf.value, d.value

    @property
    def handle(self) -> C.c_void_p:
        if self._h is None:
            raise RuntimeError("mesh is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().sls_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def smooth(self, max_iter: int, tol: float = 0.0) -> dict:
        info = Info()
        _check(lib().sls_smooth(self.handle, int(max_iter), float(tol), C.byref(info)), "sls_smooth")
        return info.as_dict()

    def smooth_noalloc(self, xy_in, xy_out, max_iter: int, tol: float = 0.0, stream=None) -> dict:
        """Passes on two caller-owned float64 CUDA tensors of shape (n, 2),
        allocating nothing (``sls_smooth_noalloc``): xy_in holds the start
        and is clobbered, xy_out receives the result."""
        import torch
        for t in (xy_in, xy_out):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == 2 * self.n):
                raise ValueError("coordinates must be contiguous float64 CUDA tensors with 2n elements")
        info = Info()
        _check(lib().sls_smooth_noalloc(self.handle, C.c_void_p(xy_in.data_ptr()), C.c_void_p(xy_out.data_ptr()),
                                        int(max_iter), float(tol), None if stream is None else C.c_void_p(int(stream)),
                                        C.byref(info)), "sls_smooth_noalloc")
        return info.as_dict()

    def coords(self, out=None) -> np.ndarray:
        """Current coordinates as a (n, 2) float64 array (written into `out`
        when given, e.g. a pinned buffer)."""
        if out is None:
            out = np.empty((self.n, 2), np.float64)
        elif not (out.dtype == np.float64 and out.flags.c_contiguous and out.size == 2 * self.n):
            raise ValueError("out must be a contiguous float64 array with 2n elements")
        _check(lib().sls_get_coords(self.handle, _p(out), 0), "sls_get_coords")
        return out

    def coords_device(self, out=None):
        """Current coordinates as a (n, 2) float64 torch CUDA tensor."""
        import torch
        if out is None:
            out = torch.empty((self.n, 2), dtype=torch.float64, device="cuda")
        if not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() == 2 * self.n):
            raise ValueError("out must be a contiguous float64 CUDA tensor with 2n elements")
        _check(lib().sls_get_coords(self.handle, C.c_void_p(out.data_ptr()), 1), "sls_get_coords")
        return out

    def set_coords(self, xy):
        """Overwrite the coordinates from a (n, 2) array, or from a float64 torch CUDA tensor."""
        if hasattr(xy, "is_cuda") and xy.is_cuda:
            import torch
            if not (xy.dtype == torch.float64 and xy.is_contiguous() and xy.numel() == 2 * self.n):
                raise ValueError("xy must be a contiguous float64 CUDA tensor with 2n elements")
            _check(lib().sls_set_coords(self.handle, C.c_void_p(xy.data_ptr()), 1), "sls_set_coords")
            return
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        if xy.shape[0] != self.n:
            raise ValueError("wrong number of nodes")
        _check(lib().sls_set_coords(self.handle, _p(xy), 0), "sls_set_coords")

    def gather(self, idx, out):
        """Current coordinates of the nodes idx (int32 CUDA tensor) into out
        (float64 CUDA tensor of shape (k, 2))."""
        _check(lib().sls_gather_coords(self.handle, C.c_void_p(idx.data_ptr()), int(idx.numel()),
                                       C.c_void_p(out.data_ptr())), "sls_gather_coords")
        return out

    def scatter(self, idx, values):
        """Overwrite the coordinates of the nodes idx (int32 CUDA tensor) with
        values (float64 CUDA tensor of shape (k, 2))."""
        _check(lib().sls_scatter_coords(self.handle, C.c_void_p(idx.data_ptr()), int(idx.numel()),
                                        C.c_void_p(values.data_ptr())), "sls_scatter_coords")

    def accept_mask(self) -> np.ndarray:
        out = np.empty(self.n, np.uint8)
        _check(lib().sls_get_accept(self.handle, _p(out)), "sls_get_accept")
        return out

    def histogram(self, nbins: int = 20, lo: float = -1.0, hi: float = 1.0):
        counts = np.empty(nbins, np.int64)
        qmin, qmean = C.c_double(), C.c_double()
        _check(lib().sls_quality_histogram(self.handle, int(nbins), float(lo), float(hi), _p(counts),
                                           C.byref(qmin), C.byref(qmean)), "sls_quality_histogram")
        return counts, qmin.value, qmean.value


class Batch:
    """Many meshes smoothed together (``sls_batch``)."""

    def __init__(self, meshes, iters, tols=None, **options):
        L = lib()
        k = len(meshes)
        arr = (C.c_void_p * k)(*[m.handle.value for m in meshes])
        it = np.ascontiguousarray(iters, dtype=np.int32)
        tl = None if tols is None else np.ascontiguousarray(tols, dtype=np.float64)
        self.options = make_options(**options)
        h = C.c_void_p()
        _check(L.sls_batch_create(arr, k, _p(it), _p(tl), C.byref(self.options), C.byref(h)),
               "sls_batch_create")
        self._h = h
        self.k = k
        self.sizes = [m.n for m in meshes]

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def smooth(self) -> list[dict]:
        infos = (Info * self.k)()
        _check(lib().sls_batch_smooth(self._h, infos), "sls_batch_smooth")
        return [i.as_dict() for i in infos]

    def coords(self, j: int) -> np.ndarray:
        out = np.empty((self.sizes[j], 2), np.float64)
        _check(lib().sls_batch_get_coords(self._h, int(j), _p(out)), "sls_batch_get_coords")
        return out

    def reset(self):
        _check(lib().sls_batch_reset(self._h), "sls_batch_reset")

    @property
    def shape(self) -> tuple[int, int]:
        """(threads per block, warp chunk) of the launches."""
        b, c = C.c_int32(), C.c_int64()
        _check(lib().sls_batch_shape(self._h, C.byref(b), C.byref(c)), "sls_batch_shape")
        return b.value, c.value

    def set_shape(self, block: int, chunk: int):
        _check(lib().sls_batch_set_shape(self._h, int(block), int(chunk)), "sls_batch_set_shape")

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().sls_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching smoothing server (``sls_server``)."""

    def __init__(self, hbm_budget: int = 0, max_queue: int = 0, **options):
        self.options = make_options(**options)
        h = C.c_void_p()
        _check(lib().sls_server_create(int(hbm_budget), int(max_queue), C.byref(self.options),
                                       C.byref(h)), "sls_server_create")
        self._h = h
        self._sizes: dict[int, int] = {}

    def submit(self, xy, tri, boundary=None, max_iter: int = 100, tol: float = 0.0) -> int:
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
        bnd = None if boundary is None else np.ascontiguousarray(boundary, dtype=np.uint8)
        job = C.c_uint64()
        _check(lib().sls_submit(self._h, _p(xy), xy.shape[0], _p(tri), tri.shape[0], _p(bnd),
                                int(max_iter), float(tol), C.byref(job)), "sls_submit")
        self._sizes[job.value] = xy.shape[0]
        return job.value

    def wait(self, job: int, timeout: float = -1.0, want_coords: bool = True):
        info = Info()
        n = self._sizes.get(job)
        out = np.empty((n, 2), np.float64) if (want_coords and n is not None) else None
        _check(lib().sls_wait(self._h, C.c_uint64(job), float(timeout), _p(out), C.byref(info)),
               "sls_wait")
        self._sizes.pop(job, None)
        return out, info.as_dict()

    def try_wait(self, job: int, out: np.ndarray):
        """Non-blocking sls_wait: None while the job runs; once it is done,
        fills `out` (a contiguous (n, 2) float64 array) and returns its info."""
        info = Info()
        code = lib().sls_wait(self._h, C.c_uint64(job), 0.0, _p(out), C.byref(info))
        if code == 5:  # SLS_ERR_TIMEOUT: not finished yet
            return None
        _check(code, "sls_wait")
        self._sizes.pop(job, None)
        return info.as_dict()

    def stats(self) -> dict:
        p50, p99, nups = C.c_double(), C.c_double(), C.c_double()
        done = C.c_int64()
        _check(lib().sls_server_stats(self._h, C.byref(p50), C.byref(p99), C.byref(nups),
                                      C.byref(done)), "sls_server_stats")
        return dict(p50_ms=p50.value, p99_ms=p99.value, node_updates_per_s=nups.value,
                    completed=done.value)

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().sls_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
