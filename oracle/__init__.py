"""Plain FP64 CPU oracle for 2-D Smart Laplacian smoothing (ctypes wrapper).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library under
test never imports it, and it never imports the library: the two share no
code.  The arithmetic lives in ``oracle.c``; this file compiles it with
``gcc -O2 -ffp-contract=off`` (sequential build, plus an OpenMP build of the
same source) and marshals numpy arrays.

Functions and the part of the paper they follow:
  * ``alpha``            - element quality, Lee and Lo's alpha (Section 3.3.1)
  * ``OracleMesh``       - neighbours / incident triangles (Section 3.3.2) and
                           boundary constraints (Section 3.3.3)
  * ``OracleMesh.sweep`` - one Form-A pass (Eq. 2) with the smart accept test
                           (Sections 2.1 and 3.3.4)
  * ``OracleMesh.smooth``- the iteration loop with the copy-back of Form A
  * ``OracleMesh.colouring`` - Jones-Plassmann colouring of the free nodes
  * ``OracleMesh.smooth(form="B")`` - Form B (Eq. 3) as multicolour
                           Gauss-Seidel: colour classes in turn, in place
  * ``OracleMesh.smooth(precision=32)`` - both forms in binary32, the
                           paper's precision (Section 4, reading R11)
  * ``OracleMesh.histogram`` - quality histogram of all triangles

Parity pins (tests/test_oracle_*.py): closed forms of alpha, the regular
hexagon worked case, the fixed point of a symmetric dyadic grid, boundary
invariance, exact-rational brute force of the accept decisions on tiny
meshes, permutation invariance.  The alpha formula itself is pinned only to
its textbook values (the paper names the measure but prints no value):
"parity unpinned" against the paper for that one definition.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build")
_LIBS: dict[bool, C.CDLL] = {}
_LOCK = threading.Lock()

STATUS = {0: "ok", 1: "invalid", 2: "nonmanifold", 3: "nomem"}

# seed of the colouring priorities, splitmix64(COLOUR_SEED + i)
COLOUR_SEED = 150200355


def _lib_path(openmp: bool) -> str:
    return os.path.join(_OUT, "liboracle_omp.so" if openmp else "liboracle.so")


def build(force: bool = False) -> None:
    """Compile the sequential and the OpenMP oracle libraries."""
    os.makedirs(_OUT, exist_ok=True)
    for omp in (False, True):
        out = _lib_path(omp)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               _SRC, "-o", out + ".tmp", "-lm"]
        if omp:
            cmd.insert(1, "-fopenmp")
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)


def _lib(openmp: bool = False) -> C.CDLL:
    with _LOCK:
        if openmp not in _LIBS:
            build()
            lib = C.CDLL(_lib_path(openmp))
            P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
            lib.orc_alpha.restype = D
            lib.orc_alpha.argtypes = [D] * 6
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [I64, I64, P, P, P, C.POINTER(C.c_int)]
            lib.orc_free.argtypes = [P]
            for f in ("orc_n", "orc_m", "orc_nnz"):
                getattr(lib, f).restype = I64
                getattr(lib, f).argtypes = [P]
            lib.orc_diag.restype = D
            lib.orc_diag.argtypes = [P]
            lib.orc_get_adjacency.argtypes = [P] * 6
            lib.orc_sweep.argtypes = [P, P, P, C.c_int, P, P, P]
            lib.orc_update_nodes.argtypes = [P, P, C.c_int, I64, P, P, P, P, P, P, P]
            lib.orc_smooth.restype = C.c_int
            lib.orc_smooth.argtypes = [P, P, I32, D, C.c_int, P, P, P, P, P]
            lib.orc_histogram.argtypes = [P, P, I32, D, D, P, P, P]
            lib.orc_colour.restype = C.c_int
            lib.orc_colour.argtypes = [P, C.c_uint64, P, P, P]
            lib.orc_sweep_coloured.argtypes = [P, P, P, I32, C.c_int, P, P, P]
            lib.orc_smooth_coloured.restype = C.c_int
            lib.orc_smooth_coloured.argtypes = [P, P, P, I32, I32, D, C.c_int, P, P, P, P, P]
            lib.orc32_alpha.restype = C.c_float
            lib.orc32_alpha.argtypes = [C.c_float] * 6
            lib.orc32_sweep.argtypes = [P, P, P, P, I32, C.c_int, P, P, P]
            lib.orc32_smooth.restype = C.c_int
            lib.orc32_smooth.argtypes = [P, P, P, I32, I32, D, C.c_int, P, P, P, P, P]
            _LIBS[openmp] = lib
        return _LIBS[openmp]


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def alpha(ax, ay, bx, by, cx, cy) -> float:
    """Lee and Lo's alpha of triangle (a, b, c) in that vertex order (Section 3.3.1)."""
    return _lib().orc_alpha(ax, ay, bx, by, cx, cy)


def alpha32(ax, ay, bx, by, cx, cy) -> np.float32:
    """The same alpha in binary32 arithmetic (R11); arguments are rounded to float."""
    return np.float32(_lib().orc32_alpha(*[float(np.float32(v)) for v in (ax, ay, bx, by, cx, cy)]))


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle mesh rejected: {STATUS.get(code, code)}")
        self.code = code


class OracleMesh:
    """Mesh plus adjacency as the oracle builds it (Sections 3.3.2-3.3.3)."""

    def __init__(self, xy, tri, boundary=None, openmp: bool = False):
        self._lib = _lib(openmp)
        self.xy0 = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
        bnd = None if boundary is None else np.ascontiguousarray(boundary, dtype=np.uint8)
        st = C.c_int(0)
        h = self._lib.orc_create(self.xy0.shape[0], self.tri.shape[0], _ptr(self.xy0),
                                 _ptr(self.tri), _ptr(bnd), C.byref(st))
        if not h:
            raise OracleError(st.value)
        self._h = C.c_void_p(h)
        self.n = int(self._lib.orc_n(self._h))
        self.m = int(self._lib.orc_m(self._h))
        self.diag = float(self._lib.orc_diag(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_free(h)
            self._h = None

    def adjacency(self):
        """(nbr_ptr, nbr, tri_ptr, tri_of, fixed): N(i) in canonical order, T(i) ascending."""
        nnz = int(self._lib.orc_nnz(self._h))
        nbr_ptr = np.empty(self.n + 1, np.int64)
        nbr = np.empty(max(nnz, 1), np.int32)
        tri_ptr = np.empty(self.n + 1, np.int64)
        tri_of = np.empty(3 * self.m, np.int32)
        fixed = np.empty(self.n, np.uint8)
        self._lib.orc_get_adjacency(self._h, _ptr(nbr_ptr), _ptr(nbr), _ptr(tri_ptr),
                                    _ptr(tri_of), _ptr(fixed))
        return nbr_ptr, nbr[:nnz], tri_ptr, tri_of, fixed

    def sweep(self, xy, strict: bool = False):
        """One Form-A pass from xy.  Returns (xy_next, accept, maxd2, nacc)."""
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        nxt = np.empty_like(xy)
        acc = np.empty(self.n, np.uint8)
        maxd2 = C.c_double(0.0)
        nacc = C.c_int64(0)
        self._lib.orc_sweep(self._h, _ptr(xy), _ptr(nxt), int(strict), _ptr(acc),
                            C.byref(maxd2), C.byref(nacc))
        return nxt, acc, maxd2.value, nacc.value

    def update_nodes(self, xy, idx, strict: bool = False):
        """The pass-(q+1) update of the listed nodes from xy = X^q.
        Returns (xy_out[k,2], accept[k], d2[k], q_old[k], q_new[k], centre[k,2])."""
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        k = idx.size
        out = np.empty((k, 2), np.float64)
        acc = np.empty(k, np.uint8)
        d2 = np.empty(k, np.float64)
        qo = np.empty(k, np.float64)
        qn = np.empty(k, np.float64)
        cand = np.empty((k, 2), np.float64)
        self._lib.orc_update_nodes(self._h, _ptr(xy), int(strict), k, _ptr(idx), _ptr(out),
                                   _ptr(acc), _ptr(d2), _ptr(qo), _ptr(qn), _ptr(cand))
        return out, acc, d2, qo, qn, cand

    def colouring(self, seed: int = COLOUR_SEED):
        """Jones-Plassmann colouring of the free nodes.  Returns (colour[n]
        with -1 for fixed nodes, number of colours, number of rounds)."""
        col = np.empty(self.n, np.int32)
        nc = C.c_int32(0)
        rounds = C.c_int32(0)
        rc = self._lib.orc_colour(self._h, C.c_uint64(seed), _ptr(col), C.byref(nc), C.byref(rounds))
        if rc != 0:
            raise OracleError(rc)
        return col, nc.value, rounds.value

    def sweep_coloured(self, xy, colour, ncolours: int, strict: bool = False):
        """One Form-B sweep (colour classes in turn, in place) from xy.
        Returns (xy_next, accept, maxd2, nacc)."""
        xy = np.array(xy, dtype=np.float64, copy=True).reshape(-1, 2)
        colour = np.ascontiguousarray(colour, dtype=np.int32)
        acc = np.empty(self.n, np.uint8)
        maxd2 = C.c_double(0.0)
        nacc = C.c_int64(0)
        self._lib.orc_sweep_coloured(self._h, _ptr(xy), _ptr(colour), int(ncolours), int(strict), _ptr(acc),
                                     C.byref(maxd2), C.byref(nacc))
        return xy, acc, maxd2.value, nacc.value

    def smooth(self, xy, max_iter: int, tol: float = 0.0, strict: bool = False, form: str = "A",
               precision: int = 64):
        """Iterate from xy (Form A, or Form B in colour order; FP64, or binary32
        with xy rounded to float first).  Returns (xy_final as float64 --
        binary32 values widened exactly --, info dict, accept mask of the last
        pass)."""
        acc = np.zeros(self.n, np.uint8)
        it = C.c_int32(0)
        conv = C.c_int32(0)
        nacc = C.c_int64(0)
        maxd2 = C.c_double(0.0)
        if precision == 32:
            x32 = np.array(xy, dtype=np.float64).reshape(-1, 2).astype(np.float32)
            col, nc = (None, 0) if form == "A" else self.colouring()[:2]
            rc = self._lib.orc32_smooth(self._h, _ptr(x32), _ptr(col), int(nc), int(max_iter), float(tol),
                                        int(strict), _ptr(acc), C.byref(it), C.byref(conv), C.byref(nacc),
                                        C.byref(maxd2))
            if rc != 0:
                raise OracleError(rc)
            info = dict(iterations=it.value, converged=conv.value, accepted_last=nacc.value,
                        maxd2_last=maxd2.value)
            return x32.astype(np.float64), info, acc
        if precision != 64:
            raise ValueError(precision)
        xy = np.array(xy, dtype=np.float64, copy=True).reshape(-1, 2)
        if form == "A":
            rc = self._lib.orc_smooth(self._h, _ptr(xy), int(max_iter), float(tol), int(strict),
                                      _ptr(acc), C.byref(it), C.byref(conv), C.byref(nacc),
                                      C.byref(maxd2))
        elif form == "B":
            col, nc, _ = self.colouring()
            rc = self._lib.orc_smooth_coloured(self._h, _ptr(xy), _ptr(col), int(nc), int(max_iter),
                                               float(tol), int(strict), _ptr(acc), C.byref(it),
                                               C.byref(conv), C.byref(nacc), C.byref(maxd2))
        else:
            raise ValueError(form)
        if rc != 0:
            raise OracleError(rc)
        info = dict(iterations=it.value, converged=conv.value, accepted_last=nacc.value,
                    maxd2_last=maxd2.value)
        return xy, info, acc

    def histogram(self, xy, nbins: int = 20, lo: float = -1.0, hi: float = 1.0):
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        counts = np.empty(nbins, np.int64)
        qmin = C.c_double(0.0)
        qmean = C.c_double(0.0)
        self._lib.orc_histogram(self._h, _ptr(xy), int(nbins), float(lo), float(hi),
                                _ptr(counts), C.byref(qmin), C.byref(qmean))
        return counts, qmin.value, qmean.value
