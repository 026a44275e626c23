"""CPU oracle for the sparse tensor-times-vector product (paper Sec. 3.3, Eq. 3),
the MTTKRP built on it (named in Sec. 3.3 and Sec. 5), and the paper's two
simple kernels, the dense dot product (Eq. 1) and matrix-vector product (Eq. 2).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it; the CUDA
library (``paper_2510_01495_gb300``) neither imports nor links it, and this
package imports nothing from the library.

``ttv``, ``mttkrp``, ``dot`` and ``matvec`` wrap the plain C statements in ``ttv_oracle.c``
(built with gcc and ``-ffp-contract=off``).  It upcasts float32 inputs to float64 exactly before
the call, so an FP32-stored tensor is evaluated as the exact FP64 values it
holds.  Parity status of every function here: pinned (see tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ttv_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libttv_oracle.so")
_MAX_D = 16
_lock = threading.Lock()
_lib = None

ERRORS = {
    0: "ok",
    -1: "invalid argument",
    -2: "invalid or repeated mode",
    -3: "vector length differs from the mode size",
    -4: "subscript out of range",
    -5: "out of memory",
}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle_ttv failed: {ERRORS.get(code, code)} ({code})")
        self.code = code


class _Out(ctypes.Structure):
    _fields_ = [
        ("order", ctypes.c_int32),
        ("shape", ctypes.c_int64 * _MAX_D),
        ("nnz", ctypes.c_int64),
        ("subs", ctypes.POINTER(ctypes.c_int64)),
        ("vals", ctypes.POINTER(ctypes.c_double)),
    ]


def compile_library(src: str = _SRC, out_path: str = _LIB_PATH, extra_flags=()) -> str:
    """Compile the C oracle into a shared library (plain gcc, no CUDA)."""
    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    tmp = out_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           *extra_flags, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, out_path)
    return out_path


def build() -> str:
    """Build the oracle library if it is missing or older than its source."""
    if (not os.path.exists(_LIB_PATH)
            or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        compile_library()
    return _LIB_PATH


def load_library(path: str):
    lib = ctypes.CDLL(path)
    lib.oracle_ttv.restype = ctypes.c_int
    lib.oracle_ttv.argtypes = [
        ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
        ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
        ctypes.POINTER(ctypes.POINTER(ctypes.c_double)), ctypes.c_int32,
        ctypes.POINTER(_Out)]
    lib.oracle_free.restype = None
    lib.oracle_free.argtypes = [ctypes.POINTER(_Out)]
    lib.oracle_mttkrp.restype = ctypes.c_int
    lib.oracle_mttkrp.argtypes = [
        ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
        ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.POINTER(ctypes.c_double)),
        ctypes.POINTER(ctypes.c_double)]
    lib.oracle_dot.restype = ctypes.c_int
    lib.oracle_dot.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)]
    lib.oracle_matvec.restype = ctypes.c_int
    lib.oracle_matvec.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                  ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    return lib


def _get_lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _as_f64(a) -> np.ndarray:
    a = np.asarray(a)
    if a.dtype not in (np.float64, np.float32):
        raise TypeError(f"values must be float64 or float32, got {a.dtype}")
    return np.ascontiguousarray(a, dtype=np.float64)   # float32 -> float64 is exact


def ttv(subs, vals, shape, modes, vecs, dense: bool = False, lib=None):
    """Sparse TTV by the plain definition.

    subs  : (nnz, d) integer array of 0-based subscripts (any memory order)
    vals  : (nnz,) float64 or float32
    shape : d mode sizes
    modes : contracted modes (a single int or a sequence), any order
    vecs  : one vector per entry of ``modes`` (float64 or float32)
    dense : return a dense array of shape[R] instead of COO

    Returns (newsubs (nnz_out, d - n_v) int64, newvals (nnz_out,) float64,
    newshape tuple) -- for ``dense`` newsubs is None and newvals has shape
    newshape (a 0-d array when every mode is contracted).
    """
    lib = lib or _get_lib()
    if np.isscalar(modes):
        modes, vecs = [int(modes)], [vecs]
    shape = np.ascontiguousarray(np.asarray(shape, dtype=np.int64).reshape(-1))
    d = int(shape.size)
    subs = np.ascontiguousarray(np.asarray(subs, dtype=np.int64).reshape(-1, d))
    vals = _as_f64(vals).reshape(-1)
    if subs.shape[0] != vals.shape[0]:
        raise ValueError("subs and vals disagree on nnz")
    modes_a = np.ascontiguousarray(np.asarray(modes, dtype=np.int32).reshape(-1))
    vec_arrs = [_as_f64(v).reshape(-1) for v in vecs]
    if len(vec_arrs) != modes_a.size:
        raise ValueError("one vector per contracted mode")
    lens = np.ascontiguousarray(np.array([v.size for v in vec_arrs], dtype=np.int64))
    ptr_arr = (ctypes.POINTER(ctypes.c_double) * max(1, len(vec_arrs)))(
        *[v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for v in vec_arrs])
    out = _Out()
    rc = lib.oracle_ttv(
        d, shape.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(vals.size),
        subs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        int(modes_a.size), modes_a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        lens.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ptr_arr,
        1 if dense else 0, ctypes.byref(out))
    if rc != 0:
        raise OracleError(rc)
    try:
        order = out.order
        newshape = tuple(int(out.shape[j]) for j in range(order))
        n = int(out.nnz)
        vals_out = np.ctypeslib.as_array(out.vals, shape=(max(n, 1),))[:n].copy()
        if dense:
            return None, vals_out.reshape(newshape), newshape
        if order > 0 and n > 0:
            subs_out = np.ctypeslib.as_array(out.subs, shape=(n * order,)).copy().reshape(n, order)
        else:
            subs_out = np.zeros((n, order), dtype=np.int64)
        return subs_out, vals_out, newshape
    finally:
        lib.oracle_free(ctypes.byref(out))


def mttkrp(subs, vals, shape, mode: int, factors, lib=None) -> np.ndarray:
    """MTTKRP along ``mode`` by the plain definition: ``factors`` holds one
    (shape[m], rank) matrix per mode (the entry for ``mode`` is ignored and may
    be None); returns the (shape[mode], rank) float64 result."""
    lib = lib or _get_lib()
    shape = np.ascontiguousarray(np.asarray(shape, dtype=np.int64).reshape(-1))
    d = int(shape.size)
    subs = np.ascontiguousarray(np.asarray(subs, dtype=np.int64).reshape(-1, d))
    vals = _as_f64(vals).reshape(-1)
    if subs.shape[0] != vals.shape[0]:
        raise ValueError("subs and vals disagree on nnz")
    mode = int(mode)
    rank = None
    mats = []
    for m in range(d):
        if m == mode:
            mats.append(None)
            continue
        a = _as_f64(factors[m])
        if a.ndim != 2 or a.shape[0] != shape[m]:
            raise ValueError(f"factor {m} must be ({shape[m]}, rank)")
        if rank is None:
            rank = a.shape[1]
        if a.shape[1] != rank:
            raise ValueError("factors disagree on the rank")
        mats.append(np.ascontiguousarray(a))
    if rank is None:
        raise ValueError("no factor matrices")
    nullp = ctypes.POINTER(ctypes.c_double)()
    ptr_arr = (ctypes.POINTER(ctypes.c_double) * d)(
        *[nullp if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in mats])
    out = np.zeros((int(shape[mode]), rank), dtype=np.float64)
    rc = lib.oracle_mttkrp(d, shape.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(vals.size),
                           subs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                           vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), mode, rank, ptr_arr,
                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise OracleError(rc)
    return out


def dot(x, y, lib=None) -> float:
    """x . y by the plain definition (Eq. 1): rounded products summed in index
    order with Neumaier's compensation."""
    lib = lib or _get_lib()
    x = _as_f64(x).reshape(-1)
    y = _as_f64(y).reshape(-1)
    if x.size != y.size:
        raise ValueError("vectors of different lengths")
    out = ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.oracle_dot(int(x.size), x.ctypes.data_as(dp), y.ctypes.data_as(dp), ctypes.byref(out))
    if rc != 0:
        raise OracleError(rc)
    return float(out.value)


def matvec(A, x, lib=None) -> np.ndarray:
    """A x by the plain definition (Eq. 2): row i is the dot product of A's row
    i with x.  ``A`` is read in its own memory order (C or Fortran)."""
    lib = lib or _get_lib()
    A = np.asarray(A)
    if A.ndim != 2:
        raise ValueError("A must be a matrix")
    if A.dtype != np.float64:
        A = _as_f64(A)
    n1, n2 = A.shape
    x = _as_f64(x).reshape(-1)
    if x.size != n2:
        raise ValueError("x length differs from the number of columns")
    if A.strides[0] % 8 or A.strides[1] % 8:
        A = np.ascontiguousarray(A)
    y = np.zeros(n1, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.oracle_matvec(n1, n2, A.ctypes.data_as(dp), A.strides[0] // 8, A.strides[1] // 8,
                           x.ctypes.data_as(dp), y.ctypes.data_as(dp))
    if rc != 0:
        raise OracleError(rc)
    return y


# ---- the same TTV definition on all host cores (OpenMP), for the benchmark's
# multi-core CPU baseline; bit-identical to ``ttv`` (tests/test_oracle_pins.py)

_OMP_SRC = os.path.join(_HERE, "ttv_oracle_omp.c")
_OMP_LIB_PATH = os.path.join(_BUILD_DIR, "libttv_oracle_omp.so")
_omp_lib = None


def build_parallel() -> str:
    """Build the OpenMP statement if it is missing or older than its source."""
    if (not os.path.exists(_OMP_LIB_PATH)
            or os.path.getmtime(_OMP_LIB_PATH) < os.path.getmtime(_OMP_SRC)):
        compile_library(_OMP_SRC, _OMP_LIB_PATH, extra_flags=("-fopenmp",))
    return _OMP_LIB_PATH


def _get_omp_lib():
    global _omp_lib
    with _lock:
        if _omp_lib is None:
            lib = ctypes.CDLL(build_parallel())
            lib.oracle_ttv_omp.restype = ctypes.c_int
            lib.oracle_ttv_omp.argtypes = [
                ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                ctypes.POINTER(ctypes.POINTER(ctypes.c_double)), ctypes.c_int32, ctypes.c_int32,
                ctypes.POINTER(_Out)]
            lib.oracle_omp_free.restype = None
            lib.oracle_omp_free.argtypes = [ctypes.POINTER(_Out)]
            lib.oracle_omp_max_threads.restype = ctypes.c_int
            _omp_lib = lib
    return _omp_lib


def parallel_threads() -> int:
    """Threads the OpenMP statement uses by default (all allowed cores)."""
    return int(_get_omp_lib().oracle_omp_max_threads())


def ttv_parallel(subs, vals, shape, modes, vecs, dense: bool = False, threads: int = 0):
    """``ttv`` on ``threads`` host cores (0: all); same result, bit for bit."""
    lib = _get_omp_lib()
    if np.isscalar(modes):
        modes, vecs = [int(modes)], [vecs]
    shape = np.ascontiguousarray(np.asarray(shape, dtype=np.int64).reshape(-1))
    d = int(shape.size)
    subs = np.ascontiguousarray(np.asarray(subs, dtype=np.int64).reshape(-1, d))
    vals = _as_f64(vals).reshape(-1)
    if subs.shape[0] != vals.shape[0]:
        raise ValueError("subs and vals disagree on nnz")
    modes_a = np.ascontiguousarray(np.asarray(modes, dtype=np.int32).reshape(-1))
    vec_arrs = [_as_f64(v).reshape(-1) for v in vecs]
    if len(vec_arrs) != modes_a.size:
        raise ValueError("one vector per contracted mode")
    lens = np.ascontiguousarray(np.array([v.size for v in vec_arrs], dtype=np.int64))
    ptr_arr = (ctypes.POINTER(ctypes.c_double) * max(1, len(vec_arrs)))(
        *[v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for v in vec_arrs])
    out = _Out()
    rc = lib.oracle_ttv_omp(
        d, shape.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(vals.size),
        subs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), vals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        int(modes_a.size), modes_a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        lens.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ptr_arr, 1 if dense else 0, int(threads),
        ctypes.byref(out))
    if rc != 0:
        raise OracleError(rc)
    try:
        order = out.order
        newshape = tuple(int(out.shape[j]) for j in range(order))
        n = int(out.nnz)
        vals_out = np.ctypeslib.as_array(out.vals, shape=(max(n, 1),))[:n].copy()
        if dense:
            return None, vals_out.reshape(newshape), newshape
        if order > 0 and n > 0:
            subs_out = np.ctypeslib.as_array(out.subs, shape=(n * order,)).copy().reshape(n, order)
        else:
            subs_out = np.zeros((n, order), dtype=np.int64)
        return subs_out, vals_out, newshape
    finally:
        lib.oracle_omp_free(ctypes.byref(out))
