"""Sparse tensor-times-vector product (TTV) on GB300: Python binding.

Thin ctypes marshalling over the C ABI in ``include/ttv.h`` (library
``_lib/libttv_gb300.so``, built for sm_103a by ``_build.build()``).  Every
step of the computation runs in the library's CUDA kernels; PyTorch only
provides device memory and the stream.  There is no CPU fallback: without the
compiled library or a CUDA device every call raises.

The operation (paper Sec. 3.3, Eq. 3): for a sparse COO tensor with int64
``subs`` (nnz x d) and ``vals`` and dense vectors ``vecs[i]`` on modes
``modes[i]``,

    B(i_R) = sum_{k : subs[k, R] = i_R} vals[k] * prod_i vecs[i][subs[k, modes[i]]]

over the surviving modes R (increasing).  Sparse results are canonical COO
(ascending lexicographic rows, one per distinct surviving tuple present in the
input); dense results are row-major arrays of shape[R].
"""
from __future__ import annotations

import atexit
import ctypes
import os
import sys
import threading
import weakref

import numpy as np

import torch

from . import _build

TTV_MAX_D = 8
_LIB_PATH = _build.LIB
_lock = threading.Lock()
_lib = None

ERR = {
    0: "TTV_OK", -1: "TTV_ERR_ARG", -2: "TTV_ERR_MODE", -3: "TTV_ERR_VEC_LEN", -4: "TTV_ERR_SUBSCRIPT",
    -5: "TTV_ERR_KEY_OVERFLOW", -6: "TTV_ERR_BUDGET", -7: "TTV_ERR_TIMEOUT", -8: "TTV_ERR_CUDA",
    -9: "TTV_ERR_CAPACITY", -10: "TTV_ERR_NOMEM", -11: "TTV_ERR_UNSUPPORTED",
}
FMT = {"sparse": 0, "dense": 1, "auto": 2}
PATH = {"auto": 0, "dense": 1, "sort": 2, "hash": 3, "bucket": 4}
ACCUM = {"fp64": 0, "compensated": 1, "exact": 2}
DTYPE = {torch.float64: 0, torch.float32: 1}


class TTVError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR.get(code, code)}: {msg}")
        self.code = code
        self.name = ERR.get(code, str(code))


class Tensor(ctypes.Structure):
    _fields_ = [("subs", ctypes.c_void_p), ("stride_nz", ctypes.c_int64), ("stride_mode", ctypes.c_int64),
                ("vals", ctypes.c_void_p), ("val_dtype", ctypes.c_int), ("nnz", ctypes.c_int64),
                ("shape", ctypes.POINTER(ctypes.c_int64)), ("d", ctypes.c_int32)]


class Out(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("shape", ctypes.c_int64 * TTV_MAX_D), ("nnz", ctypes.c_int64),
                ("subs", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("subs_capacity", ctypes.c_int64),
                ("vals_capacity", ctypes.c_int64), ("dtype", ctypes.c_int), ("is_dense", ctypes.c_int32),
                ("internal", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("fmt", ctypes.c_int32), ("path", ctypes.c_int32), ("accum", ctypes.c_int32),
                ("deterministic", ctypes.c_int32), ("async_", ctypes.c_int32), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t)]


def _declare(lib):
    P = ctypes.POINTER
    lib.ttv_opts_init.argtypes = [P(Opts)]
    lib.ttv_opts_init.restype = None
    lib.ttv_last_error.restype = ctypes.c_char_p
    lib.ttv_last_error.argtypes = []
    lib.ttv_single.argtypes = [P(Tensor), ctypes.c_int32, ctypes.c_void_p, ctypes.c_int, P(Out), P(Opts), ctypes.c_void_p]
    lib.ttv_single.restype = ctypes.c_int
    lib.ttv_multi.argtypes = [P(Tensor), P(ctypes.c_int32), ctypes.c_int32, P(ctypes.c_void_p), ctypes.c_int,
                              P(Out), P(Opts), ctypes.c_void_p]
    lib.ttv_multi.restype = ctypes.c_int
    lib.ttv_multi_checked.argtypes = [P(Tensor), P(ctypes.c_int32), ctypes.c_int32, P(ctypes.c_void_p),
                                      P(ctypes.c_int64), ctypes.c_int, P(Out), P(Opts), ctypes.c_void_p]
    lib.ttv_multi_checked.restype = ctypes.c_int
    lib.ttv_out_capacity.argtypes = [P(Tensor), P(ctypes.c_int32), ctypes.c_int32, P(Opts), P(ctypes.c_int64),
                                     P(ctypes.c_int64)]
    lib.ttv_out_capacity.restype = ctypes.c_int
    lib.ttv_workspace_size.argtypes = [P(Tensor), P(ctypes.c_int32), ctypes.c_int32, ctypes.c_int, P(Opts),
                                       P(ctypes.c_size_t)]
    lib.ttv_workspace_size.restype = ctypes.c_int
    lib.ttv_out_sync.argtypes = [P(Out)]
    lib.ttv_out_sync.restype = ctypes.c_int
    lib.ttv_out_free.argtypes = [P(Out)]
    lib.ttv_out_free.restype = None
    return lib


def build(verbose: bool = False) -> str:
    """Compile the CUDA library for sm_103a (nvcc) and return its path."""
    return _build.build(verbose=verbose)


def load(path: str | None = None):
    """Load the compiled library (building it first if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or _LIB_PATH
            if not os.path.exists(p):
                p = build()
            _lib = _declare(ctypes.CDLL(p))
    return _lib


def _check(lib, rc: int):
    if rc != 0:
        raise TTVError(rc, lib.ttv_last_error().decode(errors="replace"))


def _stream_handle(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_tensor(subs: torch.Tensor, vals: torch.Tensor, shape):
    """C descriptor for a (nnz, d) subscript view of any strides (AoS when
    row-major, SoA when it is the transpose of a (d, nnz) contiguous array)."""
    if not subs.is_cuda or not vals.is_cuda:
        raise ValueError("subs and vals must be CUDA tensors")
    if subs.dtype != torch.int64:
        raise TypeError("subs must be int64")
    if vals.dtype not in DTYPE:
        raise TypeError("vals must be float64 or float32")
    d = len(shape)
    if subs.dim() != 2 or subs.shape[1] != d or subs.shape[0] != vals.shape[0]:
        raise ValueError("subs must be (nnz, d) and match vals")
    if vals.dim() != 1 or (vals.numel() > 1 and vals.stride(0) != 1):
        raise ValueError("vals must be a contiguous vector")
    shp = (ctypes.c_int64 * max(1, d))(*[int(s) for s in shape])
    t = Tensor(subs.data_ptr(), subs.stride(0), subs.stride(1), vals.data_ptr(), DTYPE[vals.dtype],
               vals.shape[0], ctypes.cast(shp, ctypes.POINTER(ctypes.c_int64)), d)
    t._keep = (shp, subs, vals)
    return t


def make_opts(fmt="sparse", path="auto", accum="fp64", deterministic=False, async_=False,
              workspace: torch.Tensor | None = None):
    o = Opts()
    load().ttv_opts_init(ctypes.byref(o))
    o.fmt = FMT[fmt]
    o.path = PATH[path]
    o.accum = ACCUM[accum]
    o.deterministic = int(bool(deterministic))
    o.async_ = int(bool(async_))
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o


def workspace_size(subs, vals, shape, modes, vec_dtype=torch.float64, **opt) -> int:
    lib = load()
    t = make_tensor(subs, vals, shape)
    m = (ctypes.c_int32 * len(modes))(*modes)
    o = make_opts(**opt)
    n = ctypes.c_size_t()
    _check(lib, lib.ttv_workspace_size(ctypes.byref(t), m, len(modes), DTYPE[vec_dtype], ctypes.byref(o), ctypes.byref(n)))
    return int(n.value)


def out_capacity(subs, vals, shape, modes, **opt):
    lib = load()
    t = make_tensor(subs, vals, shape)
    m = (ctypes.c_int32 * len(modes))(*modes)
    o = make_opts(**opt)
    r, v = ctypes.c_int64(), ctypes.c_int64()
    _check(lib, lib.ttv_out_capacity(ctypes.byref(t), m, len(modes), ctypes.byref(o), ctypes.byref(r), ctypes.byref(v)))
    return int(r.value), int(v.value)


class Result:
    """Result of a TTV call: ``subs`` (nnz, order) int64 (None when dense),
    ``vals`` (nnz,) or a dense array of ``shape``, all on the device."""

    def __init__(self, subs, vals, shape, is_dense):
        self.subs, self.vals, self.shape, self.is_dense = subs, vals, tuple(shape), is_dense

    def __iter__(self):
        return iter((self.subs, self.vals, self.shape))

    def to_sptensor_arrays(self):
        """Host arrays in pyttb's sptensor layout: ``subs`` (nnz, order) int64,
        ``vals`` (nnz, 1) float64 and the shape.  A dense result is returned
        as its nonzero cells in the same row-major order."""
        if self.is_dense:
            flat = self.vals.reshape(-1)
            idx = torch.nonzero(flat, as_tuple=False).reshape(-1)
            subs = torch.stack(torch.unravel_index(idx, self.shape), dim=1) if self.shape else \
                torch.zeros((idx.numel(), 0), dtype=torch.int64, device=flat.device)
            return subs.cpu().numpy(), flat[idx].reshape(-1, 1).cpu().numpy(), self.shape
        return self.subs.cpu().numpy(), self.vals.reshape(-1, 1).cpu().numpy(), self.shape


def ttv_multi(subs: torch.Tensor, vals: torch.Tensor, shape, modes, vecs, *, fmt="sparse", path="auto",
              accum="fp64", deterministic=False, out_subs: torch.Tensor | None = None,
              out_vals: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None) -> Result:
    """TTV of a COO tensor with one vector per mode in ``modes`` (any order).

    ``out_subs`` / ``out_vals`` / ``workspace`` may be preallocated (see
    ``out_capacity`` and ``workspace_size``); otherwise they are allocated here
    with torch.  Synchronises the stream once to learn the result size."""
    lib = load()
    modes = [int(m) for m in modes]
    if len(vecs) != len(modes):
        raise ValueError("one vector per mode")
    vdt = vecs[0].dtype if vecs else torch.float64
    for v in vecs:
        if not v.is_cuda or v.dtype != vdt or v.dim() != 1 or (v.numel() > 1 and v.stride(0) != 1):
            raise ValueError("vectors must be contiguous CUDA vectors of one dtype")
    if vdt not in DTYPE:
        raise TypeError("vectors must be float64 or float32")
    t = make_tensor(subs, vals, shape)
    m = (ctypes.c_int32 * len(modes))(*modes)
    vp = (ctypes.c_void_p * len(vecs))(*[v.data_ptr() for v in vecs])
    lens = (ctypes.c_int64 * len(vecs))(*[v.numel() for v in vecs])
    d = len(shape)
    if fmt == "auto" and out_subs is None and out_vals is None:
        # the library allocates the result, so that it can turn it dense
        o = make_opts(fmt=fmt, path=path, accum=accum, deterministic=deterministic,
                      workspace=workspace if workspace is not None else None)
        res = Out()
        rc = lib.ttv_multi_checked(ctypes.byref(t), m, len(modes), vp, lens, DTYPE[vdt], ctypes.byref(res),
                                   ctypes.byref(o), _stream_handle(stream))
        if rc != 0:
            msg = lib.ttv_last_error().decode(errors="replace")
            lib.ttv_out_free(ctypes.byref(res))
            raise TTVError(rc, msg)
        return _take_result(lib, res)
    rows, nvals = ctypes.c_int64(), ctypes.c_int64()
    if workspace is None:
        o0 = make_opts(fmt=fmt, path=path, accum=accum, deterministic=deterministic)
        _check(lib, lib.ttv_out_capacity(ctypes.byref(t), m, len(modes), ctypes.byref(o0), ctypes.byref(rows), ctypes.byref(nvals)))
        nbytes = ctypes.c_size_t()
        _check(lib, lib.ttv_workspace_size(ctypes.byref(t), m, len(modes), DTYPE[vdt], ctypes.byref(o0), ctypes.byref(nbytes)))
        workspace = torch.empty(max(1, nbytes.value), dtype=torch.uint8, device=subs.device)
    else:
        o0 = make_opts(fmt=fmt, path=path, accum=accum, deterministic=deterministic)
        _check(lib, lib.ttv_out_capacity(ctypes.byref(t), m, len(modes), ctypes.byref(o0), ctypes.byref(rows), ctypes.byref(nvals)))
    order = d - len(modes)
    if out_vals is None:
        out_vals = torch.empty(max(1, nvals.value), dtype=torch.float64, device=subs.device)
    if out_subs is None and fmt != "dense" and order > 0:
        out_subs = torch.empty((max(1, rows.value), order), dtype=torch.int64, device=subs.device)
    o = make_opts(fmt=fmt, path=path, accum=accum, deterministic=deterministic, workspace=workspace)
    res = Out()
    res.vals = out_vals.data_ptr()
    res.vals_capacity = out_vals.numel()
    if out_subs is not None:
        res.subs = out_subs.data_ptr()
        res.subs_capacity = out_subs.shape[0]
    else:
        res.subs = None
        res.subs_capacity = 0
    try:
        rc = lib.ttv_multi_checked(ctypes.byref(t), m, len(modes), vp, lens, DTYPE[vdt], ctypes.byref(res),
                                   ctypes.byref(o), _stream_handle(stream))
        _check(lib, rc)
        newshape = tuple(int(res.shape[j]) for j in range(res.order))
        n = int(res.nnz)
        if res.is_dense:
            return Result(None, out_vals[:n].view(newshape), newshape, True)
        vals_out = out_vals[:n]
        subs_out = out_subs[:n] if out_subs is not None else torch.zeros((n, 0), dtype=torch.int64, device=subs.device)
        return Result(subs_out, vals_out, newshape, False)
    finally:
        lib.ttv_out_free(ctypes.byref(res))


def ttv_single(subs, vals, shape, mode: int, v: torch.Tensor, **kw) -> Result:
    """TTV with one vector along ``mode`` (paper Eq. 3)."""
    return ttv_multi(subs, vals, shape, [mode], [v], **kw)


def resolve_dims(d: int, nvec: int, dims=None, exclude_dims=None):
    """pyttb's mode specification for ttv: ``dims`` lists the modes to
    contract, ``exclude_dims`` the modes to keep (never both); neither means
    every mode.  Returns the modes in increasing order and, for each, the
    index of its vector: with one vector per tensor mode (nvec == d) mode m
    takes vectors[m]; otherwise there is one vector per listed mode, paired
    with the modes in the order they were listed."""
    if dims is not None and exclude_dims is not None:
        raise ValueError("give dims or exclude_dims, not both")
    if dims is None and exclude_dims is None:
        listed = list(range(d))
    elif exclude_dims is not None:
        ex = [exclude_dims] if isinstance(exclude_dims, int) else [int(m) for m in exclude_dims]
        if any(m < 0 or m >= d for m in ex) or len(set(ex)) != len(ex):
            raise ValueError(f"exclude_dims {ex} invalid for a {d}-way tensor")
        listed = [m for m in range(d) if m not in ex]
    else:
        listed = [dims] if isinstance(dims, int) else [int(m) for m in dims]
    if any(m < 0 or m >= d for m in listed) or len(set(listed)) != len(listed):
        raise ValueError(f"modes {listed} invalid for a {d}-way tensor")
    order = sorted(range(len(listed)), key=lambda j: listed[j])
    modes = [listed[j] for j in order]
    if nvec > d:
        raise ValueError(f"{nvec} vectors for a {d}-way tensor")
    if nvec == d:
        return modes, list(modes)
    if nvec != len(listed):
        raise ValueError(f"{nvec} vectors for {len(listed)} modes")
    return modes, order


def ttv(subs, vals, shape, vectors, dims=None, exclude_dims=None, *, fmt="auto", **kw):
    """TTV with pyttb's calling convention (sptensor.ttv): ``vectors`` is one
    vector or a list, the modes come from ``dims`` / ``exclude_dims`` (see
    ``resolve_dims``), the result is dense when more than half its cells are
    nonzero (``fmt="auto"``), and an order-0 result is returned as a float."""
    vecs = [vectors] if isinstance(vectors, torch.Tensor) else list(vectors)
    modes, vidx = resolve_dims(len(shape), len(vecs), dims, exclude_dims)
    r = ttv_multi(subs, vals, shape, modes, [vecs[i] for i in vidx], fmt=fmt, **kw)
    if r.shape == ():
        return float(r.vals.reshape(-1)[0])
    return r


# ---- measurement hooks (per-kernel CUDA-event timing, launch counts) --------

def _declare_prof(lib):
    if getattr(lib, "_prof_declared", False):
        return lib
    lib.ttv_launch_count.restype = ctypes.c_longlong
    lib.ttv_launch_count.argtypes = []
    lib.ttv_profile_enable.argtypes = [ctypes.c_int]
    lib.ttv_profile_enable.restype = None
    lib.ttv_profile_collect.restype = ctypes.c_int
    lib.ttv_profile_collect.argtypes = []
    lib.ttv_profile_get.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    lib.ttv_profile_get.restype = ctypes.c_int
    lib.ttv_profile_names.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    lib.ttv_profile_names.restype = ctypes.c_int
    lib.ttv_profile_reset.argtypes = []
    lib.ttv_profile_reset.restype = None
    lib._prof_declared = True
    return lib


def launch_count() -> int:
    """Kernel launches the library has issued since it was loaded."""
    return int(_declare_prof(load()).ttv_launch_count())


def test_set_wait_polls(polls: int):
    """Test hook (ttv_test_set_wait_polls): the sort's look-back waits and the
    staged dense kernel's pipeline waits give up after ``polls`` polls;
    ``polls < 0`` restores their own limits."""
    lib = load()
    lib.ttv_test_set_wait_polls.argtypes = [ctypes.c_longlong]
    lib.ttv_test_set_wait_polls.restype = ctypes.c_int
    _check(lib, lib.ttv_test_set_wait_polls(int(polls)))


def test_wait_probe(kind: int, polls: int) -> str:
    """Test hook (ttv_test_wait_probe): one wait that nothing satisfies, on an
    mbarrier (kind 0) or a device word (kind 1); returns the status name
    ("TTV_ERR_TIMEOUT" when the wait ran out)."""
    lib = load()
    lib.ttv_test_wait_probe.argtypes = [ctypes.c_int, ctypes.c_uint]
    lib.ttv_test_wait_probe.restype = ctypes.c_int
    rc = lib.ttv_test_wait_probe(int(kind), int(polls))
    return "TTV_OK" if rc == 0 else ERR.get(rc, str(rc))


def profile_enable(on: bool = True):
    _declare_prof(load()).ttv_profile_enable(1 if on else 0)


def profile_collect():
    lib = _declare_prof(load())
    _check(lib, lib.ttv_profile_collect())


def profile_reset():
    _declare_prof(load()).ttv_profile_reset()


def profile_get(kernel: str):
    """(total milliseconds, launches) of one kernel since the last reset."""
    lib = _declare_prof(load())
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    lib.ttv_profile_get(kernel.encode(), ctypes.byref(ms), ctypes.byref(n))
    return float(ms.value), int(n.value)


def profile_names():
    lib = _declare_prof(load())
    need = lib.ttv_profile_names(None, 0)
    buf = ctypes.create_string_buffer(max(1, need))
    lib.ttv_profile_names(buf, len(buf))
    return [x for x in buf.value.decode().split("\n") if x]


# ---- prepared tensors -------------------------------------------------------------

def _declare_prep(lib):
    if getattr(lib, "_prep_declared", False):
        return lib
    P = ctypes.POINTER
    lib.ttv_prepare.argtypes = [P(Tensor), P(ctypes.c_int32), ctypes.c_int32, P(ctypes.c_void_p), ctypes.c_void_p]
    lib.ttv_prepare.restype = ctypes.c_int
    lib.ttv_prepared_run.argtypes = [ctypes.c_void_p, P(ctypes.c_void_p), P(ctypes.c_int64), ctypes.c_int, P(Out),
                                     P(Opts), ctypes.c_void_p]
    lib.ttv_prepared_run.restype = ctypes.c_int
    lib.ttv_prepared_info.argtypes = [ctypes.c_void_p, P(ctypes.c_int64), P(ctypes.c_int32), P(ctypes.c_size_t)]
    lib.ttv_prepared_info.restype = ctypes.c_int
    lib.ttv_prepared_workspace_size.argtypes = [ctypes.c_void_p, P(ctypes.c_size_t)]
    lib.ttv_prepared_workspace_size.restype = ctypes.c_int
    lib.ttv_prepared_free.argtypes = [ctypes.c_void_p]
    lib.ttv_prepared_free.restype = None
    lib.ttv_mttkrp_prepared.argtypes = [ctypes.c_void_p, P(ctypes.c_void_p), ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    lib.ttv_mttkrp_prepared.restype = ctypes.c_int
    lib.ttv_mttkrp_workspace_size.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_size_t)]
    lib.ttv_mttkrp_workspace_size.restype = ctypes.c_int
    lib.ttv_mttkrp.argtypes = [P(Tensor), ctypes.c_int32, P(ctypes.c_void_p), ctypes.c_int32, ctypes.c_void_p,
                               ctypes.c_void_p]
    lib.ttv_mttkrp.restype = ctypes.c_int
    lib._prep_declared = True
    return lib


class Prepared:
    """A tensor prepared for repeated TTVs along ``modes`` (see ttv_prepare):
    ``run(vecs)`` takes one vector per mode, in the order of ``modes``."""

    def __init__(self, subs: torch.Tensor, vals: torch.Tensor, shape, modes, stream=None):
        self._lib = _declare_prep(load())
        self.modes = [int(m) for m in modes]
        self.shape = tuple(int(x) for x in shape)
        self.device = subs.device
        t = make_tensor(subs, vals, shape)
        m = (ctypes.c_int32 * len(self.modes))(*self.modes)
        h = ctypes.c_void_p()
        _check(self._lib, self._lib.ttv_prepare(ctypes.byref(t), m, len(self.modes), ctypes.byref(h),
                                                _stream_handle(stream)))
        self._h = h
        nnz_out, order, nbytes = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_size_t()
        _check(self._lib, self._lib.ttv_prepared_info(h, ctypes.byref(nnz_out), ctypes.byref(order),
                                                      ctypes.byref(nbytes)))
        self.nnz_out, self.order, self.device_bytes = int(nnz_out.value), int(order.value), int(nbytes.value)
        ws = ctypes.c_size_t()
        _check(self._lib, self._lib.ttv_prepared_workspace_size(h, ctypes.byref(ws)))
        self.workspace_bytes = int(ws.value)

    def run(self, vecs, *, fmt="sparse", accum="fp64", out_subs=None, out_vals=None, workspace=None,
            stream=None) -> Result:
        if self._h is None:
            raise RuntimeError("prepared tensor released")
        if len(vecs) != len(self.modes):
            raise ValueError("one vector per prepared mode")
        vdt = vecs[0].dtype
        for v in vecs:
            if not v.is_cuda or v.dtype != vdt or v.dim() != 1 or (v.numel() > 1 and v.stride(0) != 1):
                raise ValueError("vectors must be contiguous CUDA vectors of one dtype")
        if vdt not in DTYPE:
            raise TypeError("vectors must be float64 or float32")
        vp = (ctypes.c_void_p * len(vecs))(*[v.data_ptr() for v in vecs])
        lens = (ctypes.c_int64 * len(vecs))(*[v.numel() for v in vecs])
        surv = [self.shape[m] for m in range(len(self.shape)) if m not in self.modes]
        dense = fmt == "dense" or not surv
        ncells = 1
        for x in surv:
            ncells *= x
        if workspace is None:
            workspace = torch.empty(max(1, self.workspace_bytes), dtype=torch.uint8, device=self.device)
        if out_vals is None:
            out_vals = torch.empty(max(1, ncells if dense else self.nnz_out), dtype=torch.float64, device=self.device)
        if out_subs is None and not dense:
            out_subs = torch.empty((max(1, self.nnz_out), self.order), dtype=torch.int64, device=self.device)
        o = make_opts(fmt=fmt, accum=accum, workspace=workspace)
        res = Out()
        res.vals = out_vals.data_ptr()
        res.vals_capacity = out_vals.numel()
        if out_subs is not None:
            res.subs = out_subs.data_ptr()
            res.subs_capacity = out_subs.shape[0]
        try:
            _check(self._lib, self._lib.ttv_prepared_run(self._h, vp, lens, DTYPE[vdt], ctypes.byref(res),
                                                         ctypes.byref(o), _stream_handle(stream)))
            newshape = tuple(int(res.shape[j]) for j in range(res.order))
            n = int(res.nnz)
            if res.is_dense:
                return Result(None, out_vals[:n].view(newshape), newshape, True)
            subs_out = out_subs[:n] if out_subs is not None else torch.zeros((n, 0), dtype=torch.int64,
                                                                               device=self.device)
            return Result(subs_out, out_vals[:n], newshape, False)
        finally:
            self._lib.ttv_out_free(ctypes.byref(res))

    def mttkrp(self, factors, *, out=None, workspace=None, stream=None) -> torch.Tensor:
        """MTTKRP along the one mode not prepared: ``factors`` are (shape[m],
        rank) float64 CUDA matrices, one per prepared mode in their order."""
        if self._h is None:
            raise RuntimeError("prepared tensor released")
        if len(factors) != len(self.modes):
            raise ValueError("one factor per prepared mode")
        rank = int(factors[0].shape[1])
        for f, m in zip(factors, self.modes):
            if (not f.is_cuda or f.dtype != torch.float64 or f.dim() != 2 or not f.is_contiguous()
                    or f.shape != (self.shape[m], rank)):
                raise ValueError("factors must be contiguous (shape[m], rank) float64 CUDA matrices")
        n = [m for m in range(len(self.shape)) if m not in self.modes]
        if len(n) != 1:
            raise ValueError("MTTKRP needs a tensor prepared for every mode but one")
        rows = self.shape[n[0]]
        if out is None:
            out = torch.empty((rows, rank), dtype=torch.float64, device=self.device)
        if workspace is None:
            nb = ctypes.c_size_t()
            _check(self._lib, self._lib.ttv_mttkrp_workspace_size(self._h, rank, ctypes.byref(nb)))
            workspace = torch.empty(max(1, nb.value), dtype=torch.uint8, device=self.device)
        fp = (ctypes.c_void_p * len(factors))(*[f.data_ptr() for f in factors])
        _check(self._lib, self._lib.ttv_mttkrp_prepared(self._h, fp, rank, out.data_ptr(), workspace.data_ptr(),
                                                        workspace.numel(), _stream_handle(stream)))
        return out

    def close(self):
        if self._h is not None:
            self._lib.ttv_prepared_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mttkrp(subs, vals, shape, mode: int, factors, stream=None) -> torch.Tensor:
    """MTTKRP along ``mode`` (ttv_mttkrp): ``factors`` holds one (shape[m],
    rank) float64 CUDA matrix per mode (the entry for ``mode`` is ignored)."""
    lib = _declare_prep(load())
    d = len(shape)
    rank = int(next(f for m, f in enumerate(factors) if m != mode).shape[1])
    fp = (ctypes.c_void_p * d)(*[0 if (m == mode or factors[m] is None) else factors[m].data_ptr()
                                  for m in range(d)])
    out = torch.empty((int(shape[mode]), rank), dtype=torch.float64, device=subs.device)
    t = make_tensor(subs, vals, shape)
    _check(lib, lib.ttv_mttkrp(ctypes.byref(t), int(mode), fp, rank, out.data_ptr(), _stream_handle(stream)))
    return out


# ---- dense dot product (Eq. 1) and matrix-vector product (Eq. 2) -----------------

def _declare_dense(lib):
    if getattr(lib, "_dense_declared", False):
        return lib
    P = ctypes.POINTER
    lib.ttv_dot.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    lib.ttv_dot.restype = ctypes.c_int
    lib.ttv_dot_workspace_size.argtypes = [ctypes.c_int64, P(ctypes.c_size_t)]
    lib.ttv_dot_workspace_size.restype = ctypes.c_int
    lib.ttv_matvec.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                               ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                               ctypes.c_void_p]
    lib.ttv_matvec.restype = ctypes.c_int
    lib.ttv_matvec_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                              P(ctypes.c_size_t)]
    lib.ttv_matvec_workspace_size.restype = ctypes.c_int
    lib._dense_declared = True
    return lib


def _dense_operand(t: torch.Tensor, what: str):
    if not t.is_cuda or t.dtype not in DTYPE:
        raise ValueError(f"{what} must be a float64 or float32 CUDA tensor")


def dot(x: torch.Tensor, y: torch.Tensor, *, out: torch.Tensor | None = None, workspace=None,
        stream=None) -> torch.Tensor:
    """x . y (ttv_dot, paper Eq. 1) of two contiguous CUDA vectors of one
    dtype; returns a one-element float64 CUDA tensor (asynchronous)."""
    lib = _declare_dense(load())
    _dense_operand(x, "x")
    _dense_operand(y, "y")
    if x.dtype != y.dtype or x.numel() != y.numel() or not x.is_contiguous() or not y.is_contiguous():
        raise ValueError("x and y must be contiguous, of one dtype and length")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=x.device)
    nb = workspace.numel() if workspace is not None else 0
    _check(lib, lib.ttv_dot(x.data_ptr(), y.data_ptr(), x.numel(), DTYPE[x.dtype], out.data_ptr(),
                            workspace.data_ptr() if workspace is not None else None, nb, _stream_handle(stream)))
    return out


def matvec(A: torch.Tensor, x: torch.Tensor, *, out: torch.Tensor | None = None, workspace=None,
           stream=None) -> torch.Tensor:
    """A x (ttv_matvec, paper Eq. 2) for a CUDA matrix in row-major or
    column-major storage (any strides with one of them 1) and a contiguous
    vector of the same dtype; returns float64 (asynchronous)."""
    lib = _declare_dense(load())
    _dense_operand(A, "A")
    _dense_operand(x, "x")
    if A.dim() != 2 or x.dim() != 1 or x.numel() != A.shape[1] or A.dtype != x.dtype or not x.is_contiguous():
        raise ValueError("A must be (n1, n2) and x a contiguous (n2,) vector of the same dtype")
    n1, n2 = A.shape
    if out is None:
        out = torch.empty(n1, dtype=torch.float64, device=A.device)
    nb = workspace.numel() if workspace is not None else 0
    _check(lib, lib.ttv_matvec(A.data_ptr(), n1, n2, A.stride(0), A.stride(1), DTYPE[A.dtype], x.data_ptr(),
                               out.data_ptr(), workspace.data_ptr() if workspace is not None else None, nb,
                               _stream_handle(stream)))
    return out


def matvec_workspace_size(A: torch.Tensor) -> int:
    lib = _declare_dense(load())
    nb = ctypes.c_size_t()
    _check(lib, lib.ttv_matvec_workspace_size(A.shape[0], A.shape[1], A.stride(0), A.stride(1), ctypes.byref(nb)))
    return nb.value


def dot_workspace_size(n: int) -> int:
    lib = _declare_dense(load())
    nb = ctypes.c_size_t()
    _check(lib, lib.ttv_dot_workspace_size(int(n), ctypes.byref(nb)))
    return nb.value


# ---- autotuner ------------------------------------------------------------------

TUNE_MAX = 16
PATH_NAME = {v: k for k, v in PATH.items()}


class TuneResult(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("items_per_thread", ctypes.c_int32),
                ("ms", ctypes.c_double), ("n_candidates", ctypes.c_int32), ("cand_path", ctypes.c_int32 * TUNE_MAX),
                ("cand_ctas", ctypes.c_int32 * TUNE_MAX), ("cand_items", ctypes.c_int32 * TUNE_MAX),
                ("cand_ms", ctypes.c_double * TUNE_MAX)]


def _declare_tune(lib):
    if getattr(lib, "_tune_declared", False):
        return lib
    P = ctypes.POINTER
    lib.ttv_autotune.argtypes = [P(Tensor), P(ctypes.c_int32), ctypes.c_int32, P(ctypes.c_void_p), ctypes.c_int,
                                 P(Opts), ctypes.c_int32, P(TuneResult), ctypes.c_void_p]
    lib.ttv_autotune.restype = ctypes.c_int
    lib.ttv_tune_save.argtypes = [ctypes.c_char_p]
    lib.ttv_tune_save.restype = ctypes.c_int
    lib.ttv_tune_load.argtypes = [ctypes.c_char_p]
    lib.ttv_tune_load.restype = ctypes.c_int
    lib.ttv_tune_clear.argtypes = []
    lib.ttv_tune_clear.restype = None
    lib.ttv_tune_count.argtypes = []
    lib.ttv_tune_count.restype = ctypes.c_int
    lib.ttv_tune_lookup.argtypes = [P(Tensor), P(ctypes.c_int32), ctypes.c_int32, P(Opts), P(ctypes.c_int32),
                                    P(ctypes.c_int32), P(ctypes.c_int32)]
    lib.ttv_tune_lookup.restype = ctypes.c_int
    lib.ttv_tune_set.argtypes = [P(Tensor), P(ctypes.c_int32), ctypes.c_int32, P(Opts), ctypes.c_int32,
                                 ctypes.c_int32, ctypes.c_int32]
    lib.ttv_tune_set.restype = ctypes.c_int
    lib._tune_declared = True
    return lib


def autotune(subs, vals, shape, modes, vecs, *, fmt="sparse", trials=5, deterministic=False, stream=None) -> dict:
    """Times every applicable (path, CTAs per SM) plan on this problem and
    records the fastest for its problem class (see ttv_autotune)."""
    lib = _declare_tune(load())
    vdt = vecs[0].dtype
    t = make_tensor(subs, vals, shape)
    m = (ctypes.c_int32 * len(modes))(*[int(x) for x in modes])
    vp = (ctypes.c_void_p * len(vecs))(*[v.data_ptr() for v in vecs])
    o = make_opts(fmt=fmt, deterministic=deterministic)
    r = TuneResult()
    _check(lib, lib.ttv_autotune(ctypes.byref(t), m, len(modes), vp, DTYPE[vdt], ctypes.byref(o), int(trials),
                                 ctypes.byref(r), _stream_handle(stream)))
    cands = [{"path": PATH_NAME[r.cand_path[i]], "ctas_per_sm": r.cand_ctas[i], "items_per_thread": r.cand_items[i],
              "ms": r.cand_ms[i]} for i in range(r.n_candidates)]
    return {"path": PATH_NAME[r.path], "ctas_per_sm": r.ctas_per_sm, "items_per_thread": r.items_per_thread,
            "ms": r.ms, "candidates": cands}


def tune_lookup(subs, vals, shape, modes, *, fmt="sparse"):
    """(path name, CTAs per SM, items per thread) recorded for this problem's
    class, or None."""
    lib = _declare_tune(load())
    t = make_tensor(subs, vals, shape)
    m = (ctypes.c_int32 * len(modes))(*[int(x) for x in modes])
    o = make_opts(fmt=fmt)
    pth, ctas, items = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    rc = lib.ttv_tune_lookup(ctypes.byref(t), m, len(modes), ctypes.byref(o), ctypes.byref(pth), ctypes.byref(ctas),
                             ctypes.byref(items))
    if rc < 0:
        _check(lib, rc)
    return (PATH_NAME[pth.value], ctas.value, items.value) if rc == 1 else None


def tune_set(subs, vals, shape, modes, path: str, ctas_per_sm: int = 0, items_per_thread: int = 0, *,
             fmt="sparse"):
    """Records a plan for this problem's class by hand (ttv_tune_set)."""
    lib = _declare_tune(load())
    t = make_tensor(subs, vals, shape)
    m = (ctypes.c_int32 * len(modes))(*[int(x) for x in modes])
    o = make_opts(fmt=fmt)
    _check(lib, lib.ttv_tune_set(ctypes.byref(t), m, len(modes), ctypes.byref(o), PATH[path], int(ctas_per_sm),
                                 int(items_per_thread)))


def tune_save(path: str):
    lib = _declare_tune(load())
    _check(lib, lib.ttv_tune_save(os.fsencode(path)))


def tune_load(path: str):
    lib = _declare_tune(load())
    _check(lib, lib.ttv_tune_load(os.fsencode(path)))


def tune_clear():
    _declare_tune(load()).ttv_tune_clear()


def tune_count() -> int:
    return int(_declare_tune(load()).ttv_tune_count())


# ---- allocation-free dense TTV -----------------------------------------------

def ttv_dense_noalloc(subs: torch.Tensor, vals: torch.Tensor, shape, modes, vecs, out: torch.Tensor,
                      stream=None) -> torch.Tensor:
    """Dense-result TTV into ``out`` (a float64 CUDA buffer of at least
    prod(shape[R]) values) without any device allocation by the library.

    For callers that must not allocate (their host application owns all
    device memory, or they run where the allocator's locks and
    synchronisation are not allowed): the scratch is a fixed array inside the
    library.  Synchronous; calls that overlap on the GPU race on that array,
    so serialise them.  The first call on a device must precede any stream
    capture.  Returns ``out[:prod].view(shape[R])``."""
    lib = load()
    if not getattr(lib, "_noalloc_declared", False):
        P = ctypes.POINTER
        lib.ttv_dense_noalloc.argtypes = [P(Tensor), P(ctypes.c_int32), ctypes.c_int32, P(ctypes.c_void_p),
                                          P(ctypes.c_int64), ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p]
        lib.ttv_dense_noalloc.restype = ctypes.c_int
        lib._noalloc_declared = True
    modes = [int(m) for m in modes]
    if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 CUDA buffer")
    vdt = vecs[0].dtype
    t = make_tensor(subs, vals, shape)
    m = (ctypes.c_int32 * len(modes))(*modes)
    vp = (ctypes.c_void_p * len(vecs))(*[v.data_ptr() for v in vecs])
    lens = (ctypes.c_int64 * len(vecs))(*[v.numel() for v in vecs])
    rc = lib.ttv_dense_noalloc(ctypes.byref(t), m, len(modes), vp, lens, DTYPE[vdt], out.data_ptr(), out.numel(),
                               _stream_handle(stream))
    _check(lib, rc)
    rshape = tuple(int(shape[i]) for i in range(len(shape)) if i not in modes)
    n = 1
    for x in rshape:
        n *= x
    return out.view(-1)[:n].view(rshape)


# ---- batched TTV (one CUDA graph per set of problems) ------------------------

class Problem(ctypes.Structure):
    _fields_ = [("tensor", Tensor), ("modes", ctypes.POINTER(ctypes.c_int32)), ("n_v", ctypes.c_int32),
                ("vecs", ctypes.POINTER(ctypes.c_void_p)), ("v_dtype", ctypes.c_int)]


def _declare_batch(lib):
    if getattr(lib, "_batch_declared", False):
        return lib
    P = ctypes.POINTER
    lib.ttv_batch.argtypes = [P(Problem), ctypes.c_int32, P(Out), P(Opts), ctypes.c_void_p]
    lib.ttv_batch.restype = ctypes.c_int
    lib.ttv_batch_workspace_size.argtypes = [P(Problem), ctypes.c_int32, P(Opts), P(ctypes.c_size_t)]
    lib.ttv_batch_workspace_size.restype = ctypes.c_int
    lib.ttv_batch_graph_launches.argtypes = [P(Problem), ctypes.c_int32, P(Out), P(Opts)]
    lib.ttv_batch_graph_launches.restype = ctypes.c_longlong
    lib.ttv_batch_release.argtypes = []
    lib.ttv_batch_release.restype = None
    lib.ttv_outs_free.argtypes = [P(Out), ctypes.c_int32]
    lib.ttv_outs_free.restype = None
    lib._batch_declared = True
    return lib


# The ttv_out fields BatchResults needs, at their ctypes offsets.
_OUT_DTYPE = np.dtype({"names": ["order", "shape", "nnz", "is_dense"],
                       "formats": [np.int32, (np.int64, TTV_MAX_D), np.int64, np.int32],
                       "offsets": [Out.order.offset, Out.shape.offset, Out.nnz.offset, Out.is_dense.offset],
                       "itemsize": ctypes.sizeof(Out)})


class BatchResults:
    """The results of one batch run: ``Result`` views made on access."""

    def __init__(self, meta, info):
        self._meta, self._info = meta, info

    def __len__(self):
        return len(self._info)

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self[j] for j in range(*i.indices(len(self)))]
        ov, os_, _, _ = self._meta[i]
        nn, dense, order, shp = self._info[i]
        newshape = tuple(int(x) for x in shp[:order])
        if dense:
            return Result(None, ov[:nn].view(newshape), newshape, True)
        subs_out = os_[:nn] if os_ is not None else torch.zeros((nn, 0), dtype=torch.int64, device=ov.device)
        return Result(subs_out, ov[:nn], newshape, False)

    def __iter__(self):
        return (self[i] for i in range(len(self)))


class Batch:
    """Many TTVs run as one CUDA-graph launch (``ttv_batch``).

    ``problems`` is a list of ``(subs, vals, shape, modes, vecs)`` on the
    device.  Result and workspace buffers are allocated once here, so every
    ``run()`` after the first replays the cached graph."""

    def __init__(self, problems, fmt="sparse", path="auto", accum="fp64"):
        self.lib = _declare_batch(load())
        self.n = len(problems)
        self._keep = []
        self.probs = (Problem * max(1, self.n))()
        self.fmt = fmt
        self.meta = []
        for i, (subs, vals, shape, modes, vecs) in enumerate(problems):
            t = make_tensor(subs, vals, shape)
            m = (ctypes.c_int32 * len(modes))(*[int(x) for x in modes])
            vp = (ctypes.c_void_p * len(vecs))(*[v.data_ptr() for v in vecs])
            self.probs[i] = Problem(t, ctypes.cast(m, ctypes.POINTER(ctypes.c_int32)), len(modes),
                                    ctypes.cast(vp, ctypes.POINTER(ctypes.c_void_p)), DTYPE[vecs[0].dtype])
            self._keep.append((t, m, vp, subs, vals, vecs))
            rows, nvals = out_capacity(subs, vals, shape, list(modes), fmt=fmt, path=path, accum=accum)
            order = len(shape) - len(modes)
            ov = torch.empty(max(1, nvals), dtype=torch.float64, device=subs.device)
            os_ = (torch.empty((max(1, rows), order), dtype=torch.int64, device=subs.device)
                   if fmt != "dense" and order > 0 else None)
            self.meta.append((ov, os_, tuple(shape), list(modes)))
        self.opts0 = make_opts(fmt=fmt, path=path, accum=accum)
        nbytes = ctypes.c_size_t()
        _check(self.lib, self.lib.ttv_batch_workspace_size(self.probs, self.n, ctypes.byref(self.opts0),
                                                           ctypes.byref(nbytes)))
        dev = problems[0][0].device if problems else torch.device("cuda")
        self.workspace = torch.empty(max(1, nbytes.value), dtype=torch.uint8, device=dev)
        self.opts = make_opts(fmt=fmt, path=path, accum=accum, workspace=self.workspace)

    def _outs(self):
        outs = (Out * max(1, self.n))()
        for i, (ov, os_, _, _) in enumerate(self.meta):
            outs[i].vals = ov.data_ptr()
            outs[i].vals_capacity = ov.numel()
            if os_ is not None:
                outs[i].subs = os_.data_ptr()
                outs[i].subs_capacity = os_.shape[0]
        return outs

    def run(self, stream=None):
        """Launch the batch; returns one Result per problem (views of the
        batch's buffers, rewritten by the next run), formed when indexed."""
        if getattr(self, "_outs_arr", None) is None:
            self._outs_arr = self._outs()      # the same caller buffers every run
        outs = self._outs_arr
        rc = self.lib.ttv_batch(self.probs, self.n, outs, ctypes.byref(self.opts), _stream_handle(stream))
        try:
            _check(self.lib, rc)
            # nnz, is_dense, order and shape of every result in one read of the array
            a = np.frombuffer(outs, dtype=_OUT_DTYPE, count=self.n)
            return BatchResults(self.meta, list(zip(a["nnz"].tolist(), a["is_dense"].astype(bool).tolist(),
                                                    a["order"].tolist(), map(tuple, a["shape"].tolist()))))
        finally:
            self.lib.ttv_outs_free(outs, self.n)

    def graph_launches(self) -> int:
        """Kernel launches one replay of the cached graph performs."""
        return int(self.lib.ttv_batch_graph_launches(self.probs, self.n, self._outs(), ctypes.byref(self.opts)))


def batch_release():
    """Drops every cached batch graph."""
    _declare_batch(load()).ttv_batch_release()


# ---- serving (continuous batching) ------------------------------------------

class Stats(ctypes.Structure):
    _fields_ = [("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("completed", ctypes.c_longlong), ("admitted", ctypes.c_longlong),
                ("refused", ctypes.c_longlong), ("pending", ctypes.c_longlong), ("seconds", ctypes.c_double),
                ("throughput_rps", ctypes.c_double), ("throughput_gnnz_s", ctypes.c_double),
                ("bytes_in_use", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t),
                ("prepared_runs", ctypes.c_longlong), ("grouped_runs", ctypes.c_longlong)]


def _declare_serve(lib):
    if getattr(lib, "_serve_declared", False):
        return lib
    P = ctypes.POINTER
    lib.ttv_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int32, P(ctypes.c_void_p)]
    lib.ttv_server_create.restype = ctypes.c_int
    lib.ttv_server_register.argtypes = [ctypes.c_void_p, P(Tensor), P(ctypes.c_int32)]
    lib.ttv_server_register.restype = ctypes.c_int
    lib.ttv_server_prepare.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_int32), ctypes.c_int32]
    lib.ttv_server_prepare.restype = ctypes.c_int
    lib.ttv_server_submit.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_int32), ctypes.c_int32,
                                      P(ctypes.c_void_p), ctypes.c_int, P(Opts), P(ctypes.c_uint64)]
    lib.ttv_server_submit.restype = ctypes.c_int
    lib.ttv_server_wait.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, P(Out)]
    lib.ttv_server_wait.restype = ctypes.c_int
    lib.ttv_server_wait_any.argtypes = [ctypes.c_void_p, ctypes.c_int64, P(ctypes.c_uint64), P(Out)]
    lib.ttv_server_wait_any.restype = ctypes.c_int
    lib.ttv_server_stats.argtypes = [ctypes.c_void_p, P(Stats)]
    lib.ttv_server_stats.restype = ctypes.c_int
    lib.ttv_server_reset_stats.argtypes = [ctypes.c_void_p]
    lib.ttv_server_reset_stats.restype = ctypes.c_int
    lib.ttv_server_destroy.argtypes = [ctypes.c_void_p]
    lib.ttv_server_destroy.restype = None
    lib._serve_declared = True
    return lib


class _DeviceArray:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 2, "strides": None}


class _OwnedOut:
    """A library-owned result, released (ttv_out_free) when the last tensor
    viewing it is gone; torch's current stream is synchronised first, so work
    queued on the views has finished."""

    def __init__(self, lib, out: Out):
        self.lib, self.out = lib, out

    def __del__(self):
        if sys.is_finalizing():   # the runtime may be gone; the process frees everything
            return
        try:
            torch.cuda.current_stream().synchronize()
            self.lib.ttv_out_free(ctypes.byref(self.out))
        except Exception:   # noqa: BLE001
            pass


class _OwnedArray(_DeviceArray):
    def __init__(self, owner, ptr, shape, typestr):
        super().__init__(ptr, shape, typestr)
        self.owner = owner       # torch.as_tensor keeps this object, hence the result, alive


def _view_result(lib, out: Out) -> Result:
    """A library-owned result as torch views of its buffers (no copy); the
    buffers are released when the views are."""
    owner = _OwnedOut(lib, out)
    newshape = tuple(int(out.shape[j]) for j in range(out.order))
    n = int(out.nnz)
    dev = torch.device("cuda", torch.cuda.current_device())
    if n > 0 and out.vals:
        vals = torch.as_tensor(_OwnedArray(owner, out.vals, (n,), "<f8"), device=dev)
    else:
        vals = torch.zeros(n, dtype=torch.float64, device=dev)
    if out.is_dense:
        return Result(None, vals.view(newshape), newshape, True)
    if out.order > 0 and n > 0 and out.subs:
        subs = torch.as_tensor(_OwnedArray(owner, out.subs, (n, out.order), "<i8"), device=dev)
    else:
        subs = torch.zeros((n, out.order), dtype=torch.int64, device=dev)
    return Result(subs, vals, newshape, False)


def _take_result(lib, out: Out) -> Result:
    """Copies a library-owned result into torch tensors and releases it."""
    try:
        newshape = tuple(int(out.shape[j]) for j in range(out.order))
        n = int(out.nnz)
        dev = torch.device("cuda", torch.cuda.current_device())
        if n > 0 and out.vals:
            vals = torch.as_tensor(_DeviceArray(out.vals, (n,), "<f8"), device=dev).clone()
        else:
            vals = torch.zeros(n, dtype=torch.float64, device=dev)
        if out.is_dense:
            return Result(None, vals.view(newshape), newshape, True)
        if out.order > 0 and n > 0 and out.subs:
            subs = torch.as_tensor(_DeviceArray(out.subs, (n, out.order), "<i8"), device=dev).clone()
        else:
            subs = torch.zeros((n, out.order), dtype=torch.int64, device=dev)
        return Result(subs, vals, newshape, False)
    finally:
        # the copies above run on torch's stream; the result's memory returns to
        # the library's stream-ordered pool only after they have finished
        torch.cuda.current_stream().synchronize()
        lib.ttv_out_free(ctypes.byref(out))


# Servers still open when the interpreter exits are closed first (their
# scheduler threads must stop before the CUDA runtime is torn down).
_live_servers = weakref.WeakSet()


@atexit.register
def _close_servers():
    for srv in list(_live_servers):
        try:
            srv.close()
        except Exception:   # noqa: BLE001
            pass


class Server:
    """Continuous-batching TTV server (``ttv_server_*``): resident tensors,
    requests admitted by memory budget onto ``slots`` concurrent streams."""

    def __init__(self, budget_bytes: int, slots: int = 8):
        self.lib = _declare_serve(load())
        self.h = ctypes.c_void_p()
        _check(self.lib, self.lib.ttv_server_create(int(budget_bytes), int(slots), ctypes.byref(self.h)))
        _live_servers.add(self)
        self.shapes = {}

    def register(self, subs, vals, shape) -> int:
        t = make_tensor(subs, vals, shape)
        tid = ctypes.c_int32()
        _check(self.lib, self.lib.ttv_server_register(self.h, ctypes.byref(t), ctypes.byref(tid)))
        self.shapes[int(tid.value)] = tuple(shape)
        torch.cuda.synchronize()
        return int(tid.value)

    def prepare(self, tensor_id: int, modes):
        """Prepared layout of a registered tensor for TTVs along ``modes``."""
        m = (ctypes.c_int32 * len(modes))(*[int(x) for x in modes])
        _check(self.lib, self.lib.ttv_server_prepare(self.h, int(tensor_id), m, len(modes)))

    def submit(self, tensor_id: int, modes, host_vecs, fmt="sparse", accum="fp64", path="auto") -> int:
        import numpy as np
        arrs = [np.ascontiguousarray(v) for v in host_vecs]
        dt = arrs[0].dtype
        if any(a.dtype != dt for a in arrs) or dt not in (np.float64, np.float32):
            raise TypeError("host vectors must all be float64 or all float32")
        m = (ctypes.c_int32 * len(modes))(*[int(x) for x in modes])
        vp = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
        o = make_opts(fmt=fmt, accum=accum, path=path)
        rid = ctypes.c_uint64()
        _check(self.lib, self.lib.ttv_server_submit(self.h, int(tensor_id), m, len(arrs), vp,
                                                    1 if dt == np.float32 else 0, ctypes.byref(o), ctypes.byref(rid)))
        return int(rid.value)

    def wait(self, req_id: int, timeout_us: int = -1, copy: bool = True) -> Result:
        """The result of request req_id: copied into torch memory (copy=True),
        or views of the library's buffers, released with them (copy=False)."""
        out = Out()
        rc = self.lib.ttv_server_wait(self.h, int(req_id), int(timeout_us), ctypes.byref(out))
        if rc != 0:
            msg = self.lib.ttv_last_error().decode(errors="replace")
            if out.internal:
                self.lib.ttv_out_free(ctypes.byref(out))
            raise TTVError(rc, msg)
        return _take_result(self.lib, out) if copy else _view_result(self.lib, out)

    def wait_any(self, timeout_us: int = -1, copy: bool = True):
        """The next finished request, whichever it is: (request id, Result);
        copy as for wait."""
        out = Out()
        rid = ctypes.c_uint64()
        rc = self.lib.ttv_server_wait_any(self.h, int(timeout_us), ctypes.byref(rid), ctypes.byref(out))
        if rc != 0:
            msg = self.lib.ttv_last_error().decode(errors="replace")
            if out.internal:
                self.lib.ttv_out_free(ctypes.byref(out))
            raise TTVError(rc, msg)
        return int(rid.value), (_take_result(self.lib, out) if copy else _view_result(self.lib, out))

    def stats(self) -> dict:
        s = Stats()
        _check(self.lib, self.lib.ttv_server_stats(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def reset_stats(self):
        _check(self.lib, self.lib.ttv_server_reset_stats(self.h))

    def close(self):
        if self.h:
            self.lib.ttv_server_destroy(self.h)
            self.h = ctypes.c_void_p()
        _live_servers.discard(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
