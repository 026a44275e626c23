"""The allocation-free dense TTV entry point (ttv_dense_noalloc), called
through the C ABI, against the oracle and against the regular entry point
(ttv_multi, dense result) on the same inputs, twice in a row -- the second
call reuses the library's fixed scratch array left over from the first.

It serves callers that may not allocate device memory themselves or let a
library do it for them (their host application owns every allocation, or
they run where the allocator's locks and synchronisation are not allowed).
This file is collected last so that a failure here comes after every other
test has run."""
import ctypes

import numpy as np
import pytest
import torch

import synthetic as S
from parity import FLOOR, RTOL, assert_close, oracle_ttv, to_device

pytestmark = pytest.mark.gpu

# FP32 storage: both sides see the same float inputs, upcast exactly, so the
# binary64 tolerance applies against the oracle run on those inputs.


def _device_memory_state():
    """(free bytes of the device, bytes in use in its default memory pool)."""
    free, _ = torch.cuda.mem_get_info()
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    used = ctypes.c_uint64()
    CU_MEMPOOL_ATTR_USED_MEM_CURRENT = 7
    assert cu.cuMemPoolGetAttribute(pool, CU_MEMPOOL_ATTR_USED_MEM_CURRENT, ctypes.byref(used)) == 0
    return int(free), int(used.value)


def _problem(name, spec):
    if name == "allbutone":
        return S.allbutone_4way_1000(nnz=300_000)
    shape, nnz, modes = spec
    t = S.sptenrand(40 + nnz, shape, nnz, vals="u11")
    return S.Problem(t, list(modes), [S.vector(40 + nnz, m, shape[m]) for m in modes])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("case", [
    ("allbutone", None),
    ("small", ((30, 20, 10, 5), 20_000, [0, 3])),
    ("order0", ((9, 8, 7), 300, [0, 1, 2])),
    # 16384 result cells (the largest): the scratch holds 31 partial arrays,
    # so the CTA count is capped below the regular path's
    ("largest", ((128, 128, 50, 40), 3_000_000, [2, 3])),
], ids=lambda c: c[0] if isinstance(c, tuple) else str(c))
def test_noalloc_matches_oracle_and_ttv_multi_twice(cuda_lib, case, dtype):
    p = _problem(*case)
    subs, vals, vecs = to_device(p, layout="soa", val_dtype=dtype, vec_dtype=dtype)
    shape = p.tensor.shape
    ref, A = oracle_ttv(subs, vals, shape, p.modes, vecs, dense=True)
    multi = cuda_lib.ttv_multi(subs, vals, shape, p.modes, vecs, fmt="dense")
    n = max(1, multi.vals.numel())
    out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    cuda_lib.ttv_dense_noalloc(subs, vals, shape, p.modes, vecs, out)       # warm-up: first call on the device
    torch.cuda.synchronize()
    for i in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        before = _device_memory_state()
        got = cuda_lib.ttv_dense_noalloc(subs, vals, shape, p.modes, vecs, out)
        after = _device_memory_state()
        assert before == after, f"call {i}: device memory changed {before} -> {after}"
        assert tuple(got.shape) == tuple(multi.shape) == tuple(ref[2])
        assert_close(got.cpu().numpy(), ref[1], A, RTOL, FLOOR, what=f"noalloc vs oracle, call {i}")
        assert_close(got.cpu().numpy(), multi.vals.cpu().numpy(), A, RTOL, FLOOR, what=f"noalloc vs ttv_multi, call {i}")


def test_noalloc_rejects_oversize_and_bad_subscripts(cuda_lib):
    dev = "cuda"
    subs = torch.zeros((4, 3), dtype=torch.int64, device=dev)
    vals = torch.ones(4, dtype=torch.float64, device=dev)
    out = torch.empty(1 << 16, dtype=torch.float64, device=dev)
    with pytest.raises(cuda_lib.TTVError) as e:     # 200 x 200 cells: above the dense limit
        cuda_lib.ttv_dense_noalloc(subs, vals, (200, 5, 200), [1], [torch.ones(5, dtype=torch.float64, device=dev)], out)
    assert e.value.name == "TTV_ERR_UNSUPPORTED"
    with pytest.raises(cuda_lib.TTVError) as e:     # output buffer too small
        cuda_lib.ttv_dense_noalloc(subs, vals, (20, 5, 20), [1], [torch.ones(5, dtype=torch.float64, device=dev)], out[:10])
    assert e.value.name == "TTV_ERR_CAPACITY"
    with pytest.raises(ValueError):                 # a strided view is not a contiguous output buffer
        cuda_lib.ttv_dense_noalloc(subs, vals, (20, 5, 20), [1], [torch.ones(5, dtype=torch.float64, device=dev)],
                                   out.view(256, 256)[:, :200])
    bad = subs.clone()
    bad[2, 0] = 20
    with pytest.raises(cuda_lib.TTVError) as e:
        cuda_lib.ttv_dense_noalloc(bad, vals, (20, 5, 20), [1], [torch.ones(5, dtype=torch.float64, device=dev)], out)
    assert e.value.name == "TTV_ERR_SUBSCRIPT"
    # the shared scratch is usable again after an error
    got = cuda_lib.ttv_dense_noalloc(subs, vals, (20, 5, 20), [1], [torch.ones(5, dtype=torch.float64, device=dev)], out)
    assert float(got[0, 0]) == 4.0
