"""The allocation-free dense TTV entry point (ttv_dense_noalloc), called
through the C ABI, against the regular entry point (ttv_multi, dense result)
on the same inputs, twice in a row -- the second call reuses the library's
fixed scratch array left over from the first.

It serves callers that may not allocate device memory themselves or let a
library do it for them (their host application owns every allocation, or
they run where the allocator's locks and synchronisation are not allowed).
This file is collected last so that a failure here comes after every other
test has run."""
import numpy as np
import pytest
import torch

import synthetic as S
from parity import RTOL, FLOOR, to_device

pytestmark = pytest.mark.gpu


def _compare(got, want, A):
    got = got.detach().cpu().numpy().reshape(-1)
    want = want.detach().cpu().numpy().reshape(-1)
    A = A.detach().cpu().numpy().reshape(-1)
    tol = RTOL * np.maximum(np.abs(want), FLOOR * A)
    assert np.all(np.abs(got - want) <= tol), float(np.max(np.abs(got - want) - tol))


@pytest.mark.parametrize("case", [
    ("allbutone", None),
    ("small", ((30, 20, 10, 5), 20_000, [0, 3])),
    ("order0", ((9, 8, 7), 300, [0, 1, 2])),
])
def test_noalloc_matches_ttv_multi_twice(cuda_lib, case):
    name, spec = case
    if name == "allbutone":
        p = S.allbutone_4way_1000(nnz=300_000)
    else:
        shape, nnz, modes = spec
        t = S.sptenrand(40 + nnz, shape, nnz, vals="u11")
        p = S.Problem(t, list(modes), [S.vector(40 + nnz, m, shape[m]) for m in modes])
    subs, vals, vecs = to_device(p, layout="soa")
    shape = p.tensor.shape
    ref = cuda_lib.ttv_multi(subs, vals, shape, p.modes, vecs, fmt="dense")
    A = cuda_lib.ttv_multi(subs, vals.abs(), shape, p.modes, [v.abs() for v in vecs], fmt="dense")
    n = max(1, ref.vals.numel())
    for _ in range(2):
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        got = cuda_lib.ttv_dense_noalloc(subs, vals, shape, p.modes, vecs, out)
        assert tuple(got.shape) == tuple(ref.shape)
        _compare(got, ref.vals, A.vals)


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
    bad = subs.clone()
    bad[2, 0] = 20
    with pytest.raises(cuda_lib.TTVError) as e:
        cuda_lib.ttv_dense_noalloc(bad, vals, (20, 5, 20), [1], [torch.ones(5, dtype=torch.float64, device=dev)], out)
    assert e.value.name == "TTV_ERR_SUBSCRIPT"
    # the shared scratch is usable again after an error
    got = cuda_lib.ttv_dense_noalloc(subs, vals, (20, 5, 20), [1], [torch.ones(5, dtype=torch.float64, device=dev)], out)
    assert float(got[0, 0]) == 4.0
