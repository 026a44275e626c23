"""pyttb's calling convention for ttv (mode specification by dims or
exclude_dims, automatic dense result, scalar order-0 result, sptensor-layout
arrays) on the CUDA path, against the oracle."""
import numpy as np
import pytest
import torch

import paper_2510_01495_gb300 as ttv
import synthetic as S
from parity import assert_close, check_result, oracle_ttv

pytestmark = pytest.mark.gpu


def tensor(seed, shape, nnz):
    t = S.sptenrand(seed, shape, nnz, vals="u11")
    vecs = [S.vector(seed, m, n) for m, n in enumerate(shape)]
    return t, vecs


def test_exclude_dims_equals_listed_modes(cuda_lib):
    t, vecs = tensor(3, (30, 40, 50, 20), 40_000)
    subs, vals = t.subs.cuda(), t.vals.cuda()
    dv = [v.cuda() for v in vecs]
    # all-but-one along mode 2, vectors given for every mode
    r = ttv.ttv(subs, vals, t.shape, dv, exclude_dims=2, fmt="sparse")
    ref, A = oracle_ttv(t.subs, t.vals, t.shape, [0, 1, 3], [vecs[0], vecs[1], vecs[3]])
    check_result(r, ref, A, what="exclude_dims=2")
    # the same, vectors only for the contracted modes, listed out of order
    r2 = ttv.ttv(subs, vals, t.shape, [dv[3], dv[0], dv[1]], dims=[3, 0, 1], fmt="sparse")
    assert torch.equal(r.subs, r2.subs)
    check_result(r2, ref, A, what="dims=[3,0,1]")


def test_single_vector_and_auto_dense(cuda_lib):
    # 20x30x40 with 20000 nonzeros: contracting mode 2 fills most of the
    # 20x30 result, so the automatic format returns it dense
    t, vecs = tensor(4, (20, 30, 40), 20_000)
    subs, vals = t.subs.cuda(), t.vals.cuda()
    r = ttv.ttv(subs, vals, t.shape, vecs[2].cuda(), dims=2)
    ref, A = oracle_ttv(t.subs, t.vals, t.shape, [2], [vecs[2]], dense=True)
    assert r.is_dense
    check_result(r, ref, A, dense=True, what="auto dense")
    # a sparse one stays sparse, and its sptensor arrays are the oracle's rows
    t2, v2 = tensor(5, (200, 300, 400), 20_000)
    r2 = ttv.ttv(t2.subs.cuda(), t2.vals.cuda(), t2.shape, v2[0].cuda(), dims=0)
    assert not r2.is_dense
    ref2, A2 = oracle_ttv(t2.subs, t2.vals, t2.shape, [0], [v2[0]])
    s, v, shp = r2.to_sptensor_arrays()
    assert shp == (300, 400) and v.shape == (ref2[1].shape[0], 1) and np.array_equal(s, ref2[0])
    assert_close(v, ref2[1], A2, what="sptensor arrays")


def test_dense_result_as_sptensor_arrays(cuda_lib):
    t, vecs = tensor(6, (20, 30, 40), 20_000)
    r = ttv.ttv(t.subs.cuda(), t.vals.cuda(), t.shape, vecs[2].cuda(), dims=2, fmt="dense")
    s, v, shp = r.to_sptensor_arrays()
    ref, A = oracle_ttv(t.subs, t.vals, t.shape, [2], [vecs[2]])
    keep = ref[1] != 0
    assert np.array_equal(s, ref[0][keep])
    assert_close(v, ref[1][keep], A[keep], what="dense as sptensor")


def test_all_modes_returns_a_float(cuda_lib):
    t, vecs = tensor(7, (9, 8, 7), 300)
    x = ttv.ttv(t.subs.cuda(), t.vals.cuda(), t.shape, [v.cuda() for v in vecs])
    assert isinstance(x, float)
    ref, A = oracle_ttv(t.subs, t.vals, t.shape, [0, 1, 2], vecs)
    assert_close([x], ref[1], A, what="order 0")


def test_auto_format_with_caller_buffers(cuda_lib):
    """The automatic format on caller-provided buffers: converted in place
    when the value buffer holds every cell, left sparse otherwise."""
    t, vecs = tensor(8, (20, 30, 40), 20_000)
    subs, vals = t.subs.cuda(), t.vals.cuda()
    v = vecs[2].cuda()
    big = torch.empty(600, dtype=torch.float64, device="cuda")
    rows = torch.empty((600, 2), dtype=torch.int64, device="cuda")
    r = ttv.ttv_multi(subs, vals, t.shape, [2], [v], fmt="auto", out_vals=big, out_subs=rows)
    ref, A = oracle_ttv(t.subs, t.vals, t.shape, [2], [vecs[2]], dense=True)
    assert r.is_dense
    check_result(r, ref, A, dense=True, what="auto, caller buffers")
    # 600 nonzeros fill about 63 % of the 600 cells: dense by the rule, but a
    # value buffer of exactly the sparse size keeps it sparse
    t2, v2 = tensor(9, (20, 30, 40), 600)
    ref2, A2 = oracle_ttv(t2.subs, t2.vals, t2.shape, [2], [v2[2]])
    n_out = ref2[1].size
    assert 300 < n_out < 600
    small = torch.empty(n_out, dtype=torch.float64, device="cuda")
    small_rows = torch.empty((n_out, 2), dtype=torch.int64, device="cuda")
    r2 = ttv.ttv_multi(t2.subs.cuda(), t2.vals.cuda(), t2.shape, [2], [v2[2].cuda()], fmt="auto", out_vals=small,
                       out_subs=small_rows)
    assert not r2.is_dense
    check_result(r2, ref2, A2, what="auto, small caller buffers")
    r3 = ttv.ttv(t2.subs.cuda(), t2.vals.cuda(), t2.shape, v2[2].cuda(), dims=2)     # library buffers
    assert r3.is_dense
    ref3, A3 = oracle_ttv(t2.subs, t2.vals, t2.shape, [2], [v2[2]], dense=True)
    check_result(r3, ref3, A3, dense=True, what="auto, library buffers")
