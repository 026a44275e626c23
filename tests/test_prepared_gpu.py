"""Prepared tensors: one sort at preparation, then streaming reduce-by-key
runs with fresh vectors.  Each run equals the sort path bit for bit and the
oracle within the tolerance."""
import numpy as np
import pytest
import torch

import paper_2510_01495_gb300 as ttv
import synthetic as S
from parity import check_result, oracle_ttv, to_device

pytestmark = pytest.mark.gpu


def rand_problem(seed, shape, nnz, modes):
    t = S.sptenrand(seed, shape, nnz, vals="u11")
    return S.Problem(t, list(modes), [S.vector(seed, m, shape[m]) for m in modes], name=f"prep{seed}")


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("case", [
    ((7, 9, 11), 600, [1], "sparse"),
    ((300, 200, 100), 100_003, [1], "sparse"),
    ((30, 20, 10, 5), 20_000, [3, 0], "sparse"),
    ((30, 20, 10, 5), 20_001, [0, 1, 3], "dense"),
    ((5, 6, 7, 8, 9), 7_777, [4, 0, 2], "sparse"),
    ((2000, 500, 10000, 200, 50), 60_000, [2], "sparse"),
    ((9, 8, 7), 401, [0, 1, 2], "sparse"),         # order 0: one scalar
])
def test_prepared_equals_sort_path_and_oracle(cuda_lib, case, layout):
    shape, nnz, modes, fmt = case
    p = rand_problem(900 + nnz, shape, nnz, modes)
    subs, vals, vecs = to_device(p, layout=layout)
    prep = ttv.Prepared(subs, vals, shape, modes)
    r = prep.run(vecs, fmt=fmt)
    s = ttv.ttv_multi(subs, vals, shape, modes, vecs, fmt=fmt, path="sort")
    assert r.shape == s.shape
    assert torch.equal(r.vals, s.vals)
    if r.subs is not None and s.subs is not None:
        assert torch.equal(r.subs, s.subs)
    dense = fmt == "dense"
    ref, A = oracle_ttv(subs, vals, shape, modes, vecs, dense=dense)
    check_result(r, ref, A, dense=dense, what="prepared")
    # fresh vectors on the same preparation
    vecs2 = [S.vector(77, m, shape[m]).to("cuda") for m in modes]
    r2 = prep.run(vecs2, fmt=fmt)
    ref2, A2 = oracle_ttv(subs, vals, shape, modes, vecs2, dense=dense)
    check_result(r2, ref2, A2, dense=dense, what="prepared, second vectors")
    prep.close()


def test_prepared_zipf_float32_and_repeats(cuda_lib):
    shape = (2000, 500, 10000, 200, 50)
    p = S.single_5way_zipf(nnz=300_000, shape=shape)
    subs, vals, vecs = to_device(p, layout="soa", val_dtype=torch.float32, vec_dtype=torch.float32)
    prep = ttv.Prepared(subs, vals, shape, p.modes)
    ref, A = oracle_ttv(subs, vals, shape, p.modes, vecs)
    first = None
    for _ in range(3):
        r = prep.run(vecs)
        check_result(r, ref, A, what="prepared zipf fp32")
        if first is None:
            first = r.vals.clone()
        assert torch.equal(r.vals, first)   # deterministic
    assert prep.nnz_out == r.vals.numel()
    prep.close()


def test_prepared_source_arrays_may_be_freed(cuda_lib):
    p = rand_problem(5, (60, 70, 80), 30_000, [1])
    subs, vals, vecs = to_device(p)
    ref, A = oracle_ttv(subs, vals, p.tensor.shape, p.modes, vecs)
    prep = ttv.Prepared(subs, vals, p.tensor.shape, p.modes)
    subs.fill_(-1)
    vals.fill_(float("nan"))
    check_result(prep.run(vecs), ref, A, what="after the caller's arrays changed")
    prep.close()


def test_prepared_errors_and_empty(cuda_lib):
    dev = "cuda"
    subs = torch.tensor([[0, 1], [1, 2]], dtype=torch.int64, device=dev)
    vals = torch.tensor([1.0, 2.0], dtype=torch.float64, device=dev)
    with pytest.raises(ttv.TTVError) as e:
        ttv.Prepared(subs, vals, (2, 2), [0])
    assert e.value.name == "TTV_ERR_SUBSCRIPT"
    with pytest.raises(ttv.TTVError) as e:
        ttv.Prepared(subs, vals, (2, 3), [2])
    assert e.value.name == "TTV_ERR_MODE"
    prep = ttv.Prepared(subs, vals, (2, 3), [1])
    with pytest.raises(ttv.TTVError) as e:
        prep.run([torch.ones(4, dtype=torch.float64, device=dev)])
    assert e.value.name == "TTV_ERR_VEC_LEN"
    prep.close()
    empty = ttv.Prepared(torch.zeros((0, 3), dtype=torch.int64, device=dev),
                         torch.zeros(0, dtype=torch.float64, device=dev), (3, 4, 5), [1])
    r = empty.run([torch.ones(4, dtype=torch.float64, device=dev)])
    assert r.vals.numel() == 0 and r.shape == (3, 5)
    r = empty.run([torch.ones(4, dtype=torch.float64, device=dev)], fmt="dense")
    assert r.vals.shape == (3, 5) and float(r.vals.abs().sum()) == 0.0
    empty.close()


@pytest.mark.parametrize("case", [
    ((300, 200, 100), 100_003, [1]),
    ((30, 20, 10, 5), 20_000, [0, 3]),
    ((2, 5000, 80), 400_001, [1, 2]),           # two rows of 200 000 nonzeros: runs across many tiles
])
def test_prepared_compensated_matches_oracle(cuda_lib, case):
    shape, nnz, modes = case
    t = S.sptenrand(61 + nnz, shape, nnz, vals="u11")
    vecs = [S.vector(61 + nnz, m, shape[m]) for m in modes]
    subs = t.subs.t().contiguous().t().cuda()
    dv = [v.cuda() for v in vecs]
    prep = ttv.Prepared(subs, t.vals.cuda(), shape, modes)
    r1 = prep.run(dv, accum="compensated")
    r2 = prep.run(dv, accum="compensated")
    assert torch.equal(r1.subs, r2.subs) and torch.equal(r1.vals, r2.vals)       # fixed order
    ref, A = oracle_ttv(t.subs, t.vals, shape, modes, vecs)
    check_result(r1, ref, A, what=f"prepared compensated {case}")
    rp = prep.run(dv)                                                             # plain binary64 unchanged
    rs = ttv.ttv_multi(subs, t.vals.cuda(), shape, modes, dv, path="sort")
    assert torch.equal(rp.subs, rs.subs) and torch.equal(rp.vals, rs.vals)
    prep.close()


def test_prepared_compensated_recovers_cancelled_terms(cuda_lib):
    """One result row of 4e5 terms repeating (2^53, 1, -2^53, 1): a plain
    binary64 sum loses every 1 that meets 2^53, the compensated run sums
    carry it through the thread, tile, group and scan stages: exactly 2e5."""
    n = 400_000
    pattern = np.array([2.0 ** 53, 1.0, -(2.0 ** 53), 1.0])
    vals = torch.from_numpy(np.tile(pattern, n // 4)).cuda()
    subs = torch.stack([torch.zeros(n, dtype=torch.int64), torch.arange(n, dtype=torch.int64)], dim=1).cuda()
    prep = ttv.Prepared(subs, vals, (1, n), [1])
    x = torch.ones(n, dtype=torch.float64, device="cuda")
    rc = prep.run([x], accum="compensated")
    assert rc.vals.cpu().tolist() == [n / 2]
    (_, ref_vals, _), _ = oracle_ttv(subs.cpu(), vals.cpu(), (1, n), [1], [x.cpu()])
    assert ref_vals.tolist() == [n / 2]
    prep.close()
