"""Parity at the benchmark sizes, in the launch configuration bench.py times
(SoA subscripts, AUTO path, binary64, preallocated workspace and results).

Where the oracle finishes in seconds (all-but-one 1000^4, 1e7 nonzeros) every
result cell is compared.  For the 1e8-nonzero Zipf TTV the oracle computes
sampled result rows one by one (the oracle over exactly the nonzeros whose
surviving tuple is a sampled row gives those rows), and properties that hold
at any size are checked on all of it with torch alone: the row count equals
the number of distinct surviving tuples, rows ascend strictly, and the total
equals the sum of all terms.  The batch of 512 problems is checked element by
element on sampled problems and by row counts on all of them."""
import numpy as np
import pytest
import torch

import paper_2510_01495_gb300 as ttv
import synthetic as S
from parity import check_result, oracle_ttv

pytestmark = pytest.mark.gpu


def soa(subs):
    return subs.t().contiguous().t()


def run_like_bench(subs, vals, shape, modes, vecs, fmt):
    ws = torch.empty(max(1, ttv.workspace_size(subs, vals, shape, modes, fmt=fmt)), dtype=torch.uint8,
                     device="cuda")
    rows, nv = ttv.out_capacity(subs, vals, shape, modes, fmt=fmt)
    order = len(shape) - len(modes)
    ov = torch.empty(nv, dtype=torch.float64, device="cuda")
    os_ = torch.empty((max(1, rows), max(1, order)), dtype=torch.int64, device="cuda") if fmt != "dense" else None
    return ttv.ttv_multi(subs, vals, shape, modes, vecs, fmt=fmt, workspace=ws, out_vals=ov, out_subs=os_)


def surviving_keys(subs, shape, modes):
    """Row-major keys of the surviving subscripts, with torch int64 ops."""
    key = torch.zeros(subs.shape[0], dtype=torch.int64, device=subs.device)
    for m in range(len(shape)):
        if m not in modes:
            key = key * shape[m] + subs[:, m]
    return key


def test_allbutone_4way_1000_full(cuda_lib):
    p = S.allbutone_4way_1000(device="cuda")
    t = p.tensor
    subs = soa(t.subs)
    r = run_like_bench(subs, t.vals, t.shape, p.modes, p.vecs, "dense")
    ref, A = oracle_ttv(subs, t.vals, t.shape, p.modes, p.vecs, dense=True)
    check_result(r, ref, A, dense=True, what="allbutone 1e7, every cell")


def test_single_5way_zipf_full(cuda_lib):
    p = S.single_5way_zipf(device="cuda")
    t = p.tensor
    assert t.nnz == 100_000_000
    subs = soa(t.subs)
    modes, shape = p.modes, t.shape
    r = run_like_bench(subs, t.vals, shape, modes, p.vecs, "sparse")
    n_out = r.vals.numel()

    # row count = distinct surviving tuples; rows ascend strictly
    keys_in = surviving_keys(t.subs, shape, modes)
    assert n_out == torch.unique(keys_in).numel()
    rshape = [shape[m] for m in range(len(shape)) if m not in modes]
    keys_out = torch.zeros(n_out, dtype=torch.int64, device="cuda")
    for j, n in enumerate(rshape):
        keys_out = keys_out * n + r.subs[:, j]
    assert bool((keys_out[1:] > keys_out[:-1]).all())

    # total = sum of all terms (both sides within the summation bound)
    terms = t.vals * p.vecs[0][t.subs[:, modes[0]]]
    total, abs_total = float(terms.sum()), float(terms.abs().sum())
    assert abs(float(r.vals.sum()) - total) <= 1e-11 * abs_total

    # 512 sampled rows, exactly against the oracle on their nonzeros
    g = torch.Generator(device="cpu").manual_seed(11)
    pick = torch.randint(0, n_out, (512,), generator=g).unique().to("cuda")
    mask = torch.isin(keys_in, keys_out[pick])
    sub_subs, sub_vals = t.subs[mask], t.vals[mask]
    ref, A = oracle_ttv(sub_subs, sub_vals, shape, modes, p.vecs)
    got = type(r)(r.subs[pick], r.vals[pick], r.shape, False)
    check_result(got, ref, A, what="zipf 1e8, sampled rows")

    # the prepared form of the same TTV equals it bit for bit
    prep = ttv.Prepared(subs, t.vals, shape, modes)
    rp = prep.run(p.vecs)
    assert torch.equal(rp.subs, r.subs) and torch.equal(rp.vals, r.vals)
    prep.close()


def test_batch_512_full(cuda_lib):
    probs = S.batch_problems(seed=5, count=512, device="cuda")
    items = [(soa(q.tensor.subs), q.tensor.vals, q.tensor.shape, q.modes, q.vecs) for q in probs]
    ttv.tune_clear()
    for it in items:
        if ttv.tune_lookup(it[0], it[1], it[2], it[3]) is None:
            ttv.autotune(it[0], it[1], it[2], it[3], it[4], trials=1)
    try:
        b = ttv.Batch(items)
        b.run()
        res = b.run()            # a replay of the cached graph
        torch.cuda.synchronize()
        for q, r in zip(probs, res):
            keys = surviving_keys(q.tensor.subs, q.tensor.shape, q.modes)
            assert r.vals.numel() == torch.unique(keys).numel(), q.name
        for i in np.random.default_rng(3).choice(len(probs), 6, replace=False):
            q = probs[int(i)]
            ref, A = oracle_ttv(q.tensor.subs, q.tensor.vals, q.tensor.shape, q.modes, q.vecs)
            check_result(res[int(i)], ref, A, what=f"batch problem {i}")
    finally:
        ttv.tune_clear()
        ttv.batch_release()
