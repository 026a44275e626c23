"""ttv_batch (one CUDA graph for many TTVs) against the oracle, and the
replayed graph against the first launch."""
import numpy as np
import pytest
import torch

import synthetic as S
from parity import check_result, oracle_ttv

pytestmark = pytest.mark.gpu


def _problems(count, seed, scale=0.002):
    ps = S.batch_problems(seed=seed, count=count, scale=scale)
    return ps


@pytest.mark.parametrize("fmt", ["sparse"])
def test_batch_matches_oracle_and_replays(cuda_lib, fmt):
    ps = _problems(24, 7)
    dev = "cuda"
    items = []
    for p in ps:
        t = p.tensor
        items.append((t.subs.to(dev), t.vals.to(dev), t.shape, p.modes, [v.to(dev) for v in p.vecs]))
    b = cuda_lib.Batch(items, fmt=fmt)
    r1 = b.run()
    torch.cuda.synchronize()
    first = [(x.subs.clone() if x.subs is not None else None, x.vals.clone()) for x in r1]
    assert b.graph_launches() > 0
    for p, (subs, vals, shape, modes, vecs), res in zip(ps, items, r1):
        ref, A = oracle_ttv(subs, vals, shape, modes, vecs, dense=(fmt == "dense"))
        check_result(res, ref, A, dense=(fmt == "dense"), what=p.name)
    n0 = cuda_lib.launch_count()
    r2 = b.run()
    assert cuda_lib.launch_count() - n0 == b.graph_launches()
    for (s1, v1), res in zip(first, r2):
        assert torch.equal(v1, res.vals)
        if s1 is not None:
            assert torch.equal(s1, res.subs)


def test_batch_mixed_orders_and_dense(cuda_lib):
    dev = "cuda"
    g = np.random.default_rng(5)
    items, refs = [], []
    for i in range(12):
        d = 2 + i % 4
        shape = tuple(int(x) for x in g.integers(3, 12, size=d))
        nnz = int(g.integers(1, 600))
        t = S.sptenrand(300 + i, shape, min(nnz, int(np.prod(shape)) // 2 + 1), vals="u11")
        nv = 1 + i % (d - 1) if d > 1 else 1
        modes = [int(m) for m in g.permutation(d)[:nv]]
        vecs = [S.vector(300 + i, m, shape[m]) for m in modes]
        items.append((t.subs.to(dev), t.vals.to(dev), shape, modes, [v.to(dev) for v in vecs]))
    for fmt in ("dense", "sparse"):
        b = cuda_lib.Batch(items, fmt=fmt)
        res = b.run()
        for (subs, vals, shape, modes, vecs), r in zip(items, res):
            ref, A = oracle_ttv(subs, vals, shape, modes, vecs, dense=(fmt == "dense"))
            check_result(r, ref, A, dense=(fmt == "dense"))


def _items(ps, dev="cuda", soa_every=0):
    """Device copies; every soa_every-th problem gets d contiguous columns
    (an odd nnz gives an odd column stride: the key kernel's any-stride form)."""
    items = []
    for j, p in enumerate(ps):
        t = p.tensor
        subs = t.subs.to(dev)
        if soa_every and j % soa_every == 0:
            subs = subs.t().contiguous().t()
        items.append((subs, t.vals.to(dev), t.shape, p.modes, [v.to(dev) for v in p.vecs]))
    return items


@pytest.mark.parametrize("accum", ["fp64", "compensated"])
def test_batch_stagewise_sort_path(cuda_lib, accum):
    """Sort-path problems run stage by stage: the whole batch is a fixed
    handful of kernel launches (key kernels per order and layout class: 3
    orders x 3 classes here; one histogram scan, at most 8 digit passes, 4
    reduce-by-key stages), every result matches the oracle, and a replay is
    bit-identical."""
    ps = _problems(40, 11, scale=0.003)
    items = _items(ps, soa_every=3)
    soa = [it[0].stride(1) for it in items if it[0].stride(0) == 1]
    assert any(s % 2 for s in soa) and any(s % 2 == 0 for s in soa)
    b = cuda_lib.Batch(items, fmt="sparse", path="sort", accum=accum)
    r1 = b.run()
    assert 0 < b.graph_launches() <= 9 + 1 + 8 + 4, b.graph_launches()
    for p, it, r in zip(ps, items, r1):
        ref, A = oracle_ttv(*it, dense=False)
        check_result(r, ref, A, dense=False, what=p.name)
    first = [(r.subs.clone(), r.vals.clone()) for r in r1]
    r2 = b.run()
    for (s1, v1), r in zip(first, r2):
        assert torch.equal(s1, r.subs) and torch.equal(v1, r.vals)


def test_batch_stagewise_mixed_with_other_paths(cuda_lib):
    """Sort-path problems of uneven size beside small dense-path ones in one
    graph: each result matches the oracle."""
    ps = _problems(16, 13, scale=0.01)
    items = _items(ps, soa_every=2)
    g = np.random.default_rng(9)
    for i in range(6):
        shape = tuple(int(x) for x in g.integers(4, 20, size=3))
        t = S.sptenrand(700 + i, shape, int(np.prod(shape)) // 3, vals="u11")
        items.append((t.subs.cuda(), t.vals.cuda(), shape, [i % 3], [S.vector(700 + i, i % 3, shape[i % 3]).cuda()]))
    b = cuda_lib.Batch(items, fmt="sparse")
    res = b.run()
    for it, r in zip(items, res):
        ref, A = oracle_ttv(*it, dense=False)
        check_result(r, ref, A, dense=False)


def test_batch_stagewise_subscript_error(cuda_lib):
    """A subscript outside its mode in one problem of a stage-wise batch
    makes the batch report TTV_ERR_SUBSCRIPT; the context stays usable."""
    from paper_2510_01495_gb300 import TTVError
    ps = _problems(8, 17, scale=0.002)
    items = _items(ps)
    subs, vals, shape, modes, vecs = items[3]
    bad = subs.clone()
    bad[bad.shape[0] // 2, 0] = shape[0]
    items[3] = (bad, vals, shape, modes, vecs)
    b = cuda_lib.Batch(items, fmt="sparse", path="sort")
    with pytest.raises(TTVError) as ei:
        b.run()
    assert ei.value.name == "TTV_ERR_SUBSCRIPT"
    good = _items(ps[:3])
    res = cuda_lib.Batch(good, fmt="sparse", path="sort").run()
    for it, r in zip(good, res):
        ref, A = oracle_ttv(*it, dense=False)
        check_result(r, ref, A, dense=False)


def test_batch_stagewise_f32_tiny_and_order2(cuda_lib):
    """FP32 values and vectors on the stage-wise path (both sides see the
    same float values, upcast exactly: the FP64 tolerance), beside problems
    of 0, 1, 2 and 3 nonzeros and order-2 tensors."""
    g = np.random.default_rng(23)
    items = []
    for i, p in enumerate(_problems(10, 19, scale=0.004)):
        t = p.tensor
        subs = t.subs.cuda()
        if i % 2:
            subs = subs.t().contiguous().t()
        items.append((subs, t.vals.float().cuda(), t.shape, p.modes, [v.float().cuda() for v in p.vecs]))
    for i, nnz in enumerate([0, 1, 2, 3, 5000, 777]):
        d = 2 if i >= 4 else 3
        shape = tuple(int(x) for x in g.integers(200, 3000, size=d))
        t = S.sptenrand(900 + i, shape, nnz, vals="u11")
        m = int(g.integers(0, d))
        items.append((t.subs.cuda(), t.vals.cuda(), shape, [m], [S.vector(900 + i, m, shape[m]).cuda()]))
    b = cuda_lib.Batch(items, fmt="sparse", path="sort")
    res = b.run()
    for it, r in zip(items, res):
        subs, vals, shape, modes, vecs = it
        ref, A = oracle_ttv(subs, vals.double(), shape, modes, [v.double() for v in vecs], dense=False)
        check_result(r, ref, A, dense=False)


def test_batch_stagewise_capacity_error(cuda_lib):
    """A result buffer with fewer rows than a stage-wise problem's result
    makes the batch report TTV_ERR_CAPACITY (rows past the buffer are not
    written)."""
    from paper_2510_01495_gb300 import TTVError
    ps = _problems(6, 29, scale=0.003)
    items = _items(ps)
    b = cuda_lib.Batch(items, fmt="sparse", path="sort")
    ov, os_, shape, modes = b.meta[2]
    half = max(1, ov.numel() // 2)
    guard = torch.full((half + 64,), 7.0, dtype=torch.float64, device=ov.device)
    b.meta[2] = (guard[:half], os_[:half], shape, modes)
    with pytest.raises(TTVError) as ei:
        b.run()
    assert ei.value.name == "TTV_ERR_CAPACITY"
    assert torch.all(guard[half:] == 7.0)
