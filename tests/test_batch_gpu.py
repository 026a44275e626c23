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
