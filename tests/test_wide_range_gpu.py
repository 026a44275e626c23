"""Parity at the edges of the binary64 range (Eq. 3's product chain).

Values and vector entries are rescaled by seeded powers of two (2^0 for most,
2^+-300, 2^+-350, 2^+-600, 2^-700 for the rest), so that some products of
three factors overflow part-way through the chain, some underflow to zero
part-way, some land among the subnormals and some groups mix very large and
very small terms.  Eq. 3 forms each term as a chain of binary64 products in
increasing mode order; every path must give the oracle's value for it: the
same infinity or nan, and finite values within the FP64 tolerance, which for a
lone subnormal term means the same bits.
"""
import pytest
import torch

import synthetic as S
from parity import check_result, oracle_ttv, to_device

pytestmark = pytest.mark.gpu


def wide_problem(seed, shape, nnz, modes, dist="uniform"):
    t = S.sptenrand(seed, shape, nnz, dist=dist, vals="u11")
    vecs = [S.vector(seed, m, shape[m]) for m in modes]
    return S.widen(S.Problem(t, list(modes), vecs, name=f"wide{seed}_{shape}_{nnz}_{modes}"), seed)


def check(ttv, p, layout="aos", fmt="sparse", what="", **kw):
    subs, vals, vecs = to_device(p, layout=layout)
    dense = fmt == "dense"
    ref, A = oracle_ttv(subs, vals, p.tensor.shape, p.modes, vecs, dense=dense)
    res = ttv.ttv_multi(subs, vals, p.tensor.shape, p.modes, vecs, fmt=fmt, **kw)
    check_result(res, ref, A, dense=dense, what=what or p.name)
    return ref


@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_dense_default_kernel(cuda_lib, layout):
    # three vectors: the register-loading dense kernel with integer products
    p = wide_problem(21, (30, 20, 50, 40), 40_000, [0, 1, 3])
    check(cuda_lib, p, layout=layout, fmt="dense", path="dense")
    check(cuda_lib, p, layout=layout, fmt="sparse", path="dense")


def test_dense_generic_kernel(cuda_lib):
    # SoA with an odd column stride is served by the generic dense kernel
    p = wide_problem(22, (30, 20, 50, 40), 40_001, [0, 1])
    check(cuda_lib, p, layout="soa", fmt="sparse", path="dense")


def test_dense_bulk_staged_kernel(cuda_lib):
    p = wide_problem(23, (100, 80, 25, 40), 1_400_000, [0, 1, 3])
    subs, vals, vecs = to_device(p, layout="soa")
    cuda_lib.tune_clear()
    try:
        cuda_lib.tune_set(subs, vals, p.tensor.shape, p.modes, "dense", 1, 4, fmt="dense")
        check(cuda_lib, p, layout="soa", fmt="dense")
    finally:
        cuda_lib.tune_clear()


@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_dense_exact_accumulation(cuda_lib, layout):
    p = wide_problem(24, (30, 20, 50, 40), 40_000, [0, 1, 3])
    check(cuda_lib, p, layout=layout, fmt="dense", path="dense", accum="exact")


def test_dense_exact_without_infinities(cuda_lib):
    # no term overflows: the fixed-point path runs to the end (no hand-over)
    t = S.sptenrand(25, (30, 20, 50, 40), 40_000, vals="u11")
    vecs = [S.vector(25, m, t.shape[m]) for m in (0, 1, 3)]
    p = S.Problem(t, [0, 1, 3], vecs)
    ev = S.wide_exponents(25, 9, t.nnz)
    ev = torch.where(ev > 0, -ev, ev)          # only downward moves: no overflow
    vals = torch.ldexp(t.vals, ev.to(torch.float64))
    q = S.Problem(S.SparseTensor(t.subs, vals, t.shape), p.modes,
                  [torch.ldexp(v, torch.where(S.wide_exponents(25, 10 + j, v.shape[0]) > 0, 0,
                                              S.wide_exponents(25, 10 + j, v.shape[0])).to(torch.float64))
                   for j, v in enumerate(vecs)], name="wide_down_only")
    check(cuda_lib, q, fmt="dense", path="dense", accum="exact")


def test_dense_compensated(cuda_lib):
    p = wide_problem(30, (30, 20, 50, 40), 40_000, [0, 1, 3])
    check(cuda_lib, p, fmt="dense", path="dense", accum="compensated")


@pytest.mark.parametrize("path", ["sort", "hash", "bucket"])
def test_sparse_paths(cuda_lib, path):
    p = wide_problem(26, (2000, 500, 10000, 200, 50), 300_000, [2, 4], dist="zipf")
    check(cuda_lib, p, layout="soa", path=path)


def test_sort_compensated(cuda_lib):
    p = wide_problem(27, (300, 200, 100, 50), 200_000, [1, 2])
    check(cuda_lib, p, path="sort", accum="compensated")


def test_single_mode(cuda_lib):
    p = wide_problem(28, (300, 200, 100), 100_000, [1])
    check(cuda_lib, p, path="sort")
    check(cuda_lib, p, path="hash")


def test_prepared_runs(cuda_lib):
    p = wide_problem(29, (2000, 500, 10000, 200, 50), 300_000, [2, 4], dist="zipf")
    subs, vals, vecs = to_device(p, layout="soa")
    ref, A = oracle_ttv(subs, vals, p.tensor.shape, p.modes, vecs)
    prep = cuda_lib.Prepared(subs, vals, p.tensor.shape, p.modes)
    try:
        for accum in ("fp64", "compensated"):
            res = prep.run(vecs, accum=accum)
            check_result(res, ref, A, what=f"prepared {accum}")
    finally:
        prep.close()
