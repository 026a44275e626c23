"""MTTKRP on the GPU (prepared tensor, chunked warps, fixed-order fix-up)
against the CPU oracle, element by element."""
import numpy as np
import pytest
import torch

import oracle
import paper_2510_01495_gb300 as ttv
import synthetic as S

pytestmark = pytest.mark.gpu


def mttkrp_case(seed, shape, nnz, rank, dist="uniform"):
    t = S.sptenrand(seed, shape, nnz, vals="u11", dist=dist)
    g = np.random.default_rng(seed)
    facs = [g.uniform(-1, 1, (n, rank)) for n in shape]
    return t, facs


def check(M, subs, vals, shape, mode, facs, what):
    ref = oracle.mttkrp(subs, vals, shape, mode, facs)
    A = oracle.mttkrp(subs, np.abs(vals), shape, mode, [np.abs(f) for f in facs])
    got = M.cpu().numpy()
    assert got.shape == ref.shape, what
    err = np.abs(got - ref)
    tol = 1e-12 * np.maximum(np.abs(ref), 1e-3 * A)
    bad = np.argwhere(err > tol)
    assert bad.size == 0, f"{what}: {bad.shape[0]} entries off, first {bad[0]}: {got[tuple(bad[0])]} vs {ref[tuple(bad[0])]}"


@pytest.mark.parametrize("case", [
    ((30, 40, 50), 20_000, 0, 8),
    ((300, 200, 100), 100_003, 1, 16),
    ((30, 20, 10, 5), 20_000, 3, 32),
    ((5, 6, 7, 8, 9), 7_777, 2, 33),
    ((2000, 50, 60), 200_000, 0, 64),
    ((200, 300), 30_000, 1, 100),
    ((7, 9, 11), 601, 2, 1),
])
def test_mttkrp_vs_oracle(cuda_lib, case):
    shape, nnz, mode, rank = case
    t, facs = mttkrp_case(700 + nnz, shape, nnz, rank)
    subs = t.subs.t().contiguous().t().cuda()
    vals = t.vals.cuda()
    fd = [torch.from_numpy(f).cuda() for f in facs]
    M = ttv.mttkrp(subs, vals, shape, mode, fd)
    check(M, t.subs.numpy(), t.vals.numpy(), shape, mode, facs, f"mttkrp {case}")


def test_mttkrp_rows_over_many_chunks(cuda_lib):
    """Two rows of about 2.5e6 nonzeros each: the fix-up takes whole aligned
    runs of 64 and 4096 chunks from their sums, the rest chunk by chunk."""
    t, facs = mttkrp_case(77, (2, 3000, 3000), 5_000_000, 3)
    subs = t.subs.t().contiguous().t().cuda()
    fd = [torch.from_numpy(f).cuda() for f in facs]
    M1 = ttv.mttkrp(subs, t.vals.cuda(), t.shape, 0, fd)
    M2 = ttv.mttkrp(subs, t.vals.cuda(), t.shape, 0, fd)
    assert torch.equal(M1, M2)
    check(M1, t.subs.numpy(), t.vals.numpy(), t.shape, 0, facs, "two long rows")


def test_mttkrp_prepared_repeats_zipf_and_float32(cuda_lib):
    shape = (2000, 500, 10000, 200, 50)
    p = S.single_5way_zipf(nnz=300_000, shape=shape)
    t = p.tensor
    mode, rank = 2, 16
    g = np.random.default_rng(4)
    facs = [g.uniform(-1, 1, (n, rank)) for n in shape]
    modes = [m for m in range(5) if m != mode][::-1]           # any order
    subs = t.subs.t().contiguous().t().cuda()
    vals32 = t.vals.to(torch.float32).cuda()
    prep = ttv.Prepared(subs, vals32, shape, modes)
    fd = [torch.from_numpy(facs[m]).cuda() for m in modes]
    M1 = prep.mttkrp(fd).clone()
    M2 = prep.mttkrp(fd)
    assert torch.equal(M1, M2)                                  # deterministic
    check(M1, t.subs.numpy(), vals32.cpu().numpy(), shape, mode, facs, "zipf fp32 values")
    prep.close()


def test_mttkrp_rank_one_is_all_but_one_ttv(cuda_lib):
    t, facs = mttkrp_case(31, (60, 70, 80), 50_000, 1)
    subs, vals = t.subs.cuda(), t.vals.cuda()
    mode = 1
    others = [m for m in range(3) if m != mode]
    M = ttv.mttkrp(subs, vals, t.shape, mode, [torch.from_numpy(f).cuda() for f in facs])
    r = ttv.ttv_multi(subs, vals, t.shape, others, [torch.from_numpy(facs[m][:, 0]).cuda() for m in others],
                      fmt="dense")
    assert torch.allclose(M[:, 0], r.vals, rtol=1e-12, atol=1e-14)


def test_mttkrp_errors_and_empty(cuda_lib):
    dev = "cuda"
    subs = torch.zeros((0, 3), dtype=torch.int64, device=dev)
    vals = torch.zeros(0, dtype=torch.float64, device=dev)
    f = [torch.ones((n, 4), dtype=torch.float64, device=dev) for n in (3, 4, 5)]
    M = ttv.mttkrp(subs, vals, (3, 4, 5), 1, f)
    assert M.shape == (4, 4) and float(M.abs().sum()) == 0.0
    t, facs = mttkrp_case(5, (10, 11, 12), 500, 4)
    prep = ttv.Prepared(t.subs.cuda(), t.vals.cuda(), t.shape, [1])     # two surviving modes
    with pytest.raises(ValueError):
        prep.mttkrp([torch.from_numpy(facs[1]).cuda()])
    prep.close()
    with pytest.raises(ttv.TTVError) as e:
        ttv.mttkrp(t.subs.cuda(), t.vals.cuda(), t.shape, 0, [torch.ones((n, 200), dtype=torch.float64,
                                                                          device=dev) for n in t.shape])
    assert e.value.name == "TTV_ERR_ARG"                               # rank above the maximum
