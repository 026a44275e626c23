"""The seeded input generators (no GPU): the SplitMix64 output function
against its published definition written out with Python integers, the
counter-based streams, and the properties the workloads claim (distinct
subscripts in range, truncated Zipf frequencies, value ranges)."""
import numpy as np
import torch

import synthetic as S

MASK = (1 << 64) - 1


def splitmix64_reference(state: int, count: int):
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) with Python integers:
    state += 0x9E3779B97F4A7C15, then the two xor-shift-multiply rounds."""
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


def test_mix64_is_splitmix64():
    # counter k of a stream with base b feeds mix64(k * golden + b): with
    # b = golden that is the SplitMix64 sequence from state 0
    k = torch.arange(0, 16, dtype=torch.int64)
    got = S.mix64(k * S._GOLDEN + S._GOLDEN)
    want = splitmix64_reference(0, 16)
    assert [int(x) & MASK for x in got] == want


def test_streams_are_counter_based_and_seeded():
    a = S.rand_bits(7, 3, 0, 100)
    assert torch.equal(a[40:], S.rand_bits(7, 3, 40, 60))     # any window of the same counters
    assert torch.equal(a, S.rand_bits(7, 3, 0, 100))
    assert not torch.equal(a, S.rand_bits(8, 3, 0, 100))
    assert not torch.equal(a, S.rand_bits(7, 4, 0, 100))


def test_uniform_ranges_and_moments():
    u = S.uniform(1, 1, 200_000).numpy()
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005
    v = S.uniform(1, 2, 200_000, -1.0, 1.0).numpy()
    assert v.min() >= -1.0 and v.max() < 1.0 and abs(v.mean()) < 0.01
    z = S.normal(1, 3, 200_000).numpy()
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    i = S.uniform_int(1, 4, 200_000, 7).numpy()
    assert i.min() == 0 and i.max() == 6 and np.all(np.abs(np.bincount(i) / 200_000 - 1 / 7) < 0.005)


def test_truncated_zipf_frequencies():
    n, s = 100, 1.2
    r = S.zipf_int(2, 5, 400_000, n, s).numpy()
    assert r.min() >= 0 and r.max() <= n - 1
    f = np.bincount(r, minlength=n) / r.size
    p = np.arange(1, n + 1, dtype=np.float64) ** (-s)
    p /= p.sum()
    assert np.all(np.abs(f[:10] - p[:10]) < 0.005)
    assert abs(f[0] / f[1] - 2.0 ** s) < 0.05


def test_sptenrand_distinct_in_range_and_deterministic():
    for dist in ("uniform", "zipf"):
        t = S.sptenrand(11, (50, 40, 30), 20_000, dist=dist, vals="u11")
        assert t.subs.shape == (20_000, 3) and t.vals.shape == (20_000,)
        assert t.subs.min() >= 0 and all(int(t.subs[:, m].max()) < n for m, n in enumerate((50, 40, 30)))
        assert torch.unique(t.subs, dim=0).shape[0] == 20_000
        t2 = S.sptenrand(11, (50, 40, 30), 20_000, dist=dist, vals="u11")
        assert torch.equal(t.subs, t2.subs) and torch.equal(t.vals, t2.vals)
    dense = S.sptenrand(12, (10, 10, 10), 900)         # nearly full: permutation of the cells
    assert torch.unique(dense.subs, dim=0).shape[0] == 900


def test_workload_recipes():
    p = S.allbutone_4way_1000(nnz=10_000)
    assert p.tensor.shape == (1000,) * 4 and p.modes == [0, 1, 3] and p.dense
    assert [v.numel() for v in p.vecs] == [1000, 1000, 1000]
    z = S.single_5way_zipf(nnz=20_000)
    assert z.tensor.shape == S.ZIPF5_SHAPE and z.modes == [2] and z.vecs[0].numel() == S.ZIPF5_SHAPE[2]
    assert int(torch.mode(z.tensor.subs[:, 0]).values) == 0           # Zipf: subscript 0 most frequent
    q = S.paper_sweep(100)
    assert q.tensor.shape == (100, 100, 100) and q.tensor.nnz == 10_000 and q.modes == [1]
    b = S.batch_problems(count=6, nnz_hi=2e4)
    for pr in b:
        d = pr.tensor.d
        assert 3 <= d <= 5 and len(pr.modes) == 1 and 0 <= pr.modes[0] < d
        assert all(50 <= n <= 50_000 for n in pr.tensor.shape)
        assert pr.tensor.nnz <= 0.5 * float(np.prod([float(n) for n in pr.tensor.shape]))


def test_widened_inputs_reach_every_edge_of_the_range():
    """widen() really produces the cases the wide-range parity tests need:
    chains of three factors that overflow part-way while the whole product is
    finite, chains that underflow part-way while the product is not tiny, and
    products in the subnormal range (exponents from frexp, no TTV arithmetic)."""
    p = S.widen(S.Problem(S.sptenrand(21, (30, 20, 50, 40), 40_000, vals="u11"), [0, 1, 3],
                          [S.vector(21, m, n) for m, n in ((0, 30), (1, 20), (3, 40))]), 21)
    s = p.tensor.subs.numpy()
    e = [np.frexp(p.tensor.vals.numpy())[1].astype(np.int64)]
    for j, m in enumerate(p.modes):
        e.append(np.frexp(p.vecs[j].numpy()[s[:, m]])[1].astype(np.int64))
    part = np.cumsum(np.vstack(e), axis=0)[1:]     # frexp exponents of the partial products
    total = part[-1]
    assert np.any((part.max(axis=0) > 1030) & (total < 1000))
    assert np.any((part.min(axis=0) < -1080) & (total > -1000))
    assert np.any((total < -1030) & (total > -1070) & (part[:-1].min(axis=0) > -1020))
    # scaling is exact: the significands are those of the unscaled inputs
    base = S.sptenrand(21, (30, 20, 50, 40), 40_000, vals="u11").vals.numpy()
    assert np.array_equal(np.frexp(p.tensor.vals.numpy())[0], np.frexp(base)[0])
