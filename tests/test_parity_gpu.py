"""CUDA path vs the CPU oracle, element by element, on seeded inputs that span
several tiles with a ragged tail, plus the degenerate cases."""
import numpy as np
import pytest
import torch

import synthetic as S
from parity import check_result, oracle_ttv, to_device

pytestmark = pytest.mark.gpu


def run_case(ttv, problem, path="auto", fmt="sparse", layout="aos", val_dtype=torch.float64,
             vec_dtype=torch.float64, accum="fp64", what=""):
    subs, vals, vecs = to_device(problem, layout=layout, val_dtype=val_dtype, vec_dtype=vec_dtype)
    dense = fmt == "dense"
    ref, A = oracle_ttv(subs, vals, problem.tensor.shape, problem.modes, vecs, dense=dense)
    res = ttv.ttv_multi(subs, vals, problem.tensor.shape, problem.modes, vecs, fmt=fmt, path=path, accum=accum)
    check_result(res, ref, A, dense=dense, what=what or problem.name)
    return res


def rand_problem(seed, shape, nnz, modes, dist="uniform", vals="u11"):
    t = S.sptenrand(seed, shape, nnz, dist=dist, vals=vals)
    vecs = [S.vector(seed, m, shape[m]) for m in modes]
    return S.Problem(t, list(modes), vecs, name=f"rand{seed}_{shape}_{nnz}_{modes}")


@pytest.mark.parametrize("path", ["auto", "dense", "sort"])
def test_single_3way_100(cuda_lib, path):
    run_case(cuda_lib, S.single_3way_100(), path=path)


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("path", ["dense", "sort"])
@pytest.mark.parametrize("case", [
    ((7, 9, 11), 600, [1]),
    ((30, 20, 10, 5), 20_000, [0, 3]),
    ((50, 40, 30), 9_001, [2]),
    ((5, 6, 7, 8, 9), 7_777, [4, 0, 2]),
    ((1000,), 999, [0]),
    ((40, 50), 1_999, [1]),
])
def test_random_small(cuda_lib, case, path, layout):
    shape, nnz, modes = case
    p = rand_problem(11 + nnz, shape, nnz, modes)
    run_case(cuda_lib, p, path=path, layout=layout)


@pytest.mark.parametrize("path", ["dense", "sort"])
def test_dense_format(cuda_lib, path):
    p = rand_problem(5, (20, 30, 40), 5_000, [0])
    run_case(cuda_lib, p, path=path, fmt="dense")


def test_allbutone_4way_reduced(cuda_lib):
    p = S.allbutone_4way_1000(nnz=300_000)
    run_case(cuda_lib, p, fmt="dense")
    run_case(cuda_lib, p, fmt="dense", path="sort")


def test_zipf_5way_reduced(cuda_lib):
    shape = (2000, 500, 10000, 200, 50)
    p = S.single_5way_zipf(nnz=400_000, shape=shape)
    res = run_case(cuda_lib, p, path="sort")
    assert res.vals.numel() > 100_000


@pytest.mark.parametrize("path", ["dense", "sort"])
def test_float32_storage(cuda_lib, path):
    p = rand_problem(21, (60, 70, 80), 30_000, [1])
    run_case(cuda_lib, p, path=path, val_dtype=torch.float32, vec_dtype=torch.float32)


@pytest.mark.parametrize("path", ["dense", "sort"])
def test_compensated(cuda_lib, path):
    p = rand_problem(22, (60, 70, 80), 30_000, [1])
    run_case(cuda_lib, p, path=path, accum="compensated")


def test_order0_scalar(cuda_lib):
    p = rand_problem(23, (9, 8, 7), 300, [0, 1, 2])
    res = run_case(cuda_lib, p)
    assert res.vals.numel() == 1 and res.shape == ()


def test_empty(cuda_lib):
    dev = "cuda"
    subs = torch.zeros((0, 3), dtype=torch.int64, device=dev)
    vals = torch.zeros(0, dtype=torch.float64, device=dev)
    v = torch.ones(4, dtype=torch.float64, device=dev)
    r = cuda_lib.ttv_single(subs, vals, (3, 4, 5), 1, v)
    assert r.shape == (3, 5) and r.vals.numel() == 0 and r.subs.shape == (0, 2)
    r = cuda_lib.ttv_single(subs, vals, (3, 4, 5), 1, v, fmt="dense")
    assert r.vals.shape == (3, 5) and float(r.vals.abs().sum()) == 0.0
    r = cuda_lib.ttv_multi(subs, vals, (3, 4, 5), [0, 1, 2],
                           [torch.ones(n, dtype=torch.float64, device=dev) for n in (3, 4, 5)])
    assert r.shape == () and r.vals.numel() == 1 and float(r.vals[0]) == 0.0


@pytest.mark.parametrize("path", ["dense", "sort"])
def test_duplicates_and_heavy_segments(cuda_lib, path):
    # one surviving tuple repeated 5000 times (long segment), duplicates of input subs
    g = np.random.default_rng(3)
    n = 12_000
    subs = np.stack([g.integers(0, 3, n), g.integers(0, 50, n), g.integers(0, 2, n)], axis=1)
    subs[:5000, 0] = 1
    subs[:5000, 2] = 1
    vals = g.uniform(-1, 1, n)
    x = g.uniform(-1, 1, 50)
    p = S.Problem(S.SparseTensor(torch.from_numpy(subs), torch.from_numpy(vals), (3, 50, 2)), [1],
                  [torch.from_numpy(x)], name="heavy")
    run_case(cuda_lib, p, path=path)


def test_sort_is_deterministic(cuda_lib):
    p = rand_problem(31, (300, 200, 100), 200_000, [1])
    subs, vals, vecs = to_device(p)
    r1 = cuda_lib.ttv_multi(subs, vals, p.tensor.shape, p.modes, vecs, path="sort")
    r2 = cuda_lib.ttv_multi(subs, vals, p.tensor.shape, p.modes, vecs, path="sort")
    assert torch.equal(r1.subs, r2.subs) and torch.equal(r1.vals, r2.vals)


def test_errors(cuda_lib):
    dev = "cuda"
    subs = torch.tensor([[0, 1], [1, 2]], dtype=torch.int64, device=dev)
    vals = torch.tensor([1.0, 2.0], dtype=torch.float64, device=dev)
    with pytest.raises(cuda_lib.TTVError) as e:
        cuda_lib.ttv_single(subs, vals, (2, 2), 0, torch.ones(2, dtype=torch.float64, device=dev))
    assert e.value.name == "TTV_ERR_SUBSCRIPT"
    subs = torch.tensor([[0, 1], [1, 0]], dtype=torch.int64, device=dev)
    with pytest.raises(cuda_lib.TTVError) as e:
        cuda_lib.ttv_single(subs, vals, (2, 2), 2, torch.ones(2, dtype=torch.float64, device=dev))
    assert e.value.name == "TTV_ERR_MODE"
    with pytest.raises(cuda_lib.TTVError) as e:
        cuda_lib.ttv_multi(subs, vals, (2, 2), [0, 0], [torch.ones(2, dtype=torch.float64, device=dev)] * 2)
    assert e.value.name == "TTV_ERR_MODE"
    with pytest.raises(cuda_lib.TTVError) as e:
        cuda_lib.ttv_single(subs, vals, (2, 2), 0, torch.ones(3, dtype=torch.float64, device=dev))
    assert e.value.name == "TTV_ERR_VEC_LEN"
    big = (1 << 32, 1 << 32, 2)
    with pytest.raises(cuda_lib.TTVError) as e:
        cuda_lib.ttv_single(torch.zeros((1, 3), dtype=torch.int64, device=dev), vals[:1], big, 2,
                            torch.ones(2, dtype=torch.float64, device=dev))
    assert e.value.name == "TTV_ERR_KEY_OVERFLOW"


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("case", [
    ((7, 9, 11), 600, [1], "sparse"),
    ((30, 20, 10, 5), 20_000, [0, 3], "sparse"),
    ((30, 20, 10, 5), 20_001, [0, 1, 3], "dense"),
    ((5, 6, 7, 8, 9), 7_777, [4, 0, 2], "dense"),
    ((9, 8, 7), 401, [0, 1, 2], "sparse"),
])
def test_exact_fixed_point(cuda_lib, case, layout):
    shape, nnz, modes, fmt = case
    p = rand_problem(101 + nnz, shape, nnz, modes)
    run_case(cuda_lib, p, path="dense", fmt=fmt, layout=layout, accum="exact")


def test_exact_is_deterministic_and_float32(cuda_lib):
    p = S.allbutone_4way_1000(nnz=400_000)
    subs, vals, vecs = to_device(p, layout="soa")
    r1 = cuda_lib.ttv_multi(subs, vals, p.tensor.shape, p.modes, vecs, fmt="dense", accum="exact")
    r2 = cuda_lib.ttv_multi(subs, vals, p.tensor.shape, p.modes, vecs, fmt="dense", accum="exact")
    assert torch.equal(r1.vals, r2.vals)
    run_case(cuda_lib, p, fmt="dense", accum="exact", layout="soa")
    run_case(cuda_lib, p, fmt="dense", accum="exact", val_dtype=torch.float32, vec_dtype=torch.float32)


def test_nonfinite_inputs_propagate(cuda_lib):
    # inf / nan in the values: the exact path hands over to binary64 arithmetic
    p = rand_problem(7, (20, 30, 40), 3_000, [0, 2])
    subs, vals, vecs = to_device(p)
    vals[5] = float("inf")
    vals[9] = float("nan")
    ref, A = oracle_ttv(subs, vals, p.tensor.shape, p.modes, vecs)
    for accum in ("fp64", "exact"):
        r = cuda_lib.ttv_multi(subs, vals, p.tensor.shape, p.modes, vecs, accum=accum)
        got = r.vals.cpu().numpy()
        assert np.array_equal(r.subs.cpu().numpy(), ref[0])
        assert np.array_equal(np.isnan(got), np.isnan(ref[1]))
        assert np.array_equal(np.isinf(got), np.isinf(ref[1]))
        fin = np.isfinite(ref[1])
        assert np.array_equal(got[~fin & ~np.isnan(got)], ref[1][~fin & ~np.isnan(ref[1])])
        err = np.abs(got[fin] - ref[1][fin])
        assert np.all(err <= 1e-12 * np.maximum(np.abs(ref[1][fin]), 1e-3 * A[fin]))


# ---- bucket path (splitter partition + on-chip sort) ------------------------------

@pytest.mark.parametrize("layout", ["soa", "aos"])
def test_bucket_path_zipf(cuda_lib, layout):
    shape = (2000, 500, 10000, 200, 50)
    p = S.single_5way_zipf(nnz=400_000, shape=shape)
    run_case(cuda_lib, p, path="bucket", layout=layout)


@pytest.mark.parametrize("layout", ["soa", "aos"])
def test_partition_path_runs_without_fallback(cuda_lib, layout):
    # the partition path itself (not the sort path it falls back to) produced the result
    p = S.single_5way_zipf(nnz=2_000_000, shape=(2000, 500, 10000, 200, 50))
    subs, vals, vecs = to_device(p, layout=layout)
    ref, A = oracle_ttv(subs, vals, p.tensor.shape, p.modes, vecs)
    cuda_lib.profile_reset()
    cuda_lib.profile_enable(True)
    try:
        res = cuda_lib.ttv_multi(subs, vals, p.tensor.shape, p.modes, vecs, path="bucket")
    finally:
        cuda_lib.profile_enable(False)
    cuda_lib.profile_collect()
    names = cuda_lib.profile_names()
    assert "part_scatter" in names and "part_process" in names, names
    assert "rbk_emit" not in names, names
    check_result(res, ref, A, what="partition path")


def test_bucket_path_large_uniform(cuda_lib):
    # 1.5e6 uniform nonzeros, 3-way result of 1.2e9 cells
    p = rand_problem(77, (1000, 1200, 50, 1000), 1_500_000, [2])
    run_case(cuda_lib, p, path="bucket", layout="soa")
    run_case(cuda_lib, p, layout="soa")


def test_bucket_heavy_keys_and_oversized_buckets(cuda_lib):
    # 40 surviving tuples carry half of 600k nonzeros (7.5k each): heavy keys that
    # the sample isolates, or buckets larger than the on-chip capacity that are
    # split by key sub-ranges; the rest is spread thinly
    g = np.random.default_rng(9)
    n = 600_000
    s0 = g.integers(0, 50, n)
    s1 = g.integers(0, 1000, n)
    s2 = g.integers(0, 2000, n)
    heavy = g.integers(0, 40, n // 2)
    s0[: n // 2] = heavy % 50
    s2[: n // 2] = (heavy * 37) % 2000
    perm = g.permutation(n)
    subs = np.stack([s0, s1, s2], axis=1)[perm]
    vals = g.uniform(-1, 1, n)
    x = g.uniform(-1, 1, 1000)
    p = S.Problem(S.SparseTensor(torch.from_numpy(subs), torch.from_numpy(vals), (50, 1000, 2000)), [1],
                  [torch.from_numpy(x)], name="bucket_heavy")
    run_case(cuda_lib, p, path="bucket", layout="soa")
    run_case(cuda_lib, p, path="bucket", layout="aos")


def test_bucket_dense_cluster_split(cuda_lib):
    # 200k distinct keys packed into a narrow key range next to a sparse tail:
    # quantile buckets are uneven and some exceed the on-chip capacity
    g = np.random.default_rng(11)
    n = 300_000
    lin = np.concatenate([g.choice(250_000, size=250_000, replace=False),
                          g.integers(0, 10**12, 50_000)])
    shape = (10**6, 10**6, 7)
    s0 = lin // 10**6
    s1 = lin % 10**6
    s2 = g.integers(0, 7, n)
    subs = np.stack([s0, s1, s2], axis=1)[g.permutation(n)]
    vals = g.uniform(-1, 1, n)
    x = g.uniform(-1, 1, 7)
    p = S.Problem(S.SparseTensor(torch.from_numpy(subs), torch.from_numpy(vals), shape), [2],
                  [torch.from_numpy(x)], name="bucket_cluster")
    run_case(cuda_lib, p, path="bucket", layout="soa")


def test_bucket_near_heavy_keys_at_range_top(cuda_lib):
    # keys repeated just under one quantile step (~4k times) are not isolated and
    # end up at the top of an oversized bucket's key range
    g = np.random.default_rng(21)
    nh = 60
    mult = g.integers(3000, 4090, nh)
    heavy_keys = g.choice(5_000_000, size=nh, replace=False)
    lin = np.concatenate([np.repeat(heavy_keys, mult), g.integers(0, 5_000_000, 400_000)])
    n = lin.size
    s0, s2 = lin // 1000, lin % 1000
    s1 = g.integers(0, 30, n)
    subs = np.stack([s0, s1, s2], axis=1)[g.permutation(n)]
    vals = g.uniform(-1, 1, n)
    x = g.uniform(-1, 1, 30)
    p = S.Problem(S.SparseTensor(torch.from_numpy(subs), torch.from_numpy(vals), (5000, 30, 1000)), [1],
                  [torch.from_numpy(x)], name="bucket_near_heavy")
    run_case(cuda_lib, p, path="bucket", layout="soa")


# ---- hash path (direct-indexed or open-addressing table in HBM) --------------------

@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("case", [
    # direct table: key space <= 4 x the table bound (no sort)
    ((300, 300, 300), 100_003, [0], "sparse"),
    ((300, 300, 300), 100_003, [0], "dense"),
    ((60, 70, 80, 90), 250_001, [1, 3], "sparse"),
    # hashed table: large key space, distinct keys sorted afterwards
    ((200, 300, 400, 500), 200_001, [1], "sparse"),
    ((100, 1000, 1000), 1_001, [0], "dense"),
    ((5, 6, 7, 8, 9), 7_777, [4], "sparse"),
    ((2000, 500, 10000, 200, 50), 50_000, [2], "sparse"),
])
def test_hash_path(cuda_lib, case, layout):
    shape, nnz, modes, fmt = case
    p = rand_problem(301 + nnz, shape, nnz, modes)
    run_case(cuda_lib, p, path="hash", fmt=fmt, layout=layout)


@pytest.mark.parametrize("shape", [(3, 50, 2), (3000, 50, 2000)])
def test_hash_duplicates_and_heavy_keys(cuda_lib, shape):
    # 5000 copies of one surviving tuple, duplicate input subscripts, keys that
    # repeat inside a warp (warp-combined before the table)
    g = np.random.default_rng(4)
    n = 40_000
    subs = np.stack([g.integers(0, 3, n), g.integers(0, 50, n), g.integers(0, 2, n)], axis=1)
    subs[:5000, 0] = 1
    subs[:5000, 2] = 1
    subs[20_000:20_064] = subs[20_000]
    vals = g.uniform(-1, 1, n)
    x = g.uniform(-1, 1, 50)
    p = S.Problem(S.SparseTensor(torch.from_numpy(subs), torch.from_numpy(vals), shape), [1],
                  [torch.from_numpy(x)], name="hash_heavy")
    run_case(cuda_lib, p, path="hash")
    run_case(cuda_lib, p, path="hash", fmt="dense")


def test_hash_zipf_reduced(cuda_lib):
    shape = (2000, 500, 10000, 200, 50)
    p = S.single_5way_zipf(nnz=400_000, shape=shape)
    res = run_case(cuda_lib, p, path="hash", layout="soa")
    assert res.vals.numel() > 100_000


def test_hash_float32_and_order0(cuda_lib):
    p = rand_problem(41, (600, 70, 800), 60_000, [1])
    run_case(cuda_lib, p, path="hash", val_dtype=torch.float32, vec_dtype=torch.float32)
    p = rand_problem(42, (9, 8, 7), 300, [0, 1, 2])
    res = run_case(cuda_lib, p, path="hash")
    assert res.vals.numel() == 1


@pytest.mark.parametrize("shape", [(200, 300, 400, 500), (300, 300, 300)])   # hashed, direct
def test_hash_capacity_and_subscript_errors(cuda_lib, shape):
    p = rand_problem(43, shape, 20_000, [1])
    subs, vals, vecs = to_device(p)
    small_subs = torch.empty((10, len(shape) - 1), dtype=torch.int64, device="cuda")
    small_vals = torch.empty(10, dtype=torch.float64, device="cuda")
    with pytest.raises(cuda_lib.TTVError) as e:
        cuda_lib.ttv_multi(subs, vals, p.tensor.shape, p.modes, vecs, path="hash",
                           out_subs=small_subs, out_vals=small_vals)
    assert e.value.name == "TTV_ERR_CAPACITY"
    bad = subs.clone()
    bad[77, 0] = shape[0]
    with pytest.raises(cuda_lib.TTVError) as e:
        cuda_lib.ttv_multi(bad, vals, p.tensor.shape, p.modes, vecs, path="hash")
    assert e.value.name == "TTV_ERR_SUBSCRIPT"


def test_hash_empty(cuda_lib):
    dev = "cuda"
    subs = torch.zeros((0, 3), dtype=torch.int64, device=dev)
    vals = torch.zeros(0, dtype=torch.float64, device=dev)
    v = torch.ones(400, dtype=torch.float64, device=dev)
    r = cuda_lib.ttv_single(subs, vals, (300, 400, 500), 1, v, path="hash")
    assert r.vals.numel() == 0 and r.subs.shape == (0, 2)


# ---- one-pass reduce-by-key after the sort -------------------------------------------

@pytest.mark.parametrize("fmt", ["sparse", "dense"])
def test_sort_segments_spanning_many_tiles(cuda_lib, fmt):
    # one surviving tuple 300 000 times (73 tiles of 4096 pairs: the look-back
    # folds more tiles than it keeps in registers), a second long run, and
    # singletons around them; bit-identical from run to run
    g = np.random.default_rng(8)
    n = 500_000
    subs = np.stack([g.integers(0, 40, n), g.integers(0, 30, n), g.integers(0, 20, n)], axis=1)
    subs[:300_000, 0] = 7
    subs[:300_000, 2] = 3
    subs[300_000:350_000, 0] = 39
    subs[300_000:350_000, 2] = 19
    vals = g.uniform(-1, 1, n)
    x = g.uniform(-1, 1, 30)
    p = S.Problem(S.SparseTensor(torch.from_numpy(subs), torch.from_numpy(vals), (40, 30, 20)), [1],
                  [torch.from_numpy(x)], name="long_runs")
    r1 = run_case(cuda_lib, p, path="sort", fmt=fmt)
    subs_d, vals_d, vecs_d = to_device(p)
    r2 = cuda_lib.ttv_multi(subs_d, vals_d, p.tensor.shape, p.modes, vecs_d, path="sort", fmt=fmt)
    assert torch.equal(r1.vals, r2.vals)


@pytest.mark.parametrize("nnz", [1, 2, 4095, 4096, 4097, 8192, 12_289])
def test_sort_tile_edges(cuda_lib, nnz):
    p = rand_problem(500 + nnz, (300, 200, 100), nnz, [1])
    run_case(cuda_lib, p, path="sort")


# ---- extremes: the largest order, keys above 2^63 ---------------------------------------

@pytest.mark.parametrize("path", ["auto", "sort", "hash", "bucket"])
def test_order_8(cuda_lib, path):
    p = rand_problem(808, (5, 4, 6, 3, 7, 4, 5, 6), 30_000, [2, 5])
    run_case(cuda_lib, p, path=path, layout="soa")
    q = rand_problem(809, (5, 4, 6, 3, 7, 4, 5, 6), 20_000, [0, 1, 2, 3, 4, 6, 7])
    run_case(cuda_lib, q, path=path, fmt="dense" if path == "auto" else "sparse")


@pytest.mark.parametrize("path", ["sort", "hash", "bucket"])
def test_keys_above_2_63(cuda_lib, path):
    # surviving key space 65535 * 65536^3 ~ 1.8e19: keys use the top bit of
    # uint64 and must be ordered as unsigned everywhere
    g = np.random.default_rng(12)
    n = 40_000
    shape = (65535, 65536, 65536, 65536, 7)
    subs = np.stack([g.integers(0, s, n) for s in shape], axis=1)
    subs[: n // 2, 0] = g.integers(32768, 65535, n // 2)       # half the keys >= 2^63
    subs[100:140] = subs[100]                                   # a repeated tuple
    vals = g.uniform(-1, 1, n)
    x = g.uniform(-1, 1, 7)
    p = S.Problem(S.SparseTensor(torch.from_numpy(subs), torch.from_numpy(vals), shape), [4],
                  [torch.from_numpy(x)], name="top_bit_keys")
    run_case(cuda_lib, p, path=path, layout="soa")


@pytest.mark.parametrize("layout", ["soa", "aos"])
@pytest.mark.parametrize("case", [
    ((60, 70, 80, 50), 700_001, [0, 1, 3], "dense"),
    ((60, 70, 80, 50), 1_234_567, [0, 2, 3], "sparse"),      # presence bitmap: sparse result off the dense path
    ((300, 200, 100), 900_002, [1, 2], "dense"),
    ((30, 40, 50, 60, 70), 1_000_003, [0, 1, 3, 4], "dense"),
])
def test_dense_staged_kernel(cuda_lib, case, layout):
    """Sizes above the point where the dense path switches to the
    bulk-staged persistent kernel: ragged last tiles, odd counts (the element
    past the last 16-byte unit is read directly), both layouts."""
    shape, nnz, modes, fmt = case
    p = rand_problem(31 + nnz, shape, nnz, modes)
    with staged_dense_plan(cuda_lib, p, fmt, layout):
        run_case(cuda_lib, p, path="auto", fmt=fmt, layout=layout)


class staged_dense_plan:
    """Pins the bulk-staged dense kernel (DENSE, items 4) for the problem's
    class for the duration of a block, through a hand-set tuning record."""

    def __init__(self, ttv, problem, fmt, layout, val_dtype=torch.float64):
        self.ttv = ttv
        subs, vals, _ = to_device(problem, layout=layout, val_dtype=val_dtype)
        self.args = (subs, vals, problem.tensor.shape, problem.modes)
        self.fmt = fmt

    def __enter__(self):
        self.ttv.tune_clear()
        self.ttv.tune_set(*self.args, "dense", 1, 4, fmt=self.fmt)
        assert self.ttv.tune_lookup(*self.args, fmt=self.fmt) == ("dense", 1, 4)

    def __exit__(self, *exc):
        self.ttv.tune_clear()


def test_dense_staged_kernel_float32(cuda_lib):
    p = rand_problem(41, (60, 70, 80, 50), 800_003, [0, 1, 3])
    with staged_dense_plan(cuda_lib, p, "dense", "soa", torch.float32):
        run_case(cuda_lib, p, path="auto", fmt="dense", layout="soa", val_dtype=torch.float32)
    with staged_dense_plan(cuda_lib, p, "dense", "aos", torch.float32):
        run_case(cuda_lib, p, path="auto", fmt="dense", layout="aos", val_dtype=torch.float32)
