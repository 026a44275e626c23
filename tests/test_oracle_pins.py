"""The CPU oracle against its pins (no GPU)."""
import numpy as np
import pytest

import oracle
import oracle_pins as P


@pytest.mark.parametrize("check", P.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(check):
    check(oracle.ttv)


def test_errors():
    subs = np.array([[0, 1], [1, 0]], dtype=np.int64)
    vals = np.array([1.0, 2.0])
    with pytest.raises(oracle.OracleError) as e:
        oracle.ttv(subs, vals, (2, 2), [2], [np.ones(2)])
    assert e.value.code == -2
    with pytest.raises(oracle.OracleError) as e:
        oracle.ttv(subs, vals, (2, 2), [0, 0], [np.ones(2), np.ones(2)])
    assert e.value.code == -2
    with pytest.raises(oracle.OracleError) as e:
        oracle.ttv(subs, vals, (2, 2), [0], [np.ones(3)])
    assert e.value.code == -3
    with pytest.raises(oracle.OracleError) as e:
        oracle.ttv(np.array([[0, 2]]), np.array([1.0]), (2, 2), [0], [np.ones(2)])
    assert e.value.code == -4


def test_empty_and_scalar():
    s, v, sh = oracle.ttv(np.zeros((0, 3), np.int64), np.zeros(0), (2, 3, 4), [1], [np.ones(3)])
    assert sh == (2, 4) and s.shape == (0, 2) and v.shape == (0,)
    s, v, sh = oracle.ttv(np.zeros((0, 2), np.int64), np.zeros(0), (2, 3), [0, 1], [np.ones(2), np.ones(3)])
    assert sh == () and list(v) == [0.0]
    _, dv, sh = oracle.ttv(np.zeros((0, 2), np.int64), np.zeros(0), (2, 3), [0], [np.ones(2)], dense=True)
    assert sh == (3,) and list(dv) == [0.0, 0.0, 0.0]


def test_float32_inputs_are_upcast_exactly():
    g = np.random.default_rng(3)
    subs = np.stack([g.integers(0, 5, 40), g.integers(0, 4, 40)], axis=1)
    v32 = g.uniform(-1, 1, 40).astype(np.float32)
    x32 = g.uniform(-1, 1, 4).astype(np.float32)
    a = oracle.ttv(subs, v32, (5, 4), [1], [x32])
    b = oracle.ttv(subs, v32.astype(np.float64), (5, 4), [1], [x32.astype(np.float64)])
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_duplicates_summed_in_input_order():
    # 0.1 + 0.2 + 0.3 in one group: compensated sum gives the double nearest the exact sum
    subs = np.array([[0, 0], [0, 1], [0, 2]], dtype=np.int64)
    s, v, _ = oracle.ttv(subs, np.array([0.1, 0.2, 0.3]), (1, 3), [1], [np.ones(3)])
    from fractions import Fraction
    exact = Fraction(0.1) + Fraction(0.2) + Fraction(0.3)
    assert v[0] == float(exact)


def test_nonfinite_terms_follow_ieee_sum():
    """Eq. 3 is a plain sum: one +inf term gives +inf, +inf and -inf give nan,
    a nan term gives nan -- compensation must not change a non-finite sum."""
    inf, nan = float("inf"), float("nan")
    subs = np.array([[0, 0], [0, 1], [1, 0], [1, 1], [2, 0], [2, 1], [3, 0]], dtype=np.int64)
    vals = np.array([inf, 1.0, inf, -inf, nan, 2.0, -inf])
    s, v, _ = oracle.ttv(subs, vals, (4, 2), [1], [np.ones(2)])
    assert v[0] == inf and np.isnan(v[1]) and np.isnan(v[2]) and v[3] == -inf


def test_product_chain_rounds_each_step():
    """Eq. 3 forms vals[k] * x_m[.] one factor at a time in increasing mode
    order, each step rounded to binary64.  Closed forms where that chain and
    the exact product part: a partial product above the largest double stays
    infinite, one below the smallest subnormal stays zero, and a product in
    the subnormal range keeps only the bits that range holds."""
    big, small = 2.0 ** 600, 2.0 ** -600
    subs = np.zeros((1, 3), dtype=np.int64)
    # val * x0 overflows before x1 brings it back
    _, v, _ = oracle.ttv(subs, np.array([big]), (1, 1, 1), [0, 1], [np.array([big]), np.array([small])])
    assert v[0] == float("inf")
    # the same factors given in the other mode order: the chain order is fixed by the modes, not the list
    _, v, _ = oracle.ttv(subs, np.array([big]), (1, 1, 1), [1, 0], [np.array([small]), np.array([big])])
    assert v[0] == float("inf")
    # small factors first: underflow to zero, then scaled back up it stays zero
    _, v, _ = oracle.ttv(subs, np.array([-small]), (1, 1, 1), [0, 1], [np.array([small]), np.array([big])])
    assert v[0] == 0.0
    # big factor first: no partial leaves the range, the result is exact
    _, v, _ = oracle.ttv(subs, np.array([small]), (1, 1, 1), [0, 1], [np.array([big]), np.array([small])])
    assert v[0] == small
    # subnormal result: 3 * 2^-1062 is representable exactly
    _, v, _ = oracle.ttv(subs, np.array([0.75 * 2.0 ** -1000]), (1, 1, 1), [2], [np.array([2.0 ** -60])])
    assert v[0] == 3 * 2.0 ** -1062
    # subnormal result keeps 2^-1074 steps: (1 + 2^-52) * 2^-1060 rounds to 2^-1060
    _, v, _ = oracle.ttv(subs, np.array([(1 + 2.0 ** -52) * 2.0 ** -1000]), (1, 1, 1), [2],
                         [np.array([2.0 ** -60])])
    assert v[0] == 2.0 ** -1060
    # and a tie at the subnormal grid rounds to even: (1 + 2^-14) * 2^-1060 -> 2^-1060
    _, v, _ = oracle.ttv(subs, np.array([(1 + 2.0 ** -15) * 2.0 ** -1000]), (1, 1, 1), [2],
                         [np.array([2.0 ** -60])])
    assert v[0] == 2.0 ** -1060


@pytest.mark.parametrize("check", P.MTTKRP_CHECKS, ids=lambda c: c.__name__)
def test_mttkrp_pin(check):
    check(oracle.mttkrp, oracle.ttv)


def test_mttkrp_errors_and_empty():
    subs = np.array([[0, 1], [1, 0]], dtype=np.int64)
    vals = np.array([1.0, 2.0])
    facs = [np.ones((2, 3)), np.ones((2, 3))]
    with pytest.raises(oracle.OracleError) as e:
        oracle.mttkrp(np.array([[0, 2]]), np.array([1.0]), (2, 2), 0, facs)
    assert e.value.code == -4
    M = oracle.mttkrp(np.zeros((0, 2), np.int64), np.zeros(0), (2, 2), 1, facs)
    assert M.shape == (2, 3) and not M.any()
    M = oracle.mttkrp(subs, vals, (2, 2), 1, facs)
    assert M.tolist() == [[2.0] * 3, [1.0] * 3]


@pytest.mark.parametrize("check", P.DENSE_CHECKS, ids=lambda c: c.__name__)
def test_dense_kernel_pin(check):
    check(oracle.dot, oracle.matvec, oracle.ttv)


def test_dense_kernels_errors_and_empty():
    with pytest.raises(ValueError):
        oracle.dot(np.ones(3), np.ones(4))
    with pytest.raises(ValueError):
        oracle.matvec(np.ones((2, 3)), np.ones(2))
    assert oracle.dot(np.zeros(0), np.zeros(0)) == 0.0
    assert oracle.matvec(np.zeros((3, 0)), np.zeros(0)).tolist() == [0.0, 0.0, 0.0]
    assert oracle.matvec(np.zeros((0, 4)), np.ones(4)).shape == (0,)


@pytest.mark.parametrize("threads", [1, 2, 3, 8])
def test_parallel_statement_is_bit_identical(threads):
    """The OpenMP statement (the benchmark's multi-core CPU baseline) returns
    the one-core oracle's result bit for bit: same terms, same order, same
    compensated sums."""
    for seed in range(12):
        g = np.random.default_rng(900 + seed)
        d = 2 + seed % 4
        shape = tuple(int(x) for x in g.integers(2, 9, size=d))
        nnz = int(g.integers(0, 3000))
        subs = np.stack([g.integers(0, n, size=nnz) for n in shape], axis=1).astype(np.int64)
        vals = g.uniform(-1, 1, size=nnz)
        modes = sorted(g.choice(d, size=int(g.integers(1, d + 1)), replace=False).tolist())
        vecs = [g.uniform(-1, 1, size=shape[m]) for m in modes]
        for dense in (False, True):
            a = oracle.ttv(subs, vals, shape, modes, vecs, dense=dense)
            b = oracle.ttv_parallel(subs, vals, shape, modes, vecs, dense=dense, threads=threads)
            assert a[2] == b[2]
            assert np.array_equal(a[1], b[1]) and (dense or np.array_equal(a[0], b[0])), (seed, dense)
