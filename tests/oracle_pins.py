"""Pins for the CPU oracle: checks against facts the paper and the mathematics
fix, independent of the oracle's own code.  Every check takes the TTV callable
to test (``ttv(subs, vals, shape, modes, vecs, dense=False)``) so that the
mutation tests can run the same checks against deliberately broken oracles.

Sources of truth used here:
  * Eq. 3 written out as a brute-force contraction over a DENSE tensor in
    exact rational arithmetic (fractions.Fraction) -- a different algorithm
    from the oracle's sort-and-group;
  * Eq. 1: a 1-way tensor times a vector is the dot product (math.fsum);
  * Eq. 2: a 2-way tensor times a vector along its second mode is the
    matrix-vector product (math.fsum per row);
  * linearity of Eq. 3 in the vector and in the values; the all-ones vector
    gives the sum over the contracted mode;
  * contracting every mode gives the multilinear form;
  * contracting the modes one at a time, in every order, gives the same
    result as contracting them together;
  * the result's support is the set of distinct surviving tuples in the
    input, in ascending lexicographic order (the "unique" rows of Sec. 3.3).
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np

EPS = 2.0 ** -53


def rng(seed):
    return np.random.default_rng(seed)


def random_case(seed, d, max_n=4, nnz=None, dup=True, dyadic=False):
    """Tiny random COO tensor (duplicates allowed when dup) and per-mode vectors."""
    g = rng(seed)
    shape = tuple(int(x) for x in g.integers(1, max_n + 1, size=d))
    cells = int(np.prod(shape))
    if nnz is None:
        nnz = int(g.integers(0, 2 * cells + 2))
    if dup:
        subs = np.stack([g.integers(0, n, size=nnz) for n in shape], axis=1).astype(np.int64)
    else:
        nnz = min(nnz, cells)
        lin = g.choice(cells, size=nnz, replace=False)
        subs = np.stack(np.unravel_index(lin, shape), axis=1).astype(np.int64)
    if dyadic:
        vals = g.integers(-8, 9, size=nnz).astype(np.float64) / 4.0
        vecs = [g.integers(-8, 9, size=n).astype(np.float64) / 8.0 for n in shape]
    else:
        vals = g.uniform(-1, 1, size=nnz)
        vecs = [g.uniform(-1, 1, size=n) for n in shape]
    return subs.reshape(nnz, d), vals, shape, vecs


def brute_force(subs, vals, shape, modes, vecs):
    """Eq. 3 over the dense tensor, exactly: returns {tuple(i_R): Fraction}
    for the structurally present tuples, plus the surviving shape."""
    d = len(shape)
    modes = list(modes)
    dense = np.empty(shape, dtype=object)
    for idx in np.ndindex(*shape):
        dense[idx] = Fraction(0)
    for k in range(len(vals)):
        dense[tuple(int(s) for s in subs[k])] += Fraction(float(vals[k]))
    R = [m for m in range(d) if m not in modes]
    vec_of = {m: v for m, v in zip(modes, vecs)}
    present = sorted({tuple(int(subs[k, r]) for r in R) for k in range(len(vals))})
    res = {}
    for out_idx in present:
        acc = Fraction(0)
        for cidx in itertools.product(*[range(shape[m]) for m in sorted(modes)]):
            full = [0] * d
            for r, i in zip(R, out_idx):
                full[r] = i
            for m, i in zip(sorted(modes), cidx):
                full[m] = i
            term = dense[tuple(full)]
            if term == 0:
                continue
            for m, i in zip(sorted(modes), cidx):
                term *= Fraction(float(vec_of[m][i]))
            acc += term
        res[out_idx] = acc
    return res, tuple(shape[r] for r in R)


def check_bruteforce_exact(ttv, seeds=range(40)):
    """Dyadic inputs: every product and sum is exact in binary64, so the
    oracle must equal the rational brute force bit for bit."""
    for seed in seeds:
        d = 1 + seed % 4
        subs, vals, shape, vecs = random_case(seed, d, dyadic=True)
        g = rng(1000 + seed)
        nv = int(g.integers(1, d + 1))
        modes = [int(m) for m in g.permutation(d)[:nv]]
        mv = [vecs[m] for m in modes]
        ref, rshape = brute_force(subs, vals, shape, modes, mv)
        s, v, sh = ttv(subs, vals, shape, modes, mv)
        assert sh == rshape, (seed, sh, rshape)
        keys = sorted(ref)
        if len(rshape) == 0:
            want = [float(ref[()]) if ref else 0.0]
            assert list(v) == want, (seed, v, want)
            continue
        assert [tuple(int(x) for x in row) for row in s] == keys, seed
        assert list(v) == [float(ref[k]) for k in keys], seed


def check_bruteforce_rounded(ttv, seeds=range(40)):
    """General doubles: within the error bound of rounded products and a
    compensated sum, |x - exact| <= (n_v + 2) u A + 2 u |exact|."""
    for seed in seeds:
        d = 1 + seed % 4
        subs, vals, shape, vecs = random_case(seed + 77, d)
        g = rng(2000 + seed)
        nv = int(g.integers(1, d + 1))
        modes = [int(m) for m in g.permutation(d)[:nv]]
        mv = [vecs[m] for m in modes]
        ref, rshape = brute_force(subs, vals, shape, modes, mv)
        absref, _ = brute_force(subs, np.abs(vals), shape, modes, [np.abs(x) for x in mv])
        s, v, sh = ttv(subs, vals, shape, modes, mv)
        assert sh == rshape
        keys = sorted(ref) if rshape else [()]
        if rshape:
            assert [tuple(int(x) for x in row) for row in s] == keys
        for key, x in zip(keys, v):
            exact = ref.get(key, Fraction(0))
            A = absref.get(key, Fraction(0))
            bound = (nv + 2) * EPS * float(A) + 2 * EPS * abs(float(exact))
            assert abs(Fraction(float(x)) - exact) <= Fraction(bound) * (1 + 1e-12), (seed, key, x, float(exact))


def check_dot_product(ttv):
    """d = 1: A x_0 v is the dot product of Eq. 1 (scalar result)."""
    g = rng(11)
    for n in (1, 7, 1000, 4096):
        a = g.uniform(-1, 1, size=n)
        x = g.uniform(-1, 1, size=n)
        subs = np.arange(n, dtype=np.int64).reshape(n, 1)
        s, v, sh = ttv(subs, a, (n,), [0], [x])
        assert sh == () and v.shape == (1,)
        want = math.fsum(float(a[i] * x[i]) for i in range(n))
        A = math.fsum(abs(float(a[i] * x[i])) for i in range(n))
        # same rounded products on both sides; Neumaier vs correctly rounded sum
        assert abs(v[0] - want) <= 2 * EPS * abs(want) + 4 * n * EPS * EPS * A + 1e-300


def check_matvec(ttv):
    """d = 2, vector along the second mode (paper's k = 2): the matrix-vector
    product of Eq. 2, one sum per row."""
    g = rng(12)
    for n1, n2 in ((3, 5), (17, 1), (1, 33), (40, 60)):
        M = g.uniform(-1, 1, size=(n1, n2))
        x = g.uniform(-1, 1, size=n2)
        subs = np.array([(i, j) for i in range(n1) for j in range(n2)], dtype=np.int64)
        vals = np.array([M[i, j] for i in range(n1) for j in range(n2)])
        s, v, sh = ttv(subs, vals, (n1, n2), [1], [x])
        assert sh == (n1,)
        assert [int(r[0]) for r in s] == list(range(n1))
        for i in range(n1):
            want = math.fsum(float(M[i, j] * x[j]) for j in range(n2))
            assert abs(v[i] - want) <= 2 * EPS * abs(want) + 1e-300, (n1, n2, i)


def check_ones_vector_is_mode_sum(ttv):
    """x = all ones: the result is the sum of the tensor over the mode."""
    g = rng(13)
    for d in (2, 3, 4):
        shape = tuple(int(x) for x in g.integers(2, 6, size=d))
        nnz = 60
        subs = np.stack([g.integers(0, n, size=nnz) for n in shape], axis=1).astype(np.int64)
        vals = g.integers(-50, 50, size=nnz).astype(np.float64)      # integer: exact sums
        for m in range(d):
            s, v, sh = ttv(subs, vals, shape, [m], [np.ones(shape[m])])
            dense = np.zeros(shape)
            np.add.at(dense, tuple(subs.T), vals)
            msum = dense.sum(axis=m)
            R = [r for r in range(d) if r != m]
            for row, x in zip(s, v):
                assert x == msum[tuple(row)], (d, m)
            assert len(s) == len({tuple(subs[k, R]) for k in range(nnz)})


def check_linearity(ttv):
    """Eq. 3 is linear in the vector and in the values."""
    g = rng(14)
    shape = (5, 4, 6)
    nnz = 80
    subs = np.stack([g.integers(0, n, size=nnz) for n in shape], axis=1).astype(np.int64)
    vals = g.uniform(-1, 1, size=nnz)
    vals2 = g.uniform(-1, 1, size=nnz)
    for m in range(3):
        x1 = g.uniform(-1, 1, size=shape[m])
        x2 = g.uniform(-1, 1, size=shape[m])
        a, b = 0.75, -2.5
        s1, v1, _ = ttv(subs, vals, shape, [m], [x1])
        s2, v2, _ = ttv(subs, vals, shape, [m], [x2])
        s3, v3, _ = ttv(subs, vals, shape, [m], [a * x1 + b * x2])
        assert np.array_equal(s1, s3) and np.array_equal(s2, s3)
        Aabs = ttv(subs, np.abs(vals), shape, [m], [abs(a) * np.abs(x1) + abs(b) * np.abs(x2)])[1]
        assert np.all(np.abs(v3 - (a * v1 + b * v2)) <= 16 * EPS * Aabs + 1e-300), m
        t1 = ttv(subs, vals, shape, [m], [x1])[1]
        t2 = ttv(subs, vals2, shape, [m], [x1])[1]
        t3 = ttv(subs, a * vals + b * vals2, shape, [m], [x1])[1]
        Aabs2 = ttv(subs, abs(a) * np.abs(vals) + abs(b) * np.abs(vals2), shape, [m], [np.abs(x1)])[1]
        assert np.all(np.abs(t3 - (a * t1 + b * t2)) <= 16 * EPS * Aabs2 + 1e-300), m


def check_all_modes_multilinear(ttv):
    """Contracting every mode gives sum_k vals[k] prod_m x_m[subs[k, m]]."""
    g = rng(15)
    for d in (1, 2, 3, 5):
        shape = tuple(int(x) for x in g.integers(1, 7, size=d))
        nnz = 50
        subs = np.stack([g.integers(0, n, size=nnz) for n in shape], axis=1).astype(np.int64)
        vals = g.uniform(-1, 1, size=nnz)
        vecs = [g.uniform(-1, 1, size=n) for n in shape]
        s, v, sh = ttv(subs, vals, shape, list(range(d))[::-1], vecs[::-1])
        assert sh == () and v.shape == (1,)
        exact = sum((Fraction(float(vals[k])) * math.prod(Fraction(float(vecs[m][subs[k, m]])) for m in range(d))
                     for k in range(nnz)), Fraction(0))
        A = sum(abs(float(vals[k])) * math.prod(abs(float(vecs[m][subs[k, m]])) for m in range(d)) for k in range(nnz))
        assert abs(Fraction(float(v[0])) - exact) <= Fraction((d + 2) * EPS * A + 2 * EPS * abs(float(exact)))


def _contract_sequential(ttv, subs, vals, shape, order, vec_of):
    """Contract modes one at a time in the given order (tracking renumbering)."""
    cur_modes = list(range(len(shape)))       # original mode of each current mode
    s, v, sh = subs, vals, tuple(shape)
    for m in order:
        pos = cur_modes.index(m)
        s, v, sh = ttv(s, v, sh, [pos], [vec_of[m]])
        cur_modes.pop(pos)
    return s, v, sh


def check_mode_order_independence(ttv):
    """All-but-one TTV equals sequential single-mode TTVs in any order,
    and the order of `modes` in one call does not matter."""
    g = rng(16)
    for d in (3, 4):
        shape = tuple(int(x) for x in g.integers(2, 6, size=d))
        nnz = 70
        subs = np.stack([g.integers(0, n, size=nnz) for n in shape], axis=1).astype(np.int64)
        vals = g.uniform(-1, 1, size=nnz)
        vec_of = {m: g.uniform(-1, 1, size=shape[m]) for m in range(d)}
        keep = int(g.integers(0, d))
        S = [m for m in range(d) if m != keep]
        s0, v0, sh0 = ttv(subs, vals, shape, S, [vec_of[m] for m in S])
        A = ttv(subs, np.abs(vals), shape, S, [np.abs(vec_of[m]) for m in S])[1]
        for perm in itertools.permutations(S):
            s1, v1, sh1 = ttv(subs, vals, shape, list(perm), [vec_of[m] for m in perm])
            assert sh1 == sh0 and np.array_equal(s1, s0) and np.array_equal(v1, v0)
            s2, v2, sh2 = _contract_sequential(ttv, subs, vals, shape, perm, vec_of)
            assert sh2 == sh0 and np.array_equal(s2, s0), perm
            assert np.all(np.abs(v2 - v0) <= 8 * d * EPS * A + 1e-300), perm


def check_support_and_order(ttv):
    """Support = distinct surviving tuples, ascending lexicographic; entries
    that cancel to zero stay; duplicates are summed."""
    subs = np.array([[1, 2, 0], [0, 0, 1], [1, 2, 1], [0, 0, 0], [2, 1, 0], [2, 1, 1]], dtype=np.int64)
    vals = np.array([1.0, 2.0, 3.0, 4.0, 5.0, -5.0])
    s, v, sh = ttv(subs, vals, (3, 3, 2), [2], [np.ones(2)])
    assert sh == (3, 3)
    assert [tuple(r) for r in s] == [(0, 0), (1, 2), (2, 1)]
    assert list(v) == [6.0, 4.0, 0.0]
    s, v, sh = ttv(subs, vals, (3, 3, 2), [0], [np.array([1.0, 10.0, 100.0])])
    assert [tuple(r) for r in s] == [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)]
    assert list(v) == [4.0, 2.0, 500.0, -500.0, 10.0, 30.0]
    # a lone infinity stays infinite (the compensation must not make it nan)
    s, v, sh = ttv(np.array([[0, 0], [0, 1]], dtype=np.int64), np.array([float("inf"), 1.0]), (1, 2), [1], [np.ones(2)])
    assert v[0] == float("inf")
    # compensated summation: 1e16 + 1 - 1e16 in one group is exactly 1
    subs = np.array([[0, 0], [0, 1], [0, 2]], dtype=np.int64)
    s, v, sh = ttv(subs, np.array([1e16, 1.0, -1e16]), (1, 3), [1], [np.ones(3)])
    assert list(v) == [1.0]


def check_dense_matches_sparse(ttv):
    g = rng(17)
    shape = (4, 3, 5)
    nnz = 30
    subs = np.stack([g.integers(0, n, size=nnz) for n in shape], axis=1).astype(np.int64)
    vals = g.uniform(-1, 1, size=nnz)
    x = g.uniform(-1, 1, size=3)
    s, v, sh = ttv(subs, vals, shape, [1], [x])
    _, dv, dsh = ttv(subs, vals, shape, [1], [x], dense=True)
    assert dsh == sh and dv.shape == sh
    want = np.zeros(sh)
    for row, x_ in zip(s, v):
        want[tuple(row)] = x_
    assert np.array_equal(dv, want)


ALL_CHECKS = [
    check_bruteforce_exact, check_bruteforce_rounded, check_dot_product, check_matvec,
    check_ones_vector_is_mode_sum, check_linearity, check_all_modes_multilinear,
    check_mode_order_independence, check_support_and_order, check_dense_matches_sparse,
]


# ---- MTTKRP (named in Sec. 3.3 and Sec. 5; the standard definition) ----------------

def mttkrp_case(seed, d, rank, dyadic=False):
    subs, vals, shape, _ = random_case(seed, d, dyadic=dyadic)
    g = rng(5000 + seed)
    if dyadic:
        facs = [g.integers(-8, 9, size=(n, rank)).astype(np.float64) / 8.0 for n in shape]
    else:
        facs = [g.uniform(-1, 1, size=(n, rank)) for n in shape]
    mode = int(g.integers(0, d))
    return subs, vals, shape, facs, mode


def mttkrp_brute_force(subs, vals, shape, mode, facs):
    """M(i, r) exactly, term by term over the nonzeros (duplicates included)."""
    rank = facs[(mode + 1) % len(shape)].shape[1]
    out = [[Fraction(0)] * rank for _ in range(shape[mode])]
    for k in range(len(vals)):
        for r in range(rank):
            t = Fraction(float(vals[k]))
            for m in range(len(shape)):
                if m != mode:
                    t *= Fraction(float(facs[m][int(subs[k, m]), r]))
            out[int(subs[k, mode])][r] += t
    return out


def check_mttkrp_equals_ttv_columns(mttkrp, ttv):
    """Column r of the MTTKRP is the all-but-one TTV with the factor columns
    A_m(:, r) as vectors: same products, same groups, same summation order,
    so equal bit for bit."""
    for seed in range(30):
        d = 2 + seed % 4
        subs, vals, shape, facs, mode = mttkrp_case(seed, d, rank=1 + seed % 5)
        M = mttkrp(subs, vals, shape, mode, facs)
        modes = [m for m in range(d) if m != mode]
        for r in range(M.shape[1]):
            _, col, _ = ttv(subs, vals, shape, modes, [facs[m][:, r] for m in modes], dense=True)
            assert np.array_equal(M[:, r], col), (seed, r)


def check_mttkrp_bruteforce_exact(mttkrp, ttv=None):
    for seed in range(30):
        d = 1 + seed % 4
        if d == 1:
            d = 2
        subs, vals, shape, facs, mode = mttkrp_case(seed + 300, d, rank=3, dyadic=True)
        M = mttkrp(subs, vals, shape, mode, facs)
        ref = mttkrp_brute_force(subs, vals, shape, mode, facs)
        assert M.shape == (shape[mode], 3)
        assert [[Fraction(float(x)) for x in row] for row in M] == ref, seed


def check_mttkrp_bruteforce_rounded(mttkrp, ttv=None):
    for seed in range(30):
        d = 2 + seed % 3
        subs, vals, shape, facs, mode = mttkrp_case(seed + 600, d, rank=4)
        M = mttkrp(subs, vals, shape, mode, facs)
        ref = mttkrp_brute_force(subs, vals, shape, mode, facs)
        absref = mttkrp_brute_force(subs, np.abs(vals), shape, mode, [np.abs(f) for f in facs])
        for i in range(shape[mode]):
            for r in range(4):
                bound = (d + 1) * EPS * float(absref[i][r]) + 2 * EPS * abs(float(ref[i][r]))
                assert abs(Fraction(float(M[i, r])) - ref[i][r]) <= Fraction(bound) * (1 + 1e-12), (seed, i, r)


def check_mttkrp_linear_in_each_factor(mttkrp, ttv=None):
    """M is linear in every factor matrix: with dyadic entries small enough
    that every product and sum is exact, M(.., A_m + B_m, ..) equals
    M(.., A_m, ..) + M(.., B_m, ..) bit for bit, and scaling A_m by 2 scales M
    by 2."""
    for seed in range(20):
        d = 2 + seed % 3
        subs, vals, shape, facs, mode = mttkrp_case(seed + 900, d, rank=3, dyadic=True)
        m = (mode + 1 + seed % (d - 1)) % d
        g = rng(9100 + seed)
        other = g.integers(-8, 9, size=facs[m].shape).astype(np.float64) / 8.0
        base = mttkrp(subs, vals, shape, mode, facs)
        alt = list(facs)
        alt[m] = other
        plus = list(facs)
        plus[m] = facs[m] + other
        twice = list(facs)
        twice[m] = 2.0 * facs[m]
        assert np.array_equal(mttkrp(subs, vals, shape, mode, plus), base + mttkrp(subs, vals, shape, mode, alt)), seed
        assert np.array_equal(mttkrp(subs, vals, shape, mode, twice), 2.0 * base), seed


MTTKRP_CHECKS = [check_mttkrp_equals_ttv_columns, check_mttkrp_bruteforce_exact, check_mttkrp_bruteforce_rounded,
                 check_mttkrp_linear_in_each_factor]


# ---- dense dot product (Eq. 1) and matrix-vector product (Eq. 2) --------------------

def _dyadic(g, size):
    return g.integers(-16, 17, size=size).astype(np.float64) / 16.0


def check_dot_exact_dyadic(dot, matvec=None, ttv=None):
    """Sums of exactly representable products with exact partial sums: the
    result is the exact rational value."""
    for seed in range(40):
        g = rng(7000 + seed)
        n = int(g.integers(0, 300))
        x, y = _dyadic(g, n), _dyadic(g, n)
        want = sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y)), Fraction(0))
        assert Fraction(dot(x, y)) == want, seed


def check_dot_rounded_bound(dot, matvec=None, ttv=None):
    """Random doubles: within one rounding per product plus the compensated
    sum's bound of the exact value."""
    for seed in range(40):
        g = rng(7100 + seed)
        n = int(g.integers(1, 400))
        x, y = g.uniform(-1, 1, n), g.uniform(-1, 1, n)
        exact = sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y)), Fraction(0))
        A = float(np.sum(np.abs(x) * np.abs(y)))
        bound = EPS * A * (1 + 1e-9) + 2 * EPS * abs(float(exact))
        assert abs(Fraction(dot(x, y)) - exact) <= Fraction(bound), seed


def check_dot_closed_forms(dot, matvec=None, ttv=None):
    """sum i = n(n-1)/2 and sum i^2 = (n-1)n(2n-1)/6 (exact in binary64 here)."""
    for n in (1, 2, 7, 1000, 100_000):
        i = np.arange(n, dtype=np.float64)
        assert dot(i, np.ones(n)) == n * (n - 1) // 2
        assert dot(i, i) == (n - 1) * n * (2 * n - 1) // 6
    assert dot(np.zeros(0), np.zeros(0)) == 0.0


def check_dot_is_order0_ttv(dot, matvec=None, ttv=None):
    """Eq. 1 is Eq. 3 with d = 1 and the one mode contracted: the vector x as a
    1-way COO tensor (subscripts 0..n-1 in order) times y, same products and
    same summation order, so equal bit for bit."""
    for seed in range(20):
        g = rng(7200 + seed)
        n = int(g.integers(1, 500))
        x, y = g.uniform(0, 1, n), g.uniform(-1, 1, n)
        _, v, sh = ttv(np.arange(n, dtype=np.int64).reshape(n, 1), x, (n,), [0], [y])
        assert sh == () and v[0] == dot(x, y), seed


def check_matvec_rows_are_dots(dot, matvec, ttv=None):
    """Row i of A x is the dot product of row i with x, bit for bit, whatever
    the storage order of A."""
    for seed in range(20):
        g = rng(7300 + seed)
        n1, n2 = int(g.integers(1, 40)), int(g.integers(1, 40))
        A = g.uniform(-1, 1, (n1, n2))
        x = g.uniform(-1, 1, n2)
        want = np.array([dot(np.ascontiguousarray(A[i]), x) for i in range(n1)])
        for M in (A, np.asfortranarray(A), np.ascontiguousarray(A.T).T):
            assert np.array_equal(matvec(M, x), want), seed


def check_matvec_is_mode1_ttv(dot, matvec, ttv):
    """Eq. 2 is Eq. 3 with d = 2 contracted along the second mode: the dense
    matrix as a COO tensor listed row by row gives the same groups in the same
    order, so the same bits."""
    for seed in range(20):
        g = rng(7400 + seed)
        n1, n2 = int(g.integers(1, 30)), int(g.integers(1, 30))
        A = g.uniform(0, 1, (n1, n2))
        x = g.uniform(0, 1, n2)
        subs = np.array([[i, j] for i in range(n1) for j in range(n2)], dtype=np.int64)
        _, v, sh = ttv(subs, A.reshape(-1), (n1, n2), [1], [x], dense=True)
        assert sh == (n1,) and np.array_equal(v, matvec(A, x)), seed


def check_matvec_exact_dyadic(dot, matvec, ttv=None):
    for seed in range(20):
        g = rng(7500 + seed)
        n1, n2 = int(g.integers(1, 25)), int(g.integers(1, 25))
        A, x = _dyadic(g, (n1, n2)), _dyadic(g, n2)
        y = matvec(np.asfortranarray(A), x)
        for i in range(n1):
            want = sum((Fraction(float(A[i, j])) * Fraction(float(x[j])) for j in range(n2)), Fraction(0))
            assert Fraction(float(y[i])) == want, (seed, i)


DENSE_CHECKS = [check_dot_exact_dyadic, check_dot_rounded_bound, check_dot_closed_forms, check_dot_is_order0_ttv,
                check_matvec_rows_are_dots, check_matvec_is_mode1_ttv, check_matvec_exact_dyadic]
