"""Seeded synthetic sparse tensors shaped like the paper's TTV workloads.

This module only draws random inputs; it holds none of the TTV arithmetic.
Both sides of every parity check (the CUDA library and the CPU oracle) take
their inputs from here.

Random numbers come from a counter-based generator (the SplitMix64 output
function of Steele, Lea and Flood, OOPSLA 2014, applied to seed-mixed
counters), written with int64 torch operations whose results are bit-identical
on the CPU and on a CUDA device.  Uniform doubles take the top 53 bits.  Normal
variates use the Box-Muller transform, whose last bit can differ between
devices (full-size checks therefore copy device-made inputs to the host).

Distinct subscripts ("sptenrand"-like, paper Sec. 3.3 and Sec. 4.3): draws are
deduplicated by a 64-bit hash of the row, keeping first occurrences in draw
order, and more are drawn until nnz rows are distinct.  A hash collision can
only drop a row that was distinct; it never keeps a duplicate.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

_GOLDEN = -7046029254386353131        # 0x9E3779B97F4A7C15 as int64
_M1 = -4658895280553007687            # 0xBF58476D1CE4E5B9
_M2 = -7723592293110705685            # 0x94D049BB133111EB


def _srl(x: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def mix64(x: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output function on int64 bit patterns (wrapping arithmetic)."""
    z = x
    z = (z ^ _srl(z, 30)) * _M1
    z = (z ^ _srl(z, 27)) * _M2
    return z ^ _srl(z, 31)


def _stream_base(seed: int, stream: int) -> int:
    t = torch.tensor([_wrap64(seed * 1_000_003 + stream)], dtype=torch.int64)
    return int(mix64(mix64(t) + _GOLDEN)[0])


def rand_bits(seed: int, stream: int, start: int, n: int, device="cpu") -> torch.Tensor:
    """n pseudo-random 64-bit words (int64) for counters start..start+n-1."""
    base = _stream_base(seed, stream)
    ctr = torch.arange(start, start + n, dtype=torch.int64, device=device)
    return mix64(ctr * _GOLDEN + base)


def uniform(seed, stream, n, lo=0.0, hi=1.0, start=0, device="cpu") -> torch.Tensor:
    """U[lo, hi) float64 from 53 random bits."""
    u = _srl(rand_bits(seed, stream, start, n, device), 11).to(torch.float64) * (2.0 ** -53)
    if lo == 0.0 and hi == 1.0:
        return u
    return lo + (hi - lo) * u


def normal(seed, stream, n, start=0, device="cpu") -> torch.Tensor:
    """N(0, 1) float64 by Box-Muller on two uniform streams."""
    u1 = uniform(seed, stream, n, start=start, device=device)
    u2 = uniform(seed, stream + 7919, n, start=start, device=device)
    r = torch.sqrt(-2.0 * torch.log1p(-u1))          # 1 - u1 in (0, 1]
    return r * torch.cos(2.0 * math.pi * u2)


def uniform_int(seed, stream, n, hi: int, start=0, device="cpu") -> torch.Tensor:
    """Integers uniform in [0, hi) (hi <= 2^31) by the multiply-shift map."""
    w = _srl(rand_bits(seed, stream, start, n, device), 32)      # 32 random bits
    return (w * hi) >> 32


def zipf_cdf(n: int, s: float) -> np.ndarray:
    """CDF of the truncated Zipf law p(r) ~ r^-s, r = 1..n, in float64 (host)."""
    w = np.arange(1, n + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_int(seed, stream, n, size: int, s: float, start=0, device="cpu") -> torch.Tensor:
    """Subscripts r - 1 with r ~ truncated Zipf(s) on 1..size, by inverse CDF."""
    cdf = torch.from_numpy(zipf_cdf(size, s)).to(device)
    u = uniform(seed, stream, n, start=start, device=device)
    return torch.searchsorted(cdf, u, right=True).clamp_(max=size - 1)


def _wrap64(x: int) -> int:
    """Python int -> the int64 with the same low 64 bits."""
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >= (1 << 63) else x


def _row_hash(subs: torch.Tensor) -> torch.Tensor:
    h = torch.full((subs.shape[0],), 0x2545F491, dtype=torch.int64, device=subs.device)
    for m in range(subs.shape[1]):
        h = mix64(h ^ (subs[:, m] + _wrap64((m + 1) * _GOLDEN)))
    return h


def distinct_subs(seed: int, shape, nnz: int, dist: str = "uniform", zipf_s: float = 1.2,
                  device="cpu", max_rounds: int = 64) -> torch.Tensor:
    """(nnz, d) int64 distinct subscripts, in draw order after deduplication."""
    d = len(shape)
    total = 1
    for n in shape:
        total *= int(n)
    if nnz > total:
        raise ValueError("more distinct nonzeros than cells")
    if nnz == 0:
        return torch.zeros((0, d), dtype=torch.int64, device=device)
    if nnz > total // 4 and total <= 50_000_000:
        # dense-ish: a seeded random permutation of all cells, first nnz kept
        order = torch.argsort(rand_bits(seed, 99, 0, total, device), stable=True)[:nnz]
        cols = []
        rem = order
        for n in reversed(shape):
            cols.append(rem % int(n))
            rem = rem // int(n)
        return torch.stack(cols[::-1], dim=1).contiguous()
    kept = None
    drawn = 0
    batch = max(16, int(nnz * 1.05) + 16)
    for _ in range(max_rounds):
        cols = []
        for m, n in enumerate(shape):
            if dist == "uniform":
                cols.append(uniform_int(seed, 100 + m, batch, int(n), start=drawn, device=device))
            elif dist == "zipf":
                cols.append(zipf_int(seed, 100 + m, batch, int(n), zipf_s, start=drawn, device=device))
            else:
                raise ValueError(dist)
        new = torch.stack(cols, dim=1)
        drawn += batch
        cand = new if kept is None else torch.cat([kept, new], dim=0)
        h = _row_hash(cand)
        uniq, inv = torch.unique(h, sorted=True, return_inverse=True)
        first = torch.full((uniq.numel(),), cand.shape[0], dtype=torch.int64, device=device)
        first.scatter_reduce_(0, inv, torch.arange(cand.shape[0], device=device), reduce="amin")
        first, _ = torch.sort(first)
        kept = cand[first]
        del cand, h, uniq, inv, first, new
        if kept.shape[0] >= nnz:
            return kept[:nnz].contiguous()
        missing = nnz - kept.shape[0]
        batch = max(16, int(missing * 1.6 * drawn / max(1, kept.shape[0])) + 16)
    raise RuntimeError("could not draw enough distinct subscripts")


@dataclass
class SparseTensor:
    """COO tensor: subs (nnz, d) int64, vals (nnz,), shape tuple."""
    subs: torch.Tensor
    vals: torch.Tensor
    shape: tuple

    @property
    def nnz(self) -> int:
        return int(self.vals.shape[0])

    @property
    def d(self) -> int:
        return len(self.shape)

    def to(self, device) -> "SparseTensor":
        return SparseTensor(self.subs.to(device), self.vals.to(device), self.shape)

    def soa(self) -> torch.Tensor:
        """Subscripts as d contiguous columns (d, nnz): pyttb's column-major layout."""
        return self.subs.t().contiguous()


@dataclass
class Problem:
    """One TTV request: tensor, contracted modes, vectors, output format."""
    tensor: SparseTensor
    modes: list
    vecs: list
    dense: bool = False
    name: str = ""
    meta: dict = field(default_factory=dict)


def sptenrand(seed: int, shape, nnz: int, dist="uniform", vals="u01", device="cpu",
              zipf_s: float = 1.2) -> SparseTensor:
    """Random sparse tensor with nnz distinct subscripts (like pyttb.sptenrand)."""
    subs = distinct_subs(seed, shape, nnz, dist=dist, zipf_s=zipf_s, device=device)
    if vals == "u01":
        v = uniform(seed, 1, nnz, device=device)
    elif vals == "u11":
        v = uniform(seed, 1, nnz, -1.0, 1.0, device=device)
    elif vals == "normal":
        v = normal(seed, 1, nnz, device=device)
    else:
        raise ValueError(vals)
    return SparseTensor(subs, v, tuple(int(s) for s in shape))


def vector(seed: int, stream: int, n: int, kind="u11", device="cpu") -> torch.Tensor:
    if kind == "u11":
        return uniform(seed, 5000 + stream, n, -1.0, 1.0, device=device)
    if kind == "u01":
        return uniform(seed, 5000 + stream, n, device=device)
    raise ValueError(kind)


# Exponent offsets for wide-range inputs: most entries keep their scale, the
# rest move by powers of two chosen so that chained products of three factors
# overflow, underflow to zero, or land among the subnormals.
WIDE_EXPONENTS = (0, 0, 0, 0, 0, 0, 300, -300, 600, -600, 350, -350, -700)


def wide_exponents(seed: int, stream: int, n: int, device="cpu") -> torch.Tensor:
    """n seeded exponent offsets drawn from WIDE_EXPONENTS (int64)."""
    idx = uniform_int(seed, stream, n, len(WIDE_EXPONENTS), device=device)
    return torch.tensor(WIDE_EXPONENTS, dtype=torch.int64, device=device)[idx]


def widen(problem: "Problem", seed: int) -> "Problem":
    """The same problem with values and vector entries multiplied by 2^e,
    e drawn per entry from WIDE_EXPONENTS (exact: only the exponent moves,
    while it stays in the binary64 range)."""
    t = problem.tensor
    ev = wide_exponents(seed, 7001, t.nnz, device=t.vals.device)
    vals = torch.ldexp(t.vals.to(torch.float64), ev.to(torch.float64))
    vecs = []
    for j, v in enumerate(problem.vecs):
        e = wide_exponents(seed, 7100 + j, v.shape[0], device=v.device)
        vecs.append(torch.ldexp(v.to(torch.float64), e.to(torch.float64)))
    return Problem(SparseTensor(t.subs, vals, t.shape), list(problem.modes), vecs, dense=problem.dense,
                   name=problem.name + "_wide", meta=dict(problem.meta))


# ----------------------------------------------------------------------------
# Workloads.  Sizes follow the TTV configurations the library is measured on
# and the paper's own sweep (Sec. 4.3: 3-way, n in {100..1200}, density 1 %,
# vector along the second mode, values U[0,1]).
# ----------------------------------------------------------------------------

def single_3way_100(seed=1, device="cpu") -> Problem:
    """Single TTV, mode 0, 100x100x100, 10,000 distinct uniform nonzeros,
    values U[0,1), vector U[-1,1]; sparse 100x100 result."""
    t = sptenrand(seed, (100, 100, 100), 10_000, vals="u01", device=device)
    return Problem(t, [0], [vector(seed, 0, 100, device=device)], name="single_3way_100_nnz1e4_mode0")


def allbutone_4way_1000(seed=2, device="cpu", nnz=10_000_000) -> Problem:
    """All-but-one TTV (vectors on modes 0, 1, 3; mode 2 survives) on a
    1000^4 tensor with 1e7 distinct uniform nonzeros, values and vectors
    U[-1,1]; dense length-1000 result."""
    t = sptenrand(seed, (1000, 1000, 1000, 1000), nnz, vals="u11", device=device)
    vecs = [vector(seed, m, 1000, device=device) for m in (0, 1, 3)]
    return Problem(t, [0, 1, 3], vecs, dense=True, name="allbutone_4way_1000_nnz1e7")


ZIPF5_SHAPE = (20000, 5000, 100000, 2000, 500)


def single_5way_zipf(seed=3, device="cpu", nnz=100_000_000, shape=ZIPF5_SHAPE) -> Problem:
    """Single TTV, mode 2, 5-way 20000x5000x100000x2000x500, 1e8 distinct
    nonzeros with Zipf(1.2) subscripts per mode, values N(0,1), vector
    U[-1,1]; sparse 4-way result."""
    t = sptenrand(seed, shape, nnz, dist="zipf", vals="normal", device=device)
    return Problem(t, [2], [vector(seed, 2, shape[2], device=device)], name="single_5way_zipf_nnz1e8")


def paper_sweep(n: int, seed=4, device="cpu") -> Problem:
    """The paper's TTV experiment (Sec. 4.3): n x n x n, density 0.01,
    values U[0,1], dense vector along the second mode (0-based mode 1)."""
    nnz = int(round(0.01 * n ** 3))
    t = sptenrand(seed + n, (n, n, n), nnz, vals="u01", device=device)
    return Problem(t, [1], [vector(seed + n, 1, n, kind="u01", device=device)], name=f"paper_sweep_n{n}")


def batch_problems(seed=5, count=512, nnz_lo=1e3, nnz_hi=2e6, device="cpu", scale=1.0) -> list:
    """Independent 3-to-5-way tensors, nnz log-uniform in [nnz_lo, nnz_hi],
    mode sizes uniform in [50, 50000] (redrawn while nnz > half the cells),
    uniform distinct subscripts, values U[0,1), own mode U[0, d), vector U[-1,1]."""
    out = []
    for i in range(count):
        s = seed * 100_003 + i
        r = uniform(s, 9, 8).numpy()
        d = 3 + int(r[0] * 3)
        nnz = int(math.exp(math.log(nnz_lo) + r[1] * (math.log(nnz_hi) - math.log(nnz_lo))) * scale)
        nnz = max(1, nnz)
        shape = None
        for tries in range(100):
            cand = uniform_int(s, 11 + tries, d, 49_951).numpy() + 50
            cells = 1
            for c in cand:
                cells *= int(c)
            if nnz <= 0.5 * cells:
                shape = tuple(int(c) for c in cand)
                break
        if shape is None:
            raise RuntimeError("no shape found")
        mode = int(r[2] * d)
        t = sptenrand(s, shape, nnz, vals="u01", device=device)
        out.append(Problem(t, [mode], [vector(s, mode, shape[mode], device=device)], name=f"batch{i}"))
    return out
