"""Shared helpers for the GPU parity tests: run the oracle and the CUDA
library on the same seeded inputs and compare.

Tolerance (FP64): |x - ref| <= RTOL * max(|ref|, FLOOR * A) per output
entry, A = sum of |terms| in that entry's group (the oracle's TTV of |vals|
with |vectors|).  RTOL = 1e-12 relative; the floor only matters where the
group cancels to (near) zero, where a relative bound is not attainable by
any summation order.  Subscripts and counts must match bit for bit, and a
non-finite result must be the oracle's: the same infinity, or nan for nan.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

RTOL = 1e-12
FLOOR = 1e-3


def oracle_ttv(subs, vals, shape, modes, vecs, dense=False):
    s = subs.detach().cpu().numpy() if torch.is_tensor(subs) else subs
    v = vals.detach().cpu().numpy() if torch.is_tensor(vals) else vals
    vv = [x.detach().cpu().numpy() if torch.is_tensor(x) else x for x in vecs]
    ref = oracle.ttv(s, v, shape, modes, vv, dense=dense)
    absref = oracle.ttv(s, np.abs(v), shape, modes, [np.abs(x) for x in vv], dense=dense)
    return ref, absref[1]


def assert_close(x, ref, A, rtol=RTOL, floor=FLOOR, what=""):
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    A = np.asarray(A, dtype=np.float64).reshape(-1)
    assert x.shape == ref.shape, (what, x.shape, ref.shape)
    # non-finite results must match in kind: nan for nan, the same infinity
    fin = np.isfinite(ref)
    nf = np.nonzero(~fin | ~np.isfinite(x))[0]
    if nf.size:
        same = (np.isnan(x[nf]) & np.isnan(ref[nf])) | (x[nf] == ref[nf])
        if not np.all(same):
            i = nf[np.nonzero(~same)[0][0]]
            raise AssertionError(f"{what}: non-finite mismatch at {i}: got {x[i]!r} want {ref[i]!r}")
    with np.errstate(invalid="ignore"):
        err = np.where(fin, np.abs(x - ref), 0.0)
        tol = rtol * np.maximum(np.abs(ref), floor * np.where(np.isfinite(A), A, 0.0))
    bad = np.nonzero(fin & (err > tol))[0]
    if bad.size:
        i = bad[0]
        raise AssertionError(f"{what}: {bad.size} values out of tolerance; first at {i}: "
                             f"got {x[i]!r} want {ref[i]!r} (A={A[i]!r}, tol={tol[i]!r})")


def check_result(res, ref, A, dense=False, rtol=RTOL, floor=FLOOR, what=""):
    rs, rv, rsh = ref
    assert tuple(res.shape) == tuple(rsh), (what, res.shape, rsh)
    if dense:
        assert res.is_dense or len(rsh) == 0
        assert_close(res.vals.cpu().numpy(), rv, A, rtol, floor, what)
        return
    vals = res.vals.cpu().numpy()
    assert vals.shape[0] == rv.shape[0], (what, "count", vals.shape[0], rv.shape[0])
    if len(rsh) > 0:
        subs = res.subs.cpu().numpy()
        assert subs.shape == rs.shape, (what, subs.shape, rs.shape)
        if not np.array_equal(subs, rs):
            bad = np.nonzero(np.any(subs != rs, axis=1))[0]
            raise AssertionError(f"{what}: subscripts differ at {bad.size} rows, first {bad[0]}: "
                                 f"{subs[bad[0]]} vs {rs[bad[0]]}")
    assert_close(vals, rv, A, rtol, floor, what)


def to_device(problem, device="cuda", layout="aos", val_dtype=torch.float64, vec_dtype=torch.float64):
    t = problem.tensor
    if layout == "aos":
        subs = t.subs.to(device).contiguous()
    else:   # SoA: (d, nnz) contiguous, viewed as (nnz, d)
        subs = t.subs.t().contiguous().to(device).t()
    vals = t.vals.to(val_dtype).to(device)
    vecs = [v.to(vec_dtype).to(device) for v in problem.vecs]
    return subs, vals, vecs
