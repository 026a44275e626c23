"""The continuous-batching server: every result in the mix matches the oracle
and equals the result of the same TTV run alone (ttv_multi), within the FP64
tolerance; budget
admission and refusal; bounded waits."""
import threading

import numpy as np
import pytest
import torch

import synthetic as S
from parity import RTOL, FLOOR, check_result, oracle_ttv

pytestmark = pytest.mark.gpu


def _close(a, b, A):
    a = a.cpu().numpy().reshape(-1)
    b = b.cpu().numpy().reshape(-1)
    A = A.cpu().numpy().reshape(-1)
    assert a.shape == b.shape
    assert np.all(np.abs(a - b) <= RTOL * np.maximum(np.abs(b), FLOOR * A))


def test_server_mix_equals_alone(cuda_lib):
    dev = "cuda"
    g = np.random.default_rng(1)
    tensors = []
    for i, (shape, nnz) in enumerate([((300, 200, 100, 50), 200_000), ((50, 60, 70, 80), 50_000),
                                      ((1000, 900, 800, 700), 400_000), ((20, 30, 40, 50), 20_000)]):
        t = S.sptenrand(500 + i, shape, nnz, vals="u11")
        tensors.append((t.subs.to(dev), t.vals.to(dev), shape))
    srv = cuda_lib.Server(budget_bytes=8 << 30, slots=4)
    ids = [srv.register(s, v, sh) for s, v, sh in tensors]
    reqs = []
    for j in range(48):
        ti = int(g.integers(0, len(tensors)))
        shape = tensors[ti][2]
        nv = 1 + j % 2
        modes = [int(m) for m in g.permutation(4)[:nv]]
        vecs = [g.uniform(-1, 1, shape[m]) for m in modes]
        reqs.append((ti, modes, vecs))
    rids = [None] * len(reqs)

    def client(lo, hi):
        for k in range(lo, hi):
            ti, modes, vecs = reqs[k]
            rids[k] = srv.submit(ids[ti], modes, vecs)

    th = [threading.Thread(target=client, args=(a, a + 12)) for a in range(0, 48, 12)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    results = [srv.wait(r, timeout_us=60_000_000) for r in rids]
    for k, ((ti, modes, vecs), res) in enumerate(zip(reqs, results)):
        subs, vals, shape = tensors[ti]
        # every served result against the oracle ...
        ref, A = oracle_ttv(subs, vals, shape, modes, vecs)
        check_result(res, ref, A, what=f"served request {k}")
        # ... and against the same TTV run alone
        dv = [torch.from_numpy(v).to(dev) for v in vecs]
        alone = cuda_lib.ttv_multi(subs, vals, shape, modes, dv)
        check_result(alone, ref, A, what=f"request {k} alone")
        assert res.shape == alone.shape
        assert torch.equal(res.subs, alone.subs)
        _close(res.vals, alone.vals, torch.from_numpy(A))
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["pending"] == 0
    assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
    srv.close()


def test_server_float32_storage(cuda_lib):
    dev = "cuda"
    t = S.sptenrand(77, (200, 300, 400, 50), 150_000, vals="u11")
    subs, vals32 = t.subs.to(dev), t.vals.to(torch.float32).to(dev)
    srv = cuda_lib.Server(budget_bytes=4 << 30, slots=2)
    tid = srv.register(subs, vals32, t.shape)
    x = np.random.default_rng(3).uniform(-1, 1, 300).astype(np.float32)
    res = srv.wait(srv.submit(tid, [1], [x], accum="compensated"))
    ref, A = oracle_ttv(subs, vals32, t.shape, [1], [x])
    check_result(res, ref, A)
    srv.close()


@pytest.mark.parametrize("modes", [[1], [0, 3]])
def test_server_float32_error_vs_fp64_oracle(cuda_lib, modes):
    # FP32 value/vector storage with compensated binary64 accumulation against
    # the FP64 oracle on the unrounded inputs: each stored factor carries one
    # rounding of relative size <= 2^-24, so a term is perturbed by at most
    # (1 + 2^-24)^(n_v + 1) - 1 relative; binary64 products and the
    # compensated sums on both sides add at most (n_v + 4) * 2^-53 * A.
    dev = "cuda"
    t = S.sptenrand(79, (200, 300, 400, 50), 200_000, vals="u11")
    g = np.random.default_rng(5)
    x64 = [g.uniform(-1, 1, t.shape[m]) for m in modes]
    x32 = [x.astype(np.float32) for x in x64]
    srv = cuda_lib.Server(budget_bytes=4 << 30, slots=2)
    tid = srv.register(t.subs.to(dev), t.vals.to(torch.float32).to(dev), t.shape)
    res = srv.wait(srv.submit(tid, modes, x32, accum="compensated"))
    srv.close()
    ref, A = oracle_ttv(t.subs, t.vals, t.shape, modes, [torch.from_numpy(x) for x in x64])
    assert np.array_equal(res.subs.cpu().numpy(), ref[0])
    err = np.abs(res.vals.cpu().numpy() - ref[1])
    nv = len(modes)
    rel = (1 + 2.0 ** -24) ** (nv + 1) - 1 + (nv + 4) * 2.0 ** -53
    assert np.all(err <= rel * A), float(np.max(err / np.maximum(A, 1e-300)))
    # the FP32 rounding is visible: the check is not vacuous
    assert float(np.max(err / A)) > 2.0 ** -26


def test_server_budget_and_timeout(cuda_lib):
    dev = "cuda"
    t = S.sptenrand(78, (100, 100, 100), 100_000, vals="u11")
    subs, vals = t.subs.to(dev), t.vals.to(dev)
    tiny = cuda_lib.Server(budget_bytes=1 << 20, slots=1)
    with pytest.raises(cuda_lib.TTVError) as e:
        tiny.register(subs, vals, t.shape)
    assert e.value.name == "TTV_ERR_BUDGET"
    tiny.close()
    # room for the tensor but not for a request's sort workspace
    srv = cuda_lib.Server(budget_bytes=int(100_000 * 32 * 1.05), slots=1)
    tid = srv.register(subs, vals, t.shape)
    with pytest.raises(cuda_lib.TTVError) as e:
        srv.submit(tid, [0], [np.ones(100)], path="sort")
    assert e.value.name == "TTV_ERR_BUDGET"
    srv.close()
    srv = cuda_lib.Server(budget_bytes=2 << 30, slots=1)
    tid = srv.register(subs, vals, t.shape)
    rid = srv.submit(tid, [0], [np.ones(100)])
    r = srv.wait(rid, timeout_us=30_000_000)
    assert r.vals.numel() > 0
    with pytest.raises(cuda_lib.TTVError) as e:
        srv.wait(123456, timeout_us=1000)
    assert e.value.name == "TTV_ERR_TIMEOUT"
    srv.close()


def test_server_prepared_layouts(cuda_lib):
    # requests on a prepared (tensor, modes) run on the prepared layout: the
    # result equals the sort path bit for bit; other requests are unaffected
    dev = "cuda"
    t = S.sptenrand(81, (200, 300, 400, 50), 150_000, vals="u11")
    subs, vals = t.subs.to(dev), t.vals.to(dev)
    srv = cuda_lib.Server(budget_bytes=4 << 30, slots=4)
    tid = srv.register(subs, vals, t.shape)
    srv.prepare(tid, [1])
    srv.prepare(tid, [3, 0])
    g = np.random.default_rng(9)
    cases = [([1], [g.uniform(-1, 1, 300)]),
             ([0, 3], [g.uniform(-1, 1, 200), g.uniform(-1, 1, 50)]),
             ([2], [g.uniform(-1, 1, 400)])]
    rids = [srv.submit(tid, modes, xs) for modes, xs in cases]
    results = [srv.wait(r) for r in rids]
    st = srv.stats()
    assert st["prepared_runs"] == 2
    for (modes, xs), res in zip(cases, results):
        xd = [torch.from_numpy(x).to(dev) for x in xs]
        ref, A = oracle_ttv(subs, vals, t.shape, modes, xd)
        check_result(res, ref, A, what=f"server prepared {modes}")
        s = cuda_lib.ttv_multi(subs, vals, t.shape, modes, xd, path="sort")
        if modes != [2]:
            assert torch.equal(res.vals, s.vals) and torch.equal(res.subs, s.subs)
    srv.close()


@pytest.mark.parametrize("accum", ["fp64", "compensated"])
def test_server_groups_match_oracle(cuda_lib, accum):
    """A burst of requests on two slots forms groups that run as stage-wise
    batches (grouped_runs > 0); every result matches the oracle.  FP64 and
    FP32-stored tensors are mixed; requests on a prepared layout run alone."""
    dev = "cuda"
    g = np.random.default_rng(31)
    tensors = []
    for i, (shape, nnz, f32) in enumerate([((300, 200, 100, 50), 150_000, False), ((400, 30, 500, 60), 60_000, True),
                                           ((1000, 900, 800, 700), 250_000, False), ((40, 50, 60, 70), 30_000, True),
                                           ((2000, 50, 40, 3000), 5_000, False)]):
        t = S.sptenrand(600 + i, shape, nnz, vals="u11")
        v = t.vals.to(torch.float32) if f32 else t.vals
        tensors.append((t.subs.to(dev), v.to(dev), shape))
    srv = cuda_lib.Server(budget_bytes=8 << 30, slots=2)
    ids = [srv.register(s, v, sh) for s, v, sh in tensors]
    srv.prepare(ids[0], [1])
    reqs = []
    for j in range(40):
        ti = int(g.integers(0, len(tensors)))
        shape = tensors[ti][2]
        modes = [1] if (ti == 0 and j % 3 == 0) else [int(m) for m in g.permutation(4)[:1 + j % 2]]
        vecs = [g.uniform(-1, 1, shape[m]).astype(np.float32 if tensors[ti][1].dtype == torch.float32 else np.float64)
                for m in modes]
        reqs.append((ti, modes, vecs))
    rids = [srv.submit(ids[ti], modes, vecs, accum=accum) for ti, modes, vecs in reqs]
    results = [srv.wait(r, timeout_us=60_000_000) for r in rids]
    for k, ((ti, modes, vecs), res) in enumerate(zip(reqs, results)):
        subs, vals, shape = tensors[ti]
        ref, A = oracle_ttv(subs, vals.double(), shape, modes, [v.astype(np.float64) for v in vecs])
        check_result(res, ref, A, what=f"request {k}")
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["pending"] == 0
    assert st["grouped_runs"] > 0, st
    srv.close()


def test_server_wait_any_completion_order(cuda_lib):
    """wait_any hands out every finished request exactly once, whatever the
    order they finish in, each with its own result."""
    dev = "cuda"
    g = np.random.default_rng(37)
    t_big = S.sptenrand(700, (1000, 800, 600, 400), 600_000, vals="u11")
    t_small = S.sptenrand(701, (30, 40, 50, 60), 2_000, vals="u11")
    tensors = [(t_big.subs.to(dev), t_big.vals.to(dev), t_big.shape),
               (t_small.subs.to(dev), t_small.vals.to(dev), t_small.shape)]
    srv = cuda_lib.Server(budget_bytes=8 << 30, slots=2)
    ids = [srv.register(s, v, sh) for s, v, sh in tensors]
    resident = srv.stats()["bytes_in_use"]
    reqs = {}
    for j in range(16):
        ti = 0 if j % 8 == 0 else 1
        m = int(g.integers(0, 4))
        x = g.uniform(-1, 1, tensors[ti][2][m])
        reqs[srv.submit(ids[ti], [m], [x])] = (ti, m, x)
    got = {}
    for k in range(len(reqs)):
        rid, res = srv.wait_any(timeout_us=60_000_000, copy=bool(k % 2))   # views and copies
        assert rid in reqs and rid not in got
        got[rid] = res
    # every result claimed: only the resident tensors hold budget
    assert srv.stats()["bytes_in_use"] == resident
    with pytest.raises(cuda_lib.TTVError) as e:
        srv.wait_any(timeout_us=1000)
    assert e.value.name == "TTV_ERR_TIMEOUT"
    for rid, (ti, m, x) in reqs.items():
        subs, vals, shape = tensors[ti]
        ref, A = oracle_ttv(subs, vals, shape, [m], [x])
        check_result(got[rid], ref, A, what=f"request {rid}")
    srv.close()


def test_server_unclaimed_results_hold_budget_without_deadlock(cuda_lib):
    """Unclaimed results count against the budget; a client that waits by id
    for the last request while earlier results sit unclaimed still gets it
    (with nothing running, the oldest queued request is admitted)."""
    dev = "cuda"
    t = S.sptenrand(710, (400, 300, 500, 200), 300_000, vals="u11")
    subs, vals = t.subs.to(dev), t.vals.to(dev)
    probe = cuda_lib.Server(budget_bytes=8 << 30, slots=1)
    probe.register(subs, vals, t.shape)
    resident = probe.stats()["bytes_in_use"]
    probe.close()
    ws = cuda_lib.workspace_size(subs, vals, t.shape, [1])
    rows, nv = cuda_lib.out_capacity(subs, vals, t.shape, [1])
    need = ws + rows * 3 * 8 + nv * 8 + 4096
    srv = cuda_lib.Server(budget_bytes=resident + int(1.2 * need), slots=2)
    tid = srv.register(subs, vals, t.shape)
    g = np.random.default_rng(41)
    xs = [g.uniform(-1, 1, t.shape[1]) for _ in range(4)]
    rids = [srv.submit(tid, [1], [x]) for x in xs]
    for rid, x in reversed(list(zip(rids, xs))):
        res = srv.wait(rid, timeout_us=60_000_000)
        ref, A = oracle_ttv(subs, vals, t.shape, [1], [x])
        check_result(res, ref, A)
    st = srv.stats()
    assert st["completed"] == 4 and st["bytes_in_use"] == resident
    srv.close()
