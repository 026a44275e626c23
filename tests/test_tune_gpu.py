"""Autotuner on the GPU: it times the applicable plans, records the fastest
for the problem class, AUTO then runs that plan, and results still match
the oracle."""
import pytest
import torch

import paper_2510_01495_gb300 as ttv
import synthetic as S
from parity import check_result, oracle_ttv, to_device

pytestmark = pytest.mark.gpu

# kernel that shows which path ran
MARK = {"dense": "dense_accum", "sort": "keys_terms", "hash": "hash_insert", "bucket": "bkt_part1"}


@pytest.fixture()
def clean():
    ttv.tune_clear()
    yield
    ttv.tune_clear()


def kernels_of(fn):
    ttv.profile_reset()
    ttv.profile_enable(True)
    r = fn()
    torch.cuda.synchronize()
    ttv.profile_collect()
    ttv.profile_enable(False)
    return r, set(ttv.profile_names())


@pytest.mark.parametrize("case", [
    ((300, 300, 300), 200_000, [0], "sparse"),         # direct table vs sort
    ((200, 300, 400, 500), 150_000, [1], "sparse"),    # hashed table vs sort vs bucket
    ((40, 50, 60), 60_000, [0, 2], "sparse"),          # dense accumulator candidates
    ((300, 300, 300), 200_000, [1], "dense"),
])
def test_autotune_then_auto(cuda_lib, clean, case):
    shape, nnz, modes, fmt = case
    t = S.sptenrand(7 + nnz, shape, nnz, vals="u11")
    p = S.Problem(t, list(modes), [S.vector(7, m, shape[m]) for m in modes], name="tune")
    subs, vals, vecs = to_device(p, layout="soa")
    res = ttv.autotune(subs, vals, shape, modes, vecs, fmt=fmt, trials=3)
    names = {c["path"] for c in res["candidates"]}
    assert res["path"] in names and res["ms"] == min(c["ms"] for c in res["candidates"])
    assert ttv.tune_count() == 1
    r, ks = kernels_of(lambda: ttv.ttv_multi(subs, vals, shape, modes, vecs, fmt=fmt))
    assert MARK[res["path"]] in ks, (res, ks)
    dense = fmt == "dense"
    ref, A = oracle_ttv(subs, vals, shape, modes, vecs, dense=dense)
    check_result(r, ref, A, dense=dense, what=f"tuned {res['path']}")
    # a deterministic call ignores the record and sorts
    if not dense and res["path"] != "dense":
        _, ks = kernels_of(lambda: ttv.ttv_multi(subs, vals, shape, modes, vecs, fmt=fmt, deterministic=True))
        assert "keys_terms" in ks


def test_autotune_rejects_deterministic(cuda_lib, clean):
    p = S.Problem(S.sptenrand(3, (30, 40, 50), 5_000), [1], [S.vector(3, 1, 40)], name="d")
    subs, vals, vecs = to_device(p)
    with pytest.raises(ttv.TTVError) as e:
        ttv.autotune(subs, vals, (30, 40, 50), [1], vecs, deterministic=True)
    assert e.value.name == "TTV_ERR_ARG"
    assert ttv.tune_count() == 0


def test_tuned_record_survives_save_load(cuda_lib, clean, tmp_path):
    shape, modes = (300, 300, 300), [0]
    p = S.Problem(S.sptenrand(9, shape, 100_000), modes, [S.vector(9, 0, 300)], name="s")
    subs, vals, vecs = to_device(p, layout="soa")
    res = ttv.autotune(subs, vals, shape, modes, vecs, trials=2)
    f = tmp_path / "t.tune"
    ttv.tune_save(str(f))
    ttv.tune_clear()
    ttv.tune_load(str(f))
    assert ttv.tune_count() == 1
    _, ks = kernels_of(lambda: ttv.ttv_multi(subs, vals, shape, modes, vecs))
    assert MARK[res["path"]] in ks
