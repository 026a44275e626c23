"""Bounded device waits run out with an error status, not a hang.

Every wait of a kernel on another CTA's progress gives up after a poll limit
and raises a timeout bit that the call reports as TTV_ERR_TIMEOUT.  A test
hook shortens the limit to zero polls, so that the sort's decoupled look-back
and the staged dense kernel's bulk-copy pipeline must run out; the call must
fail with TTV_ERR_TIMEOUT and the next call, with the limits restored, must
match the oracle on the same context.  A probe kernel also waits on an
mbarrier and on a device word that nothing ever completes."""
import pytest

import synthetic as S
from parity import check_result, oracle_ttv, to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [0, 1], ids=["mbarrier", "word"])
def test_probe_wait_runs_out(cuda_lib, kind):
    assert cuda_lib.test_wait_probe(kind, 0) == "TTV_ERR_TIMEOUT"
    assert cuda_lib.test_wait_probe(kind, 1000) == "TTV_ERR_TIMEOUT"


def _expect_timeout_then_recover(ttv, p, layout, **kw):
    subs, vals, vecs = to_device(p, layout=layout)
    ref, A = oracle_ttv(subs, vals, p.tensor.shape, p.modes, vecs, dense=kw.get("fmt") == "dense")
    ttv.test_set_wait_polls(0)
    try:
        with pytest.raises(ttv.TTVError) as e:
            ttv.ttv_multi(subs, vals, p.tensor.shape, p.modes, vecs, **kw)
        assert e.value.name == "TTV_ERR_TIMEOUT"
    finally:
        ttv.test_set_wait_polls(-1)
    res = ttv.ttv_multi(subs, vals, p.tensor.shape, p.modes, vecs, **kw)
    check_result(res, ref, A, dense=kw.get("fmt") == "dense", what="after a timeout")


def test_sort_lookback_runs_out_then_recovers(cuda_lib):
    t = S.sptenrand(61, (300, 200, 100, 50), 200_000, vals="u11")
    p = S.Problem(t, [1, 2], [S.vector(61, m, t.shape[m]) for m in (1, 2)])
    _expect_timeout_then_recover(cuda_lib, p, "soa", path="sort")


def test_staged_dense_pipeline_runs_out_then_recovers(cuda_lib):
    t = S.sptenrand(62, (100, 80, 25, 40), 1_400_000, vals="u11")
    p = S.Problem(t, [0, 1, 3], [S.vector(62, m, t.shape[m]) for m in (0, 1, 3)])
    subs, vals, vecs = to_device(p, layout="soa")
    cuda_lib.tune_clear()
    try:
        # pin the bulk-staged persistent kernel for this problem class
        cuda_lib.tune_set(subs, vals, p.tensor.shape, p.modes, "dense", 1, 4, fmt="dense")
        _expect_timeout_then_recover(cuda_lib, p, "soa", fmt="dense")
    finally:
        cuda_lib.tune_clear()
