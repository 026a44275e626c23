"""The hand-worked examples (tests/golden/) on every CUDA path: exact small
integers, so every accumulation order gives them bit for bit."""
import json
import os

import pytest
import torch

import paper_2510_01495_gb300 as ttv

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("path", ["auto", "dense", "sort", "hash"])
@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_eq3_cases(cuda_lib, path, layout):
    g = load("hand_worked_eq3.json")
    t = g["tensor"]
    subs = torch.tensor(t["subs"], dtype=torch.int64, device="cuda")
    if layout == "soa":
        subs = subs.t().contiguous().t()
    vals = torch.tensor(t["vals"], dtype=torch.float64, device="cuda")
    for c in g["cases"]:
        vecs = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in c["vecs"]]
        r = ttv.ttv_multi(subs, vals, t["shape"], c["modes"], vecs, path=path)
        assert r.shape == tuple(c["shape"]), c["what"]
        assert r.vals.cpu().tolist() == c["vals"], (path, c["what"])
        if c["shape"]:
            assert r.subs.cpu().tolist() == c["subs"], (path, c["what"])
        if c["shape"] and len(c["modes"]) > 0:
            prep = ttv.Prepared(subs, vals, t["shape"], c["modes"])
            rp = prep.run(vecs)
            assert rp.vals.cpu().tolist() == c["vals"] and rp.subs.cpu().tolist() == c["subs"], c["what"]
            prep.close()


@pytest.mark.parametrize("path", ["auto", "dense", "sort", "hash"])
def test_duplicates_and_zero(cuda_lib, path):
    c = load("hand_worked_eq3.json")["duplicates_and_zero"]
    r = ttv.ttv_multi(torch.tensor(c["subs"], dtype=torch.int64, device="cuda"),
                      torch.tensor(c["vals"], dtype=torch.float64, device="cuda"), c["shape"], c["modes"],
                      [torch.tensor(x, dtype=torch.float64, device="cuda") for x in c["vecs"]], path=path)
    assert r.subs.cpu().tolist() == c["out_subs"] and r.vals.cpu().tolist() == c["out_vals"], path
    assert r.shape == tuple(c["out_shape"])


def test_dense_kernels_and_mttkrp(cuda_lib):
    g = load("hand_worked_dense_mttkrp.json")
    dev = "cuda"
    d = ttv.dot(torch.tensor(g["dot"]["x"], device=dev, dtype=torch.float64),
                torch.tensor(g["dot"]["y"], device=dev, dtype=torch.float64))
    assert float(d.cpu()) == g["dot"]["value"]
    A = torch.tensor(g["matvec"]["A"], device=dev, dtype=torch.float64)
    x = torch.tensor(g["matvec"]["x"], device=dev, dtype=torch.float64)
    assert ttv.matvec(A, x).cpu().tolist() == g["matvec"]["y"]
    assert ttv.matvec(A.t().contiguous().t(), x).cpu().tolist() == g["matvec"]["y"]
    m = g["mttkrp"]
    t = m["tensor"]
    facs = [torch.tensor(m["factors"][str(k)], device=dev, dtype=torch.float64) if str(k) in m["factors"] else None
            for k in range(3)]
    M = ttv.mttkrp(torch.tensor(t["subs"], dtype=torch.int64, device=dev),
                   torch.tensor(t["vals"], dtype=torch.float64, device=dev), t["shape"], m["mode"], facs)
    assert M.cpu().tolist() == m["M"]
