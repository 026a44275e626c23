"""Hand-worked examples (tests/golden/, each with its derivation and the
equation it follows) against the oracle: exact integers, so bit for bit."""
import json
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_eq3_cases():
    g = load("hand_worked_eq3.json")
    t = g["tensor"]
    subs, vals = np.array(t["subs"], dtype=np.int64), np.array(t["vals"])
    for c in g["cases"]:
        s, v, sh = oracle.ttv(subs, vals, t["shape"], c["modes"], [np.array(x) for x in c["vecs"]])
        assert sh == tuple(c["shape"]), c["what"]
        assert v.tolist() == c["vals"], c["what"]
        if c["shape"]:
            assert s.tolist() == c["subs"], c["what"]


def test_duplicates_and_zero():
    c = load("hand_worked_eq3.json")["duplicates_and_zero"]
    s, v, sh = oracle.ttv(np.array(c["subs"], dtype=np.int64), np.array(c["vals"]), c["shape"], c["modes"],
                          [np.array(x) for x in c["vecs"]])
    assert s.tolist() == c["out_subs"] and v.tolist() == c["out_vals"] and sh == tuple(c["out_shape"])


def test_dense_kernels_and_mttkrp():
    g = load("hand_worked_dense_mttkrp.json")
    assert oracle.dot(np.array(g["dot"]["x"]), np.array(g["dot"]["y"])) == g["dot"]["value"]
    assert oracle.matvec(np.array(g["matvec"]["A"]), np.array(g["matvec"]["x"])).tolist() == g["matvec"]["y"]
    m = g["mttkrp"]
    t = m["tensor"]
    facs = [np.array(m["factors"][str(k)]) if str(k) in m["factors"] else None for k in range(3)]
    M = oracle.mttkrp(np.array(t["subs"], dtype=np.int64), np.array(t["vals"]), t["shape"], m["mode"], facs)
    assert M.tolist() == m["M"]
