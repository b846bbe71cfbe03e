"""The time budget of a verify call (the bounded effort of an incremental check,
which runs until it exhausts its time, Sec. II-B): the first pass takes its tiles
in index order and stops taking them when the budget is spent; every tile taken
is finished, so the result is exact for the checked prefix [lo, checked_hi),
and a call from lo = checked_hi finishes the box. The two results merge (sums,
smallest witness, bitwise or) into the whole box's, which the FP64 oracle
fixes (the stored golden of the config-2 box, and the oracle over the prefix)."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "config2_mlp784x512x512_s6k7.json")


@pytest.fixture(scope="module")
def vb():
    import torch
    assert torch.cuda.is_available()
    import paper_1907_12933_gb300 as m
    from paper_1907_12933_gb300 import build
    build.build()
    return m


def digest(words):
    w = np.ascontiguousarray(words, dtype="<u4")
    return {"sha256": hashlib.sha256(w.tobytes()).hexdigest(), "words": int(w.size),
            "popcount": int(np.unpackbits(w.view(np.uint8)).sum())}


def run(vb, vnet, res, q, n, precision, lo=0, budget=0.0):
    try:
        s = vb.verify_query(vnet, res, q["image"], q["pixels"], q["k"], lo=lo, hi=n,
                            precision=precision, time_budget_ms=budget)
        timed_out = False
    except vb.VbmcTimeout as e:
        s, timed_out = e.summary, True
    out = {"s": s, "timed_out": timed_out, "bitmap": vb.get_verdict_bitmap(res, n),
           "ties": np.sort(vb.get_ties(res))}
    out.update(vb.get_coverage(res))
    return out


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_budget_prefix_then_resume_equals_the_whole_box(vb, precision):
    g = json.load(open(GOLDEN))
    w = synth.workload(g["workload"])
    net, q = w["net"], w["query"]
    n = g["space"]
    vnet = vb.Net(net)
    res = vb.Result(vnet, max_points=n, max_s=6, max_k=7, ties_cap=1 << 16, queue_cap=n)
    vb.verify_query(vnet, res, q["image"], q["pixels"], q["k"], precision=precision)  # warm-up
    # a budget that ends inside the first pass (the set-up before it takes a
    # fraction of a millisecond): the smallest of these that checks something
    for budget in (0.6, 1.0, 2.0, 4.0):
        a = run(vb, vnet, res, q, n, precision, budget=budget)
        if a["s"]["checked_hi"] > 0:
            break
    assert a["timed_out"], a["s"]
    cut = a["s"]["checked_hi"]
    assert 0 < cut < n and a["s"]["verdict"] == "PARTIAL" and a["s"]["n_points"] == cut
    # the prefix is exact: the oracle over [0, cut)
    o = oracle.verify(net, q, lo=0, hi=cut)
    assert a["s"]["n_adversarial"] == o["n_adv"] and a["s"]["first_witness"] == o["first_witness"]
    assert a["s"]["n_ties"] == o["n_ties"]
    nw = (cut + 31) // 32
    np.testing.assert_array_equal(a["bitmap"][:nw], o["bitmap"][:nw])
    for key in ("flip", "flip_tie", "ss", "ss_tie"):
        np.testing.assert_array_equal(a[key], o[key], err_msg=key)
    # resume from the cut without a budget, then merge the two ranges
    b = run(vb, vnet, res, q, n, precision, lo=cut)
    assert not b["timed_out"] and b["s"]["checked_hi"] == n
    firsts = [x for x in (a["s"]["first_witness"], b["s"]["first_witness"]) if x is not None]
    assert a["s"]["n_adversarial"] + b["s"]["n_adversarial"] == g["n_adversarial"]
    assert min(firsts) == g["first_witness"]
    assert a["s"]["n_ties"] + b["s"]["n_ties"] == g["n_ties"]
    assert sorted(np.concatenate([a["ties"], b["ties"]]).tolist()) == g["ties"]
    assert digest((a["bitmap"] | b["bitmap"])[:(n + 31) // 32]) == g["bitmap"]
    assert [int(x) for x in (a["flip"] | b["flip"])] == g["flip"]
    assert digest(a["ss"] | b["ss"]) == g["ss"]
    res.free()
    vnet.free()


def test_budget_spent_before_the_first_tile(vb):
    """A budget of one nanosecond is over before the first pass claims a tile: the
    call reports the empty prefix, with nothing counted."""
    w = synth.workload("mlp784x512x512_relu_s6k7", s=3)
    net, q = w["net"], w["query"]
    n = oracle.space_size(3, q["k"])
    vnet = vb.Net(net)
    res = vb.Result(vnet, max_points=n, max_s=3, max_k=q["k"], queue_cap=n)
    a = run(vb, vnet, res, q, n, "bf16", lo=40, budget=1e-6)
    assert a["timed_out"] and a["s"]["checked_hi"] == 40
    assert a["s"]["n_points"] == 0 and a["s"]["n_adversarial"] == 0 and a["s"]["first_witness"] is None
    assert not a["bitmap"].any() and not a["flip"].any()
    res.free()
    vnet.free()
