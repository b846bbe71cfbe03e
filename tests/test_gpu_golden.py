"""Full-size parity: the whole bench box of a workload, checked by the CUDA
library in each precision, against stored results of the FP64 CPU oracle over
the same box (tests/golden/make_goldens.py writes them with oracle.verify only).

Bit-exact: class D, point count, adversarial count (Eq. 10), first witness,
tie count and tie list, the verdict bitmap (SHA-256 of its words), the
sign-change masks and tie masks in full, and the SS-Cover masks (Sec. III-B)
by SHA-256 and popcount. Each precision runs its full chain of passes (screen,
split tensor pass, FP32, double-float, FP64)."""
import hashlib
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDENS = {
    "config2": os.path.join(HERE, "golden", "config2_mlp784x512x512_s6k7.json"),
    "config3": os.path.join(HERE, "golden", "config3_mlp784x1024x3_s5k15.json"),
}


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


def load(name):
    path = GOLDENS[name]
    if not os.path.exists(path):
        pytest.skip(f"{os.path.basename(path)} not generated (tests/golden/make_goldens.py {name})")
    return json.load(open(path))


def check(vb, g, precision):
    w = synth.workload(g["workload"])
    net, q = w["net"], w["query"]
    assert [int(p) for p in q["pixels"]] == g["pixels"] and int(q["k"]) == g["k"]
    n = g["space"]
    vnet = vb.Net(net)
    res = vb.Result(vnet, max_points=n, max_s=g["s"], max_k=g["k"], ties_cap=1 << 16, queue_cap=n)
    s = vb.verify_query(vnet, res, q["image"], q["pixels"], q["k"], precision=precision)
    cov = vb.get_coverage(res)
    bm = vb.get_verdict_bitmap(res, n)
    ties = vb.get_ties(res)
    res.free()
    vnet.free()
    assert s["D"] == g["D"]
    assert s["n_points"] == g["n_points"] == n
    assert s["n_adversarial"] == g["n_adversarial"], (precision, s["n_adversarial"], g["n_adversarial"])
    assert s["first_witness"] == g["first_witness"]
    assert s["n_ties"] == g["n_ties"]
    assert [int(t) for t in np.sort(ties)] == g["ties"]
    assert digest(bm[:(n + 31) // 32]) == g["bitmap"]
    assert [int(x) for x in cov["flip"]] == g["flip"]
    assert [int(x) for x in cov["flip_tie"]] == g["flip_tie"]
    assert digest(cov["ss"]) == g["ss"], precision
    assert digest(cov["ss_tie"]) == g["ss_tie"], precision
    return s


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp32", "fp8"])
def test_config2_whole_box_equals_oracle(vb, precision):
    """784-512-512-10 ReLU, s = 6, k = 7: all 11,390,625 points."""
    g = load("config2")
    check(vb, g, precision)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_config3_whole_box_equals_oracle(vb, precision):
    """784-1024-1024-1024-10 ReLU, s = 5, k = 15: all 28,629,151 points."""
    g = load("config3")
    check(vb, g, precision)


def test_golden_files_were_written_by_the_oracle_script():
    """The stored values name the oracle run that made them (not a GPU run)."""
    for name, path in GOLDENS.items():
        if os.path.exists(path):
            g = json.load(open(path))
            assert g["what"].startswith("oracle.verify over the whole box")
            assert g["n_points"] == g["space"]
