"""Wide-layer tensor-core screens (hidden layers of 256..1024 neurons, one layer
per launch): E4M3 with per-channel and per-point scales, and BF16/FP16 where the
fused 16-bit screen does not fit, against the FP64 oracle through the C ABI:
small boxes element by element, several chunks with ragged tails, a net whose
signs change (coverage and SS-Cover), agreement with the FP32 path, and the
full-size 784-1024-1024-1024-10 workload on sampled points."""

import numpy as np
import pytest

import oracle
import synth
from gpu_common import compare, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1907_12933_gb300 as m
    from paper_1907_12933_gb300 import build
    build.build()
    return m


# chunks of 384 points (three 128-point tiles; caps.wide_chunk of the result):
# many chunks, ragged tails
SMALL_CHUNK = 384


def test_accumulation_model(vb):
    """The set-up self-test picks one of the two accumulation models."""
    w = synth.workload("mlp784x1024x3_relu_s5k15", s=1)
    u = vb.fp8_accumulation_unit(vb.Net(w["net"]))
    print("fp8 accumulation unit", u)
    assert u in (2.0 ** -22, 2.0 ** -13)


@pytest.mark.parametrize("prec", ["fp8", "bf16", "fp32"])
def test_no_coverage_matches_oracle(vb, prec):
    """Without coverage the screens skip sign certainty; verdicts still exact."""
    w = synth.workload("mlp784x1024x3_relu_s5k15", s=3, k=6)
    net, q = w["net"], w["query"]
    g = run_gpu(vb, net, q, prec, coverage=False)
    compare(g, oracle.verify(net, q), net, q, coverage=False)


WIDE = ["fp8", "bf16", "fp16"]


@pytest.mark.parametrize("prec", WIDE)
def test_config3_small_box(vb, prec):
    """784-1024-1024-1024-10, s = 2, k = 15 (961 points: 8 tiles, ragged)."""
    w = synth.workload("mlp784x1024x3_relu_s5k15", s=2)
    net, q = w["net"], w["query"]
    g = run_gpu(vb, net, q, prec)
    compare(g, oracle.verify(net, q), net, q)


@pytest.mark.parametrize("prec", WIDE)
def test_config3_many_chunks(vb, prec):
    """s = 3, k = 6 (2197 points in chunks of 384) and a sub-range that starts
    and ends inside chunks."""
    w = synth.workload("mlp784x1024x3_relu_s5k15", s=3, k=6)
    net, q = w["net"], w["query"]
    compare(run_gpu(vb, net, q, prec, wide_chunk=SMALL_CHUNK), oracle.verify(net, q), net, q)
    g = run_gpu(vb, net, q, prec, lo=100, hi=2000, wide_chunk=SMALL_CHUNK)
    compare(g, oracle.verify(net, q, lo=100, hi=2000), net, q)


@pytest.mark.parametrize("prec", WIDE)
def test_active_net_coverage(vb, prec):
    """32-256-512-256-6 ReLU net (seed 94: the smallest base margin of seeds
    70..109), 3 pixels moved by up to 40 grey levels (531,441 points): sign
    changes, SS-Cover pairs and 104,011 adversarial points."""
    net = synth.make_net(94, [32, 256, 512, 256, 6], "relu", 2.0, "normal")
    q = synth.make_query(94, 0, 32, 3, 40)
    o = oracle.verify(net, q)
    assert o["flip"].any() and o["ss"].any() and o["n_adv"] > 0
    g = run_gpu(vb, net, q, prec, wide_chunk=SMALL_CHUNK)
    compare(g, o, net, q)


@pytest.mark.parametrize("prec", ["fp8", "bf16"])
def test_wide_equals_fp32_path(vb, prec):
    """s = 3, k = 15 (29,791 points): the wide tensor path and the plain FP32 path
    give identical results (both exact)."""
    w = synth.workload("mlp784x1024x3_relu_s5k15", s=3)
    net, q = w["net"], w["query"]
    vnet = vb.Net(net)
    a = run_gpu(vb, net, q, prec, vbnet=vnet)
    b = run_gpu(vb, net, q, "fp32", vbnet=vnet)
    for k in ("verdict", "D", "n_points", "n_adversarial", "first_witness", "n_ties"):
        assert a["summary"][k] == b["summary"][k], k
    for k in ("flip", "flip_tie", "ss", "ss_tie", "bitmap", "ties"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("prec", ["fp8", "bf16"])
def test_fullsize_config3_sampled(vb, prec):
    """The full 31^5 = 28,629,151-point workload in the bench's configuration;
    sampled points against the oracle one by one, plus invariants."""
    w = synth.workload("mlp784x1024x3_relu_s5k15")
    net, q = w["net"], w["query"]
    g = run_gpu(vb, net, q, prec, queue_cap=1 << 24)
    n = g["n"]
    assert n == 31 ** 5 and g["summary"]["n_points"] == n
    bm = g["bitmap"]
    bit = lambda t: (int(bm[t // 32]) >> (t % 32)) & 1  # noqa: E731
    assert bit((n - 1) // 2) == 0
    assert sum(bin(int(x)).count("1") for x in bm) == g["summary"]["n_adversarial"]
    ties = set(int(t) for t in g["ties"])
    rng = np.random.default_rng(8)
    sample = list(rng.integers(0, n, 24)) + [0, n - 1, (n - 1) // 2]
    if g["summary"]["first_witness"] is not None:
        sample.append(g["summary"]["first_witness"])
    for t in sample:
        p = oracle.eval_point(net, q, int(t))
        if abs(p["margin"]) < oracle.TAU:
            assert int(t) in ties
        else:
            assert bit(int(t)) == int(p["adversarial"]), t
    assert g["summary"]["D"] == oracle.eval_point(net, q, (n - 1) // 2)["D"]


def test_wide_rejects_unsupported_shapes(vb):
    """Hidden widths must be multiples of 256 up to 1024 (and 96 does not fit the
    fused 16-bit screen either)."""
    net = synth.make_net(5, [16, 96, 6], "relu", 2.0, "normal")
    q = synth.make_query(5, 0, 16, 2, 3)
    vnet = vb.Net(net)
    res = vb.Result(vnet, max_points=49, max_s=2, max_k=3)
    for prec in WIDE:
        with pytest.raises(vb.VbmcError):
            vb.verify_query(vnet, res, q["image"], q["pixels"], 3, precision=prec)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_no_coverage_fused_screen(vb, prec):
    """The fused 16-bit screen (784-512-512-10) without coverage: verdicts exact."""
    w = synth.workload("mlp784x512x512_relu_s6k7", s=3)
    net, q = w["net"], w["query"]
    g = run_gpu(vb, net, q, prec, coverage=False)
    compare(g, oracle.verify(net, q), net, q, coverage=False)
