"""Tensor-core (tcgen05) screens vs the FP64 oracle: BF16 and FP16 operands.

The tensor path only decides points its error bound proves; everything else
falls through to the split (3-product) tensor pass, the FP32 pass and the FP64
pass, so every output must equal the oracle's bit for bit."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import compare, run_gpu

pytestmark = pytest.mark.gpu

TC = ["bf16", "fp16"]


@pytest.fixture(scope="module")
def vb():
    import torch
    assert torch.cuda.is_available()
    import paper_1907_12933_gb300 as m
    from paper_1907_12933_gb300 import build
    build.build()
    return m


@pytest.mark.parametrize("prec", TC)
def test_kind_f16_accumulation_unit(vb, prec):
    """The set-up probe of the kind::f16 MMA (integer tiles, probe sums needing up
    to 24 significand bits, random operands against the model) picks the unit the
    screens' bounds use. On a GB300 the probe sums come back exact and every
    random output lies within the FP32 model, so the unit is 2^-22."""
    w = synth.workload("mlp784x512x512_relu_s6k7", s=1, k=1)
    vnet = vb.Net(w["net"])
    u, worst, failed = vb.tc_accumulation_unit(vnet, prec)
    print(prec, "accumulation unit", u, "worst |err| / (K sum|p|)", worst, "probes failed", bin(failed))
    assert failed == 0 and u == 2.0 ** -22, (u, worst, bin(failed))
    assert 0.0 <= worst <= u
    vnet.free()


def active_tc_case(seed=142, k=25):
    """16-64-64-8 ReLU, three pixels: sign changes in every layer, SS pairs and
    adversarial points (seed 142 picked for that); 132,651 points."""
    net = synth.make_net(seed, [16, 64, 64, 8], "relu", 2.0, "normal")
    return net, synth.make_query(seed, 0, 16, 3, k)


@pytest.mark.parametrize("prec", TC)
def test_active_small_net(vb, prec):
    net, q = active_tc_case()
    o = oracle.verify(net, q)
    assert o["n_adv"] > 0 and o["ss"].any()
    g = run_gpu(vb, net, q, prec)
    compare(g, o, net, q)


@pytest.mark.parametrize("prec", TC)
def test_config2_net_small_box(vb, prec):
    w = synth.workload("mlp784x512x512_relu_s6k7", s=3)
    net, q = w["net"], w["query"]
    compare(run_gpu(vb, net, q, prec), oracle.verify(net, q), net, q)
    g = run_gpu(vb, net, q, prec, lo=17, hi=3001)
    compare(g, oracle.verify(net, q, lo=17, hi=3001), net, q)


@pytest.mark.parametrize("prec", TC)
def test_config2_net_active_box(vb, prec):
    w = synth.workload("mlp784x512x512_relu_s6k7", s=2, k=40)
    net, q = w["net"], w["query"]
    o = oracle.verify(net, q)
    compare(run_gpu(vb, net, q, prec), o, net, q)


def test_config4_net_queries(vb):
    w = synth.workload("mlp784x256x256_relu_batch4096", nq=4, s_range=(2, 3), k_range=(3, 10))
    for q in w["queries"]:
        compare(run_gpu(vb, w["net"], q, "bf16"), oracle.verify(w["net"], q), w["net"], q)


@pytest.mark.parametrize("prec", TC)
def test_edge_cases(vb, prec):
    net, q = active_tc_case(k=4)
    for qq, lo, hi in [(dict(q, k=0), 0, 0), (dict(q, pixels=np.zeros(0, np.int32)), 0, 0),
                       (q, 50, 50), (q, 5, 6), (dict(q, pixels=q["pixels"][:1], k=127), 0, 0)]:
        g = run_gpu(vb, net, qq, prec, lo=lo, hi=hi)
        o = oracle.verify(net, qq, lo=lo, hi=hi)
        compare(g, o, net, qq)


def test_fullsize_config2_bf16_equals_fp32_path(vb):
    """The bench workload (11,390,625 points): the BF16 path and the plain FP32 path
    must give identical verdict bitmaps, counts, ties and coverage masks; sampled
    points are also checked against the oracle one by one."""
    w = synth.workload("mlp784x512x512_relu_s6k7")
    net, q = w["net"], w["query"]
    vnet = vb.Net(net)
    a = run_gpu(vb, net, q, "bf16", queue_cap=1 << 24, vbnet=vnet)
    b = run_gpu(vb, net, q, "fp32", queue_cap=1 << 24, vbnet=vnet)
    for key in ("n_adversarial", "first_witness", "n_ties", "D"):
        assert a["summary"][key] == b["summary"][key], key
    for key in ("bitmap", "flip", "flip_tie", "ss", "ss_tie", "ties"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)
    bm = a["bitmap"]
    rng = np.random.default_rng(11)
    ties = set(int(t) for t in a["ties"])
    for t in list(rng.integers(0, a["n"], 32)) + [a["summary"]["first_witness"] or 0]:
        p = oracle.eval_point(net, q, int(t))
        if abs(p["margin"]) < oracle.TAU:
            assert int(t) in ties
        else:
            assert ((int(bm[int(t) // 32]) >> (int(t) % 32)) & 1) == int(p["adversarial"])
