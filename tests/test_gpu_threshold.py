"""The misclassified literal of Eq. 11 on the GPU against the FP64 oracle, on
every path: one thread per point (small nets), the FP32 SIMT pass, the fused
BF16 tensor screen, the wide-layer E4M3/BF16 screens, the FP64 pass, the
batch, and with a point filter and the k-shell search."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import compare
from test_oracle_pins import small_relu_case
from test_oracle_threshold import reference_v

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1907_12933_gb300 as m
    from paper_1907_12933_gb300 import build
    build.build()
    return m


def run_threshold(vb, net, q, prec, vnet=None, coverage=True):
    s, k = len(q["pixels"]), int(q["k"])
    n = oracle.space_size(s, k)
    vnet = vnet or vb.Net(net)
    res = vb.Result(vnet, max_points=n, max_s=max(1, s), max_k=max(1, k), queue_cap=max(4096, n))
    summ = vb.verify_query(vnet, res, q["image"], q["pixels"], k, precision=prec, coverage=coverage,
                           bitmap=True, filter=q.get("filter", 0), l2_max=q.get("l2_max", 0),
                           threshold=q["threshold"])
    g = {"summary": summ, "n": n}
    if coverage:
        g.update(vb.get_coverage(res))
    g["bitmap"] = vb.get_verdict_bitmap(res, n)
    g["ties"] = np.sort(vb.get_ties(res))
    g["witness"] = vb.get_witness(res, s, net["dims"][0])
    res.free()
    return g


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("alpha", [0.9, 3.0, -1.0])
def test_small_net(vb, prec, alpha):
    net, q = small_relu_case(k=30)
    q = dict(q, property=1, threshold=reference_v(net, q, alpha))
    o = oracle.verify(net, q)
    assert (o["n_adv"] > 0) == (alpha > 0)
    compare(run_threshold(vb, net, q, prec), o, net, q)


def test_small_net_threshold_at_an_output(vb):
    """V equal to y_D at an Eq. 10 witness: that point is a tie of the first
    literal (the oracle and the FP64 pass both list it)."""
    net, q = small_relu_case(k=30)
    t = oracle.verify(net, q)["first_witness"]
    p = oracle.eval_point(net, q, t)
    q = dict(q, property=1, threshold=float(p["u"][-4:][p["D"]]))
    o = oracle.verify(net, q)
    assert t in set(int(x) for x in o["ties"])
    for prec in ("fp32", "fp64"):
        compare(run_threshold(vb, net, q, prec), o, net, q)


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp32"])
@pytest.mark.parametrize("coverage", [True, False])
def test_config2_net(vb, prec, coverage):
    w = synth.workload("mlp784x512x512_relu_s6k7", s=3, k=12)
    net, q = w["net"], w["query"]
    q = dict(q, property=1, threshold=reference_v(net, q, 1.5))
    o = oracle.verify(net, q, coverage=coverage)
    compare(run_threshold(vb, net, q, prec, coverage=coverage), o, net, q, coverage=coverage)


@pytest.mark.parametrize("prec", ["fp8", "bf16"])
def test_wide_net(vb, prec):
    """32-256-512-256-6 ReLU (the wide-layer screen), 3 pixels, k = 30."""
    net = synth.make_net(94, [32, 256, 512, 256, 6], "relu", 2.0, "normal")
    q0 = synth.make_query(94, 0, 32, 3, 30)
    vnet = vb.Net(net)
    for alpha in (0.9, 3.0):
        q = dict(q0, property=1, threshold=reference_v(net, q0, alpha))
        o = oracle.verify(net, q)
        assert o["n_adv"] > 0
        compare(run_threshold(vb, net, q, prec, vnet=vnet), o, net, q)


def test_with_l2_filter(vb):
    net, q = small_relu_case(k=30)
    q = dict(q, property=1, threshold=reference_v(net, q, 3.0), filter=1, l2_max=900)
    compare(run_threshold(vb, net, q, "fp32"), oracle.verify(net, q), net, q)


def test_batch_mixed_properties(vb):
    """Queries of both properties in one batch (one launch per pass)."""
    w = synth.workload("mlp784x256x256_relu_batch4096", nq=6, s_range=(2, 3), k_range=(4, 9))
    net = w["net"]
    qs = []
    for i, q in enumerate(w["queries"]):
        qs.append(dict(q, threshold=reference_v(net, q, 2.0)) if i % 2 else q)
    vnet = vb.Net(net)
    nmax = max(oracle.space_size(len(q["pixels"]), q["k"]) for q in qs)
    results = vb.result_create_batch(vnet, len(qs), max_points=nmax, max_s=3, max_k=9, queue_cap=1 << 18)
    sums = vb.verify_batch(vnet, results, qs, precision="bf16", coverage=True, bitmap=True)
    for q, r, s in zip(qs, results, sums):
        qo = dict(q, property=1) if "threshold" in q else q
        o = oracle.verify(net, qo)
        g = {"summary": s, "n": oracle.space_size(len(q["pixels"]), q["k"])}
        g.update(vb.get_coverage(r))
        g["bitmap"] = vb.get_verdict_bitmap(r, g["n"])
        g["ties"] = np.sort(vb.get_ties(r))
        g["witness"] = vb.get_witness(r, len(q["pixels"]), 784)
        compare(g, o, net, qo)
    for r in results:
        r.free()


def test_shell_search(vb):
    net, q = small_relu_case(k=30)
    V = reference_v(net, q, 3.0)
    k = q["k"]
    first, pts = None, 0
    for r in range(k + 1):
        o = oracle.verify(net, dict(q, k=r, filter=2, property=1, threshold=V))
        pts += o["n_points"]
        if o["n_adv"]:
            first = (r, o)
            break
    assert first is not None
    vnet = vb.Net(net)
    res = vb.Result(vnet, max_points=oracle.space_size(3, k), max_s=3, max_k=k, queue_cap=1 << 20)
    got = vb.shell_search(vnet, res, q["image"], q["pixels"], k, precision="fp32", threshold=V)
    r, o = first
    assert got["points_checked"] == pts
    assert got["radius"] == r and got["n_adversarial"] == o["n_adv"]
    assert got["first_witness"] == o["first_witness"]
