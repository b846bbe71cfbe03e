"""Point filters on the GPU (Euclidean ball of Eq. 9 on the grid, k-shells)
and the k-shell search, against the FP64 oracle on every path: one thread per
point (small nets), the FP32 SIMT pass, the fused BF16 tensor screen, the
wide-layer E4M3/BF16 screens, the FP64 pass and the batch."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import compare
from test_oracle_pins import small_relu_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1907_12933_gb300 as m
    from paper_1907_12933_gb300 import build
    build.build()
    return m


def run_filtered(vb, net, q, prec, vnet=None):
    s, k = len(q["pixels"]), int(q["k"])
    n = oracle.space_size(s, k)
    vnet = vnet or vb.Net(net)
    res = vb.Result(vnet, max_points=n, max_s=max(1, s), max_k=max(1, k), queue_cap=max(4096, n))
    summ = vb.verify_query(vnet, res, q["image"], q["pixels"], k, precision=prec, coverage=True,
                           bitmap=True, filter=q.get("filter", 0), l2_max=q.get("l2_max", 0))
    g = {"summary": summ, "n": n}
    g.update(vb.get_coverage(res))
    g["bitmap"] = vb.get_verdict_bitmap(res, n)
    g["ties"] = np.sort(vb.get_ties(res))
    g["witness"] = vb.get_witness(res, s, net["dims"][0])
    return g


FILTERS = [dict(filter=1, l2_max=900), dict(filter=2), dict(filter=3, l2_max=1500)]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("f", FILTERS)
def test_small_net(vb, prec, f):
    net, q = small_relu_case(k=30)
    q = dict(q, **f)
    o = oracle.verify(net, q)
    g = run_filtered(vb, net, q, prec)
    assert g["summary"]["n_points"] == o["n_points"] < oracle.space_size(3, 30)
    compare(g, o, net, q)


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("f", FILTERS)
def test_config2_net(vb, prec, f):
    w = synth.workload("mlp784x512x512_relu_s6k7", s=3, k=12)
    net, q = w["net"], dict(w["query"], **f)
    o = oracle.verify(net, q)
    compare(run_filtered(vb, net, q, prec), o, net, q)


@pytest.mark.parametrize("prec", ["fp8", "bf16"])
def test_wide_net(vb, prec):
    w = synth.workload("mlp784x1024x3_relu_s5k15", s=2)
    for f in FILTERS:
        net, q = w["net"], dict(w["query"], **f)
        compare(run_filtered(vb, net, q, prec), oracle.verify(net, q), net, q)


def test_batch_filters(vb):
    w = synth.workload("mlp784x256x256_relu_batch4096", nq=6, s_range=(2, 3), k_range=(4, 9))
    net = w["net"]
    qs = [dict(q, **FILTERS[i % 3]) for i, q in enumerate(w["queries"])]
    vnet = vb.Net(net)
    nmax = max(oracle.space_size(len(q["pixels"]), q["k"]) for q in qs)
    results = vb.result_create_batch(vnet, len(qs), max_points=nmax, max_s=3, max_k=9, queue_cap=1 << 18)
    sums = vb.verify_batch(vnet, results, qs, precision="bf16", coverage=True, bitmap=True)
    for q, r, s in zip(qs, results, sums):
        o = oracle.verify(net, q)
        g = {"summary": s, "n": oracle.space_size(len(q["pixels"]), q["k"])}
        g.update(vb.get_coverage(r))
        g["bitmap"] = vb.get_verdict_bitmap(r, g["n"])
        g["ties"] = np.sort(vb.get_ties(r))
        g["witness"] = vb.get_witness(r, len(q["pixels"]), 784)
        compare(g, o, net, q)
    for r in results:
        r.free()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_shell_search(vb, prec):
    """Shells in order: the first with a witness, its witness on the shell, and
    the points of every shell checked."""
    if prec == "fp32":
        net, q = small_relu_case(k=30)
    else:
        w = synth.workload("mlp784x512x512_relu_s6k7", s=3, k=12)
        net, q = w["net"], w["query"]
    k = q["k"]
    first = None
    pts = 0
    for r in range(k + 1):
        o = oracle.verify(net, dict(q, k=r, filter=2))
        pts += o["n_points"]
        if o["n_adv"]:
            first = (r, o)
            break
    vnet = vb.Net(net)
    s = len(q["pixels"])
    res = vb.Result(vnet, max_points=oracle.space_size(s, k), max_s=s, max_k=k, queue_cap=1 << 20)
    got = vb.shell_search(vnet, res, q["image"], q["pixels"], k, precision=prec)
    assert got["points_checked"] == pts
    if first is None:
        assert got["radius"] is None
    else:
        r, o = first
        assert got["radius"] == r and got["n_adversarial"] == o["n_adv"]
        assert got["first_witness"] == o["first_witness"]
        wit = vb.get_witness(res, s, len(q["image"]))
        assert max(abs(int(x)) for x in wit["steps"]) == r
