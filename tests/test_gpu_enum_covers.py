"""The covering methods of Sec. III-B over the enumeration (vbmc_enum_coverage):
the pairs (unperturbed image, point) of a query's box, against the FP64
oracle's pair covers on the same pairs written out, and against the sign-change
and SS masks of the verification itself."""
import numpy as np
import pytest

import oracle
import synth
from test_oracle_pins import small_relu_case

pytestmark = pytest.mark.gpu

MASKS = ("flip", "flip_tie", "ss", "ss_tie", "sv", "sv_tie", "ds", "ds_tie", "dv", "dv_tie")


@pytest.fixture(scope="module")
def vb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1907_12933_gb300 as m
    from paper_1907_12933_gb300 import build
    build.build()
    return m


def box_pairs(q, keep=None):
    """The pairs (image, perturbed image) of every point of the box, in index order;
    keep(steps) selects points (a filter), None keeps all."""
    s, k = len(q["pixels"]), int(q["k"])
    img = np.asarray(q["image"], np.int64)
    a, b = [], []
    for t in range(oracle.space_size(s, k)):
        steps = [x - k for x in oracle.digits(t, s, k)]
        x = img.copy()
        for p, st in zip(q["pixels"], steps):
            x[p] = min(255, max(0, x[p] + st))
        if keep is None or keep(img, x):
            a.append(img.astype(np.uint8))
            b.append(x.astype(np.uint8))
    return np.array(a), np.array(b)


def run(vb, net, q, g, d, **kw):
    s, k = len(q["pixels"]), int(q["k"])
    vnet = vb.Net(net)
    res = vb.Result(vnet, max_points=0, max_s=max(1, s), max_k=max(1, k))
    out = vb.enum_coverage(vnet, res, q["image"], q["pixels"], k, g=g, d=d, **kw)
    res.free()
    return out


def check(out, ref, dims):
    for key in MASKS:
        np.testing.assert_array_equal(out[key], ref[key], err_msg=key)
    assert out["ss_fraction"] == oracle.ss_covered_fraction(dims, ref["ss"])
    for key in ("ds", "dv"):
        assert out[key + "_fraction"] == oracle.layer_pair_fraction(dims, ref[key])


@pytest.mark.parametrize("k,g,d", [(16, 1.5, 0.1), (12, 1.2, 0.02), (8, 3.0, 2.0)])
def test_small_relu_box(vb, k, g, d):
    net, q = small_relu_case(k=k)
    a, b = box_pairs(q)
    ref = oracle.pairs_coverage(net, a, b, g, d)
    out = run(vb, net, q, g, d)
    assert out["n_points"] == len(a) == oracle.space_size(3, k)
    check(out, ref, net["dims"])
    if k == 16:  # sign, value and distance changes all occur
        assert out["flip"].any() and out["ds"].any() and out["dv"].any() and out["sv"].any()


def test_flip_and_ss_equal_the_verification(vb):
    net, q = small_relu_case(k=20)
    o = oracle.verify(net, q)
    out = run(vb, net, q, 2.0, 1.0)
    for key in ("flip", "flip_tie", "ss", "ss_tie"):
        np.testing.assert_array_equal(out[key], o[key], err_msg=key)


def test_l2_filter(vb):
    net, q = small_relu_case(k=10)
    l2 = 120
    a, b = box_pairs(q, keep=lambda x0, x1: int(((x1 - x0) ** 2).sum()) <= l2)
    ref = oracle.pairs_coverage(net, a, b, 1.5, 0.5)
    out = run(vb, net, q, 1.5, 0.5, filter=1, l2_max=l2)
    assert out["n_points"] == len(a)
    check(out, ref, net["dims"])


def test_sigmoid_net(vb):
    w = synth.workload("mlp25_sigmoid_s5k8", s=3, k=4)
    net, q = w["net"], w["query"]
    a, b = box_pairs(q)
    ref = oracle.pairs_coverage(net, a, b, 1.2, 0.05)
    check(run(vb, net, q, 1.2, 0.05), ref, net["dims"])


def test_wide_net_sub_range(vb):
    w = synth.workload("mlp784x512x512_relu_s6k7", s=2, k=7)
    net, q = w["net"], w["query"]
    a, b = box_pairs(q)
    lo, hi = 17, 190
    ref = oracle.pairs_coverage(net, a[lo:hi], b[lo:hi], 1.3, 0.5)
    out = run(vb, net, q, 1.3, 0.5, lo=lo, hi=hi)
    assert out["n_points"] == hi - lo
    check(out, ref, net["dims"])
