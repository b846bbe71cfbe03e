"""Covering methods over image pairs (vbmc_pair_coverage, Sec. III-B) against
the FP64 oracle: SS, SV, DS, DV, sign changes and their tie masks, and the
Eq. 3-6 fractions."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1907_12933_gb300 as m
    from paper_1907_12933_gb300 import build
    build.build()
    return m


def _pairs(seed, n, h0, moved, step):
    """n pairs: a random image and a copy with `moved` pixels shifted by up to `step`."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 256, (n, h0)).astype(np.uint8)
    b = a.copy()
    for i in range(n):
        pix = rng.choice(h0, moved, replace=False)
        b[i, pix] = np.clip(b[i, pix].astype(int) + rng.integers(-step, step + 1, moved), 0, 255)
    return a, b


@pytest.mark.parametrize("case", [
    ("relu", [16, 32, 24, 8], 60, 4, 80, 1.5, 0.3),
    ("sigmoid", [25, 10, 5], 40, 3, 60, 1.2, 0.05),
    ("relu", [784, 512, 512, 10], 12, 6, 40, 1.3, 0.5),
])
def test_pair_coverage_matches_oracle(vb, case):
    act, dims, n, moved, step, g, d = case
    net = synth.make_net(31, dims, act, 2.0 if act == "relu" else 1.0, "normal")
    a, b = _pairs(7, n, dims[0], moved, step)
    got = vb.pair_coverage(vb.Net(net), a, b, g=g, d=d)
    exp = oracle.pairs_coverage(net, a, b, g=g, d=d)
    for k, v in exp.items():
        np.testing.assert_array_equal(got[k][:len(v)], v, err_msg=k)
    assert exp["ss"].any() or exp["sv"].any() or exp["ds"].any() or exp["dv"].any()
    assert got["ss_fraction"] == oracle.ss_covered_fraction(dims, exp["ss"])
    assert got["ds_fraction"] == oracle.layer_pair_fraction(dims, exp["ds"])
    assert got["dv_fraction"] == oracle.layer_pair_fraction(dims, exp["dv"])


def test_pair_coverage_edge_cases(vb):
    """No pairs: cleared masks. A pair of identical images: nothing changes."""
    net = synth.make_net(31, [16, 32, 24, 8], "relu", 2.0, "normal")
    vnet = vb.Net(net)
    empty = np.zeros((0, 16), np.uint8)
    got = vb.pair_coverage(vnet, empty, empty)
    assert not any(got[k].any() for k in ("flip", "ss", "sv", "ds", "dv"))
    a, _ = _pairs(3, 5, 16, 2, 10)
    got = vb.pair_coverage(vnet, a, a, g=1.5, d=0.5)
    exp = oracle.pairs_coverage(net, a, a, g=1.5, d=0.5)
    for k, v in exp.items():
        np.testing.assert_array_equal(got[k][:len(v)], v, err_msg=k)
    assert not any(got[k].any() for k in ("flip", "ss", "sv", "ds", "dv"))
