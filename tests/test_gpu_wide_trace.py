"""Per-layer error of the wide-layer tensor path (E4M3, BF16) against the FP64
oracle: the operand each hidden layer hands to the next (the rounded activation
delta dh_l, dequantized) lies within the path's own proven bound R_l + E_l of
the exact dh_l, point by point and layer by layer. Prints the per-layer error
and bound relative to ||dh_l||."""
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


def relu(x):
    return np.maximum(x, 0.0)


@pytest.mark.parametrize("prec", ["fp8", "bf16"])
@pytest.mark.parametrize("case", ["config3", "active"])
def test_operands_within_bound(vb, prec, case):
    if case == "config3":
        w = synth.workload("mlp784x1024x3_relu_s5k15", s=3, k=15)
        net, q = w["net"], w["query"]
    else:
        net = synth.make_net(94, [32, 256, 512, 256, 6], "relu", 2.0, "normal")
        q = synth.make_query(94, 0, 32, 3, 40)
    dims, L = net["dims"], len(net["dims"]) - 1
    n = 96
    vnet = vb.Net(net)
    res = vb.Result(vnet, max_points=0, max_s=3, max_k=int(q["k"]), queue_cap=1 << 16)
    vals, nre = vb.wide_trace(vnet, res, q["image"], q["pixels"], int(q["k"]), prec, n)
    summ = vb.result_summary(res)
    o = oracle.verify(net, q, hi=n, bitmap=False, coverage=False)
    assert summ["n_adversarial"] == o["n_adv"] and summ["first_witness"] == o["first_witness"]
    u0 = oracle.forward(net, np.asarray(q["image"], np.float64) / 255.0)
    noff = np.concatenate([[0], np.cumsum(dims[1:])])
    rel_err = np.zeros((L - 1, n))
    rel_bnd = np.zeros((L - 1, n))
    for i in range(n):
        u = oracle.eval_point(net, q, i)["u"]
        for l in range(1, L):
            a, H = noff[l - 1], dims[l]
            dh = relu(u[a:a + H]) - relu(u0[a:a + H])
            err = float(np.linalg.norm(vals[l - 1, i, :H].astype(np.float64) - dh))
            N, R, E = (float(x) for x in nre[l - 1, i])
            assert err <= R + E + 1e-12, (l, i, err, R, E)
            assert N + E >= float(np.linalg.norm(dh)) - 1e-12
            nd = max(float(np.linalg.norm(dh)), 1e-30)
            rel_err[l - 1, i] = err / nd
            rel_bnd[l - 1, i] = (R + E) / nd
    for l in range(1, L):
        print(f"{case} {prec} layer {l}: error/||dh|| median {np.median(rel_err[l - 1]):.3e} "
              f"max {rel_err[l - 1].max():.3e}; bound/||dh|| median {np.median(rel_bnd[l - 1]):.3e} "
              f"max {rel_bnd[l - 1].max():.3e}")
    res.free()
