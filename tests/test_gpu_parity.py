"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Sizes are small enough for the oracle to finish in seconds while spanning many
tiles with ragged tails; the full-size bench workload is checked on sampled
points and invariants."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import compare, run_gpu
from test_oracle_pins import BRUTE, net222, small_relu_case

pytestmark = pytest.mark.gpu

PLAIN = ["fp64", "fp32"]


@pytest.fixture(scope="module")
def vb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1907_12933_gb300 as m
    from paper_1907_12933_gb300 import build
    build.build()
    return m


@pytest.mark.parametrize("prec", PLAIN)
def test_hand_222(vb, prec):
    net = net222()
    q = {"image": np.array([104, 100], np.uint8), "pixels": np.array([0, 1], np.int32), "k": 3}
    g = run_gpu(vb, net, q, prec)
    o = oracle.verify(net, q)
    compare(g, o, net, q)
    assert g["summary"]["verdict"] == "UNSAFE" and g["summary"]["first_witness"] == 6
    if prec == "fp32":
        # the exact zeros (ties) cannot be decided in fp32: they reach the FP64 pass
        assert g["summary"]["n_recheck"][3] >= 9


@pytest.mark.parametrize("prec", PLAIN)
@pytest.mark.parametrize("case", range(len(BRUTE)))
def test_bruteforce_fixtures(vb, prec, case):
    act, _, seed, wvar, k = BRUTE[case]
    net = synth.make_net(seed, [3, 5, 4, 3], act, wvar, "normal")
    q = synth.make_query(seed, 0, 3, 2, k)
    compare(run_gpu(vb, net, q, prec), oracle.verify(net, q), net, q)


@pytest.mark.parametrize("prec", PLAIN)
def test_active_small_relu(vb, prec):
    """6-8-6-4 ReLU, s = 3, k = 30: 226,981 points with sign changes, SS pairs and
    adversarial points; 3547 tiles of 64 with a ragged last tile."""
    net, q = small_relu_case(k=30)
    g = run_gpu(vb, net, q, prec)
    o = oracle.verify(net, q)
    assert o["n_adv"] > 0 and o["ss"].any()
    compare(g, o, net, q)


def test_config1_full(vb):
    """25-10-5 sigmoid, s = 5, k = 8: all 1,419,857 points."""
    w = synth.workload("mlp25_sigmoid_s5k8")
    g = run_gpu(vb, w["net"], w["query"], "fp32")
    compare(g, oracle.verify(w["net"], w["query"]), w["net"], w["query"])


@pytest.mark.parametrize("prec", PLAIN)
def test_config2_net_small_box(vb, prec):
    """784-512-512-10 ReLU net, s = 3, k = 7 (3375 points), plus a ragged sub-range."""
    w = synth.workload("mlp784x512x512_relu_s6k7", s=3)
    net, q = w["net"], w["query"]
    compare(run_gpu(vb, net, q, prec), oracle.verify(net, q), net, q)
    g = run_gpu(vb, net, q, prec, lo=17, hi=3001)
    o = oracle.verify(net, q, lo=17, hi=3001)
    assert g["summary"]["verdict"] == "PARTIAL"
    compare(g, o, net, q)


def test_config2_net_active_box(vb):
    """Same net, 2 pixels moved by up to 40 grey levels: hidden sign changes occur."""
    w = synth.workload("mlp784x512x512_relu_s6k7", s=2, k=40)
    net, q = w["net"], w["query"]
    o = oracle.verify(net, q)
    assert o["flip"].any()
    compare(run_gpu(vb, net, q, "fp32"), o, net, q)


def test_config3_net_small_box(vb):
    """784-1024-1024-1024-10 ReLU net, s = 2, k = 15 (961 points)."""
    w = synth.workload("mlp784x1024x3_relu_s5k15", s=2)
    net, q = w["net"], w["query"]
    compare(run_gpu(vb, net, q, "fp32"), oracle.verify(net, q), net, q)


@pytest.mark.parametrize("prec,graph,schedule", [("fp32", False, "given"), ("bf16", False, "given"),
                                                 ("bf16", True, "small_first"),
                                                 ("fp32", False, "small_first"),
                                                 ("fp64", False, "given")])
def test_config4_net_batch(vb, prec, graph, schedule):
    """784-256-256-10 ReLU net, 24 uneven queries through one vbmc_verify_batch call
    (one launch per pass over every query), each checked against the oracle; with
    the smallest-first schedule the tiles run in another order than the results."""
    w = synth.workload("mlp784x256x256_relu_batch4096", nq=24, s_range=(1, 3), k_range=(3, 10))
    net = w["net"]
    vnet = vb.Net(net)
    qs = w["queries"]
    nmax = max(oracle.space_size(len(q["pixels"]), q["k"]) for q in qs)
    results = vb.result_create_batch(vnet, len(qs), max_points=nmax, max_s=3, max_k=10,
                                     queue_cap=1 << 18)
    sums = vb.verify_batch(vnet, results, qs, precision=prec, coverage=True, bitmap=True,
                           graph=graph, schedule=schedule)
    for q, r, s in zip(qs, results, sums):
        o = oracle.verify(net, q)
        g = {"summary": s, "n": oracle.space_size(len(q["pixels"]), q["k"])}
        g.update(vb.get_coverage(r))
        g["bitmap"] = vb.get_verdict_bitmap(r, g["n"])
        g["ties"] = np.sort(vb.get_ties(r))
        g["witness"] = vb.get_witness(r, len(q["pixels"]), 784)
        compare(g, o, net, q)
        assert 0.0 < s["ms_to_verdict"] <= s["ms_device"] + 1e-3
    for r in results:
        r.free()


def batch_check(vb, net, qs, results, sums):
    for q, r, s in zip(qs, results, sums):
        o = oracle.verify(net, q)
        g = {"summary": s, "n": oracle.space_size(len(q["pixels"]), q["k"])}
        g.update(vb.get_coverage(r))
        g["bitmap"] = vb.get_verdict_bitmap(r, g["n"])
        g["ties"] = np.sort(vb.get_ties(r))
        g["witness"] = vb.get_witness(r, len(q["pixels"]), 784)
        compare(g, o, net, q)


def test_config4_wide_queries_and_graph_reuse(vb):
    """Queries of the batch workload with s = 4..6 pixels (small k), in one batch
    arena: the graph captured by the first call is relaunched by the second (same
    shapes) and captured again for a batch of other shapes; every result against
    the oracle each time."""
    w = synth.workload("mlp784x256x256_relu_batch4096", nq=20, s_range=(4, 6), k_range=(1, 2))
    net = w["net"]
    vnet = vb.Net(net)
    qs = w["queries"]
    assert {len(q["pixels"]) for q in qs} == {4, 5, 6}
    other = synth.workload("mlp784x256x256_relu_batch4096", nq=20, s_range=(3, 6), k_range=(1, 3),
                           seed=2004)["queries"]
    nmax = max(oracle.space_size(len(q["pixels"]), q["k"]) for q in qs + other)
    results = vb.result_create_batch(vnet, len(qs), max_points=nmax, max_s=6, max_k=3, queue_cap=1 << 20)
    for _ in range(2):
        sums = vb.verify_batch(vnet, results, qs, precision="bf16", coverage=True, bitmap=True,
                               graph=True, schedule="small_first")
        batch_check(vb, net, qs, results, sums)
    sums = vb.verify_batch(vnet, results, other, precision="bf16", coverage=True, bitmap=True,
                           graph=True, schedule="small_first")
    batch_check(vb, net, other, results, sums)
    for r in results:
        r.free()


@pytest.mark.parametrize("prec", PLAIN)
def test_edge_cases(vb, prec):
    net, q = small_relu_case(k=4)
    # k = 0: one point, the unperturbed image
    g = run_gpu(vb, net, dict(q, k=0), prec)
    assert g["summary"]["n_points"] == 1 and g["summary"]["verdict"] == "SAFE"
    assert not g["flip"].any()
    # s = 0: one point
    q0 = dict(q, pixels=np.zeros(0, np.int32))
    g = run_gpu(vb, net, q0, prec)
    assert g["summary"]["n_points"] == 1 and g["summary"]["n_adversarial"] == 0
    # empty range
    g = run_gpu(vb, net, q, prec, lo=50, hi=50)
    assert g["summary"]["n_points"] == 0 and g["summary"]["first_witness"] is None
    # maximum k for one pixel
    qk = dict(q, pixels=q["pixels"][:1], k=127)
    compare(run_gpu(vb, net, qk, prec), oracle.verify(net, qk), net, qk)


def test_invalid_queries_rejected(vb):
    net, q = small_relu_case(k=4)
    vnet = vb.Net(net)
    res = vb.Result(vnet, max_points=1000, max_s=4, max_k=8)
    with pytest.raises(vb.VbmcError):
        vb.verify_query(vnet, res, q["image"], [0, 0, 1], 4)          # duplicate pixel
    with pytest.raises(vb.VbmcError):
        vb.verify_query(vnet, res, q["image"], [0, 99], 4)            # out of range
    with pytest.raises(vb.VbmcError):
        vb.verify_query(vnet, res, q["image"], q["pixels"], 9)        # k above max_k
    with pytest.raises(vb.VbmcError):
        vb.verify_query(vnet, res, q["image"], q["pixels"], 4, lo=10, hi=5)
    # device-side check of a pixel list passed by device pointer
    import torch
    img = torch.tensor(q["image"], dtype=torch.uint8, device="cuda")
    pix = torch.tensor([1, 1], dtype=torch.int32, device="cuda")
    vb.verify_query_device(vnet, res, img, pix, 2)
    with pytest.raises(vb.VbmcError):
        vb.result_summary(res)


def test_range_split_equals_whole(vb):
    net, q = small_relu_case(k=20)
    n = oracle.space_size(3, 20)
    whole = run_gpu(vb, net, q, "fp32")
    cuts = [0, 33, 4096, 50000, n]
    acc = {k: np.zeros_like(whole[k]) for k in ("flip", "flip_tie", "ss", "ss_tie", "bitmap")}
    n_adv = 0
    firsts = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        p = run_gpu(vb, net, q, "fp32", lo=a, hi=b)
        n_adv += p["summary"]["n_adversarial"]
        if p["summary"]["first_witness"] is not None:
            firsts.append(p["summary"]["first_witness"])
        for k in acc:
            acc[k] |= p[k]
    assert n_adv == whole["summary"]["n_adversarial"]
    assert (min(firsts) if firsts else None) == whole["summary"]["first_witness"]
    for k in acc:
        np.testing.assert_array_equal(acc[k], whole[k])


def test_fullsize_config2_sampled(vb):
    """The bench workload at full size (11,390,625 points) in the bench's launch
    configuration; sampled points against the oracle one by one, plus invariants."""
    w = synth.workload("mlp784x512x512_relu_s6k7")
    net, q = w["net"], w["query"]
    g = run_gpu(vb, net, q, "fp32", queue_cap=1 << 24)
    n = g["n"]
    assert n == 15 ** 6
    o0 = oracle.eval_point(net, q, (n - 1) // 2)
    assert g["summary"]["D"] == o0["D"]
    bm = g["bitmap"]
    bit = lambda t: (int(bm[t // 32]) >> (t % 32)) & 1  # noqa: E731
    assert bit((n - 1) // 2) == 0
    assert sum(bin(int(x)).count("1") for x in bm) == g["summary"]["n_adversarial"]
    ties = set(int(t) for t in g["ties"])
    rng = np.random.default_rng(7)
    sample = list(rng.integers(0, n, 48)) + [0, n - 1, (n - 1) // 2]
    if g["summary"]["first_witness"] is not None:
        sample.append(g["summary"]["first_witness"])
    for t in sample:
        p = oracle.eval_point(net, q, int(t))
        if abs(p["margin"]) < oracle.TAU:
            assert int(t) in ties
        else:
            assert bit(int(t)) == int(p["adversarial"]), t


def test_autotune_cache_and_parity(vb, tmp_path):
    """Tuned launch shapes come back from the cache unchanged, and any shape gives
    the oracle's results (the tuned one and a forced wide variant)."""
    w = synth.workload("mlp784x256x256_relu_batch4096", nq=3, s_range=(2, 2), k_range=(6, 6))
    net = w["net"]
    vnet = vb.Net(net)
    path = str(tmp_path / "tuning.jsonl")
    t1 = vb.autotune(vnet, path)
    assert t1["from_cache"] == 0 and t1["ms_range"] > 0 and t1["ms_df"] > 0
    assert t1["simt_range"] in (2, 3, 4, 5, 6) and t1["simt_gather"] in (2, 3, 4, 5, 6)
    assert t1["df_ctas"] in (2, 4, 8, 16)
    t2 = vb.autotune(vb.Net(net), path)
    assert t2["from_cache"] == 1
    for f in ("simt_range", "simt_range_ctas", "simt_gather", "simt_gather_ctas", "df_ctas"):
        assert t2[f] == t1[f]
    q = w["queries"][0]
    o = oracle.verify(net, q)
    for prec in ("fp32", "bf16"):
        compare(run_gpu(vb, net, q, prec, vbnet=vnet), o, net, q)
    vb.set_tuning(vnet, simt_range=4, simt_range_ctas=1, simt_gather=4, simt_gather_ctas=2, df_ctas=3)
    compare(run_gpu(vb, net, q, "fp32", vbnet=vnet), o, net, q)


WIDTHS = {1: 32, 2: 256, 3: 512, 4: 1024, 5: 512, 6: 256}


@pytest.mark.parametrize("name,s,k", [("mlp784x256x256_relu_batch4096", 3, 8),
                                      ("mlp784x512x512_relu_s6k7", 3, 12)])
def test_every_simt_variant(vb, name, s, k):
    """Each FP32-pass variant that holds the net (forced for ranges and for queued
    points, at 1 and 2 CTAs per SM) gives the oracle's results."""
    w = synth.workload(name, s=s, k=k) if "batch" not in name else None
    if w is None:
        w = synth.workload(name, nq=1, s_range=(s, s), k_range=(k, k))
        net, q = w["net"], w["queries"][0]
    else:
        net, q = w["net"], w["query"]
    o = oracle.verify(net, q)
    vnet = vb.Net(net)
    hmax = max(net["dims"][1:])
    for var in range(1, 7):
        if WIDTHS[var] < hmax:
            continue
        for ctas in (1, 2):
            vb.set_tuning(vnet, simt_range=var, simt_range_ctas=ctas, simt_gather=var, simt_gather_ctas=ctas,
                          df_ctas=4)
            for prec in ("fp32", "bf16"):
                compare(run_gpu(vb, net, q, prec, vbnet=vnet), o, net, q)
