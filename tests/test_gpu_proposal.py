"""Learned tile proposal on the GPU, through the C ABI, against the FP64
reference in oracle/proposal_ref.py and the C oracle: gradients (the gradient
check), scores and tile orders, features, per-tile witness counts, and the
tile-ordered search."""
import numpy as np
import pytest

import oracle
import synth
from oracle import proposal_ref as pr
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _batch(seed, B, F, T):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (B, F)).astype(np.float32)
    lab = (rng.random((B, T)) < 0.2).astype(np.float32)
    lab[0] = 0.0
    lab[1] = 0.0
    lab[1, T - 1] = 1.0
    return X, lab


@pytest.mark.parametrize("dims,B", [((2352, 256, 256, 64), 48), ((70, 33, 17, 5), 13)])
def test_gradient_check_against_fp64_reference(vb, dims, B):
    """FP32 forward/backward kernels vs FP64 backpropagation on the same weights.
    Tolerance: FP32 dot products of length K <= 2352 have a relative error bound
    near K * 2^-24 = 1.4e-4 of sum |terms|; norm-wise 1e-4, element-wise 1e-3
    of the layer's largest gradient."""
    prop = vb.Proposal(dims, max_batch=64, seed=3)
    X, lab = _batch(1, B, dims[0], dims[3])
    loss = prop.grads(_dev(X), _dev(lab), bf16=False)
    P = [prop.params(l) for l in (1, 2, 3)]
    ref_loss, ref = pr.mlp_grads([(p["W"], p["b"]) for p in P], X, lab)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    for l in range(3):
        for g, r in ((P[l]["gW"], ref[l][0]), (P[l]["gb"], ref[l][1])):
            scale = np.abs(r).max()
            assert scale > 0
            assert np.linalg.norm(g - r) <= 1e-4 * np.linalg.norm(r)
            assert np.abs(g - r).max() <= 1e-3 * scale
    prop.free()


def test_train_step_lowers_the_loss(vb):
    dims = (2352, 256, 256, 64)
    prop = vb.Proposal(dims, max_batch=64, seed=4)
    X, lab = _batch(2, 64, dims[0], dims[3])
    dX, dT = _dev(X), _dev(lab)
    first = prop.grads(dX, dT, bf16=True)
    for _ in range(30):
        prop.train_step(dX, dT, 1e-3, 0.0)
    assert prop.grads(dX, dT, bf16=True) < 0.75 * first
    prop.free()


def test_scores_and_order(vb):
    """BF16 inference forward vs the FP64 forward (BF16 rounds each operand by at
    most 2^-9 relative; 5% of the score range is far above the accumulated effect
    here), and the tile order exactly as the ranking rule gives it."""
    import torch
    dims = (2352, 256, 256, 64)
    prop = vb.Proposal(dims, max_batch=256, seed=5)
    X, _ = _batch(3, 200, dims[0], dims[3])
    X = np.abs(X) * 0.3
    sc = torch.empty((200, 64), dtype=torch.float32, device="cuda")
    od = torch.empty((200, 64), dtype=torch.int32, device="cuda")
    prop.scores(_dev(X), sc, od)
    z = sc.cpu().numpy()
    order = od.cpu().numpy()
    P = [prop.params(l) for l in (1, 2, 3)]
    zr = pr.mlp_forward([(p["W"], p["b"]) for p in P], X)[-1]
    assert np.abs(z - zr).max() <= 0.05 * (np.abs(zr).max() + 1.0)
    for i in range(200):
        exp = sorted(range(64), key=lambda t: (-z[i, t], t))
        assert list(order[i]) == exp
    prop.free()


def test_features_match_reference(vb):
    import torch
    w = synth.workload("mlp784x512x512_relu_s6k7")
    net = w["net"]
    vnet = vb.Net(net)
    qs = [synth.make_query(1005, i, 784, 6, 7) for i in range(6)]
    qs.append(synth.make_query(1005, 99, 784, 3, 12))
    qs.append(dict(synth.make_query(1005, 98, 784, 1, 4)))
    from paper_1907_12933_gb300 import proposal as P
    X, reach, margin = P.features(vnet, qs, 784)
    Xh = X.cpu().numpy()
    for i, q in enumerate(qs):
        f = pr.features(net, q)
        F = f["features"]
        np.testing.assert_allclose(Xh[i, :784], F[:784], rtol=0, atol=1e-7)
        np.testing.assert_allclose(Xh[i, 784:1568], F[784:1568], rtol=1e-6, atol=0)
        np.testing.assert_allclose(Xh[i, 1568:], F[1568:], rtol=2e-3, atol=1e-5)
        assert reach[i] == pytest.approx(f["reach"], rel=2e-3)
        assert margin[i] == pytest.approx(f["margin"], rel=1e-3, abs=1e-5)
    torch.cuda.synchronize()


def _oracle_counts(o, n, T):
    bits = np.unpackbits(o["bitmap"].view(np.uint8), bitorder="little")[:n]
    return np.array([bits[slice(*pr.tile_bounds(n, T, i))].sum() for i in range(T)]), bits


@pytest.mark.parametrize("T", [64, 7, 1000])
def test_tile_counts_match_oracle(vb, T):
    net, q = small_relu_case(k=30)
    n = oracle.space_size(3, 30)
    vnet = vb.Net(net)
    res = vb.Result(vnet, max_points=n, max_s=3, max_k=30)
    vb.verify_query(vnet, res, q["image"], q["pixels"], q["k"], precision="fp32", bitmap=True)
    got = vb.tile_counts(res, T)
    o = oracle.verify(net, q)
    exp, _ = _oracle_counts(o, n, T)
    assert exp.sum() == o["n_adv"] > 0
    np.testing.assert_array_equal(got, exp)


def _check_search(vb, vnet, res, net, q, order, prec, o, T):
    n = oracle.space_size(len(q["pixels"]), q["k"])
    counts, bits = _oracle_counts(o, n, T)
    r = vb.search_query(vnet, res, q["image"], q["pixels"], q["k"], order, precision=prec)
    hits = [i for i, t in enumerate(order) if counts[t] > 0]
    if not hits:
        assert r["witness_tile"] is None and r["tiles_checked"] == T
        assert r["verdict"] == ("TIES_ONLY" if o["n_ties"] else "SAFE") and r["n_points"] == n
        assert r["n_ties"] == o["n_ties"]
        return r
    pos = hits[0]
    t = order[pos]
    lo, hi = pr.tile_bounds(n, T, t)
    assert r["witness_tile"] == t and r["tiles_checked"] == pos + 1
    assert r["verdict"] == "UNSAFE"
    assert r["n_adversarial"] == counts[t]
    assert r["first_witness"] == lo + int(np.nonzero(bits[lo:hi])[0][0])
    assert r["n_points"] == sum(np.subtract(*pr.tile_bounds(n, T, u)[::-1]) for u in order[:pos + 1])
    wit = vb.get_witness(res, len(q["pixels"]), len(q["image"]))
    assert wit["index"] == r["first_witness"]
    assert oracle.eval_point(net, q, wit["index"])["adversarial"]
    return r


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_search_follows_the_order(vb, prec):
    net, q = small_relu_case(k=30)
    n = oracle.space_size(3, 30)
    o = oracle.verify(net, q)
    vnet = vb.Net(net)
    res = vb.Result(vnet, max_points=n, max_s=3, max_k=30)
    T = 64
    rng = np.random.default_rng(11)
    for order in (list(range(T)), list(range(T))[::-1], list(rng.permutation(T))):
        _check_search(vb, vnet, res, net, q, order, prec, o, T)
    # a box without witnesses: every tile is checked, same verdict as the full check
    q2 = dict(q, k=2)
    o2 = oracle.verify(net, q2)
    assert o2["n_adv"] == 0
    r = _check_search(vb, vnet, res, net, q2, list(rng.permutation(T)), prec, o2, T)
    assert r["verdict"] in ("SAFE", "TIES_ONLY")
    # more tiles than points: empty tiles are skipped
    q3 = dict(q, pixels=q["pixels"][:1], k=10)
    o3 = oracle.verify(net, q3)
    _check_search(vb, vnet, res, net, q3, list(rng.permutation(T)), prec, o3, T)


def test_search_tensor_path(vb):
    """BF16 tensor screen under the search, on the 784-512-512-10 net (s = 3, k = 7)."""
    w = synth.workload("mlp784x512x512_relu_s6k7", s=3)
    net, q = w["net"], w["query"]
    o = oracle.verify(net, q)
    vnet = vb.Net(net)
    res = vb.Result(vnet, max_points=3375, max_s=3, max_k=7)
    rng = np.random.default_rng(12)
    for T in (64, 5):
        _check_search(vb, vnet, res, net, q, list(rng.permutation(T)), "bf16", o, T)


def test_search_rejects_bad_orders(vb):
    net, q = small_relu_case(k=4)
    vnet = vb.Net(net)
    res = vb.Result(vnet, max_points=1000, max_s=3, max_k=8)
    with pytest.raises(vb.VbmcError):
        vb.search_query(vnet, res, q["image"], q["pixels"], 4, [0, 0, 1])
    with pytest.raises(vb.VbmcError):
        vb.search_query(vnet, res, q["image"], q["pixels"], 4, [0, 2])


def test_learned_order_finds_witnesses_sooner(vb):
    """The proposal pipeline on the 784-512-512-10 net with s = 6 and k = 3
    (7^6 = 117,649 points per query, so exact labels take seconds): candidates
    filtered by first-order reach >= 0.5, per-tile labels from the exact check,
    GPU training with early stopping on a held-out fifth, then the position of
    the first witness tile in the learned order against plain index order on
    separate test queries, and the search itself on some of them."""
    import torch
    from paper_1907_12933_gb300 import proposal as P
    net = synth.workload("proposal_mlp784x512x512_s6k7")["net"]
    vnet = vb.Net(net)
    tr = synth.proposal_candidates("train", 150_000, k=3)
    te = synth.proposal_candidates("test", 40_000, k=3)
    Xtr, rtr, _ = P.features(vnet, tr, 784)
    Xte, rte, _ = P.features(vnet, te, 784)
    itr = P.select_by_reach(rtr)[:3000]
    ite = P.select_by_reach(rte)[:400]
    assert len(itr) >= 2000 and len(ite) >= 300
    qtr, qte = [tr[i] for i in itr], [te[i] for i in ite]
    Xtr = Xtr[torch.from_numpy(itr).cuda()].contiguous()
    Xte = Xte[torch.from_numpy(ite).cuda()].contiguous()
    Ttr, ctr, _ = P.labels(vnet, qtr)
    _, cte, _ = P.labels(vnet, qte)
    nv = len(qtr) // 5
    prop = vb.Proposal((2352, 256, 256, 64), max_batch=256, seed=1)
    hist = P.train(prop, Xtr[nv:].contiguous(), Ttr[nv:].contiguous(), Xtr[:nv].contiguous(),
                   ctr[:nv], max_epochs=8, lr=1e-3, weight_decay=1e-4)
    assert hist["best_epoch"] >= 0
    unsafe = cte.sum(axis=1) > 0
    assert unsafe.sum() >= 100
    plain = np.tile(np.arange(64), (len(qte), 1))
    learned = P.orders(prop, Xte)
    r_plain = P.first_witness_rank(cte, plain)[unsafe]
    r_learned = P.first_witness_rank(cte, learned)[unsafe]
    assert r_learned.mean() <= 0.5 * r_plain.mean(), (r_learned.mean(), r_plain.mean())
    # the search stops where the labels say
    idx = np.nonzero(unsafe)[0][:12]
    got = P.search_all(vnet, [qte[i] for i in idx], learned[idx])
    for i, g in zip(idx, got):
        assert g["verdict"] == "UNSAFE"
        assert g["tiles_checked"] == P.first_witness_rank(cte[i:i + 1], learned[i:i + 1])[0]
        assert cte[i, g["witness_tile"]] == g["n_adversarial"] > 0
    prop.free()
