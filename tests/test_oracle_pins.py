"""Pins of the FP64 CPU oracle against values fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself:
  * values printed in the paper (Tables I and II, tests/golden/),
  * a hand-derived 2-2-2 ReLU fixture whose verdicts, ties and coverage
    follow from closed forms,
  * exact rational arithmetic (ReLU / identity nets) and 40-digit mpmath
    arithmetic (sigmoid nets) on tiny networks, point by point,
  * closed forms for affine networks and invariants of the method.
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def bits(words, n):
    w = np.asarray(words, dtype=np.uint64)
    return {i for i in range(n) if (int(w[i // 32]) >> (i % 32)) & 1}


# --------------------------------------------------------------- decoding

@pytest.mark.parametrize("s,k", [(1, 0), (1, 3), (2, 2), (3, 1), (4, 2)])
def test_digits_follow_lexicographic_order(s, k):
    """Point index order is the lexicographic order of the digit tuple, first pixel
    most significant (the reading of the enumeration order)."""
    R = 2 * k + 1
    assert oracle.space_size(s, k) == R ** s
    for t, tup in enumerate(itertools.product(range(R), repeat=s)):
        assert oracle.digits(t, s, k) == list(tup)


def test_space_size_overflow_rejected():
    assert oracle.space_size(64, 1) == 0
    assert oracle.space_size(0, 5) == 1


# ---------------------------------------------------------- paper tables

def load_table1():
    rows = []
    for line in open(os.path.join(GOLD, "table1_preactivations.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((f[0], [float(v) for v in f[1:3]], [float(v) for v in f[3:]]))
    return rows


def table1_net():
    """An affine 2-3-2-1 network whose activation potentials reproduce every row of
    Table I (the table is affine in x2 with x1 = 1; the weights are one solution)."""
    W1 = np.array([[0.2, 0.5], [0.3, 0.7], [0.4, 0.3]], np.float32)
    W2 = np.array([[0.6, 0.5, 0.0], [0.4, 0.5, 0.6]], np.float32)
    W3 = np.array([[0.8, 0.5]], np.float32)
    b = [np.zeros(3, np.float32), np.array([0.89, 0.35], np.float32),
         np.array([-0.1], np.float32)]
    return {"dims": [2, 3, 2, 1], "W": [W1, W2, W3], "b": b, "act": "identity"}


def test_table1_forward_matches_printed_values():
    net = table1_net()
    for name, x, printed in load_table1():
        u = oracle.forward(net, x)
        np.testing.assert_allclose(u, printed, atol=6e-3, err_msg=name)


def test_table1_ss_cover_ex1_ex2():
    """Ex1 vs Ex2: only n31 changes sign in layer 1; n12 and n22 change in layer 2,
    so (n31, n12) and (n31, n22) are SS-covered (Sec. III-B discussion of Table I)."""
    rows = {r[0]: np.array(r[2]) for r in load_table1()}
    dims = [2, 3, 2, 1]
    cov = oracle.pair_coverage(dims, rows["Ex1"], rows["Ex2"])
    # neuron order: n11 n21 n31 | n12 n22 | n13
    assert bits(cov["flip"], 6) == {2, 3, 4, 5}
    # SS bits: layer1->2 block (3x2), then layer2->3 block (2x1)
    assert bits(cov["ss"], 8) == {2 * 2 + 0, 2 * 2 + 1}
    assert not bits(cov["ss_tie"], 8) and not bits(cov["flip_tie"], 6)
    # Ex2 vs Ex3: no sign change in layer 1, only n22 changes in layer 2, n13 keeps
    # its sign: no SS pair at all.
    cov = oracle.pair_coverage(dims, rows["Ex2"], rows["Ex3"])
    assert bits(cov["flip"], 6) == {4}
    assert not bits(cov["ss"], 8)
    # Ex1 vs Ex4: no sign changes anywhere.
    cov = oracle.pair_coverage(dims, rows["Ex1"], rows["Ex4"])
    assert not bits(cov["flip"], 6) and not bits(cov["ss"], 8)


def test_table2_ss_cover_and_eq3_fraction():
    """Table II: pairs {n11, n42} and {n42, n53} are SS-covered; 3 of 14 neurons
    covered, 21 %, so the Eq. 3 literal with P = 80 % is false."""
    u1, u2 = [], []
    for line in open(os.path.join(GOLD, "table2_u_vs_noisy_u.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        u1.append(float(f[3]))
        u2.append(float(f[4]))
    dims = [25, 5, 4, 5]
    cov = oracle.pair_coverage(dims, u1, u2)
    assert bits(cov["flip"], 14) == {0, 5 + 3, 9 + 4}
    # layer1->2 block: j*4+i ; layer2->3 block starts at 20: j*5+i
    assert bits(cov["ss"], 40) == {0 * 4 + 3, 20 + 3 * 5 + 4}
    frac = oracle.ss_covered_fraction(dims, cov["ss"])
    assert frac == pytest.approx(3 / 14)
    assert round(100 * frac) == 21 and frac < 0.80


# ------------------------------------------------------ hand 2-2-2 fixture

def net222():
    W1 = np.array([[255, 0], [0, 255]], np.float32)
    b1 = np.array([-100, -101], np.float32)
    W2 = np.array([[1, -1], [-1, 1]], np.float32)
    return {"dims": [2, 2, 2], "W": [W1, W2], "b": [b1, np.zeros(2, np.float32)],
            "act": "relu"}


def test_hand_222_fixture():
    """v = (104, 100), P = (0, 1), k = 3: h0 = 1 + d0, h1 = relu(d1 - 4), margin
    2 (h0 - h1). Only t = 6 (d = (0, 6)) is adversarial; t = 5 and 13 have margin 0."""
    q = {"image": np.array([104, 100], np.uint8), "pixels": np.array([0, 1], np.int32), "k": 3}
    r = oracle.verify(net222(), q, nthreads=2)
    assert r["D"] == 0 and r["base_margin"] == pytest.approx(8.0)
    assert r["n_points"] == 49
    assert r["n_adv"] == 1 and r["first_witness"] == 6
    assert list(r["ties"]) == [5, 13]
    assert bits(r["bitmap"], 49) == {6}
    # neurons: hidden 0, hidden 1, out 0, out 1
    assert bits(r["flip"], 4) == {1, 2, 3}
    # d1 = 4 makes hidden 1 exactly zero (a sign tie); t = 5, 13 make both outputs zero
    assert bits(r["flip_tie"], 4) == {1, 2, 3}
    assert bits(r["ss"], 4) == {1 * 2 + 0, 1 * 2 + 1}
    for t in range(49):
        d0, d1 = divmod(t, 7)
        p = oracle.eval_point(net222(), q, t)
        h0, h1 = 1 + d0, max(0, d1 - 4)
        assert p["margin"] == pytest.approx(2 * (h0 - h1), abs=1e-9)


def test_center_point_never_adversarial_and_k0():
    w = synth.workload("mlp25_sigmoid_s5k8")
    q = dict(w["query"])
    s, k = len(q["pixels"]), q["k"]
    center = (oracle.space_size(s, k) - 1) // 2
    p = oracle.eval_point(w["net"], q, center)
    assert not p["adversarial"]
    base = oracle.forward(w["net"], q["image"] / 255.0)
    np.testing.assert_array_equal(p["u"], base)
    q0 = dict(q, k=0)
    r = oracle.verify(w["net"], q0)
    assert r["n_points"] == 1 and r["n_adv"] == 0
    assert not r["flip"].any() and not r["ss"].any()


# ------------------------------------------- exact / high-precision brute force

def exact_eval(net, img, pixels, k, t, mode):
    """Activation potentials of point t in exact rationals (ReLU / identity) or
    40-digit mpmath (sigmoid)."""
    s = len(pixels)
    R = 2 * k + 1
    d = []
    for _ in range(s):
        t, r = divmod(t, R)
        d.append(r)
    d = d[::-1]
    v = [int(a) for a in img]
    for p in range(s):
        v[pixels[p]] = min(255, max(0, v[pixels[p]] + d[p] - k))
    if mode == "exact":
        h = [Fraction(a, 255) for a in v]
        cv = Fraction
    else:
        import mpmath
        h = [mpmath.mpf(a) / 255 for a in v]
        cv = mpmath.mpf
    us = []
    L = len(net["W"])
    for l in range(L):
        W, b = net["W"][l], net["b"][l]
        u = [sum(cv(float(W[i, j])) * h[j] for j in range(len(h))) + cv(float(b[i]))
             for i in range(W.shape[0])]
        us.extend(u)
        if l < L - 1:
            if net["act"] == "relu":
                h = [x if x > 0 else 0 * x for x in u]
            elif net["act"] == "sigmoid":
                import mpmath
                h = [1 / (1 + mpmath.exp(-x)) for x in u]
            else:
                h = u
    return us


def expected_masks(dims, ub, ut, tau):
    """Flip / SS masks of one point from high-precision potentials (the definition:
    sign(u) = [u >= 0], SS pair (j, i) iff j is the only changed neuron of its layer)."""
    n = len(ub)
    tie = [abs(ub[i]) < tau or abs(ut[i]) < tau for i in range(n)]
    fl = [((ub[i] >= 0) != (ut[i] >= 0)) and not tie[i] for i in range(n)]
    flip = {i for i in range(n) if fl[i]}
    ftie = {i for i in range(n) if tie[i]}
    ss, sst = set(), set()
    off, ssoff = 0, 0
    for l in range(1, len(dims) - 1):
        Hl, Hn = dims[l], dims[l + 1]
        F = [j for j in range(Hl) if fl[off + j]]
        T = [j for j in range(Hl) if tie[off + j]]
        cand = []
        if not T and len(F) == 1:
            cand = [(F[0], True)]
        elif T:
            cand = [(F[0], False)] if len(F) == 1 else ([(j, False) for j in T] if not F else [])
        for j, certain in cand:
            for i in range(Hn):
                ni = off + Hl + i
                if certain and fl[ni]:
                    ss.add(ssoff + j * Hn + i)
                elif fl[ni] or tie[ni]:
                    sst.add(ssoff + j * Hn + i)
        off += Hl
        ssoff += Hl * Hn
    return flip, ftie, ss, sst


# (activation, arithmetic, seed, weight variance, k): tiny 3-5-4-3 nets where two of
# the three pixels move by up to k/255, chosen so that sign changes, SS pairs and
# (for three of them) adversarial points occur.
BRUTE = [("relu", "exact", 62, 2.0, 50), ("relu", "exact", 32, 2.0, 50),
         ("identity", "exact", 32, 2.0, 50), ("identity", "exact", 12, 2.0, 50),
         ("sigmoid", "mp", 51, 8.0, 30)]


@pytest.mark.parametrize("act,mode,seed,wvar,k", BRUTE)
def test_bruteforce_high_precision(act, mode, seed, wvar, k):
    import mpmath
    mpmath.mp.dps = 40
    dims = [3, 5, 4, 3]
    net = synth.make_net(seed, dims, act, wvar, "normal")
    q = synth.make_query(seed, 0, dims[0], 2, k)
    img, pix = q["image"], [int(p) for p in q["pixels"]]
    n = (2 * k + 1) ** 2
    r = oracle.verify(net, q, nthreads=3)
    tau = Fraction(1, 10 ** 9) if mode == "exact" else mpmath.mpf("1e-9")
    ub = exact_eval(net, img, pix, k, (n - 1) // 2, mode)
    y0 = ub[-dims[-1]:]
    D = max(range(len(y0)), key=lambda i: (y0[i], -i))
    assert r["D"] == D
    flip, ftie, ss, sst = set(), set(), set(), set()
    adv, ties = set(), []
    for t in range(n):
        ut = exact_eval(net, img, pix, k, t, mode)
        y = ut[-dims[-1]:]
        m = y[D] - max(y[i] for i in range(len(y)) if i != D)
        am = max(range(len(y)), key=lambda i: (y[i], -i))
        if abs(m) < tau:
            ties.append(t)
        elif am != D:
            adv.add(t)
        a, b, c, e = expected_masks(dims, ub, ut, tau)
        flip |= a
        ftie |= b
        ss |= c
        sst |= e
    total = sum(dims[1:])
    nss = sum(dims[l] * dims[l + 1] for l in range(1, len(dims) - 1))
    assert bits(r["bitmap"], n) == adv
    assert r["n_adv"] == len(adv)
    assert r["first_witness"] == (min(adv) if adv else None)
    assert list(r["ties"]) == ties
    assert bits(r["flip"], total) == flip
    assert bits(r["flip_tie"], total) == ftie
    assert bits(r["ss"], nss) == ss
    assert bits(r["ss_tie"], nss) == sst
    # the fixtures are chosen so that the comparison is not vacuous
    assert len(flip) >= 2 and ss


def test_bruteforce_is_not_vacuous_for_adversarial():
    """Three brute-force fixtures have adversarial points."""
    n_with_adv = 0
    for act, _, seed, wvar, k in BRUTE:
        net = synth.make_net(seed, [3, 5, 4, 3], act, wvar, "normal")
        r = oracle.verify(net, synth.make_query(seed, 0, 3, 2, k))
        n_with_adv += r["n_adv"] > 0
    assert n_with_adv >= 3


# ------------------------------------------------------------ closed forms

def test_affine_single_pixel_closed_form():
    """Identity activations, one perturbed pixel: the margin is m0 + c * dv / 255 with
    dv the clipped step, so the adversarial points are an exact, countable set."""
    W1 = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]], np.float32)
    W2 = np.array([[2.0, -1.0], [0.5, 1.0]], np.float32)
    b2 = np.array([0.0, 0.0], np.float32)
    net = {"dims": [3, 2, 2], "W": [W1, W2], "b": [np.zeros(2, np.float32), b2],
           "act": "identity"}
    img = np.array([120, 102, 7], np.uint8)
    # y0 = 2 x0 - x1, y1 = 0.5 x0 + x1 ; margin (D = 1) = y1 - y0 = 2 x1 - 1.5 x0,
    # i.e. 510 * margin = 4 * 102 - 3 * v0: positive at the base v0 = 120, zero at
    # v0 = 136 (an exact tie), negative above. Pixel 0 moves x0.
    for k in (5, 13, 16, 40, 140):
        q = {"image": img, "pixels": np.array([0], np.int32), "k": k}
        r = oracle.verify(net, q)
        assert r["D"] == 1
        exp_adv, exp_tie = [], []
        for d in range(2 * k + 1):
            v0 = min(255, max(0, 120 + d - k))
            m2 = 4 * 102 - 3 * v0
            if m2 == 0:
                exp_tie.append(d)
            elif m2 < 0:
                exp_adv.append(d)
        assert r["n_adv"] == len(exp_adv)
        assert list(r["ties"]) == exp_tie
        assert r["first_witness"] == (exp_adv[0] if exp_adv else None)


# -------------------------------------------------------------- invariants

def small_relu_case(seed=66, s=3, k=6):
    """A 6-8-6-4 ReLU net where sign changes, SS pairs and adversarial points occur
    once k reaches a few tens of grey levels (seed 66 picked for that)."""
    net = synth.make_net(seed, [6, 8, 6, 4], "relu", 2.0, "normal")
    q = synth.make_query(seed, 1, 6, s, k)
    return net, q


def test_monotone_in_k():
    net, q = small_relu_case()
    prev = None
    for k in (0, 3, 8, 15, 30):
        r = oracle.verify(net, dict(q, k=k))
        if prev is not None:
            for key in ("flip", "ss"):
                assert np.all((prev[key] & ~r[key]) == 0), key
            assert r["n_adv"] >= prev["n_adv"]
        prev = r
    assert prev["flip"].any() and prev["ss"].any() and prev["n_adv"] > 0


def test_pixel_permutation_invariance():
    net, q = small_relu_case(k=25)
    r = oracle.verify(net, q)
    perm = [2, 0, 1]
    q2 = dict(q, pixels=q["pixels"][perm])
    r2 = oracle.verify(net, q2)
    for key in ("n_adv", "n_ties"):
        assert r[key] == r2[key]
    for key in ("flip", "flip_tie", "ss", "ss_tie"):
        np.testing.assert_array_equal(r[key], r2[key])
    R = 2 * q["k"] + 1
    n = R ** 3
    adv1 = bits(r["bitmap"], n)
    adv2 = bits(r2["bitmap"], n)
    assert adv1

    def remap(t):
        d = oracle.digits(t, 3, q["k"])
        d2 = [d[p] for p in perm]
        return (d2[0] * R + d2[1]) * R + d2[2]
    assert {remap(t) for t in adv1} == adv2


def test_clipped_duplicates_share_verdicts():
    """Grey level 2 with k = 6: steps -6..-2 all clip to 0; grey level 253: steps
    +2..+6 all clip to 255. Those digits give one image, so one margin."""
    net, q = small_relu_case(s=1, k=6)
    img = q["image"].copy()
    img[q["pixels"][0]] = 2
    ms = [oracle.eval_point(net, dict(q, image=img), t)["margin"] for t in range(13)]
    assert len(set(ms[0:5])) == 1
    assert len(set(ms[4:8])) == 4
    img[q["pixels"][0]] = 253
    ms = [oracle.eval_point(net, dict(q, image=img), t)["margin"] for t in range(13)]
    assert len(set(ms[8:13])) == 1
    assert len(set(ms[5:9])) == 4


def test_range_split_merges_to_whole():
    net, q = small_relu_case(k=20)
    whole = oracle.verify(net, q)
    n = whole["n_points"]
    cuts = [0, 77, 1000, 2222, n]
    parts = [oracle.verify(net, q, lo=a, hi=b) for a, b in zip(cuts[:-1], cuts[1:])]
    assert sum(p["n_adv"] for p in parts) == whole["n_adv"]
    firsts = [p["first_witness"] for p in parts if p["first_witness"] is not None]
    assert (min(firsts) if firsts else None) == whole["first_witness"]
    for key in ("flip", "flip_tie", "ss", "ss_tie", "bitmap"):
        acc = np.zeros_like(whole[key])
        for p in parts:
            acc |= p[key]
        np.testing.assert_array_equal(acc, whole[key])
