"""Pins of the oracle's misclassified literal (Eq. 11): (n_D < V) and (n_i > V)
for some output i != D, with V a reference value. Hand cases, the relation to
Eq. 10 that holds for every V, the extremes of V, and exact-rational brute
force on a small ReLU net."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from test_oracle_pins import exact_eval, small_relu_case


def _bits(mask, n):
    return [t for t in range(n) if (int(mask[t >> 5]) >> (t & 31)) & 1]


def base_outputs(net, q):
    x = np.asarray(q["image"], np.float64) / 255.0
    return oracle.forward(net, x)[-net["dims"][-1]:]


def reference_v(net, q, alpha=0.5):
    """V = y_D - alpha (y_D - y_2nd) from the unperturbed image's class output y_D
    and its runner-up (alpha < 1: between the two)."""
    y = base_outputs(net, q)
    D = int(np.argmax(y))
    second = max(y[i] for i in range(len(y)) if i != D)
    return float(y[D] - alpha * (y[D] - second))


def test_literal_hand_cases():
    y = [1.0, 2.0, 0.5]
    lit = oracle.threshold_literal
    assert lit(y, 0, 1.5) == 1    # 1 < 1.5 and 2 > 1.5
    assert lit(y, 0, 0.7) == 0    # n_D > V
    assert lit(y, 0, 2.5) == 0    # no other output above V
    assert lit(y, 1, 1.5) == 0    # the largest output is the class
    assert lit(y, 2, 0.75) == 1   # 0.5 < 0.75, 1 and 2 above
    assert lit(y, 0, 1.0) == 2    # n_D == V: the first literal is undecided
    assert lit(y, 0, 2.0) == 2    # the only candidate above V equals V
    assert lit(y, 0, 1.0 + 2e-9) == 1  # clear of the tie band on both sides
    assert lit([0.0, 0.0], 0, 0.0) == 2
    assert lit([0.0, 0.0], 0, 5e-10) == 2
    assert lit([0.0, 0.0], 0, 2e-9) == 0  # nothing above V
    # a single output can never be misclassified
    assert lit([3.0], 0, 4.0) == 0


def test_literal_and_margin_forms_agree():
    """The literal in three-valued logic and the signed distance
    max(y_D - V, V - max_{i != D} y_i): true iff <= -tau, false iff >= tau."""
    rng = np.random.default_rng(5)
    for _ in range(4000):
        n = int(rng.integers(2, 8))
        y = rng.normal(size=n)
        if rng.random() < 0.3:  # exact coincidences
            y[rng.integers(n)] = y[rng.integers(n)]
        D = int(rng.integers(n))
        V = float(rng.choice([rng.normal(), y[rng.integers(n)], y[D] + 1e-10]))
        lit = oracle.threshold_literal(y, D, V)
        m = oracle.threshold_margin(y, D, V)
        assert lit == (1 if m <= -oracle.TAU else 0 if m >= oracle.TAU else 2)
        mx = max(y[i] for i in range(n) if i != D)
        if min(abs(y[D] - V), abs(mx - V)) >= oracle.TAU:
            assert (lit == 1) == (y[D] < V and any(y[i] > V for i in range(n) if i != D))


@pytest.mark.parametrize("alpha", [0.9, 1.5, 3.0])
def test_counterexamples_of_eq11_are_counterexamples_of_eq10(alpha):
    """y_D < V < y_i puts y_i above y_D: every point that satisfies the literal
    (outside the tie bands) changes the argmax."""
    net, q = small_relu_case(k=30)
    V = reference_v(net, q, alpha)
    o10 = oracle.verify(net, q)
    o11 = oracle.verify(net, dict(q, property=1, threshold=V))
    n = oracle.space_size(3, 30)
    a10, a11 = set(_bits(o10["bitmap"], n)), set(_bits(o11["bitmap"], n))
    assert a11 and a11 <= a10
    assert o11["n_points"] == o10["n_points"] == n
    assert o11["D"] == o10["D"]
    y = base_outputs(net, q)
    assert o11["base_margin"] == pytest.approx(oracle.threshold_margin(y, o11["D"], V), abs=1e-12)
    # the coverage masks do not depend on the property
    for key in ("flip", "flip_tie", "ss", "ss_tie"):
        np.testing.assert_array_equal(o10[key], o11[key])


def test_extreme_reference_values_admit_no_counterexample():
    net, q = small_relu_case(k=30)
    for V in (-1e6, 1e6):
        o = oracle.verify(net, dict(q, property=1, threshold=V))
        assert o["n_adv"] == 0 and o["n_ties"] == 0 and o["first_witness"] is None


def test_bad_property_rejected():
    net, q = small_relu_case(k=3)
    with pytest.raises(ValueError):
        oracle.verify(net, dict(q, property=2))
    with pytest.raises(ValueError):
        oracle.verify(net, dict(q, property=1, threshold=float("nan")))


@pytest.mark.parametrize("seed,alpha", [(23, 1.5), (23, 3.0), (23, 0.9), (3, 0.9)])
def test_exact_bruteforce(seed, alpha):
    """Every point of a small box against exact rational outputs and the
    literal evaluated on them with V exact."""
    net = synth.make_net(seed, [5, 6, 4], "relu", 2.0, "normal")
    k = 20
    q = synth.make_query(seed, 1, 5, 2, k)
    img, pix = list(q["image"]), [int(p) for p in q["pixels"]]
    y0 = base_outputs(net, q)
    D = int(np.argmax(y0))
    V = reference_v(net, q, alpha)
    o = oracle.verify(net, dict(q, property=1, threshold=V))
    Vq = Fraction(V)
    n = oracle.space_size(2, k)
    exp_adv, exp_tie = [], []
    for t in range(n):
        y = exact_eval(net, img, pix, k, t, "exact")[-4:]
        a = y[D] - Vq
        b = max(y[i] for i in range(4) if i != D) - Vq
        m = max(a, -b)
        if abs(m) < Fraction(oracle.TAU):
            exp_tie.append(t)
        elif a < 0 and b > 0:
            exp_adv.append(t)
    assert _bits(o["bitmap"], n) == exp_adv
    assert list(o["ties"]) == exp_tie
    assert o["first_witness"] == (exp_adv[0] if exp_adv else None)
    assert (len(exp_adv) > 0) == (seed == 23)
    for t in exp_adv[:5]:
        p = oracle.eval_point(net, dict(q, property=1, threshold=V), t)
        assert p["adversarial"] and p["margin"] < 0
