"""Pins of the oracle's point filters: the Euclidean ball of Eq. 9 on the grid
and the k-shells (points whose largest step is exactly k). Checked against
brute force over the digits and against the unfiltered check."""
import itertools

import numpy as np

import oracle
from test_oracle_pins import small_relu_case


def _dv(q, steps):
    img = np.asarray(q["image"], np.int64)
    return [int(np.clip(img[p] + st, 0, 255) - img[p]) for p, st in zip(q["pixels"], steps)]


def _bits(mask, n):
    return [t for t in range(n) if (int(mask[t >> 5]) >> (t & 31)) & 1]


def test_shells_partition_the_box():
    """Shells r = 0..k (each checked as the box of radius r restricted to its
    boundary) hold every point once, and their adversarial points add up to
    those of the whole box."""
    net, q = small_relu_case(k=12)
    whole = oracle.verify(net, q)
    n_pts = n_adv = n_ties = 0
    for r in range(0, 13):
        o = oracle.verify(net, dict(q, k=r, filter=2))
        exp_pts = (2 * r + 1) ** 3 - (2 * r - 1) ** 3 if r else 1
        assert o["n_points"] == exp_pts
        n_pts += o["n_points"]
        n_adv += o["n_adv"]
        n_ties += o["n_ties"]
    assert n_pts == whole["n_points"] and n_adv == whole["n_adv"] > 0 and n_ties == whole["n_ties"]


def test_shell_adversarial_points_are_on_the_shell():
    net, q = small_relu_case(k=20)
    r = 17
    o = oracle.verify(net, dict(q, k=r, filter=2))
    n = oracle.space_size(3, r)
    for t in _bits(o["bitmap"], n):
        d = oracle.digits(t, 3, r)
        assert max(abs(x - r) for x in d) == r
        assert oracle.eval_point(net, dict(q, k=r), t)["adversarial"]


def test_l2_ball_against_brute_force():
    net, q = small_relu_case(k=30)
    k = 30
    for l2 in (0, 50, 900, 2000, 10 ** 9):
        o = oracle.verify(net, dict(q, filter=1, l2_max=l2))
        inside = []
        for t, steps in enumerate(itertools.product(range(-k, k + 1), repeat=3)):
            if sum(v * v for v in _dv(q, steps)) <= l2:
                inside.append(t)
        assert o["n_points"] == len(inside), l2
        if len(inside) < 5000:
            adv = [t for t in inside if oracle.eval_point(net, q, t)["adversarial"]]
            assert _bits(o["bitmap"], oracle.space_size(3, k)) == adv
    full = oracle.verify(net, q)
    assert oracle.verify(net, dict(q, filter=1, l2_max=10 ** 9))["n_adv"] == full["n_adv"]


def test_filters_combine():
    """Ball and shell together: the points in both."""
    net, q = small_relu_case(k=10)
    o = oracle.verify(net, dict(q, filter=3, l2_max=150))
    cnt = sum(1 for steps in itertools.product(range(-10, 11), repeat=3)
              if max(abs(s) for s in steps) == 10 and sum(v * v for v in _dv(q, steps)) <= 150)
    assert o["n_points"] == cnt
