"""Pins of the DS, SV and DV covers (Sec. III-B) in the oracle, against the
covered pairs the paper names for its Table I examples (the affine 2-3-2-1 net
of tests/golden/table1_preactivations.txt), plus threshold, symmetry and tie
checks."""
import numpy as np

import oracle
from test_oracle_pins import load_table1, table1_net

# neuron order of the 2-3-2-1 net: n11 n21 n31 | n12 n22 | n13 (bits 0..5)
N11, N21, N31, N12, N22, N13 = range(6)


def _u(name):
    net = table1_net()
    rows = {r[0]: r[1] for r in load_table1()}
    return oracle.forward(net, np.asarray(rows[name], np.float64))


def _bits(mask):
    return {i for i in range(32 * len(mask)) if (int(mask[i >> 5]) >> (i & 31)) & 1}


DIMS = [2, 3, 2, 1]


def test_ds_ex2_ex3():
    """No sign change in layer 1 between Ex2 and Ex3, layer-1 distance 0.18 >= d,
    and n22 changes sign: DS covers (any layer-1 neuron, n22)."""
    c = oracle.pair_covers(DIMS, _u("Ex2"), _u("Ex3"), g=1.5, d=0.1)
    assert _bits(c["ds"]) == {N22}
    assert not c["ds_tie"].any()
    assert oracle.layer_pair_fraction(DIMS, c["ds"]) == 4 / 6  # n11 n21 n31 n22
    # the distance threshold above the layer-1 distance removes the pair
    c = oracle.pair_covers(DIMS, _u("Ex2"), _u("Ex3"), g=1.5, d=0.2)
    assert not c["ds"].any()


def test_sv_ex2_ex3():
    """n22 is the only layer-2 sign change and n13 keeps its sign with a value
    ratio 0.353 / 0.176 > 2: SV covers (n22, n13)."""
    c = oracle.pair_covers(DIMS, _u("Ex2"), _u("Ex3"), g=1.5, d=0.1)
    # SS layout: layer pair (1,2) takes 3 x 2 bits, then pair (2,3): bit 6 + j * 1 + i
    assert _bits(c["sv"]) == {6 + 1 * 1 + 0}
    c = oracle.pair_covers(DIMS, _u("Ex2"), _u("Ex3"), g=2.1, d=0.1)
    assert not c["sv"].any()


def test_dv_ex1_ex4():
    """No sign changes anywhere between Ex1 and Ex4; every layer distance is
    large and every later neuron changes its value by more than 1.5x: DV covers
    (any layer-1 neuron, n12), (any, n22) and (any layer-2 neuron, n13)."""
    c = oracle.pair_covers(DIMS, _u("Ex1"), _u("Ex4"), g=1.5, d=1.0)
    assert _bits(c["dv"]) == {N12, N22, N13}
    assert not c["ds"].any() and not c["sv"].any()
    assert oracle.layer_pair_fraction(DIMS, c["dv"]) == 1.0
    # n13 changes by 4.957 / 1.417 = 3.5, n22 by 3.13, n12 by 4.29
    c = oracle.pair_covers(DIMS, _u("Ex1"), _u("Ex4"), g=3.2, d=1.0)
    assert _bits(c["dv"]) == {N12, N13}


def test_ss_ex1_ex2_is_not_ds():
    """Ex1 -> Ex2 changes the sign of n31 in layer 1: no distance change there."""
    c = oracle.pair_covers(DIMS, _u("Ex1"), _u("Ex2"), g=1.5, d=0.1)
    assert not (_bits(c["ds"]) | _bits(c["dv"])) & {N12, N22}


def test_symmetric_in_the_pair():
    for a, b in (("Ex1", "Ex2"), ("Ex2", "Ex3"), ("Ex1", "Ex4"), ("Ex3", "Ex4")):
        c1 = oracle.pair_covers(DIMS, _u(a), _u(b), g=1.5, d=0.5)
        c2 = oracle.pair_covers(DIMS, _u(b), _u(a), g=1.5, d=0.5)
        for k in c1:
            np.testing.assert_array_equal(c1[k], c2[k], err_msg=k)


def test_ties():
    """A potential inside the tie band, a ratio exactly at g and a distance
    exactly at d are undecided: the pairs they could form go to the tie masks."""
    u1 = np.array([-1.0, -2.0, -0.5, 1.0, 2.0, 3.0])
    # n11 sits in the tie band in x2; layer 2: n12 ratio exactly 2 (= g)
    u2 = np.array([0.5e-9, -2.0, -0.5, 2.0, 2.0, 3.0])
    c = oracle.pair_covers(DIMS, u1, u2, g=2.0, d=0.0)
    # layer 1 has a tie (n11) and no certain change: dc(1) only possible
    assert not c["ds"].any() and not c["dv"].any()
    assert N12 in _bits(c["dv_tie"])
    # n11 may be the only changed neuron of layer 1: SV (n11, n12) undecided
    assert 0 * 2 + 0 in _bits(c["sv_tie"]) and not c["sv"].any()
    # a clean distance exactly at d is a tie as well
    u3 = np.array([-1.0, -2.0, -0.5 - 1.0, 1.0, 2.0, 3.0])
    c = oracle.pair_covers(DIMS, u1, u3, g=1.5, d=1.0)
    assert not c["dv"].any() and not c["ds"].any()
