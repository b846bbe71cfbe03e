"""Pins of the FP64 proposal reference (oracle/proposal_ref.py) against facts
outside itself: central finite differences, the C oracle's FP64 forward pass,
closed forms and hand-computed losses."""
import numpy as np
import pytest

import oracle
import synth
from oracle import proposal_ref as pr


def _params(dims, seed):
    rng = np.random.default_rng(seed)
    return [(rng.normal(0, np.sqrt(2.0 / dims[l]), (dims[l + 1], dims[l])),
             rng.normal(0, 0.1, dims[l + 1])) for l in range(3)]


def _batch(seed, B, F, T):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (B, F))
    lab = (rng.random((B, T)) < 0.3).astype(np.float64)
    lab[0] = 0.0          # a row without witness tiles: no weight
    lab[1] = 0.0
    lab[1, T - 1] = 1.0   # a single witness tile
    return X, lab


def test_loss_hand_values():
    # equal logits: p = 1/T; one witness tile -> log T; all tiles -> log T as well
    T = 8
    Z = np.zeros((2, T))
    lab = np.zeros((2, T))
    lab[0, 3] = 1.0
    lab[1, :] = 1.0
    loss, dZ = pr.listwise_loss(Z, lab)
    assert loss == pytest.approx(np.log(T), abs=1e-15)
    # dZ = (p - q) / rows: row 0 -> 1/8 - [i == 3], row 1 -> 0
    exp0 = np.full(T, 1.0 / T)
    exp0[3] -= 1.0
    np.testing.assert_allclose(dZ[0], exp0 / 2, atol=1e-15)
    np.testing.assert_allclose(dZ[1], 0.0, atol=1e-15)
    # two logits, label on the first: loss = log(1 + e^(z1 - z0))
    loss, _ = pr.listwise_loss(np.array([[2.0, -1.0]]), np.array([[1.0, 0.0]]))
    assert loss == pytest.approx(np.log1p(np.exp(-3.0)), rel=1e-14)
    # no weighted row: zero loss, zero gradient
    loss, dZ = pr.listwise_loss(np.ones((3, 4)), np.zeros((3, 4)))
    assert loss == 0.0 and not dZ.any()


@pytest.mark.parametrize("dims", [(7, 5, 4, 3), (12, 9, 6, 5)])
def test_mlp_grads_finite_differences(dims):
    params = _params(dims, 3)
    X, lab = _batch(4, 6, dims[0], dims[3])
    _, grads = pr.mlp_grads(params, X, lab)
    h = 1e-6
    for l in range(3):
        W, b = params[l]
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            flat = arr.reshape(-1)
            gf = g.reshape(-1)
            for idx in range(0, flat.size, max(1, flat.size // 17)):
                old = flat[idx]
                flat[idx] = old + h
                lp, _ = pr.listwise_loss(pr.mlp_forward(params, X)[-1], lab)
                flat[idx] = old - h
                lm, _ = pr.listwise_loss(pr.mlp_forward(params, X)[-1], lab)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                assert gf[idx] == pytest.approx(fd, rel=1e-5, abs=1e-8), (l, idx)


def test_rows_without_witness_do_not_move_the_gradient():
    dims = (7, 5, 4, 3)
    params = _params(dims, 5)
    X, lab = _batch(6, 6, dims[0], dims[3])
    _, g1 = pr.mlp_grads(params, X, lab)
    X2 = X.copy()
    X2[0] += 10.0            # row 0 has no witness tile
    _, g2 = pr.mlp_grads(params, X2, lab)
    for a, b in zip(g1, g2):
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])


def test_input_gradient_matches_c_oracle_finite_differences():
    """dM/dx of the reference against central differences of the C oracle's FP64
    forward pass (no ReLU kink is crossed within +-h at these points)."""
    net = synth.make_net(66, [20, 16, 12, 5], "relu", 2.0, "normal")
    rng = np.random.default_rng(9)
    for _ in range(3):
        x = rng.random(20)
        M, D, r, g = pr.margin_gradient(net, x)
        u = oracle.forward(net, x)
        y = u[-5:]
        assert D == int(np.argmax(y)) and M == pytest.approx(y[D] - y[r], abs=1e-12)
        h = 1e-7
        for j in range(20):
            xp, xm = x.copy(), x.copy()
            xp[j] += h
            xm[j] -= h
            yp, ym = oracle.forward(net, xp)[-5:], oracle.forward(net, xm)[-5:]
            fd = ((yp[D] - yp[r]) - (ym[D] - ym[r])) / (2 * h)
            assert g[j] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_features_closed_forms():
    net = synth.make_net(66, [20, 16, 12, 5], "relu", 2.0, "normal")
    q = {"image": np.arange(20, dtype=np.uint8) * 12, "pixels": np.array([7, 2, 19], np.int32),
         "k": 4}
    f = pr.features(net, q)
    F = f["features"]
    np.testing.assert_array_equal(F[:20], np.arange(20) * 12 / 255.0)
    mask = F[20:40]
    assert mask[7] == 1.0 and mask[2] == pytest.approx(1 / 9) and mask[19] == pytest.approx(1 / 81)
    assert np.count_nonzero(mask) == 3
    grad = F[40:]
    assert np.count_nonzero(grad) <= 3
    scale = (4 / 255.0) / f["margin"]
    assert grad[7] == pytest.approx(np.clip(f["grad"][7] * scale, -16, 16))
    assert f["reach"] == pytest.approx(sum(abs(f["grad"][j]) * scale for j in (7, 2, 19)))
    # D is the class the C oracle gives the unperturbed image (centre point of the box)
    n = oracle.space_size(3, 4)
    assert f["D"] == oracle.eval_point(net, q, (n - 1) // 2)["D"]


def test_tile_bounds_cover_the_space_once():
    for n, T in ((15 ** 6, 64), (3375, 64), (10, 64), (64, 64), (1, 3)):
        covered = np.zeros(n, np.int32)
        for i in range(T):
            lo, hi = pr.tile_bounds(n, T, i)
            assert 0 <= lo <= hi <= n
            covered[lo:hi] += 1
        assert (covered == 1).all()
    assert pr.tile_bounds(15 ** 6, 64, 1) == (177_979, 355_958)
