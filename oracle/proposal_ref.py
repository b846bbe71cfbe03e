"""FP64 reference of the learned tile proposal: query features, the proposal
MLP's forward pass, its listwise loss and the gradients of that loss.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU leg of the
benchmark use this module; the CUDA library never does. It imports nothing
from the CUDA package. Every quantity is written out from its definition in
double precision, with numpy's matmul as the only library step.

Definitions (the CUDA side documents the same ones in its C header):

  tiles      the index space [0, n) of a query, n = R^s, R = 2k + 1, cut into
             T contiguous tiles of ceil(n / T) points (the last ragged)
  features   3 x H_0 per query: x_j = v_j / 255; m_j = R^-p at the p-th
             listed pixel (the place value of its digit in the point index,
             relative to the leading digit), else 0; g_j = clip(m_j * dM/dx_j *
             (k / 255) / max(M, 1e-6), -16, 16), where M = y_D - y_r is the
             margin of the unperturbed image (Eq. 10's class D against the
             runner-up r) and dM/dx its input gradient through the ReLU layers
             (Eq. 1 for the potentials)
  reach      sum over the listed pixels of |dM/dx_j| * (k / 255) / max(M, 1e-6)
  MLP        z = W3 relu(W2 relu(W1 X + b1) + b2) + b3
  loss       mean over rows with at least one witness tile of
             -sum_i (t_i / sum t) log softmax(z)_i  (rows without one: weight 0)

Parity pins (tests/test_oracle_proposal.py): the gradients against central
finite differences of the loss, the input gradient against central finite
differences of the oracle C library's FP64 forward pass, the place values
against their closed form, and the loss against hand values.
"""
from __future__ import annotations

import numpy as np

FEAT_CLIP = 16.0
MARGIN_EPS = 1e-6


def relu(a):
    return np.maximum(a, 0.0)


def net_forward(net: dict, x: np.ndarray) -> list:
    """Potentials u_l = W_l h_{l-1} + b_l of layers 1..L (Eq. 1); ReLU between."""
    us = []
    h = np.asarray(x, dtype=np.float64)
    L = len(net["W"])
    for l in range(L):
        u = net["W"][l].astype(np.float64) @ h + net["b"][l].astype(np.float64)
        us.append(u)
        h = relu(u) if l < L - 1 else u
    return us


def class_and_runner_up(y: np.ndarray) -> tuple[int, int]:
    """Argmax (lowest index on ties) and the best other class (lowest index on ties)."""
    D = int(np.argmax(y))
    others = [i for i in range(len(y)) if i != D]
    r = max(others, key=lambda i: (y[i], -i))
    return D, r


def margin_gradient(net: dict, x: np.ndarray) -> tuple[float, int, int, np.ndarray]:
    """Margin M = y_D - y_r at x and dM/dx by backpropagation through the ReLU layers."""
    us = net_forward(net, x)
    y = us[-1]
    D, r = class_and_runner_up(y)
    g = np.zeros(len(y))
    g[D], g[r] = 1.0, -1.0
    for l in range(len(net["W"]) - 1, -1, -1):
        g = net["W"][l].astype(np.float64).T @ g
        if l > 0:
            g = g * (us[l - 1] > 0)
    return float(y[D] - y[r]), D, r, g


def features(net: dict, query: dict) -> dict:
    """The 3 x H_0 feature row of a query, its reach and its margin."""
    img = np.asarray(query["image"], dtype=np.float64)
    H0 = len(img)
    x = img / 255.0
    M, D, r, g = margin_gradient(net, x)
    k = int(query["k"])
    R = 2 * k + 1
    scale = (k / 255.0) / max(M, MARGIN_EPS)
    mask = np.zeros(H0)
    grad = np.zeros(H0)
    reach = 0.0
    for p, j in enumerate(np.asarray(query["pixels"], dtype=np.int64)):
        pv = float(R) ** (-p)
        mask[j] = pv
        grad[j] = np.clip(pv * g[j] * scale, -FEAT_CLIP, FEAT_CLIP)
        reach += abs(g[j] * scale)
    return {"features": np.concatenate([x, mask, grad]), "reach": reach, "margin": M, "D": D,
            "r": r, "grad": g}


def tile_bounds(n: int, n_tiles: int, i: int) -> tuple[int, int]:
    """[lo, hi) of tile i of [0, n) cut into n_tiles tiles of ceil(n / n_tiles) points."""
    t = -(-n // n_tiles)
    lo = min(n, i * t)
    return lo, min(n, lo + t)


def mlp_forward(params: list, X: np.ndarray) -> list:
    """Activations [X, a1, a2, z] of the proposal MLP; params = [(W1, b1), (W2, b2), (W3, b3)]."""
    acts = [np.asarray(X, dtype=np.float64)]
    for l, (W, b) in enumerate(params):
        a = acts[-1] @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        acts.append(relu(a) if l < len(params) - 1 else a)
    return acts


def listwise_loss(Z: np.ndarray, T: np.ndarray) -> tuple[float, np.ndarray]:
    """Loss and dLoss/dZ of the listwise softmax cross-entropy (rows without a
    witness tile carry no weight; the loss is the mean over the others)."""
    Z = np.asarray(Z, np.float64)
    T = np.asarray(T, np.float64)
    ts = T.sum(axis=1)
    w = ts > 0
    n = int(w.sum())
    dZ = np.zeros_like(Z)
    if n == 0:
        return 0.0, dZ
    mx = Z.max(axis=1, keepdims=True)
    lse = mx + np.log(np.exp(Z - mx).sum(axis=1, keepdims=True))
    logp = Z - lse
    q = np.where(w[:, None], T / np.where(ts > 0, ts, 1.0)[:, None], 0.0)
    loss = float(-(q * logp).sum() / n)
    dZ[w] = (np.exp(logp[w]) - q[w]) / n
    return loss, dZ


def mlp_grads(params: list, X: np.ndarray, T: np.ndarray) -> tuple[float, list]:
    """Loss and [(dW1, db1), (dW2, db2), (dW3, db3)] by backpropagation."""
    acts = mlp_forward(params, X)
    loss, d = listwise_loss(acts[-1], T)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W = np.asarray(params[l][0], np.float64)
        grads[l] = (d.T @ acts[l], d.sum(axis=0))
        if l > 0:
            d = (d @ W) * (acts[l] > 0)
    return loss, grads
