"""Learned tile proposal: label generation, GPU training and tile-ordered search.

The pipeline, end to end on the GPU through the C ABI:
  1. features: vbmc_proposal_features for every query (image, place-value
     mask, normalised input gradient of the margin);
  2. labels: vbmc_verify_query with the verdict bitmap over each training
     query's whole space, then vbmc_tile_counts: a tile is labelled 1 iff it
     holds an adversarial point (the exact check decides every label);
  3. training: vbmc_proposal_train_step over shuffled mini-batches (forward,
     listwise loss, backward and AdamW in the library's kernels);
  4. inference: vbmc_proposal_scores gives each query's tile order, and
     vbmc_search_query checks the tiles in that order, stopping at the first
     tile that holds a witness.
This module only moves arrays between the host, torch's device memory and the
library; PyTorch is used for allocation and for row gathers of mini-batches.
"""
from __future__ import annotations

import time

import numpy as np

from . import (Net, Proposal, Result, proposal_features, search_query, tile_counts,
               verify_query)

N_TILES = 64


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the proposal pipeline needs a CUDA device (no CPU fallback)")
    return torch


def query_arrays(queries: list, h0: int):
    """Pack queries into device tensors: images [n, H0] u8, pixels [n, smax] i32, s, k."""
    torch = _torch()
    n = len(queries)
    smax = max(1, max(len(q["pixels"]) for q in queries))
    img = np.zeros((n, h0), np.uint8)
    pix = np.zeros((n, smax), np.int32)
    s = np.zeros(n, np.int32)
    k = np.zeros(n, np.int32)
    for i, q in enumerate(queries):
        img[i] = q["image"]
        p = np.asarray(q["pixels"], np.int32)
        pix[i, :len(p)] = p
        s[i] = len(p)
        k[i] = q["k"]
    dev = "cuda"
    return (torch.from_numpy(img).to(dev), torch.from_numpy(pix).to(dev),
            torch.from_numpy(s).to(dev), torch.from_numpy(k).to(dev))


def features(vnet: Net, queries: list, h0: int, chunk: int = 8192):
    """Feature rows [n, 3 H0] (device), reach [n] and margin [n] (host)."""
    torch = _torch()
    n = len(queries)
    X = torch.empty((n, 3 * h0), dtype=torch.float32, device="cuda")
    reach = torch.empty(n, dtype=torch.float32, device="cuda")
    margin = torch.empty(n, dtype=torch.float32, device="cuda")
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        img, pix, s, k = query_arrays(queries[a:b], h0)
        proposal_features(vnet, img, pix, s, k, X[a:b], reach[a:b], margin[a:b])
    torch.cuda.synchronize()
    return X, reach.cpu().numpy(), margin.cpu().numpy()


def labels(vnet: Net, queries: list, n_tiles: int = N_TILES, precision: str = "bf16",
           queue_cap: int = 1 << 24):
    """0/1 witness labels per tile [n, n_tiles] (device) and per-tile counts (host),
    from the exact check of each query's whole space."""
    torch = _torch()
    smax = max(len(q["pixels"]) for q in queries)
    kmax = max(int(q["k"]) for q in queries)
    nmax = max((2 * int(q["k"]) + 1) ** len(q["pixels"]) for q in queries)
    res = Result(vnet, max_points=nmax, max_s=smax, max_k=kmax, queue_cap=queue_cap)
    counts = np.zeros((len(queries), n_tiles), np.int64)
    t0 = time.perf_counter()
    for i, q in enumerate(queries):
        verify_query(vnet, res, q["image"], q["pixels"], q["k"], precision=precision,
                     coverage=False, bitmap=True)
        counts[i] = tile_counts(res, n_tiles)
    secs = time.perf_counter() - t0
    res.free()
    T = torch.from_numpy((counts > 0).astype(np.float32)).to("cuda")
    return T, counts, secs


def _snapshot(prop: Proposal) -> list:
    return [(d["W"], d["b"]) for d in (prop.params(l) for l in (1, 2, 3))]


def _restore(prop: Proposal, snap: list) -> None:
    for l, (W, b) in enumerate(snap, start=1):
        prop.set_params(l, W, b)


def mean_rank(prop: Proposal, X, counts: np.ndarray) -> float:
    """Mean 1-based position of the first witness tile over queries that hold one."""
    has = counts.sum(axis=1) > 0
    if not has.any():
        return 0.0
    return float(first_witness_rank(counts, orders(prop, X))[has].mean())


def train(prop: Proposal, X, T, X_val=None, counts_val=None, max_epochs: int = 16,
          batch: int = 128, lr: float = 1e-3, weight_decay: float = 1e-4, seed: int = 0,
          patience: int = 3, log=None) -> dict:
    """Mini-batch AdamW on the rows that hold at least one witness tile. With a
    validation set, the weights of the epoch with the lowest mean first-witness
    rank on it are kept (early stopping: longer training memorises the
    training queries and ranks held-out ones worse)."""
    torch = _torch()
    keep = torch.nonzero(T.sum(dim=1) > 0).flatten()
    Xk, Tk = X.index_select(0, keep).contiguous(), T.index_select(0, keep).contiguous()
    n = Xk.shape[0]
    if n == 0:
        raise ValueError("no training query holds a witness")
    rng = np.random.default_rng(seed)
    b = min(batch, prop.max_batch, n)
    hist = {"loss": [], "val_rank": [], "best_epoch": -1}
    best, best_snap, bad = None, None, 0
    for ep in range(max_epochs):
        perm = torch.from_numpy(rng.permutation(n)).to("cuda")
        last_loss = 0.0
        starts = list(range(0, n - b + 1, b))
        for i, a in enumerate(starts):
            idx = perm[a:a + b]
            l = prop.train_step(Xk.index_select(0, idx).contiguous(),
                                Tk.index_select(0, idx).contiguous(), lr, weight_decay,
                                want_loss=i == len(starts) - 1)
            if l is not None:
                last_loss = l
        hist["loss"].append(last_loss)
        if X_val is not None:
            r = mean_rank(prop, X_val, counts_val)
            hist["val_rank"].append(r)
            if best is None or r < best:
                best, best_snap, bad = r, _snapshot(prop), 0
                hist["best_epoch"] = ep
            else:
                bad += 1
            if log:
                log(f"epoch {ep}: loss {last_loss:.4f} val rank {r:.3f}")
            if bad >= patience:
                break
        elif log:
            log(f"epoch {ep}: loss {last_loss:.4f}")
    if best_snap is not None:
        _restore(prop, best_snap)
    torch.cuda.synchronize()
    return hist


def orders(prop: Proposal, X):
    """Tile order [n, T] (host int32) from the proposal's scores."""
    torch = _torch()
    n = X.shape[0]
    T = prop.dims[3]
    out = torch.empty((n, T), dtype=torch.int32, device="cuda")
    sc = torch.empty((n, T), dtype=torch.float32, device="cuda")
    for a in range(0, n, prop.max_batch):
        b = min(n, a + prop.max_batch)
        prop.scores(X[a:b].contiguous(), sc[a:b], out[a:b])
    return out.cpu().numpy()


def search_all(vnet: Net, queries: list, tile_orders, precision: str = "bf16",
               queue_cap: int = 1 << 24) -> list:
    """vbmc_search_query for each query with its tile order."""
    smax = max(len(q["pixels"]) for q in queries)
    kmax = max(int(q["k"]) for q in queries)
    nmax = max((2 * int(q["k"]) + 1) ** len(q["pixels"]) for q in queries)
    res = Result(vnet, max_points=nmax, max_s=smax, max_k=kmax, queue_cap=queue_cap)
    out = []
    for q, o in zip(queries, tile_orders):
        out.append(search_query(vnet, res, q["image"], q["pixels"], q["k"], o,
                                precision=precision))
    res.free()
    return out


def select_by_reach(reach: np.ndarray, threshold: float = 0.5) -> np.ndarray:
    """Indices of queries whose first-order reach (the fraction of the margin the
    box can use up, to first order) is at least `threshold`: a cheap filter that
    drops queries far from the decision boundary before the exact labelling."""
    return np.nonzero(np.asarray(reach) >= threshold)[0]


def first_witness_rank(counts: np.ndarray, tile_orders) -> np.ndarray:
    """1-based position of the first tile holding a witness in each order (0: none)."""
    out = np.zeros(len(counts), np.int64)
    for i, (c, o) in enumerate(zip(counts, tile_orders)):
        hits = np.nonzero(c[np.asarray(o)] > 0)[0]
        out[i] = hits[0] + 1 if len(hits) else 0
    return out
