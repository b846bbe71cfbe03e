"""Counter-based random streams and the five synthetic workloads.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: value i of stream (seed, stream) is mix(key + (i+1)*G) with
key = mix(seed + stream*G2). Normals use the Box-Muller transform in float64.

The paper's benchmark (5x5 vowel images and a trained 25-5-4-5 sigmoid MLP,
Section IV-A) is not available, so every network and image here is drawn from
these streams. Weights are drawn in float64 and rounded once to float32; both
the CUDA path and the oracle consume those float32 values.
"""
from __future__ import annotations

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_G2 = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, stream: int, n: int) -> np.ndarray:
    """n uint64 values of stream `stream` under `seed`."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([np.uint64(seed % 2**64) + np.uint64(stream % 2**64) * _G2],
                            dtype=np.uint64))[0]
        ctr = np.arange(1, n + 1, dtype=np.uint64) * _G + key
    return _mix(ctr)


def uniform01(seed: int, stream: int, n: int) -> np.ndarray:
    """Uniform float64 in [0, 1) with 53 random bits."""
    return (splitmix64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normal float64 via Box-Muller on two interleaved uniforms."""
    m = (n + 1) // 2
    u = uniform01(seed, stream, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
    return z[:n]


def randint(seed: int, stream: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive)."""
    span = hi - lo + 1
    return lo + np.floor(uniform01(seed, stream, n) * span).astype(np.int64)


def distinct(seed: int, stream: int, n: int, s: int) -> np.ndarray:
    """s distinct indices from range(n), in draw order (partial Fisher-Yates)."""
    perm = np.arange(n, dtype=np.int64)
    u = uniform01(seed, stream, s)
    for i in range(s):
        j = i + int(u[i] * (n - i))
        perm[i], perm[j] = perm[j], perm[i]
    return perm[:s].astype(np.int32)


def make_net(seed: int, dims, hidden_act: str, w_var: float, bias: str = "normal") -> dict:
    """MLP with W_l ~ N(0, w_var / fan_in); biases N(0, w_var / fan_in) or zero.

    W[l] has shape (dims[l+1], dims[l]): row i holds the weights of output
    neuron i, matching u = sum_j w_j * i_j + b (Eq. 1).
    """
    dims = [int(d) for d in dims]
    Ws, bs = [], []
    for l in range(len(dims) - 1):
        fan_in, fan_out = dims[l], dims[l + 1]
        sd = np.sqrt(w_var / fan_in)
        w = (normal(seed, 1000 + 2 * l, fan_in * fan_out) * sd).astype(np.float32)
        Ws.append(w.reshape(fan_out, fan_in))
        if bias == "normal":
            bs.append((normal(seed, 1001 + 2 * l, fan_out) * sd).astype(np.float32))
        else:
            bs.append(np.zeros(fan_out, dtype=np.float32))
    return {"dims": dims, "W": Ws, "b": bs, "act": hidden_act}


def make_query(seed: int, qid: int, h0: int, s: int, k: int) -> dict:
    """Base image with grey levels uniform in {0..255}, s distinct pixels, step bound k."""
    img = randint(seed, 10_000 + 3 * qid, h0, 0, 255).astype(np.uint8)
    pix = distinct(seed, 10_001 + 3 * qid, h0, s)
    return {"image": img, "pixels": pix, "k": int(k)}


def make_queries(seed: int, n: int, h0: int, s_range, k_range) -> list:
    """n queries with s ~ U{s_range} and k ~ U{k_range}, each with its own image."""
    ss = randint(seed, 20_000, n, s_range[0], s_range[1])
    ks = randint(seed, 20_001, n, k_range[0], k_range[1])
    return [make_query(seed, q, h0, int(ss[q]), int(ks[q])) for q in range(n)]


# The five workloads. Seeds are fixed here once and for all.
WORKLOADS = {
    "mlp25_sigmoid_s5k8": dict(seed=1001, dims=[25, 10, 5], act="sigmoid", w_var=1.0,
                               bias="normal", s=5, k=8),
    "mlp784x512x512_relu_s6k7": dict(seed=1002, dims=[784, 512, 512, 10], act="relu",
                                     w_var=2.0, bias="zero", s=6, k=7),
    "mlp784x1024x3_relu_s5k15": dict(seed=1003, dims=[784, 1024, 1024, 1024, 10], act="relu",
                                     w_var=2.0, bias="zero", s=5, k=15),
    "mlp784x256x256_relu_batch4096": dict(seed=1004, dims=[784, 256, 256, 10], act="relu",
                                          w_var=2.0, bias="zero", nq=4096,
                                          s_range=(2, 6), k_range=(3, 10)),
    # the 784-512-512-10 net above (net_seed 1002); training queries from seed
    # 1005, held-out queries from seed 1006; 64 contiguous tiles per query
    "proposal_mlp784x512x512_s6k7": dict(seed=1005, net_seed=1002, test_seed=1006,
                                         dims=[784, 512, 512, 10], act="relu", w_var=2.0,
                                         bias="zero", s=6, k=7, n_tiles=64),
    # coverage over a dataset of image pairs (Sec. III-B): the 784-512-512-10 net
    # (net_seed 1002); pair i is a random image and a noisy copy (every pixel
    # moved by a uniform integer in [-noise, noise], clipped); covers with value
    # ratio g and distance threshold d
    "pairs_mlp784x512x512_n65536": dict(seed=1007, net_seed=1002, dims=[784, 512, 512, 10],
                                        act="relu", w_var=2.0, bias="zero", n_pairs=65536,
                                        noise=16, g=2.0, d=1.0),
}


def make_pairs(seed: int, n: int, h0: int, noise: int):
    """n image pairs (uint8 [n, h0] each): uniform grey levels and a noisy copy."""
    a = randint(seed, 30_000, n * h0, 0, 255).reshape(n, h0)
    e = randint(seed, 30_001, n * h0, -noise, noise).reshape(n, h0)
    b = np.clip(a + e, 0, 255)
    return a.astype(np.uint8), b.astype(np.uint8)


def workload(name: str, **override) -> dict:
    """Net plus query (or queries) of a named workload; keyword overrides shrink it."""
    cfg = dict(WORKLOADS[name])
    cfg.update(override)
    net = make_net(cfg.get("net_seed", cfg["seed"]), cfg["dims"], cfg["act"], cfg["w_var"],
                   cfg["bias"])
    out = {"name": name, "net": net, "cfg": cfg}
    if "n_pairs" in cfg:
        out["pairs"] = make_pairs(cfg["seed"], cfg["n_pairs"], cfg["dims"][0], cfg["noise"])
    elif "nq" in cfg:
        out["queries"] = make_queries(cfg["seed"], cfg["nq"], cfg["dims"][0],
                                      cfg["s_range"], cfg["k_range"])
    else:
        out["query"] = make_query(cfg["seed"], 0, cfg["dims"][0], cfg["s"], cfg["k"])
    return out


def proposal_candidates(split: str, n: int, start: int = 0, **override) -> list:
    """Candidate queries of the tile-proposal workload: 'train' or 'test' split,
    queries start .. start + n - 1, each with its own image and s pixels."""
    cfg = dict(WORKLOADS["proposal_mlp784x512x512_s6k7"])
    cfg.update(override)
    seed = cfg["seed"] if split == "train" else cfg["test_seed"]
    return [make_query(seed, i, cfg["dims"][0], cfg["s"], cfg["k"]) for i in range(start, start + n)]
