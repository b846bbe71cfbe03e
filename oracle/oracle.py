"""ctypes binding of the plain C oracle in vbmc_oracle.c.

Test infrastructure only: see the header of vbmc_oracle.c for what the oracle
computes and which passages of the paper each step follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vbmc_oracle.c")
LIB = os.path.join(HERE, "liborc.so")
TAU = 1e-9
ACTS = {"identity": 0, "sigmoid": 1, "relu": 2}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE double: no fast-math)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread",
                               "-fno-fast-math", "-ffp-contract=off",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Net(C.Structure):
    _fields_ = [("L", C.c_int), ("dims", C.POINTER(C.c_int)),
                ("W", C.POINTER(C.POINTER(C.c_float))), ("b", C.POINTER(C.POINTER(C.c_float))),
                ("act", C.c_int)]


class _Query(C.Structure):
    _fields_ = [("image", C.POINTER(C.c_uint8)), ("s", C.c_int), ("pixels", C.POINTER(C.c_int)),
                ("k", C.c_int), ("lo", C.c_uint64), ("hi", C.c_uint64), ("tau", C.c_double),
                ("bitmap", C.POINTER(C.c_uint32)), ("flip", C.POINTER(C.c_uint32)),
                ("flip_tie", C.POINTER(C.c_uint32)), ("ss", C.POINTER(C.c_uint32)),
                ("ss_tie", C.POINTER(C.c_uint32)), ("ties", C.POINTER(C.c_uint64)),
                ("ties_cap", C.c_uint64), ("D", C.c_int), ("base_margin", C.c_double),
                ("n_points", C.c_uint64), ("n_adv", C.c_uint64), ("first_witness", C.c_uint64),
                ("n_ties", C.c_uint64), ("filter", C.c_int), ("l2max", C.c_longlong),
                ("property", C.c_int), ("V", C.c_double)]


def configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    lib.orc_verify.argtypes = [C.POINTER(_Net), C.POINTER(_Query), C.c_int]
    lib.orc_verify.restype = C.c_int
    lib.orc_eval_point.argtypes = [C.POINTER(_Net), C.POINTER(C.c_uint8), C.c_int,
                                   C.POINTER(C.c_int), C.c_int, C.c_uint64,
                                   C.POINTER(C.c_double), C.POINTER(C.c_int),
                                   C.POINTER(C.c_double), C.POINTER(C.c_int)]
    lib.orc_pair_coverage.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.c_double] + \
        [C.POINTER(C.c_uint32)] * 4
    lib.orc_pair_covers.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.c_double, C.c_double, C.c_double] + \
        [C.POINTER(C.c_uint32)] * 6
    lib.orc_pair_covers.restype = None
    lib.orc_layer_pair_fraction.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_uint32)]
    lib.orc_layer_pair_fraction.restype = C.c_double
    lib.orc_ss_covered_fraction.argtypes = [C.c_int, C.POINTER(C.c_int),
                                            C.POINTER(C.c_uint32)]
    lib.orc_ss_covered_fraction.restype = C.c_double
    lib.orc_threshold_literal.argtypes = [C.POINTER(C.c_double), C.c_int, C.c_int, C.c_double,
                                          C.c_double]
    lib.orc_threshold_literal.restype = C.c_int
    lib.orc_threshold_margin.argtypes = [C.POINTER(C.c_double), C.c_int, C.c_int, C.c_double]
    lib.orc_threshold_margin.restype = C.c_double
    lib.orc_space_size.argtypes = [C.c_int, C.c_int]
    lib.orc_space_size.restype = C.c_uint64
    lib.orc_digits.argtypes = [C.c_uint64, C.c_int, C.c_int, C.POINTER(C.c_int)]
    lib.orc_ss_bits.argtypes = [C.c_int, C.POINTER(C.c_int)]
    lib.orc_ss_bits.restype = C.c_uint64
    lib.orc_forward.argtypes = [C.POINTER(_Net)] + [C.POINTER(C.c_double)] * 4
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = configure(C.CDLL(build()))
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


class _NetHandle:
    """Keeps the numpy buffers alive while the C struct points at them."""

    def __init__(self, net: dict):
        self.dims = np.ascontiguousarray(net["dims"], dtype=np.int32)
        self.W = [np.ascontiguousarray(w, dtype=np.float32) for w in net["W"]]
        self.b = [np.ascontiguousarray(b, dtype=np.float32) for b in net["b"]]
        L = len(self.W)
        self.Wp = (C.POINTER(C.c_float) * L)(*[_ptr(w, C.c_float) for w in self.W])
        self.bp = (C.POINTER(C.c_float) * L)(*[_ptr(b, C.c_float) for b in self.b])
        act = net["act"] if isinstance(net["act"], int) else ACTS[net["act"]]
        self.c = _Net(L, _ptr(self.dims, C.c_int), self.Wp, self.bp, act)


def mask_words(dims) -> tuple[int, int]:
    """(flip mask words, SS mask words) for a net with sizes dims."""
    L = len(dims) - 1
    total = sum(dims[1:])
    ss = sum(dims[l] * dims[l + 1] for l in range(1, L))
    return (total + 31) // 32, max(1, (ss + 31) // 32)


def space_size(s: int, k: int) -> int:
    return int(_load().orc_space_size(s, k))


def digits(t: int, s: int, k: int) -> list[int]:
    d = (C.c_int * max(1, s))()
    _load().orc_digits(t, s, k, d)
    return [d[i] for i in range(s)]


def verify(net: dict, query: dict, lo: int = 0, hi: int = 0, coverage: bool = True,
           bitmap: bool = True, nthreads: int | None = None, ties_cap: int = 1 << 16) -> dict:
    """Exhaustive FP64 check of points [lo, hi) (hi = 0: all R^s points)."""
    lib = _load()
    nh = _NetHandle(net)
    img = np.ascontiguousarray(query["image"], dtype=np.uint8)
    pix = np.ascontiguousarray(query["pixels"], dtype=np.int32)
    s, k = len(pix), int(query["k"])
    n = space_size(s, k)
    fw, sw = mask_words(net["dims"])
    bm = np.zeros(((n + 31) // 32) if bitmap else 1, dtype=np.uint32)
    masks = [np.zeros(fw, np.uint32), np.zeros(fw, np.uint32), np.zeros(sw, np.uint32),
             np.zeros(sw, np.uint32)]
    ties = np.zeros(max(1, ties_cap), dtype=np.uint64)
    q = _Query()
    q.image = _ptr(img, C.c_uint8)
    q.s = s
    q.pixels = _ptr(pix, C.c_int)
    q.k = k
    q.lo, q.hi, q.tau = lo, hi, TAU
    q.filter = int(query.get("filter", 0))
    q.l2max = int(query.get("l2_max", 0))
    q.property = int(query.get("property", 0))
    q.V = float(query.get("threshold", 0.0))
    q.bitmap = _ptr(bm, C.c_uint32) if bitmap else None
    if coverage:
        q.flip, q.flip_tie, q.ss, q.ss_tie = [_ptr(m, C.c_uint32) for m in masks]
    q.ties = _ptr(ties, C.c_uint64)
    q.ties_cap = ties_cap
    rc = lib.orc_verify(C.byref(nh.c), C.byref(q), nthreads or os.cpu_count() or 1)
    if rc != 0:
        raise ValueError("oracle rejected the query")
    out = {"D": q.D, "base_margin": q.base_margin, "n_points": q.n_points, "n_adv": q.n_adv,
           "first_witness": None if q.first_witness == 2**64 - 1 else int(q.first_witness),
           "n_ties": q.n_ties, "ties": np.sort(ties[:min(q.n_ties, ties_cap)]).astype(np.int64),
           "bitmap": bm if bitmap else None}
    if coverage:
        out.update(flip=masks[0], flip_tie=masks[1], ss=masks[2], ss_tie=masks[3])
    return out


def eval_point(net: dict, query: dict, t: int) -> dict:
    """FP64 activation potentials (all layers), class D, margin and verdict at point t
    (Eq. 10, or Eq. 11 when query["property"] == 1)."""
    lib = _load()
    nh = _NetHandle(net)
    img = np.ascontiguousarray(query["image"], dtype=np.uint8)
    pix = np.ascontiguousarray(query["pixels"], dtype=np.int32)
    u = np.zeros(sum(net["dims"][1:]), dtype=np.float64)
    D, adv, m = C.c_int(), C.c_int(), C.c_double()
    lib.orc_eval_point(C.byref(nh.c), _ptr(img, C.c_uint8), len(pix), _ptr(pix, C.c_int),
                       int(query["k"]), t, _ptr(u, C.c_double), C.byref(D), C.byref(m),
                       C.byref(adv))
    out = {"u": u, "D": D.value, "margin": m.value, "adversarial": bool(adv.value)}
    if int(query.get("property", 0)) == 1:  # Eq. 11 with V = query["threshold"]
        HL = int(net["dims"][-1])
        y = np.ascontiguousarray(u[-HL:])
        V = float(query["threshold"])
        lit = lib.orc_threshold_literal(_ptr(y, C.c_double), HL, D.value, V, TAU)
        out.update(margin=lib.orc_threshold_margin(_ptr(y, C.c_double), HL, D.value, V),
                   adversarial=lit == 1, tie=lit == 2)
    return out


def forward(net: dict, x) -> np.ndarray:
    """FP64 activation potentials of layers 1..L for an arbitrary input vector x."""
    lib = _load()
    nh = _NetHandle(net)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    u = np.zeros(sum(net["dims"][1:]), dtype=np.float64)
    hmax = max(net["dims"])
    h0, h1 = np.zeros(hmax), np.zeros(hmax)
    lib.orc_forward(C.byref(nh.c), _ptr(xx, C.c_double), _ptr(u, C.c_double),
                    _ptr(h0, C.c_double), _ptr(h1, C.c_double))
    return u


def pair_coverage(dims, u1, u2, tau: float = TAU) -> dict:
    """Sign-change and SS-Cover masks of one input pair from its activation potentials."""
    lib = _load()
    d = np.ascontiguousarray(dims, dtype=np.int32)
    a = np.ascontiguousarray(u1, dtype=np.float64)
    b = np.ascontiguousarray(u2, dtype=np.float64)
    fw, sw = mask_words(list(dims))
    masks = [np.zeros(fw, np.uint32), np.zeros(fw, np.uint32), np.zeros(sw, np.uint32),
             np.zeros(sw, np.uint32)]
    lib.orc_pair_coverage(len(dims) - 1, _ptr(d, C.c_int), _ptr(a, C.c_double),
                          _ptr(b, C.c_double), tau, *[_ptr(m, C.c_uint32) for m in masks])
    return dict(flip=masks[0], flip_tie=masks[1], ss=masks[2], ss_tie=masks[3])


def ss_covered_fraction(dims, ss) -> float:
    """Eq. 3's covered fraction from an SS mask."""
    d = np.ascontiguousarray(dims, dtype=np.int32)
    m = np.ascontiguousarray(ss, dtype=np.uint32)
    return float(_load().orc_ss_covered_fraction(len(dims) - 1, _ptr(d, C.c_int),
                                                 _ptr(m, C.c_uint32)))


def pair_covers(dims, u1, u2, g: float, d: float, tau: float = TAU) -> dict:
    """DS, DV (per layer-(k+1) neuron bit) and SV (SS layout) masks of one input
    pair, each with its tie mask (Sec. III-B)."""
    lib = _load()
    dd = np.ascontiguousarray(dims, dtype=np.int32)
    a = np.ascontiguousarray(u1, dtype=np.float64)
    b = np.ascontiguousarray(u2, dtype=np.float64)
    fw, sw = mask_words(list(dims))
    m = [np.zeros(fw, np.uint32) for _ in range(4)] + [np.zeros(sw, np.uint32) for _ in range(2)]
    lib.orc_pair_covers(len(dims) - 1, _ptr(dd, C.c_int), _ptr(a, C.c_double), _ptr(b, C.c_double),
                        tau, g, d, *[_ptr(x, C.c_uint32) for x in m])
    return dict(ds=m[0], ds_tie=m[1], dv=m[2], dv_tie=m[3], sv=m[4], sv_tie=m[5])


def layer_pair_fraction(dims, mask) -> float:
    """Eq. 4 / Eq. 6 covered fraction from a DS or DV mask."""
    dd = np.ascontiguousarray(dims, dtype=np.int32)
    m = np.ascontiguousarray(mask, dtype=np.uint32)
    return float(_load().orc_layer_pair_fraction(len(dims) - 1, _ptr(dd, C.c_int), _ptr(m, C.c_uint32)))


def pairs_coverage(net: dict, images1, images2, g: float, d: float, tau: float = TAU) -> dict:
    """Every cover (sign changes, SS, DS, SV, DV and their tie masks) ORed over a set
    of input pairs, from the FP64 potentials of each image."""
    dims = net["dims"]
    fw, sw = mask_words(list(dims))
    acc = {k: np.zeros(fw, np.uint32) for k in ("flip", "flip_tie", "ds", "ds_tie", "dv", "dv_tie")}
    acc.update({k: np.zeros(sw, np.uint32) for k in ("ss", "ss_tie", "sv", "sv_tie")})
    for x1, x2 in zip(images1, images2):
        u1 = forward(net, np.asarray(x1, np.float64) / 255.0)
        u2 = forward(net, np.asarray(x2, np.float64) / 255.0)
        for k, v in pair_coverage(dims, u1, u2, tau).items():
            acc[k] |= v
        for k, v in pair_covers(dims, u1, u2, g, d, tau).items():
            acc[k] |= v
    return acc


def threshold_literal(y, D: int, V: float, tau: float = TAU) -> int:
    """Eq. 11 on output vector y in three-valued logic: 1 true, 0 false, 2 tie."""
    lib = _load()
    a = np.ascontiguousarray(y, dtype=np.float64)
    return int(lib.orc_threshold_literal(_ptr(a, C.c_double), len(a), int(D), float(V), tau))


def threshold_margin(y, D: int, V: float) -> float:
    """max(y_D - V, V - max_{i != D} y_i): negative iff Eq. 11 holds."""
    lib = _load()
    a = np.ascontiguousarray(y, dtype=np.float64)
    return float(lib.orc_threshold_margin(_ptr(a, C.c_double), len(a), int(D), float(V)))
