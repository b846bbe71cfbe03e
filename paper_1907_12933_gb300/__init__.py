"""Python binding of libvbmc (include/vbmc.h): argument marshalling only.

Every step of the verification runs in the CUDA library. PyTorch supplies the
CUDA stream (and, for the device-resident entry point, device memory). There
is no CPU fallback: importing this package without the built library, or
calling it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvbmc.so")

PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3, "fp8": 4}
ACTS = {"identity": 0, "sigmoid": 1, "relu": 2}
VERDICTS = {0: "SAFE", 1: "UNSAFE", 2: "TIES_ONLY", 3: "PARTIAL"}
NO_WITNESS = 2**64 - 1
MAX_S, MAX_K = 16, 127


class VbmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"vbmc status {status}: {msg}")
        self.status = status


class VbmcTimeout(VbmcError):
    """VBMC_ERR_TIMEOUT: the time budget ran out; `summary` is the result of the
    checked prefix [lo, summary["checked_hi"])."""

    def __init__(self, status: int, msg: str, summary: dict):
        super().__init__(status, msg)
        self.summary = summary


class _MlpDesc(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("dims", C.POINTER(C.c_int32)),
                ("W", C.POINTER(C.POINTER(C.c_float))), ("b", C.POINTER(C.POINTER(C.c_float))),
                ("hidden_act", C.c_int32)]


class _Query(C.Structure):
    _fields_ = [("image", C.POINTER(C.c_uint8)), ("s", C.c_int32),
                ("pixels", C.POINTER(C.c_int32)), ("k", C.c_int32), ("lo", C.c_uint64),
                ("hi", C.c_uint64), ("filter", C.c_int32), ("l2_max", C.c_int64),
                ("property", C.c_int32), ("threshold", C.c_double)]


FILTER_L2, FILTER_SHELL = 1, 2
PROP_ARGMAX, PROP_THRESHOLD = 0, 1


def _query(img, pix, k, lo=0, hi=0, filter=0, l2_max=0, threshold=None) -> _Query:
    """vbmc_query over numpy buffers; threshold=None checks Eq. 10, a number V the
    misclassified literal of Eq. 11 (y_D < V and y_i > V for some i != D)."""
    prop = PROP_ARGMAX if threshold is None else PROP_THRESHOLD
    return _Query(_ptr(img, C.c_uint8), len(pix), _ptr(pix, C.c_int32), int(k), int(lo), int(hi),
                  int(filter), int(l2_max), prop, 0.0 if threshold is None else float(threshold))


def l2_max_of(radius: float) -> int:
    """l2_max for a Euclidean radius on the [0, 1] pixel scale (Eq. 9)."""
    return int(np.floor((255.0 * radius) ** 2 + 1e-9))


class _Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("coverage", C.c_int32), ("bitmap", C.c_int32),
                ("graph", C.c_int32), ("schedule", C.c_int32), ("time_budget_ms", C.c_double)]


SCHEDULES = {"given": 0, "small_first": 1}


class _Caps(C.Structure):
    _fields_ = [("max_points", C.c_uint64), ("max_s", C.c_int32), ("max_k", C.c_int32),
                ("ties_cap", C.c_uint32), ("queue_cap", C.c_uint64), ("wide_chunk", C.c_int64)]


class _Summary(C.Structure):
    _fields_ = [("verdict", C.c_int32), ("D", C.c_int32), ("base_margin", C.c_double),
                ("n_points", C.c_uint64), ("n_adversarial", C.c_uint64),
                ("first_witness", C.c_uint64), ("n_ties", C.c_uint64),
                ("n_recheck", C.c_uint64 * 4), ("ms_device", C.c_double),
                ("ms_prologue", C.c_double), ("ms_screen", C.c_double),
                ("ms_recheck", C.c_double), ("ms_to_verdict", C.c_double),
                ("ms_pass", C.c_double * 4), ("checked_hi", C.c_uint64)]


class _SearchOut(C.Structure):
    _fields_ = [("tiles_checked", C.c_int32), ("witness_tile", C.c_int32),
                ("points_checked", C.c_uint64), ("ms_to_witness", C.c_double)]


class _Tuning(C.Structure):
    _fields_ = [("simt_range", C.c_int32), ("simt_range_ctas", C.c_int32),
                ("simt_gather", C.c_int32), ("simt_gather_ctas", C.c_int32),
                ("df_ctas", C.c_int32), ("from_cache", C.c_int32), ("ms_range", C.c_double),
                ("ms_gather", C.c_double), ("ms_df", C.c_double)]


class _CoverParams(C.Structure):
    _fields_ = [("g", C.c_double), ("d", C.c_double)]


PAIR_MASKS = ("flip", "flip_tie", "ss", "ss_tie", "sv", "sv_tie", "ds", "ds_tie", "dv", "dv_tie")


class _PairMasks(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in PAIR_MASKS]


class _ShellOut(C.Structure):
    _fields_ = [("radius", C.c_int32), ("points_checked", C.c_uint64), ("n_ties", C.c_uint64),
                ("ms_device", C.c_double)]


class _NoallocOut(C.Structure):
    _fields_ = [("counters", C.c_void_p), ("flip", C.c_void_p), ("flip_tie", C.c_void_p),
                ("ss", C.c_void_p), ("ss_tie", C.c_void_p), ("bitmap", C.c_void_p),
                ("bitmap_bits", C.c_uint64), ("ties", C.c_void_p), ("ties_cap", C.c_uint32)]


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                              "(no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        vp, st = C.c_void_p, C.c_int
        sig = {
            "vbmc_net_create": [C.POINTER(_MlpDesc), C.POINTER(vp)],
            "vbmc_net_free": [vp],
            "vbmc_net_prepare": [vp, C.c_int32],
            "vbmc_result_create": [vp, C.POINTER(_Caps), C.POINTER(vp)],
            "vbmc_result_free": [vp],
            "vbmc_result_create_batch": [vp, C.POINTER(_Caps), C.c_int32, C.POINTER(vp)],
            "vbmc_verify_query": [vp, C.POINTER(_Query), C.POINTER(_Options), vp, vp],
            "vbmc_verify_query_device": [vp, vp, C.c_int32, vp, C.c_int32, C.c_uint64,
                                         C.c_uint64, C.POINTER(_Options), vp, vp],
            "vbmc_verify_batch": [vp, C.POINTER(_Query), C.c_int32, C.POINTER(_Options),
                                  C.POINTER(vp), vp],
            "vbmc_result_summary": [vp, C.POINTER(_Summary)],
            "vbmc_get_witness": [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_uint8), C.POINTER(C.c_double)],
            "vbmc_get_coverage": [vp, C.POINTER(C.c_uint32), C.c_size_t, C.POINTER(C.c_uint32),
                                  C.POINTER(C.c_uint32), C.c_size_t, C.POINTER(C.c_uint32),
                                  C.POINTER(C.c_double)],
            "vbmc_mask_words": [vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)],
            "vbmc_get_verdict_bitmap": [vp, C.POINTER(C.c_uint32), C.c_size_t],
            "vbmc_get_ties": [vp, C.POINTER(C.c_uint64), C.c_size_t, C.POINTER(C.c_uint64)],
            "vbmc_verify_range_fp64_noalloc": [vp, vp, C.c_int32, vp, C.c_int32, C.c_uint64,
                                               C.c_uint64, C.POINTER(_NoallocOut), vp],
            "vbmc_search_query": [vp, C.POINTER(_Query), C.c_int32, C.POINTER(C.c_int32),
                                  C.POINTER(_Options), vp, C.POINTER(_SearchOut), vp],
            "vbmc_tile_counts": [vp, C.c_int32, C.POINTER(C.c_uint64)],
            "vbmc_shell_search": [vp, C.POINTER(_Query), C.POINTER(_Options), vp, C.POINTER(_ShellOut), vp],
            "vbmc_autotune": [vp, C.c_char_p, C.POINTER(_Tuning)],
            "vbmc_fp8_accumulation_unit": [vp, C.POINTER(C.c_double)],
            "vbmc_tc_accumulation_unit": [vp, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_int32)],
            "vbmc_pair_coverage": [vp, vp, vp, C.c_int32, C.POINTER(_CoverParams),
                                   C.POINTER(_PairMasks), vp],
            "vbmc_covered_fraction": [vp, C.c_int32, C.POINTER(C.c_uint32), C.POINTER(C.c_double)],
            "vbmc_wide_trace": [vp, C.POINTER(_Query), C.c_int32, C.c_int32, C.POINTER(C.c_float),
                                C.POINTER(C.c_float), vp, vp],
            "vbmc_enum_coverage": [vp, C.POINTER(_Query), C.POINTER(_CoverParams), C.POINTER(_PairMasks), vp,
                                   C.POINTER(C.c_uint64), vp],
            "vbmc_set_tuning": [vp, C.POINTER(_Tuning)],
            "vbmc_proposal_create": [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                     C.c_uint64, C.POINTER(vp)],
            "vbmc_proposal_free": [vp],
            "vbmc_proposal_features": [vp, vp, vp, vp, vp, C.c_int32, C.c_int32, vp, vp, vp, vp],
            "vbmc_proposal_scores": [vp, vp, C.c_int32, vp, vp, vp],
            "vbmc_proposal_grads": [vp, vp, vp, C.c_int32, C.c_int32, C.POINTER(C.c_float), vp],
            "vbmc_proposal_train_step": [vp, vp, vp, C.c_int32, C.c_float, C.c_float,
                                         C.POINTER(C.c_float), vp],
            "vbmc_proposal_params": [vp, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                     C.POINTER(C.c_float), C.POINTER(C.c_float)],
            "vbmc_proposal_set_params": [vp, C.c_int32, C.POINTER(C.c_float),
                                         C.POINTER(C.c_float)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = st
        L.vbmc_last_error.restype = C.c_char_p
        L.vbmc_last_error.argtypes = []
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise VbmcError(rc, lib().vbmc_last_error().decode())


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def current_stream() -> int:
    """cudaStream_t of torch's current stream (0 when torch has no CUDA)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:  # noqa: BLE001 - no torch: legacy default stream
        pass
    return 0


class Net:
    """vbmc_net_create / vbmc_net_free. `net` has dims, W (list of (H_out, H_in)
    float32), b, act ('sigmoid' | 'relu' | 'identity')."""

    def __init__(self, net: dict):
        self.dims = [int(d) for d in net["dims"]]
        W = [np.ascontiguousarray(w, dtype=np.float32) for w in net["W"]]
        b = [np.ascontiguousarray(x, dtype=np.float32) for x in net["b"]]
        L = len(W)
        dims = np.ascontiguousarray(self.dims, dtype=np.int32)
        Wp = (C.POINTER(C.c_float) * L)(*[_ptr(w, C.c_float) for w in W])
        bp = (C.POINTER(C.c_float) * L)(*[_ptr(x, C.c_float) for x in b])
        act = net["act"] if isinstance(net["act"], int) else ACTS[net["act"]]
        desc = _MlpDesc(L, _ptr(dims, C.c_int32), Wp, bp, act)
        h = C.c_void_p()
        _check(lib().vbmc_net_create(C.byref(desc), C.byref(h)))
        self.h = h

    def mask_words(self) -> tuple[int, int]:
        fw, sw = C.c_size_t(), C.c_size_t()
        _check(lib().vbmc_mask_words(self.h, C.byref(fw), C.byref(sw)))
        return fw.value, sw.value

    def free(self):
        if getattr(self, "h", None):
            lib().vbmc_net_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


class Result:
    """vbmc_result_create / vbmc_result_free: a reusable workspace."""

    def __init__(self, net: Net, max_points: int = 0, max_s: int = MAX_S, max_k: int = 32,
                 ties_cap: int = 1 << 16, queue_cap: int = 1 << 22, wide_chunk: int = 0):
        caps = _Caps(max_points, max_s, max_k, ties_cap, queue_cap, wide_chunk)
        h = C.c_void_p()
        _check(lib().vbmc_result_create(net.h, C.byref(caps), C.byref(h)))
        self.h = h
        self.net = net

    def free(self):
        if getattr(self, "h", None):
            lib().vbmc_result_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


def result_create_batch(net: Net, nq: int, max_points: int = 0, max_s: int = MAX_S,
                        max_k: int = 32, ties_cap: int = 1 << 12, queue_cap: int = 1 << 24,
                        wide_chunk: int = 0) -> list:
    """vbmc_result_create_batch: nq workspaces that vbmc_verify_batch serves together."""
    caps = _Caps(max_points, max_s, max_k, ties_cap, queue_cap, wide_chunk)
    hs = (C.c_void_p * nq)()
    _check(lib().vbmc_result_create_batch(net.h, C.byref(caps), nq, hs))
    out = []
    for i in range(nq):
        r = Result.__new__(Result)
        r.h = C.c_void_p(hs[i])
        r.net = net
        out.append(r)
    return out


def _options(precision, coverage, bitmap, graph=False, schedule="given", time_budget_ms=0.0):
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    sc = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    return _Options(p, int(bool(coverage)), int(bool(bitmap)), int(bool(graph)), sc,
                    float(time_budget_ms))


def _summary_dict(s: _Summary) -> dict:
    return {"verdict": VERDICTS.get(s.verdict, s.verdict), "D": s.D, "base_margin": s.base_margin,
            "n_points": s.n_points, "n_adversarial": s.n_adversarial,
            "first_witness": None if s.first_witness == NO_WITNESS else int(s.first_witness),
            "n_ties": s.n_ties, "n_recheck": list(s.n_recheck), "ms_device": s.ms_device,
            "ms_prologue": s.ms_prologue, "ms_screen": s.ms_screen, "ms_recheck": s.ms_recheck,
            "ms_to_verdict": s.ms_to_verdict, "ms_pass": list(s.ms_pass),
            "checked_hi": int(s.checked_hi)}


def verify_query(net: Net, res: Result, image, pixels, k: int, lo: int = 0, hi: int = 0,
                 precision="fp32", coverage: bool = True, bitmap: bool = True,
                 filter: int = 0, l2_max: int = 0, threshold: float | None = None,
                 stream: int | None = None, wait: bool = True,
                 time_budget_ms: float = 0.0) -> dict | None:
    """vbmc_verify_query: host inputs; with wait (default) blocks until the result
    is final and returns its summary, else returns once the work is enqueued.
    filter: FILTER_L2 (with l2_max) and/or FILTER_SHELL; threshold V: check Eq. 11."""
    img = np.ascontiguousarray(image, dtype=np.uint8)
    pix = np.ascontiguousarray(pixels, dtype=np.int32)
    q = _query(img, pix, k, lo, hi, filter, l2_max, threshold)
    opt = _options(precision, coverage, bitmap, time_budget_ms=time_budget_ms)
    st = current_stream() if stream is None else stream
    rc = lib().vbmc_verify_query(net.h, C.byref(q), C.byref(opt), res.h, C.c_void_p(st))
    if rc == -4:  # VBMC_ERR_TIMEOUT: the result holds the checked prefix
        raise VbmcTimeout(rc, lib().vbmc_last_error().decode(), result_summary_partial(res))
    _check(rc)
    return result_summary(res) if wait else None


def verify_query_device(net: Net, res: Result, d_image, d_pixels, k: int, lo: int = 0,
                        hi: int = 0, precision="fp32", coverage: bool = True, bitmap: bool = True,
                        stream: int | None = None) -> None:
    """vbmc_verify_query_device: image (uint8) and pixels (int32) are CUDA tensors;
    enqueues on `stream` (default: torch's current stream) and returns."""
    opt = _options(precision, coverage, bitmap)
    st = current_stream() if stream is None else stream
    _check(lib().vbmc_verify_query_device(net.h, C.c_void_p(d_image.data_ptr()),
                                          int(d_pixels.numel()), C.c_void_p(d_pixels.data_ptr()),
                                          int(k), int(lo), int(hi), C.byref(opt), res.h,
                                          C.c_void_p(st)))


def verify_batch(net: Net, results: list, queries: list, precision="fp32",
                 coverage: bool = True, bitmap: bool = False, graph: bool = False,
                 schedule="given", stream: int | None = None) -> list:
    """vbmc_verify_batch: queries are dicts with image, pixels, k (and optional lo, hi,
    filter, l2_max, threshold); schedule 'given' or 'small_first' (tiles of smaller
    spaces first)."""
    keep = []
    qs = (_Query * len(queries))()
    for i, qd in enumerate(queries):
        img = np.ascontiguousarray(qd["image"], dtype=np.uint8)
        pix = np.ascontiguousarray(qd["pixels"], dtype=np.int32)
        keep += [img, pix]
        qs[i] = _query(img, pix, qd["k"], qd.get("lo", 0), qd.get("hi", 0), qd.get("filter", 0),
                       qd.get("l2_max", 0), qd.get("threshold"))
    hs = (C.c_void_p * len(results))(*[r.h for r in results])
    opt = _options(precision, coverage, bitmap, graph, schedule)
    st = current_stream() if stream is None else stream
    _check(lib().vbmc_verify_batch(net.h, qs, len(queries), C.byref(opt), hs, C.c_void_p(st)))
    return [result_summary(r) for r in results]


def result_summary_partial(res: Result) -> dict:
    """vbmc_result_summary of a call that timed out (the summary of its prefix)."""
    s = _Summary()
    lib().vbmc_result_summary(res.h, C.byref(s))
    return _summary_dict(s)


def result_summary(res: Result) -> dict:
    s = _Summary()
    _check(lib().vbmc_result_summary(res.h, C.byref(s)))
    return _summary_dict(s)


def get_witness(res: Result, s: int, h0: int) -> dict | None:
    """vbmc_get_witness: first adversarial index, its steps, image and FP64 margin."""
    idx = C.c_uint64()
    steps = np.zeros(max(1, s), dtype=np.int32)
    img = np.zeros(h0, dtype=np.uint8)
    m = C.c_double()
    _check(lib().vbmc_get_witness(res.h, C.byref(idx), _ptr(steps, C.c_int32),
                                  _ptr(img, C.c_uint8), C.byref(m)))
    if idx.value == NO_WITNESS:
        return None
    return {"index": int(idx.value), "steps": steps[:s], "image": img, "margin": m.value}


def get_coverage(res: Result) -> dict:
    """vbmc_get_coverage: sign-change and SS masks (uint32 words) and Eq. 3's fraction."""
    fw, sw = res.net.mask_words()
    f, ft = np.zeros(fw, np.uint32), np.zeros(fw, np.uint32)
    s, stt = np.zeros(sw, np.uint32), np.zeros(sw, np.uint32)
    frac = C.c_double()
    _check(lib().vbmc_get_coverage(res.h, _ptr(f, C.c_uint32), fw, _ptr(ft, C.c_uint32),
                                   _ptr(s, C.c_uint32), sw, _ptr(stt, C.c_uint32),
                                   C.byref(frac)))
    return {"flip": f, "flip_tie": ft, "ss": s, "ss_tie": stt, "covered_fraction": frac.value}


def get_verdict_bitmap(res: Result, n_points: int) -> np.ndarray:
    w = np.zeros(max(1, (n_points + 31) // 32), np.uint32)
    _check(lib().vbmc_get_verdict_bitmap(res.h, _ptr(w, C.c_uint32), len(w)))
    return w


def get_ties(res: Result, cap: int = 1 << 16) -> np.ndarray:
    n = C.c_uint64()
    out = np.zeros(max(1, cap), np.uint64)
    _check(lib().vbmc_get_ties(res.h, _ptr(out, C.c_uint64), cap, C.byref(n)))
    return out[:min(n.value, cap)].astype(np.int64)


def verify_range_fp64_noalloc(net: Net, d_image, d_pixels, k: int, lo: int, hi: int, counters,
                              flip=None, flip_tie=None, ss=None, ss_tie=None, bitmap=None,
                              ties=None, stream: int | None = None) -> None:
    """vbmc_verify_range_fp64_noalloc: the FP64 check of [lo, hi) for callers that
    cannot allocate device memory. Every argument is a CUDA tensor the caller owns
    (counters: 4 x int64; masks and bitmap: int32 words; ties: int64); the library
    allocates nothing. Enqueued on `stream`; read the outputs after it finishes."""
    def ptr(t):
        return None if t is None else t.data_ptr()
    out = _NoallocOut(ptr(counters), ptr(flip), ptr(flip_tie), ptr(ss), ptr(ss_tie), ptr(bitmap),
                      0 if bitmap is None else 32 * bitmap.numel(), ptr(ties),
                      0 if ties is None else ties.numel())
    st = current_stream() if stream is None else stream
    _check(lib().vbmc_verify_range_fp64_noalloc(net.h, C.c_void_p(d_image.data_ptr()),
                                                int(d_pixels.numel()),
                                                C.c_void_p(d_pixels.data_ptr()), int(k), int(lo),
                                                int(hi), C.byref(out), C.c_void_p(st)))


def fp8_accumulation_unit(net: Net) -> float:
    """vbmc_fp8_accumulation_unit: the per-product accumulation error the FP8 bound uses."""
    u = C.c_double()
    _check(lib().vbmc_fp8_accumulation_unit(net.h, C.byref(u)))
    return u.value


def net_prepare(net: Net, precision: str) -> None:
    """vbmc_net_prepare: build a tensor precision's operands now (no later allocation)."""
    _check(lib().vbmc_net_prepare(net.h, PRECISIONS[precision]))


def tc_accumulation_unit(net: Net, precision: str = "bf16") -> tuple[float, float, int]:
    """vbmc_tc_accumulation_unit: (unit, worst, probes_failed) of the kind::f16
    accumulator self-test."""
    u, w, f = C.c_double(), C.c_double(), C.c_int32()
    _check(lib().vbmc_tc_accumulation_unit(net.h, PRECISIONS[precision], C.byref(u), C.byref(w),
                                           C.byref(f)))
    return u.value, w.value, f.value


def autotune(net: Net, cache_path: str | None = None) -> dict:
    """vbmc_autotune: time the FP32 and double-float pass launch shapes on a sample
    box of the net, apply the fastest, and cache them (JSON lines) in cache_path."""
    t = _Tuning()
    _check(lib().vbmc_autotune(net.h, None if cache_path is None else cache_path.encode(),
                               C.byref(t)))
    return {f: getattr(t, f) for f, _ in _Tuning._fields_}


def set_tuning(net: Net, **fields) -> None:
    """vbmc_set_tuning: apply launch shapes (missing fields: the built-in choice)."""
    t = _Tuning(**{k: int(v) for k, v in fields.items() if k in dict(_Tuning._fields_)})
    _check(lib().vbmc_set_tuning(net.h, C.byref(t)))


def search_query(net: Net, res: Result, image, pixels, k: int, order, precision="bf16",
                 coverage: bool = False, bitmap: bool = False, filter: int = 0, l2_max: int = 0,
                 threshold: float | None = None, stream: int | None = None) -> dict:
    """vbmc_search_query: check the len(order) contiguous tiles of the query's space in
    the given order and stop after the first tile holding a witness. Returns the
    search record merged into the result summary."""
    img = np.ascontiguousarray(image, dtype=np.uint8)
    pix = np.ascontiguousarray(pixels, dtype=np.int32)
    o = np.ascontiguousarray(order, dtype=np.int32)
    q = _query(img, pix, k, 0, 0, filter, l2_max, threshold)
    opt = _options(precision, coverage, bitmap)
    out = _SearchOut()
    st = current_stream() if stream is None else stream
    _check(lib().vbmc_search_query(net.h, C.byref(q), len(o), _ptr(o, C.c_int32), C.byref(opt),
                                   res.h, C.byref(out), C.c_void_p(st)))
    d = result_summary(res)
    d.update(tiles_checked=out.tiles_checked,
             witness_tile=None if out.witness_tile < 0 else out.witness_tile,
             points_checked=int(out.points_checked), ms_to_witness=out.ms_to_witness)
    return d


def tile_counts(res: Result, n_tiles: int) -> np.ndarray:
    """vbmc_tile_counts: adversarial points per contiguous tile of the last full check."""
    out = np.zeros(n_tiles, np.uint64)
    _check(lib().vbmc_tile_counts(res.h, int(n_tiles), _ptr(out, C.c_uint64)))
    return out.astype(np.int64)


def proposal_features(net: Net, d_images, d_pixels, d_s, d_k, d_features, d_reach=None,
                      d_margin=None, stream: int | None = None) -> None:
    """vbmc_proposal_features on CUDA tensors: images uint8 [nq, H0], pixels int32
    [nq, stride], s and k int32 [nq]; features float32 [nq, 3 * H0]; optional reach
    and margin float32 [nq]."""
    nq, stride = int(d_pixels.shape[0]), int(d_pixels.shape[1])
    st = current_stream() if stream is None else stream
    _check(lib().vbmc_proposal_features(
        net.h, C.c_void_p(d_images.data_ptr()), C.c_void_p(d_pixels.data_ptr()),
        C.c_void_p(d_s.data_ptr()), C.c_void_p(d_k.data_ptr()), stride, nq,
        C.c_void_p(d_features.data_ptr()),
        None if d_reach is None else C.c_void_p(d_reach.data_ptr()),
        None if d_margin is None else C.c_void_p(d_margin.data_ptr()), C.c_void_p(st)))


class Proposal:
    """vbmc_proposal_*: the tile-ranking MLP with its GPU training step."""

    def __init__(self, dims=(2352, 256, 256, 64), max_batch: int = 256, seed: int = 1):
        self.dims = tuple(int(d) for d in dims)
        self.max_batch = int(max_batch)
        h = C.c_void_p()
        _check(lib().vbmc_proposal_create(*self.dims, self.max_batch, int(seed), C.byref(h)))
        self.h = h

    def scores(self, d_X, d_scores, d_order=None, stream: int | None = None) -> None:
        st = current_stream() if stream is None else stream
        _check(lib().vbmc_proposal_scores(
            self.h, C.c_void_p(d_X.data_ptr()), int(d_X.shape[0]), C.c_void_p(d_scores.data_ptr()),
            None if d_order is None else C.c_void_p(d_order.data_ptr()), C.c_void_p(st)))

    def grads(self, d_X, d_T, bf16: bool = False, stream: int | None = None) -> float:
        loss = C.c_float()
        st = current_stream() if stream is None else stream
        _check(lib().vbmc_proposal_grads(self.h, C.c_void_p(d_X.data_ptr()),
                                         C.c_void_p(d_T.data_ptr()), int(d_X.shape[0]),
                                         int(bool(bf16)), C.byref(loss), C.c_void_p(st)))
        return loss.value

    def train_step(self, d_X, d_T, lr: float, weight_decay: float = 0.0,
                   want_loss: bool = False, stream: int | None = None):
        loss = C.c_float()
        st = current_stream() if stream is None else stream
        _check(lib().vbmc_proposal_train_step(
            self.h, C.c_void_p(d_X.data_ptr()), C.c_void_p(d_T.data_ptr()), int(d_X.shape[0]),
            float(lr), float(weight_decay), C.byref(loss) if want_loss else None, C.c_void_p(st)))
        return loss.value if want_loss else None

    def params(self, layer: int) -> dict:
        n_out, n_in = self.dims[layer], self.dims[layer - 1]
        W = np.zeros((n_out, n_in), np.float32)
        b = np.zeros(n_out, np.float32)
        gW = np.zeros((n_out, n_in), np.float32)
        gb = np.zeros(n_out, np.float32)
        _check(lib().vbmc_proposal_params(self.h, layer, _ptr(W, C.c_float), _ptr(b, C.c_float),
                                          _ptr(gW, C.c_float), _ptr(gb, C.c_float)))
        return {"W": W, "b": b, "gW": gW, "gb": gb}

    def set_params(self, layer: int, W, b) -> None:
        Wc = np.ascontiguousarray(W, dtype=np.float32)
        bc = np.ascontiguousarray(b, dtype=np.float32)
        assert Wc.shape == (self.dims[layer], self.dims[layer - 1]) and bc.shape == (self.dims[layer],)
        _check(lib().vbmc_proposal_set_params(self.h, layer, _ptr(Wc, C.c_float), _ptr(bc, C.c_float)))

    def free(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            lib().vbmc_proposal_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def pair_coverage(net: Net, images1, images2, g: float = 2.0, d: float = 1.0,
                  stream: int | None = None) -> dict:
    """vbmc_pair_coverage over n image pairs (uint8 arrays [n, H0]): every cover
    mask (flip, SS, SV, DS, DV and their tie masks, uint32 words) and the Eq. 3-6
    fractions of SS, SV, DS and DV."""
    import torch
    a = np.ascontiguousarray(images1, dtype=np.uint8)
    b = np.ascontiguousarray(images2, dtype=np.uint8)
    assert a.shape == b.shape
    fw, sw = net.mask_words()
    words = {k: (fw if k in ("flip", "flip_tie", "ds", "ds_tie", "dv", "dv_tie") else sw) for k in PAIR_MASKS}
    dev = {k: torch.zeros(max(1, n), dtype=torch.int32, device="cuda") for k, n in words.items()}
    da = torch.from_numpy(a).to("cuda")
    db = torch.from_numpy(b).to("cuda")
    masks = _PairMasks(*[dev[k].data_ptr() for k in PAIR_MASKS])
    params = _CoverParams(float(g), float(d))
    st = current_stream() if stream is None else stream
    _check(lib().vbmc_pair_coverage(net.h, C.c_void_p(da.data_ptr()), C.c_void_p(db.data_ptr()),
                                    int(a.shape[0]) if a.ndim > 1 else 0, C.byref(params),
                                    C.byref(masks), C.c_void_p(st)))
    torch.cuda.synchronize()
    out = {k: dev[k].cpu().numpy().view(np.uint32)[:words[k]] for k in PAIR_MASKS}
    for name, layout in (("ss", 0), ("sv", 0), ("ds", 1), ("dv", 1)):
        m = np.ascontiguousarray(out[name]) if len(out[name]) else np.zeros(1, np.uint32)
        f = C.c_double()
        _check(lib().vbmc_covered_fraction(net.h, layout, _ptr(m, C.c_uint32), C.byref(f)))
        out[name + "_fraction"] = f.value
    return out


def _masks_out(net: Net, dev: dict) -> dict:
    """Host copies of device masks and the Eq. 3-6 fractions of SS, SV, DS, DV."""
    import torch
    torch.cuda.synchronize()
    fw, sw = net.mask_words()
    words = {k: (fw if k in ("flip", "flip_tie", "ds", "ds_tie", "dv", "dv_tie") else sw) for k in PAIR_MASKS}
    out = {k: dev[k].cpu().numpy().view(np.uint32)[:words[k]] for k in PAIR_MASKS}
    for name, layout in (("ss", 0), ("sv", 0), ("ds", 1), ("dv", 1)):
        m = np.ascontiguousarray(out[name]) if len(out[name]) else np.zeros(1, np.uint32)
        f = C.c_double()
        _check(lib().vbmc_covered_fraction(net.h, layout, _ptr(m, C.c_uint32), C.byref(f)))
        out[name + "_fraction"] = f.value
    return out


def enum_coverage(net: Net, res: Result, image, pixels, k: int, g: float = 2.0, d: float = 1.0,
                  lo: int = 0, hi: int = 0, filter: int = 0, l2_max: int = 0,
                  stream: int | None = None) -> dict:
    """vbmc_enum_coverage: every cover (flip, SS, SV, DS, DV and their tie masks) over
    the pairs (unperturbed image, point) of the query's box, FP64; the masks, the
    Eq. 3-6 fractions and the number of points checked."""
    img = np.ascontiguousarray(image, dtype=np.uint8)
    pix = np.ascontiguousarray(pixels, dtype=np.int32)
    q = _query(img, pix, k, lo, hi, filter, l2_max)
    dev = pair_masks_device(net)
    masks = _PairMasks(*[dev[kk].data_ptr() for kk in PAIR_MASKS])
    params = _CoverParams(float(g), float(d))
    npts = C.c_uint64()
    st = current_stream() if stream is None else stream
    _check(lib().vbmc_enum_coverage(net.h, C.byref(q), C.byref(params), C.byref(masks), res.h, C.byref(npts),
                                    C.c_void_p(st)))
    out = _masks_out(net, dev)
    out["n_points"] = int(npts.value)
    return out


def wide_trace(net: Net, res: Result, image, pixels, k: int, precision: str, n_points: int,
               stream: int | None = None) -> tuple:
    """vbmc_wide_trace: per hidden layer the operand rows the wide-layer tensor path
    consumed for points 0..n_points-1 (float32 [L-1, n, H_max]) and their N, R, E
    ([L-1, n, 3]): ||operand - exact dh_l|| <= R + E."""
    img = np.ascontiguousarray(image, dtype=np.uint8)
    pix = np.ascontiguousarray(pixels, dtype=np.int32)
    q = _query(img, pix, k)
    L, hmax = len(net.dims) - 1, max(net.dims[1:])
    vals = np.zeros((L - 1, n_points, hmax), dtype=np.float32)
    nre = np.zeros((L - 1, n_points, 3), dtype=np.float32)
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    st = current_stream() if stream is None else stream
    _check(lib().vbmc_wide_trace(net.h, C.byref(q), p, int(n_points), _ptr(vals, C.c_float), _ptr(nre, C.c_float),
                                 res.h, C.c_void_p(st)))
    return vals, nre


def pair_masks_device(net: Net) -> dict:
    """Zeroed device buffers (int32 tensors) for every mask of vbmc_pair_coverage."""
    import torch
    fw, sw = net.mask_words()
    return {k: torch.zeros(max(1, fw if k in ("flip", "flip_tie", "ds", "ds_tie", "dv", "dv_tie") else sw),
                           dtype=torch.int32, device="cuda") for k in PAIR_MASKS}


def pair_coverage_device(net: Net, d_images1, d_images2, masks: dict, g: float = 2.0, d: float = 1.0,
                         stream: int | None = None) -> None:
    """vbmc_pair_coverage on device-resident pairs (uint8 CUDA tensors [n, H0]) into
    the device masks of pair_masks_device; enqueues on `stream` and returns."""
    n = int(d_images1.shape[0]) if d_images1.dim() > 1 else 0
    pm = _PairMasks(*[masks[k].data_ptr() for k in PAIR_MASKS])
    params = _CoverParams(float(g), float(d))
    st = current_stream() if stream is None else stream
    _check(lib().vbmc_pair_coverage(net.h, C.c_void_p(d_images1.data_ptr()), C.c_void_p(d_images2.data_ptr()),
                                    n, C.byref(params), C.byref(pm), C.c_void_p(st)))


def shell_search(net: Net, res: Result, image, pixels, k: int, precision="bf16",
                 coverage: bool = False, bitmap: bool = False, filter: int = 0, l2_max: int = 0,
                 threshold: float | None = None, stream: int | None = None) -> dict:
    """vbmc_shell_search: shells r = 0..k in order, stopping at the first one that
    holds a witness; the record merged into the last shell's summary."""
    img = np.ascontiguousarray(image, dtype=np.uint8)
    pix = np.ascontiguousarray(pixels, dtype=np.int32)
    q = _query(img, pix, k, 0, 0, filter, l2_max, threshold)
    opt = _options(precision, coverage, bitmap)
    out = _ShellOut()
    st = current_stream() if stream is None else stream
    _check(lib().vbmc_shell_search(net.h, C.byref(q), C.byref(opt), res.h, C.byref(out), C.c_void_p(st)))
    d = result_summary(res)
    d.update(radius=None if out.radius < 0 else out.radius, points_checked=int(out.points_checked),
             ties_total=int(out.n_ties), ms_total=out.ms_device)
    return d
