"""The allocation-free entry point, for callers that cannot call cudaMalloc
(code living in another runtime's memory pool, or whose allocator must not be
re-entered): vbmc_verify_range_fp64_noalloc keeps its scratch in a fixed array
inside the library and writes only into the caller's buffers. Its results must
equal those of vbmc_verify_query in FP64 and of the FP64 CPU oracle, on two
calls in a row (the second call reuses the same scratch), on a sub-range, with
no tie buffer, and it must flag an invalid pixel list instead of checking it."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

BAD_PIXELS, TIES_CUT = 1, 4  # flags in the high word of counters[3]


@pytest.fixture(scope="module")
def vb():
    import torch
    assert torch.cuda.is_available()
    import paper_1907_12933_gb300 as m
    from paper_1907_12933_gb300 import build
    build.build()
    return m


def reference(vb, vnet, q, n):
    res = vb.Result(vnet, max_points=n, max_s=len(q["pixels"]), max_k=q["k"], queue_cap=n)
    s = vb.verify_query(vnet, res, q["image"], q["pixels"], q["k"], precision="fp64")
    cov = vb.get_coverage(res)
    bm = vb.get_verdict_bitmap(res, n)
    ties = np.sort(vb.get_ties(res))
    res.free()
    return s, cov, bm, ties


class Buffers:
    def __init__(self, vnet, nmax, ties_cap=1024):
        import torch
        fw, sw = vnet.mask_words()
        dev = torch.device("cuda")
        self.counters = torch.zeros(4, dtype=torch.int64, device=dev)
        self.masks = [torch.zeros(w, dtype=torch.int32, device=dev) for w in (fw, fw, sw, sw)]
        self.bitmap = torch.zeros((nmax + 31) // 32, dtype=torch.int32, device=dev)
        self.ties = torch.zeros(ties_cap, dtype=torch.int64, device=dev) if ties_cap else None

    def run(self, vb, vnet, q, lo=0, hi=0):
        import torch
        img = torch.tensor(q["image"], dtype=torch.uint8, device="cuda")
        pix = torch.tensor(q["pixels"], dtype=torch.int32, device="cuda")
        vb.verify_range_fp64_noalloc(vnet, img, pix, q["k"], lo, hi, self.counters, *self.masks,
                                     bitmap=self.bitmap, ties=self.ties)
        torch.cuda.synchronize()
        c = self.counters.cpu().numpy().astype(np.uint64)
        first = None if int(c[1]) == 2**64 - 1 else int(c[1])
        out = {"n_adv": int(c[0]), "first_witness": first, "n_ties": int(c[2]),
               "D": int(c[3]) & 0xFFFFFFFF, "flags": int(c[3]) >> 32,
               "bitmap": self.bitmap.cpu().numpy().view(np.uint32)}
        for m, key in zip(self.masks, ("flip", "flip_tie", "ss", "ss_tie")):
            out[key] = m.cpu().numpy().view(np.uint32)
        if self.ties is not None:
            out["ties"] = np.sort(self.ties.cpu().numpy()[:min(int(c[2]), self.ties.numel())])
        return out


def check_against_oracle(g, o, n, lo=0):
    assert g["D"] == o["D"]
    assert g["n_adv"] == o["n_adv"]
    assert g["first_witness"] == o["first_witness"]
    assert g["n_ties"] == o["n_ties"]
    if "ties" in g:
        np.testing.assert_array_equal(g["ties"], o["ties"])
    for key in ("flip", "flip_tie", "ss", "ss_tie"):
        np.testing.assert_array_equal(g[key], o[key], err_msg=key)
    bits_g = np.unpackbits(g["bitmap"].view(np.uint8), bitorder="little")[:n]
    bits_o = np.unpackbits(o["bitmap"].view(np.uint8), bitorder="little")[:n]
    np.testing.assert_array_equal(bits_g[lo:], bits_o[lo:])
    assert not bits_g[:lo].any()


def test_noalloc_equals_verify_query_and_oracle_on_two_calls(vb):
    net = synth.make_net(66, [6, 8, 6, 4], "relu", 2.0, "normal")
    queries = [synth.make_query(66, 1, 6, 3, 12), synth.make_query(66, 2, 6, 2, 20)]
    vnet = vb.Net(net)
    nmax = max(oracle.space_size(len(q["pixels"]), q["k"]) for q in queries)
    buf = Buffers(vnet, nmax)
    for q in queries:
        n = oracle.space_size(len(q["pixels"]), q["k"])
        ref_s, ref_cov, ref_bm, ref_ties = reference(vb, vnet, q, n)
        g = buf.run(vb, vnet, q)
        assert g["flags"] == 0
        # the existing entry point
        assert g["n_adv"] == ref_s["n_adversarial"]
        assert g["first_witness"] == ref_s["first_witness"]
        assert g["n_ties"] == ref_s["n_ties"] and g["D"] == ref_s["D"]
        for key in ("flip", "flip_tie", "ss", "ss_tie"):
            np.testing.assert_array_equal(g[key], ref_cov[key])
        nw = (n + 31) // 32
        np.testing.assert_array_equal(g["bitmap"][:nw], ref_bm[:nw])
        np.testing.assert_array_equal(g["ties"], ref_ties)
        # the FP64 CPU oracle
        check_against_oracle(g, oracle.verify(net, q), n)
        assert ref_s["n_adversarial"] > 0 or ref_cov["flip"].any()
    vnet.free()


def test_noalloc_subrange_and_no_tie_buffer(vb):
    """The hand-checkable 2-2-2 ReLU net (ties at t = 5 and 13, witness t = 6):
    a sub-range with lo > 0, then the whole box without a tie buffer, where the
    tie count stays exact and the truncation flag is the only flag set."""
    W1 = np.array([[255, 0], [0, 255]], np.float32)
    net = {"dims": [2, 2, 2], "W": [W1, np.array([[1, -1], [-1, 1]], np.float32)],
           "b": [np.array([-100, -101], np.float32), np.zeros(2, np.float32)], "act": "relu"}
    q = {"image": np.array([104, 100], np.uint8), "pixels": np.array([0, 1], np.int32), "k": 3}
    vnet = vb.Net(net)
    n = 49
    buf = Buffers(vnet, n)
    lo, hi = 6, 40
    g = buf.run(vb, vnet, q, lo, hi)
    o = oracle.verify(net, q, lo=lo, hi=hi)
    assert g["flags"] == 0 and g["n_ties"] == 1 and g["first_witness"] == 6
    check_against_oracle(g, o, n, lo)
    nobuf = Buffers(vnet, n, ties_cap=0)
    g = nobuf.run(vb, vnet, q)
    o = oracle.verify(net, q)
    assert g["flags"] == TIES_CUT and g["n_ties"] == 2 == o["n_ties"]
    check_against_oracle(g, o, n)
    vnet.free()


def test_noalloc_flags_invalid_pixel_list(vb):
    """A repeated pixel index is not a box of s distinct pixels: the call returns,
    the flag says so, and nothing is read outside the image."""
    net = synth.make_net(66, [6, 8, 6, 4], "relu", 2.0, "normal")
    vnet = vb.Net(net)
    q = synth.make_query(66, 1, 6, 3, 4)
    buf = Buffers(vnet, oracle.space_size(3, 4))
    for pixels in ([1, 1, 2], [0, 2, 6]):  # duplicate; index past H_0 = 6
        bad = dict(q, pixels=np.array(pixels, np.int32))
        g = buf.run(vb, vnet, bad)
        assert g["flags"] & BAD_PIXELS
    g = buf.run(vb, vnet, q)  # a valid call afterwards starts clean
    assert g["flags"] == 0
    check_against_oracle(g, oracle.verify(net, q), oracle.space_size(3, 4))
    vnet.free()


def test_noalloc_rejects_oversized_query(vb):
    """More non-input neurons than the fixed scratch holds: a clear error, no work."""
    import torch
    net = synth.make_net(5, [8, 1024, 1024, 1024, 1024, 1024, 4], "relu", 2.0, "normal")
    vnet = vb.Net(net)  # 5124 non-input neurons > VBMC_NOALLOC_MAX_NEURONS
    dev = torch.device("cuda")
    counters = torch.zeros(4, dtype=torch.int64, device=dev)
    img = torch.zeros(8, dtype=torch.uint8, device=dev)
    pix = torch.arange(2, dtype=torch.int32, device=dev)
    with pytest.raises(vb.VbmcError) as e:
        vb.verify_range_fp64_noalloc(vnet, img, pix, 3, 0, 0, counters)
    assert e.value.status == -5 and "scratch" in str(e.value)
    vnet.free()
