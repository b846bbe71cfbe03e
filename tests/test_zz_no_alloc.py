"""The allocation-free entry point, for callers that cannot call cudaMalloc
(code living in another runtime's memory pool, or whose allocator must not be
re-entered): vbmc_verify_range_fp64_noalloc keeps its scratch in a fixed array
inside the library and writes only into the caller's buffers. Its results must
equal those of vbmc_verify_query in FP64, on two calls in a row (the second
call reuses the same scratch)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


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


def test_noalloc_equals_verify_query_on_two_calls(vb):
    import torch
    net = synth.make_net(66, [6, 8, 6, 4], "relu", 2.0, "normal")
    queries = [synth.make_query(66, 1, 6, 3, 12), synth.make_query(66, 2, 6, 2, 20)]
    vnet = vb.Net(net)
    fw, sw = vnet.mask_words()
    dev = torch.device("cuda")
    nmax = max(oracle.space_size(len(q["pixels"]), q["k"]) for q in queries)
    counters = torch.zeros(4, dtype=torch.int64, device=dev)
    masks = [torch.zeros(w, dtype=torch.int32, device=dev) for w in (fw, fw, sw, sw)]
    bitmap = torch.zeros((nmax + 31) // 32, dtype=torch.int32, device=dev)
    ties = torch.zeros(1024, dtype=torch.int64, device=dev)
    for q in queries:
        n = oracle.space_size(len(q["pixels"]), q["k"])
        ref_s, ref_cov, ref_bm, ref_ties = reference(vb, vnet, q, n)
        img = torch.tensor(q["image"], dtype=torch.uint8, device=dev)
        pix = torch.tensor(q["pixels"], dtype=torch.int32, device=dev)
        vb.verify_range_fp64_noalloc(vnet, img, pix, q["k"], 0, 0, counters, *masks,
                                     bitmap=bitmap, ties=ties)
        torch.cuda.synchronize()
        c = counters.cpu().numpy().astype(np.uint64)
        assert int(c[0]) == ref_s["n_adversarial"]
        first = None if int(c[1]) == 2**64 - 1 else int(c[1])
        assert first == ref_s["first_witness"]
        assert int(c[2]) == ref_s["n_ties"]
        assert int(c[3]) & 0xFFFFFFFF == ref_s["D"] and int(c[3]) >> 32 == 0
        for m, key in zip(masks, ("flip", "flip_tie", "ss", "ss_tie")):
            np.testing.assert_array_equal(m.cpu().numpy().view(np.uint32), ref_cov[key])
        nw = (n + 31) // 32
        np.testing.assert_array_equal(bitmap.cpu().numpy().view(np.uint32)[:nw], ref_bm[:nw])
        got_ties = np.sort(ties.cpu().numpy()[:int(c[2])])
        np.testing.assert_array_equal(got_ties, ref_ties)
        assert ref_s["n_adversarial"] > 0 or ref_cov["flip"].any()


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
