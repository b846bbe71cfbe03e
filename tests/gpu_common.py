"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and
compare every output with the FP64 CPU oracle."""
import numpy as np

import oracle


def run_gpu(vb, net_dict, q, precision, lo=0, hi=0, coverage=True, bitmap=True, queue_cap=None,
            vbnet=None, wide_chunk=0):
    s, k = len(q["pixels"]), int(q["k"])
    n = oracle.space_size(s, k)
    net = vbnet or vb.Net(net_dict)
    res = vb.Result(net, max_points=n if bitmap else 0, max_s=max(1, s), max_k=max(1, k),
                    ties_cap=1 << 16, queue_cap=queue_cap or max(4096, n), wide_chunk=wide_chunk)
    summ = vb.verify_query(net, res, q["image"], q["pixels"], k, lo=lo, hi=hi,
                           precision=precision, coverage=coverage, bitmap=bitmap)
    out = {"summary": summ, "n": n}
    if coverage:
        out.update(vb.get_coverage(res))
    if bitmap:
        out["bitmap"] = vb.get_verdict_bitmap(res, n)
    out["ties"] = np.sort(vb.get_ties(res))
    out["witness"] = vb.get_witness(res, s, net_dict["dims"][0])
    res.free()
    if vbnet is None:
        net.free()
    return out


def compare(g, o, net_dict, q, coverage=True, bitmap=True, margin_rel=1e-4):
    """Bit-exact on class, counts, first witness, ties, bitmap and masks; the
    witness margin within 1e-4 relative of the oracle's FP64 margin."""
    s = g["summary"]
    assert s["D"] == o["D"]
    assert abs(s["base_margin"] - o["base_margin"]) <= 1e-9 + 1e-12 * abs(o["base_margin"])
    assert s["n_points"] == o["n_points"]
    assert s["n_adversarial"] == o["n_adv"], (s, o["n_adv"])
    assert s["first_witness"] == o["first_witness"]
    assert s["n_ties"] == o["n_ties"]
    np.testing.assert_array_equal(g["ties"], o["ties"])
    if bitmap:
        nw = (g["n"] + 31) // 32
        np.testing.assert_array_equal(g["bitmap"][:nw], o["bitmap"][:nw])
    if coverage:
        for key in ("flip", "flip_tie", "ss", "ss_tie"):
            np.testing.assert_array_equal(g[key], o[key], err_msg=key)
        assert g["covered_fraction"] == oracle.ss_covered_fraction(net_dict["dims"], o["ss"])
    w = g["witness"]
    if o["first_witness"] is None:
        assert w is None
    else:
        assert w["index"] == o["first_witness"]
        p = oracle.eval_point(net_dict, q, o["first_witness"])
        assert abs(w["margin"] - p["margin"]) <= margin_rel * abs(p["margin"]) + 1e-9
        d = oracle.digits(o["first_witness"], len(q["pixels"]), q["k"])
        assert list(w["steps"]) == [x - q["k"] for x in d]
        img = np.array(q["image"], dtype=np.int64)
        for pix, st in zip(q["pixels"], w["steps"]):
            img[pix] = min(255, max(0, img[pix] + st))
        np.testing.assert_array_equal(w["image"], img.astype(np.uint8))
