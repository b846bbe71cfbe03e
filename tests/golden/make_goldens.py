"""Write the stored expected results of the full-size parity tests.

Calls only the FP64 CPU oracle (``oracle.verify``) on the seeded synthetic
workloads of ``synth``; nothing here touches the CUDA library. Each golden
holds the outputs of one exhaustive check of a whole box (Eq. 10 over every
point, the sign changes and SS-Cover of Sec. III-B with coverage on):
class D, point count, adversarial count, first witness, the tie list, and
digests of the verdict bitmap and coverage masks (SHA-256 of the uint32
words, little endian, plus their popcounts; the flip masks in full).

    python tests/golden/make_goldens.py config2      # 784-512-512-10, s=6, k=7
    python tests/golden/make_goldens.py config3      # 784-1024x3-10, s=5, k=15

Run time on 8 host cores: config2 about 10 minutes, config3 about 2 hours.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

TARGETS = {
    "config2": ("mlp784x512x512_relu_s6k7", "config2_mlp784x512x512_s6k7.json"),
    "config3": ("mlp784x1024x3_relu_s5k15", "config3_mlp784x1024x3_s5k15.json"),
}


def digest(words: np.ndarray) -> dict:
    w = np.ascontiguousarray(words, dtype="<u4")
    return {"sha256": hashlib.sha256(w.tobytes()).hexdigest(), "words": int(w.size),
            "popcount": int(np.unpackbits(w.view(np.uint8)).sum())}


def golden(workload: str) -> dict:
    w = synth.workload(workload)
    net, q = w["net"], w["query"]
    n = oracle.space_size(len(q["pixels"]), q["k"])
    t0 = time.time()
    o = oracle.verify(net, q, coverage=True, bitmap=True, ties_cap=1 << 20)
    dt = time.time() - t0
    return {
        "workload": workload,
        "what": "oracle.verify over the whole box, coverage on (Eq. 10; Sec. III-B)",
        "seconds": round(dt, 1), "threads": os.cpu_count(),
        "dims": list(net["dims"]), "s": len(q["pixels"]), "k": int(q["k"]),
        "pixels": [int(p) for p in q["pixels"]],
        "n_points": int(o["n_points"]), "space": int(n),
        "D": int(o["D"]), "base_margin": float(o["base_margin"]),
        "n_adversarial": int(o["n_adv"]),
        "first_witness": o["first_witness"],
        "n_ties": int(o["n_ties"]), "ties": [int(t) for t in o["ties"]],
        "bitmap": digest(o["bitmap"][:(n + 31) // 32]),
        "flip": [int(x) for x in o["flip"]], "flip_tie": [int(x) for x in o["flip_tie"]],
        "ss": digest(o["ss"]), "ss_tie": digest(o["ss_tie"]),
        "ss_bits_if_few": [int(i) for i in np.flatnonzero(np.unpackbits(
            o["ss"].astype("<u4").view(np.uint8), bitorder="little"))][:4096],
    }


def main(argv):
    for name in argv or ["config2"]:
        workload, fname = TARGETS[name]
        g = golden(workload)
        with open(os.path.join(HERE, fname), "w") as f:
            json.dump(g, f, indent=1)
            f.write("\n")
        print(name, g["n_adversarial"], g["first_witness"], g["n_ties"], g["seconds"], "s")


if __name__ == "__main__":
    main(sys.argv[1:])
