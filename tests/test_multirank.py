"""The multi-GPU paths on the CPU, as gloo ranks.

Range split (one query over all ranks): rank r checks a contiguous slice of
[0, R^s) and the exchange step merges the slices (sums of the counts, the
smallest first witness, bitwise or of the masks and of the verdict bitmap,
the tie lists joined). Each rank runs the FP64 oracle on its slice; the merged
result must equal the oracle's check of the whole box bit for bit.

Independent queries (weak scaling): each rank verifies its own query of the
same net; the only traffic between ranks is the step time (max) and the
checked-point count (sum)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
import oracle
import synth
from paper_1907_12933_gb300 import partition
from test_oracle_pins import net222, small_relu_case


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        net, _ = small_relu_case()
        w = {"cfg": {"seed": 66, "dims": [6, 8, 6, 4], "s": 3, "k": 9}, "query": synth.make_query(66, 0, 6, 3, 9)}
        q = bench.rank_query(w, rank)
        o = oracle.verify(net, q, nthreads=1)
        # a made-up step time per rank: the job takes the slowest
        ms = 10.0 + 5.0 * rank
        ms_max, n_all, value = bench.job_throughput(ms, int(o["n_points"]), world)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), ms_max=ms_max, n_all=n_all, value=value,
                 n_adv=o["n_adv"], first=-1 if o["first_witness"] is None else o["first_witness"],
                 image=q["image"], pixels=q["pixels"])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r = [np.load(tmp_path / f"rank{i}.npz") for i in range(world)]
    n = oracle.space_size(3, 9)
    for x in r:
        assert float(x["ms_max"]) == 15.0
        assert int(x["n_all"]) == world * n
        assert float(x["value"]) == pytest.approx(world * n / 0.015)
    # different queries per rank, each rank's verdict is its own query's
    assert not (np.array_equal(r[0]["image"], r[1]["image"]) and np.array_equal(r[0]["pixels"], r[1]["pixels"]))
    net, _ = small_relu_case()
    for i, x in enumerate(r):
        q = {"image": x["image"], "pixels": x["pixels"], "k": 9}
        o = oracle.verify(net, q)
        assert int(x["n_adv"]) == o["n_adv"]
        assert int(x["first"]) == (-1 if o["first_witness"] is None else o["first_witness"])


def test_single_rank_needs_no_collective():
    ms_max, n_all, value = bench.job_throughput(20.0, 1000, 1)
    assert (ms_max, n_all) == (20.0, 1000) and value == pytest.approx(50000.0)


# ------------------------------------------------------------ range split

CASES = {
    "relu_6_8_6_4": lambda: (small_relu_case()[0], synth.make_query(66, 0, 6, 3, 9)),
    "hand_222": lambda: (net222(), {"image": np.array([104, 100], np.uint8),
                                    "pixels": np.array([0, 1], np.int32), "k": 3}),
}


def _split_main(rank, world, port, out_dir, case):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        net, q = CASES[case]()
        n = oracle.space_size(len(q["pixels"]), q["k"])
        lo, hi = partition.rank_range(n, rank, world)
        o = oracle.verify(net, q, lo=lo, hi=hi, nthreads=1) if hi > lo else None
        fw, sw = oracle.mask_words(net["dims"])
        empty = lambda w: np.zeros(w, np.uint32)  # noqa: E731
        part = {"n_points": hi - lo, "n_adv": o["n_adv"] if o else 0, "n_ties": o["n_ties"] if o else 0,
                "first_witness": o["first_witness"] if o else None,
                "D": o["D"] if o else -1, "base_margin": o["base_margin"] if o else 0.0,
                "flip": o["flip"] if o else empty(fw), "flip_tie": o["flip_tie"] if o else empty(fw),
                "ss": o["ss"] if o else empty(sw), "ss_tie": o["ss_tie"] if o else empty(sw),
                "bitmap": o["bitmap"] if o else empty((n + 31) // 32),
                "ties": o["ties"] if o else np.zeros(0, np.int64)}
        m = partition.merge_partials(part)
        np.savez(os.path.join(out_dir, f"split{rank}.npz"), lo=lo, hi=hi,
                 counts=[m["n_points"], m["n_adv"], m["n_ties"]],
                 first=-1 if m["first_witness"] is None else m["first_witness"],
                 verdict=partition.merged_verdict(m),
                 **{k: m[k] for k in ("flip", "flip_tie", "ss", "ss_tie", "bitmap", "ties")})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("relu_6_8_6_4", 2), ("relu_6_8_6_4", 3), ("hand_222", 2)])
def test_range_split_merges_to_the_whole_box(tmp_path, case, world):
    mp.start_processes(_split_main, args=(world, _free_port(), str(tmp_path), case), nprocs=world,
                       join=True, start_method="spawn")
    net, q = CASES[case]()
    n = oracle.space_size(len(q["pixels"]), q["k"])
    whole = oracle.verify(net, q)
    r = [np.load(tmp_path / f"split{i}.npz") for i in range(world)]
    # the slices tile [0, n) in order, 32-aligned inside
    assert int(r[0]["lo"]) == 0 and int(r[-1]["hi"]) == n
    for a, b in zip(r, r[1:]):
        assert int(a["hi"]) == int(b["lo"]) and int(a["hi"]) % 32 == 0
    for x in r:  # every rank holds the same merged result: the whole box's
        assert list(x["counts"]) == [n, whole["n_adv"], whole["n_ties"]]
        assert int(x["first"]) == (-1 if whole["first_witness"] is None else whole["first_witness"])
        for key in ("flip", "flip_tie", "ss", "ss_tie"):
            np.testing.assert_array_equal(x[key], whole[key], err_msg=key)
        np.testing.assert_array_equal(x["bitmap"], whole["bitmap"])
        np.testing.assert_array_equal(x["ties"], whole["ties"])
        assert str(x["verdict"]) == ("UNSAFE" if whole["n_adv"] else
                                     "TIES_ONLY" if whole["n_ties"] else "SAFE")
    # the comparison is not vacuous: the box has witnesses or sign changes
    assert whole["n_adv"] > 0 or whole["flip"].any()


def test_rank_range_tiles_the_space():
    for n in (1, 31, 32, 33, 1000, 15 ** 6):
        for world in (1, 2, 3, 8):
            rs = [partition.rank_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert all(lo % 32 == 0 for lo, _ in rs)
    with pytest.raises(ValueError):
        partition.rank_range(10, 2, 2)
