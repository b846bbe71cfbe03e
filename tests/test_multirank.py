"""The multi-GPU path on the CPU: two gloo ranks. Each rank verifies its own
query of the same net (independent problems, weak scaling); the only traffic
between ranks is the step time (max) and the checked-point count (sum). The
ranks' results must equal what the oracle gives for each query alone."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
import oracle
import synth
from test_oracle_pins import small_relu_case


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
