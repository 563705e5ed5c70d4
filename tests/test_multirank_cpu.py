"""Multi-rank host logic on CPU: two gloo ranks shard a workload's generators
and time a step the way bench.py does on several GPUs (no GPU involved).

Each rank computes, with the oracle, the first outputs of the generators it
owns; rank 0 gathers them and checks that the shards together are exactly the
single-process result over the same global generators.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2309_16682_gb300 import inputs as I
from paper_2309_16682_gb300 import shard

WORLD = 2
PER_RANK = 2
WORKLOAD = "vmt64_m8_g32768"   # consecutive seeds: a slice error shows as a wrong seed
N_OUT = 64


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, q):
    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=WORLD)
        seeds = shard.rank_seeds(WORKLOAD, WORLD, rank, PER_RANK)
        w = I.WORKLOADS[WORKLOAD]
        v = O.VARIANTS[w["variant"]]
        outs = [O.vstream(v, w["lanes"], int(sd), N_OUT, "u64") for sd in seeds]
        gathered = [None] * WORLD
        dist.all_gather_object(gathered, (rank, [int(x) for x in seeds], [o.tolist() for o in outs]))
        shard.barrier()
        t_max = shard.max_over_ranks(1.0 + rank)     # rank times 1.0 and 2.0
        total = shard.sum_over_ranks(PER_RANK)       # generators processed by all ranks
        if rank == 0:
            q.put(("ok", gathered, t_max, total))
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent; the rank exits normally
        q.put(("error", repr(e), None, None))


def test_slices_partition_the_global_sequence():
    for world in (1, 2, 3, 8):
        got = np.concatenate([shard.rank_seeds("vmt32_m16_g65536", world, r, 5) for r in range(world)])
        assert np.array_equal(got, I.workload_seeds("vmt32_m16_g65536", 0, 5 * world))
    with pytest.raises(ValueError):
        shard.rank_slice(4, 2, 2)


def test_two_gloo_ranks_shard_and_time(oracle_polys):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    try:
        status, gathered, t_max, total = q.get(timeout=240)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert status == "ok", gathered
    assert t_max == 2.0 and total == WORLD * PER_RANK
    gathered.sort()
    seeds = [s for _, ss, _ in gathered for s in ss]
    outs = [np.array(o, np.uint64) for _, _, oo in gathered for o in oo]
    ref_seeds = I.workload_seeds(WORKLOAD, 0, WORLD * PER_RANK)
    assert seeds == [int(x) for x in ref_seeds]
    w = I.WORKLOADS[WORKLOAD]
    v = O.VARIANTS[w["variant"]]
    for sd, o in zip(ref_seeds, outs):
        assert np.array_equal(o, O.vstream(v, w["lanes"], int(sd), N_OUT, "u64"))
