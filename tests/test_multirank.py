"""The N > 1 path of bench.py on CPU: two ranks over gloo (127.0.0.1), no GPU.

Ranks run independent replicas (weak scaling): the same top-K Kraus sets on every rank (the host
library is deterministic across processes), a distinct shot seed per rank, no exchange on the data
path; the timing is the maximum over ranks and the job throughput counts every rank's shots."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import hashlib
    import json

    import numpy as np
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2504_16297_gb300 import runtime
    from workloads import config

    cfg = config(1)
    P = runtime.Ptsbe(device=-1)                 # host-only context: registration and PTS
    cid = P.register(cfg["circuit"])
    info = P.sample_kraus(cid, "topk", k=2000, total_shots=10**6)
    h = hashlib.sha256()
    for a in (info.offsets, info.sites, info.kidx, info.shots):
        h.update(np.ascontiguousarray(a).tobytes())
    digests = [None] * world
    dist.all_gather_object(digests, h.hexdigest())
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(cfg["seed"], rank))
    ms = bench.max_over_ranks(10.0 * (rank + 1), dist, torch.device("cpu"))
    value = bench.job_throughput(world, 10**8, ms)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"digests": digests, "seeds": seeds, "ms": ms, "value": value}, f)
    dist.destroy_process_group()


def test_two_ranks_replicate_sets_split_seeds_and_take_max_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import json

    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert len(set(r["digests"])) == 1          # every rank prepares the same sets
        assert len(set(r["seeds"])) == world        # and draws its own shots
        assert r["ms"] == 20.0                      # slowest rank
        assert r["value"] == pytest.approx(2 * 10**8 / 0.020)
