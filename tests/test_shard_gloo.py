"""Multi-rank sharding of independent designs, on CPU with the gloo backend
(world size 2): the longest-processing-time partition is complete, disjoint
and balanced, and per-design reports gathered over the ranks equal the
unsharded ones.  The per-design analysis here is the FP64 oracle (the GPU
library needs a device); the sharding and gather code is the one bench.py
uses under torchrun."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2511_11660_b300 import shard, synth


def test_lpt_partition_properties():
    rng = np.random.default_rng(0)
    w = np.exp(rng.uniform(np.log(5e3), np.log(5e5), 64))
    for n in (1, 2, 3, 4, 8):
        parts = shard.lpt_partition(w, n)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [w[p].sum() for p in parts]
        # greedy LPT is within (4/3 - 1/(3n)) of optimal; the mean bounds the optimum from below
        assert max(loads) <= (4 / 3) * max(w.sum() / n, w.max()) + 1e-9


def _designs():
    lib = synth.make_library(3)
    return [synth.make_design(n, 6, seed=40 + i, lib=lib, period_ns=0.8) for i, n in enumerate([60, 200, 35, 120, 90])]


def _reports(ds, idx):
    import oracle
    out = {}
    for i in idx:
        r = oracle.sta(ds[i])
        out[i] = (float(r["wns_setup"][0]), float(r["tns_setup"][0]), int(r["n_viol_setup"][0]))
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ds = _designs()
    parts = shard.lpt_partition([synth.design_stats(d)["arcs"] for d in ds], world)
    merged = shard.gather_reports(_reports(ds, parts[rank]), dist)
    q.put((rank, merged))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gather_equals_unsharded():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    want = _reports(_designs(), range(5))
    for _, merged in got:
        assert merged == want
