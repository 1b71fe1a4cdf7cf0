"""N > 1 on CPU (gloo, world size 2): the path shards by events -- each rank sums
-log P over its contiguous share and the partial NLL and gradient are all-reduced -- and
by independent problems (each rank its own data set, weak scaling, the job's time the
maximum over ranks).  Both checked with the oracle as the per-rank evaluator."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1311_1753_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from tests import oracle_models as om
    lo, hi = synth.VOIGT_RANGE
    x = synth.voigt_threshold_events(50_001, **synth.VOIGT_TRUTH, lo=lo, hi=hi, seed=31)
    bounds = np.linspace(0, len(x), world + 1).astype(int)
    m, free = om.voigt_model(nbins=2000)
    p = m.p.copy()
    p[free] *= np.array([1.00001, 1.02, 0.97, 1.05, 0.9])
    f, g = m.nll([x[bounds[rank]:bounds[rank + 1]]], p, grad=True)
    t = torch.tensor(np.concatenate([[f], g]), dtype=torch.float64)
    dist.all_reduce(t)  # one all-reduce of 1 + n_par doubles per evaluation
    # replicas: each rank its own data set and time; the job's time is the maximum
    tm = torch.tensor([1.0 + rank], dtype=torch.float64)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    if rank == 0:
        full = m.nll([x], p, grad=True)
        q.put((t.numpy(), np.concatenate([[full[0]], full[1]]), tm.item()))
    dist.barrier()
    dist.destroy_process_group()


def test_event_sharding_all_reduce_equals_full_sum():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got, full, tmax = q.get(timeout=300)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert abs(got[0] - full[0]) <= 1e-12 * abs(full[0])
    assert np.all(np.abs(got[1:] - full[1:]) <= 1e-10 * np.abs(full[1:]) + 1e-8)
    assert tmax == 2.0
