"""Replica helpers with two gloo ranks on CPU (the N > 1 path without GPUs)."""
import os
import socket

import torch.multiprocessing as mp

from paper_2501_07535_gb300 import inputs, replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world_size, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world_size),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    replicas.init("gloo")
    replicas.barrier()
    mx = replicas.max_over_ranks(float(rank + 1))
    sm = replicas.sum_over_ranks(float(10 * (rank + 1)))
    jobs = inputs.uneven_batch(n_jobs=10, seed=1)
    mine = [j.seed for j in replicas.shard(jobs, rank, world_size)]
    replicas.barrier()
    replicas.finalize()
    out[rank] = (mx, sm, mine)


def test_two_gloo_ranks():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 2.0
    assert out[0][1] == out[1][1] == 30.0
    seeds = sorted(out[0][2] + out[1][2])
    assert seeds == sorted(j.seed for j in inputs.uneven_batch(n_jobs=10, seed=1))
    assert not set(out[0][2]) & set(out[1][2])
