"""The multi-GPU path is replicas: each rank solves its own problems and only host
scalars (timings, solve counts) are reduced. Checked with world_size 2 on gloo (CPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, size, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(size), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2208_02427_gb300 import replicas
    r, s, _ = replicas.init(backend="gloo")
    units = list(replicas.shard(4097, r, s))
    replicas.barrier()
    t = replicas.reduce_scalar(10.0 + r, "max")
    total = replicas.reduce_scalar(float(len(units)), "sum")
    out[r] = (units[0], units[-1], len(units), t, total)
    replicas.finish()


def test_two_ranks_shard_and_reduce():
    port = _free_port()
    with mp.get_context("spawn").Manager() as man:  # no fork of this multi-threaded process
        out = man.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][:3] == (0, 2048, 2049) and res[1][:3] == (2049, 4096, 2048)
    for r in (0, 1):
        assert res[r][3] == 11.0 and res[r][4] == 4097.0


def test_single_process_is_identity():
    from paper_2208_02427_gb300 import replicas
    assert replicas.reduce_scalar(3.5, "max") == 3.5
    assert list(replicas.shard(5, 0, 1)) == [0, 1, 2, 3, 4]
    assert [len(replicas.shard(10, r, 3)) for r in range(3)] == [4, 3, 3]
