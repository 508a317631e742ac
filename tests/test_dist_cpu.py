"""The multi-process path of bench.py on CPU: two gloo ranks, the timing barrier and the
max over ranks (the only collectives of the replicated bench), and distinct per-rank
inputs (each replica steps its own seeded worlds)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank), OSTRICH_BENCH_GLOO="1")
    import bench
    r, ws, lr = bench.dist_init()
    bench.dist_barrier()
    m = bench.dist_max(1.0 + 1.5 * rank)
    _, states, _, _ = bench.make_inputs(4, seed=r)
    out[rank] = (r, ws, m, float(states[0].sum()))
    bench._DIST.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0][:3] == (0, 2, 2.5) and out[1][:3] == (1, 2, 2.5)
    assert out[0][3] != out[1][3]                  # each replica has its own worlds
