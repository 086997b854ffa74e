"""The benchmark's multi-rank host logic on CPU: two gloo ranks.  Each rank
times its own instance; the job-wide step time is the max over ranks and the
points are summed.  The reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    got = bench.reduce_over_ranks(ms=1.0 + rank, e2e_ms=10.0 - rank, points=100 * (rank + 1), ws=ws,
                                  device="cpu")
    # the reference arm: ranks other than 0 exit 0 without work
    ref = bench.run_reference(type("A", (), {"workload": "tiny", "cpu_sample": None, "steps": 1, "warmup": 1,
                                             "gpus": ws})()) if rank != 0 else None
    out[rank] = (got, ref)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_and_reference_arm():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        ms, e2e, pts = res[r][0]
        assert ms == 2.0 and e2e == 10.0 and pts == 300
    assert res[1][1] == 0
