"""The multi-GPU form of the benchmark runs independent replicas (the solve does
not shard): its only cross-rank step combines the slowest rank's time with the
nonzeros of all ranks.  Checked here with two gloo ranks on CPU."""
import os
import sys
from pathlib import Path

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = Path(__file__).resolve().parents[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, str(ROOT))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, nnz = [(120.0, 3.0e9), (150.0, 5.0e9)][rank]
        out[rank] = bench.combine_ranks(ms, nnz, dist, "cpu")
    finally:
        dist.destroy_process_group()


def test_two_replicas_combine_time_and_work():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    with mp.get_context("spawn").Manager() as m:   # no fork: the process may hold CUDA state
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        got = dict(out)
    for rank in (0, 1):
        max_ms, nnz_all = got[rank]
        assert max_ms == 150.0 and nnz_all == 8.0e9
    # whole-job throughput: all ranks' nonzeros over the slowest rank's time
    assert nnz_all / (max_ms * 1e-3) == pytest.approx(8.0e9 / 0.150)
