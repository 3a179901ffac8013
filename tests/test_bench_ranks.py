"""The N>1 path of the benchmark (replicas only) on CPU with gloo ranks: the
whole-job aggregation takes the slowest rank's times and the sum of all
ranks' iterations."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.distributed.barrier()
        ms, e2e_ms = 100.0 + 10.0 * rank, 120.0 - 5.0 * rank
        res = bench.reduce_over_ranks(ms, e2e_ms, 1000 + rank, 900 + 2 * rank, world)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        torch.distributed.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_reduce_over_ranks_gloo(tmp_path, world):
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        ms, e2e_ms, iters, e2e_iters = json.load(open(tmp_path / f"r{r}.json"))
        assert ms == 100.0 + 10.0 * (world - 1)          # slowest rank
        assert e2e_ms == 120.0                           # slowest e2e rank (rank 0)
        assert iters == sum(1000 + k for k in range(world))
        assert e2e_iters == sum(900 + 2 * k for k in range(world))


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    import bench
    assert bench.reduce_over_ranks(1.0, 2.0, 3, 4, 1) == (1.0, 2.0, 3, 4)
