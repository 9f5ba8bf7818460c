"""Host logic of bench.py that needs no GPU: the replica aggregation over ranks
(max of times, sum of work) with two gloo ranks, and the argument defaults."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, n = bench.reduce_max_sum(1.5 + rank, 100.0 * (rank + 1), world)
    with open(f"{out_path}.{rank}", "w") as f:
        f.write(f"{t} {n}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "agg")
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        t, n = map(float, open(f"{out}.{r}").read().split())
        assert t == 2.5          # slowest rank's time
        assert n == 300.0        # work of all ranks


def test_bench_defaults_and_workload():
    sys.path.insert(0, ROOT)
    import bench
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1
    assert a.n_qubits == 100 and a.depth == 30 and a.impl == "ours"
    assert "100-qubit" in bench.workload_name(a)
    t, n = bench.reduce_max_sum(2.0, 5.0, 1)
    assert (t, n) == (2.0, 5.0)
    assert bench.fp32_peak_tflops(152, 2070.0) == pytest.approx(80.54784)
