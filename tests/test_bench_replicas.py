"""Multi-rank bench logic on CPU (gloo, world size 2): replicas time independently, the job time
is the slowest rank's, value counts every rank's cells."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=2)
    ms_local = 100.0 if rank == 0 else 250.0
    ms, value = bench.aggregate(ms_local, cells_per_rank=1000, steps=10, dist=dist, device="cpu")
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_gloo_two_ranks():
    import multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get() for _ in range(2))
    for rank, ms, value in res:
        assert ms == 250.0                                  # max over ranks
        assert abs(value - 2 * 1000 * 10 / 0.25 / 1e6) < 1e-12


def test_profile_counts_dropped_when_kernel_sources_change(monkeypatch):
    """The roofline's flop, DRAM and FP64-pipe figures per face come from the committed ncu summary
    only while the flux kernels' sources hash to the value recorded there."""
    import bench
    flops, dram, pipe = bench.profile_numbers()
    if flops:
        assert set(flops) == {"r", "theta", "phi"} and all(v > 0 for v in flops.values())
        assert set(pipe) == {"r", "theta", "phi"} and all(0 < v <= 1 for v in pipe.values())
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.profile_numbers() == ({}, {}, {})


def test_kernel_sequence_option_maps_to_options_fused():
    """--kernels names the three values of options.fused that icarus_init accepts (0, 1, 2), the
    default is 0, and a name outside them is refused by the parser."""
    import bench
    assert bench.KERNEL_SEQUENCES == {"default": 0, "fused": 1, "separate": 2}
    assert bench.parse_args([]).kernels == "default"
    assert bench.parse_args(["--kernels", "separate"]).kernels == "separate"
    with pytest.raises(SystemExit):
        bench.parse_args(["--kernels", "other"])
