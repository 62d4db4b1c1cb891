"""The multi-rank path of bench.py on CPU: two gloo ranks, weak scaling.

Each rank runs its own source set (independent BC problems, no collective on
the data path); the whole-job figure is the units of all ranks over the
slowest rank's time.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r: 1000 ms over 5 steps (rank 1 slower), 10^9 (r+1) arcs per step
    total_ms = 1000.0 * (1 + rank)
    v, e2e, tmax = bench.combine_ranks(dist, world, total_ms, 5, 1e9 * (rank + 1), 0.5 + rank, 2e9, "cpu")
    out[rank] = (v, e2e, tmax)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_units_over_the_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(worker, args=(world, free_port(), out), nprocs=world, join=True)
    for r in range(world):
        v, e2e, tmax = out[r]
        assert tmax == 2000.0
        # (1e9 + 2e9) arcs per step / (2000 ms / 5 steps)
        assert abs(v - 3e9 / 0.4 / 1e9) < 1e-9
        assert abs(e2e - 4e9 / 1.5 / 1e9) < 1e-9


def test_ranks_draw_their_own_sources():
    _, g, s0 = bench.workload_inputs("rmat20_64src_batched", 0)
    _, _, s1 = bench.workload_inputs("rmat20_64src_batched", 1)
    assert len(s0) == len(s1) == 64 and not np.array_equal(s0, s1)
    assert np.all(g.degrees()[s1] >= 1)


def test_single_rank_has_no_collective():
    v, e2e, tmax = bench.combine_ranks(None, 1, 800.0, 4, 4e9, 2.0, 4e9)
    assert tmax == 800.0 and abs(v - 4e9 / 0.2 / 1e9) < 1e-9 and abs(e2e - 2.0) < 1e-9


def test_recorded_traffic_only_for_the_current_kernels(tmp_path, monkeypatch):
    # A traffic record counts only when workload, batch width and the hash of
    # the kernel sources all match; any kernel edit makes it stale (None).
    h = bench.kernel_source_hash()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "t.md").write_text(
        "# capture\n"
        f"traffic-record: workload=w1 width=128 sources={h} dram_bytes=1.5e11\n"
        "traffic-record: workload=w1 width=256 sources=0000000000000000 dram_bytes=9e9\n"
        f"traffic-record: workload=w3 width=128 sources={h} per_alg_byte=1.25 captured=small\n")
    csrc = os.path.join(bench.ROOT, "paper_2401_02472_gb300")
    os.symlink(csrc, tmp_path / "paper_2401_02472_gb300")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("w1", 128, 1e11)[0] == 1.5e11
    assert bench.recorded_traffic("w1", 256, 1e11)[0] is None
    assert bench.recorded_traffic("w2", 128, 1e11)[0] is None
    # a capture of a smaller launch: bytes per algorithmic byte, scaled by this launch's
    b, note = bench.recorded_traffic("w3", 128, 4e11)
    assert b == 5e11 and "small" in note
