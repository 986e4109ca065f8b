"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks.

Each rank is a replica with its own particle shard (no collective on the data
path); the only collective is the MAX of the ranks' times, and the reported
value is the whole job's particles over that time.
"""
import importlib.util
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        local = [12.5, 20.0][rank]
        ms = b.max_over_ranks(local, world, torch.device("cpu"))
        out[rank] = (ms, b.job_throughput(world, 1000, 10, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_value():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == 20.0
    assert value == pytest.approx(world * 1000 * 10 / 0.020)


def test_single_rank_needs_no_process_group():
    b = _bench()
    assert b.max_over_ranks(7.0, 1) == 7.0
    assert b.job_throughput(1, 2 ** 24, 100, 576.9) == pytest.approx(2 ** 24 * 100 / 0.5769)


def test_ranks_draw_distinct_particle_shards():
    b = _bench()
    from paper_1201_4060_gb300 import synth
    wl = dict(synth.WORKLOADS["throughput512"])
    seeds = [b.rank_particle_seed(wl, r) for r in range(4)]
    assert len(set(seeds)) == 4
    shards = [synth.clustered_particles(64, seed=s) for s in seeds[:2]]
    assert not np.array_equal(shards[0], shards[1])


def test_reference_arm_prints_nothing_on_other_ranks(monkeypatch, capsys):
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    b.run_reference(type("A", (), {"steps": 1, "warmup": 0})())
    assert capsys.readouterr().out == ""
