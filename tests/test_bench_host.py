"""Host-side logic of bench.py: the multi-rank path (world size 2 over gloo on
CPU) and the CPU reference arm."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    import pamd_inputs as inputs
    w = inputs.workload("lj500")
    ms = 10.0 + 5.0 * rank  # rank 1 is the slowest
    ms_max = b.max_over_ranks(ms)
    value = b.aggregate(w.units, world, 4, ms_max)
    out[rank] = (b.rank_seed(w, rank), ms_max, value)
    dist.destroy_process_group()


def test_two_ranks_shard_chains_and_take_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    world, port = 2, 29531
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    seeds = [out[r][0] for r in range(world)]
    assert len(set(seeds)) == world  # every rank draws its own chains
    for r in range(world):
        assert out[r][1] == 15.0  # max over ranks
    import pamd_inputs as inputs
    units = inputs.workload("lj500").units
    assert abs(out[0][2] - units * world * 4 / 15e-3) < 1e-6 * out[0][2]


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ)
    env.pop("WORLD_SIZE", None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--config", "ho3d", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "particle-timeslices/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0
