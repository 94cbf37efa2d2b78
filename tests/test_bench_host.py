"""CPU tests of bench.py's host-side logic: the JSON line of the CPU
reference arm (the oracle on a bounded sample), the rank-0-only rule, and
the max-over-ranks timing reduction with world_size 2 over gloo."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--n", "1024", "--s", "8", "--cpu-sample-n", "256"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"] > 0
    assert "256x256" in d["cpu_baseline"]["sample"]


def test_reference_arm_nonzero_rank_is_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-sample-n", "256"], capture_output=True, text=True, timeout=120,
                       cwd=ROOT, env=env)
    assert r.returncode == 0
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    bench.init_dist(world, "gloo")
    v = bench.max_over_ranks(10.0 + rank, world)
    bench.barrier(world)
    out[rank] = v
    import torch.distributed as dist

    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29600 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 11.0


def test_committed_traffic_matches_current_kernel_sources():
    """profiles/traffic.json holds DRAM bytes only for kernel sources whose
    hash it records; both captured kernels match the committed sources, and
    the operator's figure scales with n^2 to the benchmark size."""
    sys.path.insert(0, ROOT)
    import bench

    sym = bench.kernel_traffic("k_symv_df", 6144)
    gem = bench.kernel_traffic("k_sliced_umma", 16384)
    assert sym is not None and gem is not None, "ncu capture is stale: re-profile the changed kernel"
    sym16 = bench.kernel_traffic("k_symv_df", 16384)
    assert abs(sym16["dram_bytes"] / sym["dram_bytes"] - (16384 / 6144) ** 2) < 1e-12
    # algorithmic bytes of one symv at n = 6144 (triangle hi + lo, w and z); traffic within 10%
    alg = 8.0 * 6144 * 6145 / 2 + 16.0 * 6144
    assert 1.0 <= sym["dram_bytes"] / alg < 1.1
    assert bench.kernel_traffic("no_such_kernel", 100) is None
