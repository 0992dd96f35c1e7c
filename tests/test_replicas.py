"""Host logic of the N-GPU replica run (one process per GPU, independent
problems), exercised with world size 2 on the gloo backend on CPU: the
barrier, the maximum of the per-rank times, the whole-job throughput, the
per-rank seeds, and the reference arm's non-zero ranks exiting without work."""

import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2109_10687_gb300 import replicas
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w, r, lr = replicas.rank_env()
        replicas.barrier(w)
        elapsed = replicas.max_over_ranks(1.5 + rank, w)          # rank 1 is the slower one
        value = replicas.job_throughput(w, 4, elapsed)
        seeds = replicas.replica_seeds(1001, 2001, r)
        replicas.barrier(w)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
            fh.write(f"{w} {r} {lr} {elapsed} {value} {seeds[0]} {seeds[1]}\n")
    finally:
        dist.destroy_process_group()


def test_replicas_world2_gloo(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(world)]
    for r, row in enumerate(rows):
        w, rk, lr = int(row[0]), int(row[1]), int(row[2])
        elapsed, value = float(row[3]), float(row[4])
        assert (w, rk, lr) == (world, r, r)
        assert elapsed == 2.5                     # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 4 / 2.5)  # all ranks' units / max time
    seeds = {(int(row[5]), int(row[6])) for row in rows}
    assert len(seeds) == world                    # independent replicas


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert res.returncode == 0
    assert res.stdout.strip() == ""


def test_reference_arm_line_contract():
    """The reference arm (the float64 oracle on the host, a bounded sample) prints
    one JSON line with the fields the benchmark contract names."""
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    line = json.loads(res.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "solves/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 1
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"] and cpu["sample"]
    # a timed complete solve, converted to the benchmark's unit and marked so
    assert line["extrapolated"] is True and cpu["extrapolated"] is True
    m = cpu["measured"]
    assert m["all_converged"] and m["true_resid"] < 1e-10 and m["solves"] == 1
    # the per-step time is the measured one and fits inside the run
    assert line["ms_per_step"] * line["steps"] <= 1000.0 * line["wall_s"]
    assert line["e2e"] == {"value": line["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_sap_byte_model_matches_the_profiled_launch():
    """The SAP kernel's algorithmic bytes per site: the launch type that the
    ncu summary profiles (second sweep, E colour: float16 s in and out, links
    and C_inv, halo in and out, float32 b) is 680 B; the first launch has no
    halo in and reads the float32 source; the last writes no halo and the
    float32 result instead of the update."""
    import bench
    assert bench.sap_bytes_per_launch("half", 1, 0) == 52 + 144 + 144 + 96 + 96 + 96 + 52 == 680
    assert bench.sap_bytes_per_launch("half", 0, 0) == 96 + 288 + 96 + 148
    assert bench.sap_bytes_per_launch("half", bench.N_SAP, 1) == 52 + 288 + 96 + 96
    assert abs(bench.sap_bytes_per_site("half") - 659.2) < 1e-9


def test_cpu_config_oracle_jobs():
    """The host-core oracle timing jobs of the CPU configuration: a D apply
    and one SAP-BiCGStab iteration at 8^4, each timed in a spawned
    single-threaded worker, return positive seconds; the thread variables
    are restored afterwards."""
    sys.path.insert(0, ROOT)
    import bench_configs
    before = os.environ.get("OMP_NUM_THREADS")
    wall, (t_d, t_it) = bench_configs._oracle_pool([("D", (8, 8, 8, 8)), ("iter", (8, 8, 8, 8))], 1)
    assert 0 < t_d < t_it <= wall
    assert os.environ.get("OMP_NUM_THREADS") == before


def test_d_bytes_follow_the_tuned_link_format():
    """The benchmark counts the float32 D's algorithmic bytes for the link
    format the autotuner chose: 768 B per site with 18-real links, 672 with
    the 12-real variants (shape names ending in 'c')."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.D_BYTES_PER_SITE == 768 and bench.D_BYTES_PER_SITE_12 == 672
    full = ["dslash_f32_mode0_nrhs1 128x4h 0.1400 ms [128x4 0.1437, 128x4h 0.1400]"]
    comp = ["dslash_f32_mode0_nrhs1_links12 128x4hc 0.1210 ms [128x4c 0.1233, 128x4hc 0.1210]"]
    other = ["dslash_f32_mode2_nrhs1_links12 128x4hc 0.1240 ms [128x4hc 0.1240]"]
    many = ["dslash_f32_mode0_nrhs12_links12 128x4hc 1.4 ms [128x4hc 1.4]"] + full
    assert bench.d_bytes_per_site(full) == 768
    assert bench.d_bytes_per_site(comp) == 672
    assert bench.d_bytes_per_site(other) == 768  # mode 2 (A) is not the D
    assert bench.d_bytes_per_site(other, mode=2) == 672
    assert bench.d_bytes_per_site(many) == 768  # the 12-rhs key is not the single-rhs one
