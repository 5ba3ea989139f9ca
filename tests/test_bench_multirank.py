"""The benchmark's multi-process path on CPU: two gloo ranks on 127.0.0.1.

Every rank times its own replica; the job's figures are the slowest rank's time and the
work of all ranks (bench.combine_ranks), which both ranks must receive.  Under torchrun the
reference arm runs on rank 0 alone: the other ranks return at once, printing nothing."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, work = bench.combine_ranks(dist, "cpu", 10.0 + rank, 100.0 * (rank + 1))
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"ms": ms, "work": work}, f)
        assert bench.dist_env() == (rank, 0, world)
    finally:
        dist.destroy_process_group()


def test_combine_ranks_over_two_gloo_ranks(tmp_path):
    port = free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got == {"ms": 11.0, "work": 300.0}


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(None, "cpu", 3.5, 7.0) == (3.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only():
    """rank 1 of a two-process job exits 0 at once and prints nothing (no oracle work)."""
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_json_line_on_a_small_graph():
    """The reference arm (the FP64 oracle on the host) prints one JSON line with the
    contract's keys; run here on R-MAT scale 12 so it finishes in seconds."""
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "LOCAL_RANK", "WORLD_SIZE")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--scale", "12", "--er-log2", "12", "--steps", "3", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]


def test_recorded_traffic_follows_the_kernel_code_not_its_comments():
    """The committed DRAM-traffic figures apply while the kernel sources' code is the
    code that was captured: the sha ignores comments and layout, not code or literals."""
    sys.path.insert(0, ROOT)
    import bench
    a = "int f(int x) { return x + 1; }  // one\n/* block */ const char* s = \"// kept\";\n"
    b = "/* other */ int f(int x) {\n  return x + 1;  // two\n}\nconst char* s = \"// kept\";"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(a.replace("x + 1", "x + 2"))
    assert bench._code_only(a) != bench._code_only(a.replace("// kept", "// gone"))


def test_roofline_arithmetic_on_synthetic_records():
    """The roofline object from per-solve records: algorithmic bytes per launch (B of a full
    sweep, scaled by the edges a launch gathered), achieved = bytes / loop time, traffic =
    recorded bytes per gathered edge x edges per launch, and the dominant kernel = the
    variant with the larger share of solve time, reported on the R-MAT graph."""
    sys.path.insert(0, ROOT)
    import bench
    n, nnz = 1 << 24, 263_429_870
    st = {"n": n, "nnz": nnz, "rowptr_bytes": 4, "n_tma_tiles": 10}
    resident = [("rmat24", None, st), ("er24", None, dict(st, n_tma_tiles=0))]
    recs = []
    for g in ("rmat24", "er24"):
        # Jacobi: 19 iterations of nnz edges each, 0.9 ms apiece; barrier-free: one launch
        # that gathered 15.5 sweeps' worth of edges in 14 ms
        recs.append({"graph": g, "variant": "jacobi", "iterations": 19, "loop_ms": 19 * 0.9,
                     "loop_edge_visits": 19.0 * nnz, "time_to_tol_ms": 17.0})
        recs.append({"graph": g, "variant": "nonblocking", "iterations": 17, "loop_ms": 14.0,
                     "loop_edge_visits": 15.5 * nnz, "time_to_tol_ms": 16.0})
    roof, rows = bench.rooflines(recs, resident)
    B = bench.algorithmic_bytes(n, nnz, 4)
    assert B == 4 * nnz + 4 * (n + 1) + 20 * n
    by = {(r["graph"], r["variant"]): r for r in rows}
    j = by[("rmat24", "jacobi")]
    assert j["launches"] == 19
    assert j["bytes_per_launch"] == pytest.approx(B)
    assert j["achieved"] == pytest.approx(B / 0.9e-3 / 1e9)
    assert j["frac"] == pytest.approx(j["achieved"] / j["peak"])
    assert "k_rows_tma" in j["kernel"] and "k_rows_tma" not in by[("er24", "jacobi")]["kernel"]
    nb = by[("rmat24", "nonblocking")]
    assert nb["launches"] == 1
    assert nb["bytes_per_launch"] == pytest.approx(15.5 * B)
    assert nb["achieved"] == pytest.approx(15.5 * B / 14e-3 / 1e9)
    for (g, v), r in by.items():
        per_edge = bench.recorded_traffic(v, g)
        if per_edge is None:
            assert r["traffic"] is None
        else:
            assert r["traffic"] == pytest.approx(per_edge * r["bytes_per_launch"] / B * nnz)
    # Jacobi holds 34 of the 66 ms of solve time: it is the dominant kernel
    assert roof["kernel"].startswith("jacobi iteration") and roof["kernel"].endswith("on rmat24")
    assert roof["share_of_step"] == pytest.approx(34.0 / 66.0)
    assert roof["achieved"] == pytest.approx(j["achieved"]) and roof["traffic"] == j["traffic"]
    assert set(roof) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}


def test_clock_samples_summary():
    """nvidia-smi lines (csv, noheader, nounits) -> median SM clock, the maximum clock and
    every throttle reason seen Active; malformed lines are skipped."""
    sys.path.insert(0, ROOT)
    import bench
    lines = ["2070, 2070, 812.33, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "1980, 2070, 1390.02, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "2070, 2070, 901.50, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "garbage",
             "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    c = bench.ClockSampler.summarise(lines)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    hot = lines[:1] + ["1500, 2070, 1200.0, 0x0000000000000048, Active, Active, Not Active, Not Active"]
    c = bench.ClockSampler.summarise(hot)
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and c["sm_mhz"] == 1785.0
    assert bench.ClockSampler.summarise([])["reasons"] == ["no samples"]


def test_gather_ceiling_arithmetic_on_synthetic_records():
    """frac_of_ceiling = (gathers outside the L1 hub prefix per launch / the measured random
    gather rate) / the launch's time: 0.57 ms of requests in a 0.9 ms iteration is 0.633."""
    sys.path.insert(0, ROOT)
    import bench
    n, nnz = 1 << 24, 263_429_870
    hub = int(0.43 * nnz)
    st = {"n": n, "nnz": nnz, "rowptr_bytes": 4, "n_tma_tiles": 10, "hub_prefix_edges": hub}
    resident = [("rmat24", None, st)]
    recs = [{"graph": "rmat24", "variant": "jacobi", "iterations": 19, "loop_ms": 19 * 0.9,
             "loop_edge_visits": 19.0 * nnz, "time_to_tol_ms": 17.0},
            {"graph": "rmat24", "variant": "nonblocking", "iterations": 17, "loop_ms": 14.0,
             "loop_edge_visits": 15.5 * nnz, "time_to_tol_ms": 16.0}]
    rate = 303e9
    roof, rows = bench.rooflines(recs, resident, rate)
    by = {r["variant"]: r for r in rows}
    c_ms = (nnz - hub) / rate * 1e3
    assert by["jacobi"]["gather_ceiling"]["ms_per_launch"] == pytest.approx(c_ms)
    assert by["jacobi"]["gather_ceiling"]["frac_of_ceiling"] == pytest.approx(c_ms / 0.9)
    assert by["nonblocking"]["gather_ceiling"]["ms_per_launch"] == pytest.approx(15.5 * c_ms)
    assert roof["frac_of_ceiling"] == pytest.approx(c_ms / 0.9)
    assert bench.rooflines(recs, resident)[0].get("frac_of_ceiling") is None
