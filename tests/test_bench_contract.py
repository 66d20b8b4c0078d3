"""The benchmark's reference arm (the CPU oracle) runs without a GPU and prints one JSON
line with the contract's keys: the same metric and unit as the GPU arm, the oracle's
single-core and all-core rates, and an e2e object."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--config", "0"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "trajectories/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["metric"] and d["config"]["workload"].startswith("immigration_death")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["cpu_single_core"]["cores"] == 1 and d["cpu_single_core"]["value"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_profiled_counters_name_launch_shapes_and_their_capture():
    """The ncu figures the headline line reports (roofline.traffic, roofline.issue) are
    keyed by launch shapes the library has, and cite a committed profile summary; the DRAM
    traffic of a launch cannot be below its algorithmic inputs and outputs."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1608_07058_gb300 import workloads as W
    shapes = set(bench.SHAPE_NAMES)
    for (cfg, shape, block, spec), v in bench.PROFILED.items():
        assert cfg in (0, 1, 2, 3) and shape in shapes and block in (64, 128, 256)
        assert spec in (0, 1)
        w = W.config(cfg, n_traj=1)
        B = W.config(cfg).n_traj
        N, M = w.crn.n_species, w.crn.n_reactions
        algorithmic = B * (8 * N + 16 * M + 36) + B * 8 * M + B * 8  # as the line computes
        assert v["dram_bytes"] >= algorithmic * 0.9, (cfg, shape, block)
        assert v["warp_inst"] > 0 and 0.0 <= v["fp64_pipe_pct"] <= 100.0
        ref = v["source"].split("profiles/")[1].rstrip(")")
        assert os.path.exists(os.path.join(ROOT, "profiles", ref)), ref
