"""The benchmark's JSON contract on the CPU: the reference arm (the oracle on the host's cores,
on a bounded sample of the workload) prints one JSON line with the keys of the GPU arm, and both
arms name the workload with the same description."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--sample-cells", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["unit"] == "TFLOP/s" and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 0 and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    assert d["config"]["workload"] == bench.workload_text(W.CONFIGS["c5"]())


def test_workload_description_follows_the_configuration():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    full = bench.workload_text(W.CONFIGS["c3"]())
    assert full == ("c3_mixed_4k_8atom_16cube_p6: zincblende a=8.5 bohr, 8 atoms (Z 14/6), graded 16^3 cells p=6, "
                    "40 enrichment functions, MP 2x2x1 (4 k, complex), 64 vectors/k, Chebyshev degree 30")
    small = bench.workload_text(W.CONFIGS["c3small"]())
    assert "graded 8^3 cells" in small and "(2 k, complex)" in small
    large = bench.workload_text(W.CONFIGS["c5"]())
    assert large == ("c5_mixed_gamma_62atom_32cube_p6: supercell a=16.4 bohr, 62 atoms (Z 14/6), graded 32^3 cells "
                     "p=6, 310 enrichment functions, Gamma point (real), 360 vectors/k, Chebyshev degree 50")
    assert not bench.is_complex(W.CONFIGS["c5"]()) and bench.is_complex(W.CONFIGS["c3"]())
    c4 = bench.workload_text(W.CONFIGS["c4mid"]())
    assert c4 == ("c4mid_c64_8k_16atom_12cube_p6: supercell a=12 bohr, 16 atoms (Z 14/6), graded 12^3 cells p=6, "
                  "80 enrichment functions, MP 2x2x2 (8 k, complex), 97-123 vectors/k, Chebyshev degree 30")


def test_refined_cell_count_used_for_traffic_scaling():
    # the graded meshes put each of the 8 nuclei on a corner shared by 8 cells: 64 refined cells,
    # the rest single-leaf (the bench scales the captured traffic by these counts)
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    for name in ("c3", "c3small"):
        assert bench.nucleus_cells(W.CONFIGS[name]()) == 64


def test_device_potential_matches_host_potential():
    # the bench evaluates the synthetic V_eff with torch (large point sets); it must be the same input
    # the oracle side computes with numpy, a nucleus position included
    import numpy as np
    sys.path.insert(0, ROOT)
    import workloads as W
    w = W.CONFIGS["c5mid"]()
    pts = np.random.default_rng(0).uniform(0.0, w.a, (5000, 3))
    pts[:3] = w.pos[:3]
    a = W.veff(pts, w.a, w.pos, w.Z, w.sigma)
    b = W.veff_device(pts, w.a, w.pos, w.Z, w.sigma, device="cpu").numpy()
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a))
