"""The benchmark's reference arm on the CPU: one JSON line with the contract's keys, the native arm's
workload config, and a bounded oracle sample.  (The native arm needs the GPU; its aggregation over
ranks is covered in test_replicas_gloo.py.)"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--cpu-seconds", "2"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    r = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "steps", "warmup", "ms_per_step", "higher_is_better", "dtype",
              "config", "cpu_baseline", "e2e"):
        assert k in r, k
    assert r["impl"] == "reference" and r["value"] > 0 and r["higher_is_better"] is True
    assert r["e2e"]["h2d_bytes_per_step"] == 0 and r["e2e"]["d2h_bytes_per_step"] == 0
    assert r["cpu_baseline"]["kind"] == "oracle" and r["cpu_baseline"]["value"] == r["value"]
    import bench
    assert r["config"]["workload"] == bench.WORKLOAD and r["metric"] == bench.METRIC


def test_roofline_model_counts_structural_polarization_flops():
    # orthotropic tables: the roofline's algorithmic flops count the products that are not structurally zero
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from paper_1605_05712_gb300 import lattice_plan, synth
    w = synth.hashin_workload()
    assert bench.tables_orthotropic(w["stiffness"], 3)
    S = [np.array(v) for v in w["stiffness"]]
    S[2][0, 4] = S[2][4, 0] = 1e-30
    assert not bench.tables_orthotropic(S, 3)
    V2 = synth.iso_voigt(1.0, 2.0)
    V2[3, 0] = V2[0, 3] = 0.5   # outside the plane components: no effect in 2-D
    assert bench.tables_orthotropic([V2], 2)
    V2[5, 0] = V2[0, 5] = 0.5   # xx-xy coupling
    assert not bench.tables_orthotropic([V2], 2)
    P = lattice_plan([[16, 1, 0], [0, 16, 1], [0, 0, 16]])
    gen = bench.kernel_models(P, 6, "fp64", ortho=False)
    ort = bench.kernel_models(P, 6, "fp64", ortho=True)
    assert gen[0]["flops"] - ort[0]["flops"] == 6 * P.m * 2 * (36 - 12)
    assert [g["flops"] for g in gen[1:]] == [o["flops"] for o in ort[1:]]
    assert [g["bytes"] for g in gen] == [o["bytes"] for o in ort]
