"""The reference arm of the benchmark (the oracle on the host cores) runs on
the CPU and prints one JSON line with the keys the measurement contract asks
for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--workload", "lorenz63_h0.25"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == d["unit"] == "cell-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["config"]["workload"] == "lorenz63_h0.25"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_traffic_records_name_real_workloads_and_the_current_sources():
    """Every DRAM-traffic record of the bench is keyed by a workload's own name
    (the name the bench looks up), a precision and a step kernel, and carries
    the hash of the device sources it was measured on, which the bench compares
    before it reports roofline.traffic (a record of other sources reads as
    null)."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2508_13986_gb300 import workloads as W

    names = {W.config(n).name for n in ("lorenz63_h0.5", "lorenz63_h0.25", "lorenz96_6d", "lorenz96_6d_h0.5",
                                         "paper_e1", "paper_e2")}
    kernels = {"k_faces", "k_waves_list", "k_apply", "k_persistent"}
    assert bench.TRAFFIC_BYTES_PER_CELL
    for key, rec in bench.TRAFFIC_BYTES_PER_CELL.items():
        wname, prec, kern = key.split("/")
        assert wname in names and prec in ("f64", "f32") and kern in kernels, key
        assert rec["bytes_per_cell"] > 0 and len(rec["src"]) == 16, key
    h = bench.device_source_hash()
    assert len(h) == 16 and all(c in "0123456789abcdef" for c in h)
