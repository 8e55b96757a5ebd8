"""bench.py's output contract: one JSON line with the keys and types the
measurement needs, for the reference arm (the oracle, CPU) and for the GPU
arm (a short run)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def _common(d):
    for k, t in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                 ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                 ("dtype", str), ("data", str), ("config", dict)):
        assert isinstance(d[k], t), k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["config"]["workload"] == "c2_n65536_l45_fwd_inv"
    assert "vs_baseline" in d and d["vs_baseline"] is None


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"], 600)
    _common(d)
    assert d["impl"] == "reference"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_gpu_arm_line():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = _run(["--steps", "40", "--warmup", "3", "--no-cpu-baseline", "--no-batch-compare", "--no-serve",
              "--no-ablation", "--no-peak-measure", "--e2e-steps", "4", "--launch-steps", "5"], 900)
    _common(d)
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["achieved"] > 0 and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9 and 0 < r["frac"] < 1
    assert r["alg_bytes_per_launch"] in (16 * 45 * 65536, 32 * 45 * 65536)
    a = d["roofline_alu"]
    assert a["bound"] == "alu" and a["achieved"] > 0 and a["peak"] > 0
    assert abs(a["frac"] - a["achieved"] / a["peak"]) < 1e-9
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] == 45 * 65536 * 8
    if d["plan"]["kernel"] == "fused":
        assert d["gpu_launches"] == d["steps"]          # one forward + inverse launch per step
    else:
        assert d["gpu_launches"] == 2 * d["plan"]["passes"] * d["steps"]
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    # the timed configuration is the fastest of the candidates timed in the same setting
    sel = d["select_c2"]
    assert d["plan"]["chosen_by"].startswith("timed candidates")
    rows = sel["candidates"]
    assert len(rows) >= 2 and all(r["ok"] for r in rows)
    best = max(rows, key=lambda r: r["value"])
    assert d["config"]["streams"] == best["streams"] and d["config"]["ctas_per_sm"] == best["ctas_per_sm"]
    assert d["plan"]["kernel"] == best["kernel"] and d["plan"]["geometry"] == best["geometry"]


def _traffic_csv(path, kernels, read, write):
    """An ncu --csv log of one call: each kernel with its DRAM bytes and duration."""
    import csv
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"])
        i = 0
        for k in kernels:
            for m, v in (("dram__bytes_read.sum", read), ("dram__bytes_write.sum", write),
                         ("gpu__time_duration.sum", "20,000")):
                w.writerow([i, k, m, "byte", v])
                i += 1


def test_traffic_json_keys_each_per_pass_configuration(tmp_path):
    """The traffic JSON writer keeps per-pass configurations from different
    CSV logs apart: a table plan's row pass (TBL_LAST set) is keyed "table",
    an OT1 plan's "ot1", each with its own column and row launches summed."""
    sys.path.insert(0, ROOT)
    import bench
    col = "void ntt_pass_kernel<8, 4, 4, 0, 1, 1, 0, 1, 0, 1, unsigned long long, 0>(PassArgsT<T11>)"
    row_tbl = "void ntt_pass_kernel<8, 3, 4, 1, 1, 12, 1, 0, 1, 0, unsigned long long, 1>(PassArgsT<T11>)"
    row_ot1 = "void ntt_pass_kernel<8, 3, 4, 1, 1, 12, 1, 0, 1, 0, unsigned long long, 0>(PassArgsT<T11>)"
    a, b, out = tmp_path / "a.csv", tmp_path / "b.csv", tmp_path / "t.json"
    _traffic_csv(a, [col, row_tbl], "2,000,000", "1,000")
    _traffic_csv(b, [col, row_ot1], "3,000", "500")
    bench.write_traffic_json(str(out), [str(a), str(b)], "test")
    entries = json.load(open(out))["entries"]
    got = {(e["kind"], e["geometry"], e["twiddle"], e["direction"]): e["dram_bytes"] for e in entries}
    assert got == {("per_pass", 1, "table", "forward"): 4002000.0, ("per_pass", 1, "ot1", "forward"): 7000.0}
    assert all(e["source_hash"] == bench.kernel_source_hash() for e in entries)
