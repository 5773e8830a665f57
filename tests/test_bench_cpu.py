"""The benchmark's reference arm (the CPU oracle on a bounded sample) runs without a GPU and
prints one JSON line with the keys the benchmark contract requires."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("config", ["d1", "d2", "d6"])
def test_reference_arm_prints_one_contract_line(config):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", config, "--steps", "1",
                          "--warmup", "3", "--ref-sample-mb", "1"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["value"] > 0
    assert d["warmup"] >= 3 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_profiled_traffic_scales_and_refuses_what_does_not_match(tmp_path, monkeypatch):
    """roofline.traffic: the committed capture's DRAM bytes scaled to the run's text size, or
    None when the kernel sources, the launch shape or the capture's text size do not fit."""
    sys.path.insert(0, ROOT)
    import bench

    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    plan = {"warps_per_block": 24, "blocks": 152}

    def write(**kw):
        d = {"kernel_hash": "h", "config": "dx", "text_bytes": 1 << 30, "warps_per_block": 24, "blocks": 152,
             "dram_bytes_per_launch": 3 << 29}
        d.update(kw)
        (tmp_path / "profiles" / "traffic_dx.json").write_text(json.dumps(d))

    monkeypatch.setattr(bench, "kernel_hash", lambda: "h")
    write()
    assert bench.profiled_traffic("dx", 4 << 30, plan) == 6 << 30  # 1.5 B per text byte, 4 GiB
    assert bench.profiled_traffic("dx", 4 << 30, dict(plan, warps_per_block=23)) is None
    write(kernel_hash="other")
    assert bench.profiled_traffic("dx", 4 << 30, plan) is None
    write(kernel_hash="h", text_bytes=0)
    assert bench.profiled_traffic("dx", 4 << 30, plan) is None
    assert bench.profiled_traffic("none", 4 << 30, plan) is None


def test_host_cpu_names_a_model_and_the_core_count():
    sys.path.insert(0, ROOT)
    import bench

    h = bench.host_cpu()
    assert isinstance(h["model"], str) and h["model"] and h["nproc"] == os.cpu_count()
