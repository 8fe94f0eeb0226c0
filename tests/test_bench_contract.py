"""The benchmark's reference arm (the FP64 oracle on the host cores) prints
one JSON line with the keys the benchmark contract fixes; it runs on CPU."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    import bench
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_algorithmic_bytes_match_the_stated_per_volume_figures():
    """The roofline's algorithmic bytes per volume: every needed volume read
    once (interior plus the 2d face-halo layers; periodic halos rebuilt on
    chip) and the interior written once."""
    import bench
    f = bench.algorithmic_bytes_per_volume
    assert f(2, 16, 4, 4) == 36.0                    # 2D 16^2 FP32
    assert f(2, 16, 4, 8) == 72.0                    # 2D 16^2 FP64
    assert f(3, 8, 5, 4, periodic=True) == 40.0      # 3D 8^3 periodic FP32
    assert f(3, 8, 5, 2, periodic=True) == 20.0      # 3D 8^3 periodic BF16 storage
    assert f(3, 16, 5, 4) == 47.5                    # 3D 16^3 FP32
    # by hand for a small fixed patch: 3^2 interior + 4 x 3 face halo read, 3^2 written
    assert f(2, 3, 4, 8) == 4 * 8 * (9 + 12 + 9) / 9
