"""Host-side parts of bench.py on CPU: the oracle sample and crop parity
helpers, and the reference arm's JSON line on a small workload."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_oracle_sample_and_crop_parity():
    c, pos, cams, snaps = bench.make_workload("zel32_ortho256")
    nf, sec, ref = bench.oracle_sample(c, pos, cams, snaps, 64)
    assert nf > 0 and sec > 0 and ref.shape == (64, 64)
    assert bench.central_crop(cams[0], 64) == (96, 96, 64, 64)
    ok = bench.crop_parity(ref, ref.astype(np.float32))
    assert ok["pass"] and ok["max_rel_err"] <= 1e-6
    bad = ref.copy()
    bad[3, 5] += 0.01 * max(1.0, ref.max())
    assert not bench.crop_parity(ref, bad)["pass"]
    base, parity = bench.cpu_baseline(c, pos, cams, snaps, 64, gpu_crop=ref)
    assert base["kind"] == "oracle" and base["cores"] >= 1 and base["value"] > 0
    assert parity["pass"] and parity["crop"] == [96, 96, 64, 64]


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "zel32_ortho256", "--steps", "2", "--warmup", "1", "--cpu-sample-crop", "64"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "fragments/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["config"]["workload"] == "zel32_ortho256"


def test_fp32_peak_from_unit_counts_and_clock():
    peak, mhz, src = bench.fp32_peak_tflops(152)
    assert mhz > 0 and src
    assert abs(peak - 152 * 128 * 2 * mhz * 1e-6) < 1e-9


def test_raster_traffic_follows_the_captured_sources(monkeypatch):
    """The raster's DRAM traffic in the bench line is the per-frame capture
    scaled by the frames, and only while the raster's sources hash to the
    captured ones: after any change to them it reads as unmeasured."""
    cap = dict(bench.RASTER_TRAFFIC)
    monkeypatch.setattr(bench, "RASTER_TRAFFIC", dict(cap, sources_sha16=bench.raster_sources_sha16()))
    assert bench.raster_traffic(128) == cap["bytes_per_frame"] * 128
    monkeypatch.setattr(bench, "RASTER_TRAFFIC", dict(cap, sources_sha16="0" * 16))
    assert bench.raster_traffic(128) is None
    monkeypatch.setattr(bench, "RASTER_TRAFFIC", dict(cap, bytes_per_frame=None))
    assert bench.raster_traffic(128) is None

