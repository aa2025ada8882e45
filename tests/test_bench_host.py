"""Host-side pieces of bench.py (CPU): the committed ncu summaries it reads
belong to the current kernel sources, and its per-rank helpers behave."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_profiles_were_captured_on_the_current_kernel_sources():
    """The roofline's traffic and the ALU check come from committed ncu
    summaries; each names the hash of the kernel sources it was taken on."""
    h = bench.kernel_hash()
    for name in ("colour_pass_L32768_q9_traffic.md", "launches_L32768_q9.md",
                 "colour_pass_L16384_q9.md"):
        text = open(os.path.join(ROOT, "profiles", name)).read()
        m = re.search(r"(?:kernel_source_hash:|Kernel sources hash:)\s*"
                      r"([0-9a-f]{16})", text)
        assert m and m.group(1) == h, (name, m and m.group(1), h)
    assert bench.traffic_per_launch(32768) is not None
    assert bench.traffic_per_launch(16384) == bench.traffic_per_launch(32768) / 4
    ips = bench.instructions_per_site()
    assert ips is not None and 20 < ips["white"] < 60 and 20 < ips["black"] < 60


def test_replica_seeds_differ_and_reduce_max_is_identity_alone():
    seeds = {bench.replica_seed(11, r) for r in range(8)}
    assert len(seeds) == 8
    assert bench.reduce_max(1.25, 1) == 1.25


def test_measured_peaks_fall_back_when_absent(tmp_path, monkeypatch):
    hbm, kind = bench.measured_peaks()
    assert hbm > 1000 and kind in ("measured", "fallback")
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "missing.json"))
    assert bench.measured_peaks() == (6800.0, "fallback")
    p = tmp_path / "peaks.json"
    p.write_text('{"hbm_gbs": 6500.5}')
    monkeypatch.setattr(bench, "PEAKS_FILE", str(p))
    assert bench.measured_peaks() == (6500.5, "measured")
