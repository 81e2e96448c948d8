"""bench.py's host-side helpers (CPU only): the roofline's traffic and peak
sources, and the ClockSampler's verdict on a clock record."""
import json

import bench


def _traffic_file(tmp_path, sha, workload, value=123456789):
    p = tmp_path / "traffic.txt"
    p.write_text(f"# comment\nassign_src_sha256: {sha}\nworkload: {workload}\nbytes_per_launch[f32]: {value}\n")
    return str(p)


def test_traffic_only_for_the_unchanged_kernel_and_the_same_workload(tmp_path, monkeypatch):
    sha = bench.assign_sources_sha()
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _traffic_file(tmp_path, sha, "wl-a"))
    assert bench.traffic_per_launch("wl-a", "f32") == 123456789.0
    assert bench.traffic_per_launch("wl-b", "f32") is None      # other workload
    assert bench.traffic_per_launch("wl-a", "bf16") is None     # no counters for that storage
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _traffic_file(tmp_path, "0" * 64, "wl-a"))
    assert bench.traffic_per_launch("wl-a", "f32") is None      # kernel source changed since
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.traffic_per_launch("wl-a", "f32") is None


def test_traffic_of_the_schedule_in_use_and_l2_bytes(tmp_path, monkeypatch):
    sha = bench.assign_sources_sha()
    p = tmp_path / "traffic.txt"
    p.write_text(f"assign_src_sha256: {sha}\nworkload: wl\nschedule[f32]: tile_major\n"
                 "bytes_per_launch[f32]: 1000\nl2_bytes_per_launch[f32]: 5000\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(p))
    assert bench.traffic_per_launch("wl", "f32", "tile_major") == 1000.0
    assert bench.traffic_per_launch("wl", "f32", "tile_major", what="l2_bytes") == 5000.0
    assert bench.traffic_per_launch("wl", "f32", "object_major") is None   # taken under another schedule


def test_committed_traffic_file_parses():
    """The committed summary names a workload and an FP32 byte count; whether
    it applies is decided at run time by the kernel source's hash."""
    text = open(bench.TRAFFIC_FILE).read()
    assert "assign_src_sha256:" in text and "workload:" in text and "bytes_per_launch[f32]:" in text


def test_peaks_measured_then_fallback(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 1234.5}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (1234.5, "measured")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "nowhere"))
    assert bench.peaks() == (bench.FALLBACK_HBM_GBS, "fallback")


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_summary_covers_only_the_timed_window():
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    na = "Not Active"
    s.lines = [(0.5, f"0, 1000, 2070, 300, 0x0, {na}, {na}, {na}, {na}"),        # warm-up, before the window
               (1.0, f"0, 2070, 2070, 900, 0x0, {na}, {na}, {na}, {na}"),
               (1.2, f"0, 2000, 2070, 1300, 0x4, {na}, {na}, {na}, Active"),
               (1.4, f"0, 2070, 2070, 950, 0x0, {na}, {na}, {na}, {na}"),
               (1.6, "garbled line"),
               (9.0, f"0, 500, 2070, 100, 0x0, Active, {na}, {na}, {na}")]       # after the window
    assert s.stop(1.0, 1.5) == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                                "samples": 3}
    none = bench.ClockSampler(0)        # nvidia-smi could not be started
    assert none.stop(0.0, 1.0) is None
