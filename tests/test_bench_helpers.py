"""Host-side helpers of bench.py (no GPU): the launch-list summary the profiles
quote, and the rule that the recorded DRAM traffic is used only for the kernel
source it was measured on."""
import json

import bench


def _launch_csv(path, rows):
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream",
           "Block Size", "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit",
           "Metric Value"]
    with open(path, "w") as f:
        f.write(",".join(f'"{h}"' for h in hdr) + "\n")
        for i, (name, ns) in enumerate(rows):
            vals = [str(i), "1", "python", "h", f"void k_{name}(int)", "1", "7", "(256, 1, 1)",
                    "(4, 1, 1)", "0", "10.3", "Command line profiler metrics", "gpu__time_duration.sum",
                    "ns", f"{ns:,}"]
            f.write(",".join(f'"{v}"' for v in vals) + "\n")


def test_summarize_launches_per_build_and_share(tmp_path, capsys):
    p = tmp_path / "launches.csv"
    # Two builds: k_a 3 + 1 us and k_b 4 us per build.
    _launch_csv(p, [("a", 3000), ("a", 1000), ("b", 4000), ("a", 3000), ("a", 1000), ("b", 4000)])
    bench.summarize_launches(str(p), 2)
    out = capsys.readouterr().out.splitlines()
    assert out[0] == "launches 6, kernel time 0.01 ms per build"
    rows = {r.split()[0]: r.split()[1:] for r in out[2:4]}
    assert rows["k_a"] == ["4", "0.004", "50.00%"]
    assert rows["k_b"] == ["2", "0.004", "50.00%"]


def test_recorded_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"kernel": "window_scan", "source_sha256_16": bench.source_hash(str(src)),
           "dram_bytes_per_alg_byte": 3.5}
    (prof / "window_scan_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "SCAN_SOURCE", str(src))
    assert bench.recorded_traffic("window_scan") == 3.5
    assert bench.recorded_traffic("other_kernel") is None
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.recorded_traffic("window_scan") is None

