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



def test_summarize_traffic_per_build_against_the_covered_bytes(tmp_path, monkeypatch):
    # Two builds; per build k_candidates<M> reads 300 and writes 100 bytes,
    # k_hits<M> reads 50; the prune pass's own k_candidates (no template
    # argument) is not part of the window scan.
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream",
           "Block Size", "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit",
           "Metric Value"]
    rows, lid = [], 0
    for _ in range(2):
        for name, rd, wr, ns in (("k_candidates<Mersenne61>", 300, 100, 2000), ("k_hits<Mersenne61>", 50, 0, 1000),
                                 ("k_candidates", 999, 999, 5000)):
            for metric, unit, v in (("dram__bytes_read.sum", "byte", rd), ("dram__bytes_write.sum", "byte", wr),
                                    ("gpu__time_duration.sum", "ns", ns)):
                rows.append([str(lid), "1", "python", "h", f"void {name}(int)", "1", "7", "(256, 1, 1)",
                             "(4, 1, 1)", "0", "10.3", "", metric, unit, str(v)])
            lid += 1
    csv_path = tmp_path / "dram.csv"
    csv_path.write_text("\n".join(",".join(f'"{x}"' for x in r) for r in [hdr] + rows) + "\n")
    line = {"config": {"workload": "w", "n": 1000, "tau": 4, "leaf_len": 32, "levels": 3, "sum_cov_bytes": 900}}
    bj = tmp_path / "bench.json"
    bj.write_text("noise\n" + json.dumps(line) + "\n")
    src = tmp_path / "scan.cu"
    src.write_text("// scan\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "SCAN_SOURCE", str(src))
    out = tmp_path / "rec.json"
    bench.summarize_traffic(str(csv_path), str(bj), str(out), 2)
    rec = json.loads(out.read_text())
    assert rec["alg_bytes_per_build"] == 900 and rec["dram_bytes_per_build"] == 450
    assert rec["dram_bytes_per_alg_byte"] == 0.5
    assert rec["source_sha256_16"] == bench.source_hash(str(src))
    per = rec["per_kernel"]
    assert set(per) == {"k_candidates<Mersenne61>", "k_hits<Mersenne61>"}
    assert per["k_candidates<Mersenne61>"] == {"launches_per_build": 1, "dram_read_bytes": 300,
                                                "dram_write_bytes": 100, "ms": 0.002}
