"""Summarize an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel.

    python profiles/summarize_launches.py gpurun_out/launches.csv BUILDS
prints launches, total time per build and share for every kernel, and the
per-launch durations of the window-scan kernels (one build)."""
import collections
import csv
import sys


def main(path, builds):
    rows = [r for r in csv.reader(open(path)) if len(r) > 10]
    hdr, rows = rows[0], rows[1:]
    i_name, i_val = hdr.index("Kernel Name"), hdr.index("Metric Value")
    agg = collections.defaultdict(lambda: [0, 0.0])
    per = collections.defaultdict(list)
    for r in rows:
        name = r[i_name].split("(")[0].replace("void ", "").replace("(anonymous namespace)::", "")
        name = name.replace("unnamed>::", "")
        ms = float(r[i_val].replace(",", "")) / 1e6
        agg[name][0] += 1
        agg[name][1] += ms
        per[name].append(ms)
    tot = sum(v[1] for v in agg.values())
    print(f"launches {sum(v[0] for v in agg.values())}, kernel time {tot / builds:.2f} ms per build")
    print(f"{'kernel':44s} {'launches':>8s} {'ms/build':>9s} {'share':>7s}")
    for k, v in sorted(agg.items(), key=lambda x: -x[1][1])[:60]:
        print(f"{k:44s} {v[0]:8d} {v[1] / builds:9.3f} {100 * v[1] / tot:6.2f}%")
    for k in per:
        if "scan_anchor" in k or "k_candidates" in k:
            n = len(per[k]) // builds
            print(k, "per level:", " ".join(f"{x:.3f}" for x in per[k][n:2 * n]))


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else 1)
