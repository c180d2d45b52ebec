"""Write the launch-shape tuning cache (tuning_b300.txt) for the benchmark workloads.

Usage (on the GPU): python -m paper_2507_12349_b300.autotune [--out FILE] [--n-mat K] [--precision P]
Runs cos_autotune for every (order, precision, matrices per configuration) that the
workloads launch with and writes one line per case: "n precision n_mat warps ctas ms prefetch".
With --n-mat K (or --precision P) only the cases with K matrices per configuration (or that
precision) are re-tuned and merged with the lines of the current tuning file (other lines
kept); the result goes to --out.
The sample size fills the GPU: a batch per CTA for 2 CTAs per SM (one CTA per SM at orders
11-12, where one batch already holds ~0.3-0.6 s of FP64 work).
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# (order, matrices per configuration, loop weight, shifts, precision)
CASES = [
    (4, 1, 2, False, "fp64"),
    (8, 4, 1, False, "fp64"), (8, 4, 1, False, "mixed"),
    (10, 3, 1, True, "mixed"), (10, 3, 1, True, "fp64"),
    (10, 4, 1, False, "fp64"),
    (8, 4, 1, False, "df64"), (10, 3, 1, True, "df64"),
    # SU(2) with two spin blocks (determinant weights, or CoS with two flavors)
    (10, 2, 1, False, "fp64"), (10, 2, 1, False, "mixed"), (10, 2, 1, False, "df64"),
] + [(n, 1, 6, False, "fp64") for n in range(4, 13)]


def main():
    import torch
    from paper_2507_12349_b300 import binding as B
    p = argparse.ArgumentParser()
    p.add_argument("--out", default=B.TUNING_FILE)
    p.add_argument("--n-mat", type=int, default=0, help="re-tune only these cases and merge")
    p.add_argument("--precision", default="", choices=["", "fp64", "mixed", "df64"],
                   help="re-tune only this precision's cases and merge")
    args = p.parse_args()
    torch.cuda.set_device(0)
    B.lib()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    lines = []
    # configurations per lane of each precision's forward kernel (mixed: four, double-float:
    # two, FP64: one), so that the sample fills every SM with batches
    per_lane = {"fp64": 1, "mixed": 4, "df64": 2}
    seen = set()
    for n, n_mat, wt, shifts, prec in CASES:
        if (args.n_mat and n_mat != args.n_mat) or (args.precision and prec != args.precision):
            continue
        if (n, n_mat, prec) in seen:     # the shape does not depend on the loop weight
            continue
        seen.add((n, n_mat, prec))
        cpb = (32 // n_mat) * per_lane[prec]
        n_cfg = cpb * sms * (1 if n >= 11 else 2)
        w, c, pf, ms = B.cos_autotune(n, n_mat, wt, shifts, prec, n_cfg)
        line = f"{n} {B.PRECISIONS[prec]} {n_mat} {w} {c} {ms:.4f} {int(pf)}"
        print(line, f"# {prec} configs={n_cfg}", flush=True)
        lines.append(line)
    if (args.n_mat or args.precision) and os.path.exists(B.TUNING_FILE):
        fresh = {tuple(ln.split()[:3]) for ln in lines}
        kept = [ln.strip() for ln in open(B.TUNING_FILE) if ln.strip() and tuple(ln.split()[:3]) not in fresh]
        lines = kept + lines
    with open(args.out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
