"""Times the sigma kernels of one instance: `python -m paper_2601_16637_gb300.profile_sigma`.

Builds one handle for a named workload, applies sbd_sigma `--reps` times to a
normalised random vector and prints the per-kernel device times measured with
CUDA events on the launch stream (sbd_kernel_times).  Holds only the tables,
one vector, its transpose and sigma on the device, which keeps it suitable as
the command a profiler captures.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cfg3-6000")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "f32x2"])
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args()

    import torch

    from . import binding as B
    from . import workloads as W

    B.load(build_if_missing=True)
    wl = W.config(args.workload)
    g = B.SBD.from_workload(wl, timing=True)
    x = torch.from_numpy(W.random_vector(g.N, 100)[0]).cuda()
    if args.precision == "mixed":
        x = x.float()
    out = torch.empty(g.N, dtype=torch.float64, device="cuda")
    for _ in range(args.reps):
        g.sigma(x, args.precision, out=out)
    torch.cuda.synchronize()
    ms, n = g.kernel_times()
    p = args.precision
    per = {k: (ms[p][k] / n[p][k] if n[p][k] else None) for k in ms[p]}
    print(json.dumps({"workload": wl.name, "ndets": wl.ndets, "precision": p, "reps": args.reps,
                      "ms_per_launch": per, "sigma_ms": sum(v for v in per.values() if v),
                      "dets_per_s": wl.ndets / (1e-3 * sum(v for v in per.values() if v)),
                      "checksum": float(np.abs(out.cpu().numpy()).sum())}))
    g.close()


if __name__ == "__main__":
    main()
