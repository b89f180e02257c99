"""Times the sigma kernels of one instance: `python -m paper_2601_16637_gb300.profile_sigma`.

Builds one handle for a named workload, applies sbd_sigma `--reps` times to a
normalised random vector and prints the per-kernel device times measured with
CUDA events on the launch stream (sbd_kernel_times).  Holds only the tables,
one vector, its transpose and sigma on the device, which keeps it suitable as
the command a profiler captures.

With `--solve`, runs one Davidson solve of the workload instead (its own
precision, tolerance and subspace size), so that the solver's vector kernels
can be captured; `--strings n` shrinks |A| = |B| to n to keep such a capture
small.
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
    ap.add_argument("--solve", action="store_true", help="one Davidson solve instead of sigma products")
    ap.add_argument("--strings", type=int, default=0, help="override |A| = |B|")
    args = ap.parse_args()

    import torch

    from . import binding as B
    from . import workloads as W

    B.load(build_if_missing=True)
    over = {"nA": args.strings, "nB": args.strings} if args.strings > 0 else {}
    wl = W.config(args.workload, **over)
    if args.solve:
        import time
        with B.SBD.from_workload(wl, max_subspace=wl.max_subspace) as g:
            t0 = time.perf_counter()
            res = g.davidson(wl.nroots, wl.tol, wl.precision, vectors=None)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
        print(json.dumps({"workload": wl.name, "ndets": wl.ndets, "energies": [float(e) for e in res.energies],
                          "status": res.status, "seconds": sec, "report": res.report}, default=str))
        if res.status != 0:
            raise SystemExit(1)
        return
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
