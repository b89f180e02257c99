"""Runs the batched engine on the first n instances of the batched workload:
`python -m paper_2601_16637_gb300.profile_engine --n 8`.

Submits the instances to one engine, runs it to completion and prints the engine statistics and
the per-job results as one JSON line; a profiler can capture the engine's kernels from it.
"""
from __future__ import annotations

import argparse
import json
import time


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8)
    ap.add_argument("--subspace", type=int, default=20)
    ap.add_argument("--schedule", default="lockstep", choices=["lockstep", "fair"])
    args = ap.parse_args()

    import torch

    from . import binding as B
    from . import workloads as W

    B.load(build_if_missing=True)
    insts = W.batch_instances(64)[: args.n]
    t0 = time.perf_counter()
    with B.Engine(max_slots=len(insts), max_subspace=args.subspace, max_norb=26, max_strings=5000,
                  max_iter=400, schedule=args.schedule) as e:
        ids = [e.submit(w, tol=w.tol, tol_energy=w.extra["tol_energy"]) for w in insts]
        e.run()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res = [e.result(j) for j in ids]
        st = e.stats()
    print(json.dumps({"instances": len(insts), "schedule": args.schedule, "seconds": dt, "engine": st,
                      "iterations": [r["iterations"] for r in res], "status": [r["status"] for r in res],
                      "energies": [r["energy"] for r in res]}))


if __name__ == "__main__":
    main()
