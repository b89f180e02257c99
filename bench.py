#!/usr/bin/env python
"""Benchmark: selected-basis diagonalization on the norb=29 workload.

Workload (the largest single-instance configuration): norb = 29, 10 alpha +
10 beta electrons, |A| = |B| = 10,000 Gumbel-top-k strings (orbital weights
exp(-0.25 p)), 1.0e8 determinants, synthetic integrals (see
paper_2601_16637_gb300/workloads.py).  One step = one complete solve through
the C ABI: sbd_create (string sort/validation, excitation tables, string
matrix elements, Hamiltonian diagonal) + sbd_davidson (lowest root, mixed
precision sigma with FP64 defect correction, residual <= 1e-6) +
sbd_destroy.  Inputs are resident in HBM when the timed region starts.

value  = sigma=Hc determinant throughput of the whole step:
         N * (sigma vector applications in the step) / step time, summed
         over ranks (replicas: each GPU solves its own instance).
e2e    = the same through the same calls with pinned HOST inputs and the
         eigenvector written to pinned HOST memory (copies inside the timing).
roofline = the dominant kernel of the step, timed with CUDA events recorded
         by the library on the stream it launches on.
cpu_baseline = the CPU oracle (tests-only code) timed on a bounded sample of
         sigma rows of the same workload on this host's cores.

`--impl reference` times that oracle alone (the CPU reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "σ=Hc dets/s"
UNIT = "dets/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}
NUM_SMS = 152
FP32_LANES_PER_SM = 128
FP64_NOMINAL_TFLOPS = 1.25
# sigma products of the FP64 3-root solve of the 4.0e6-determinant instance (cfg2) on the GPU, the
# count the oracle Davidson time of that instance is extrapolated with
CFG2_FP64_SIGMA_COUNT = 446


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def nvsmi_gpu_id(device: int, props=None, visible: str | None = None) -> str:
    """The nvidia-smi `-i` argument for CUDA device `device` of this process.  nvidia-smi numbers GPUs
    by physical index and ignores CUDA_VISIBLE_DEVICES, so the device is named by its UUID
    ("GPU-<uuid>"); without one, a CUDA_VISIBLE_DEVICES entry is mapped back to what it names."""
    if props is None:
        try:
            import torch

            props = torch.cuda.get_device_properties(device)
        except Exception:
            props = None
    uuid = getattr(props, "uuid", None) if props is not None else None
    if uuid:
        u = str(uuid)
        return u if u.startswith(("GPU-", "MIG-")) else "GPU-" + u
    if visible is None:
        visible = os.environ.get("CUDA_VISIBLE_DEVICES")
    if visible:
        ent = [x.strip() for x in visible.split(",") if x.strip()]
        if 0 <= device < len(ent):
            return ent[device]
    return str(device)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region on the GPU that CUDA
    device `device` of this process is."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.gpu = nvsmi_gpu_id(device)
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as f:
            out = parse_clock_samples(f)
        os.unlink(self.path)
        return out


def parse_clock_samples(lines) -> dict:
    """Median SM clock, maximum SM clock and the throttle reasons seen in nvidia-smi samples
    (ClockSampler.FIELDS, csv, no header, no units); malformed lines are skipped."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def energy_error_estimates(energies, residuals, report) -> list:
    """Per root j the Kato-Temple-form error estimate residual_j^2 / (gap + E_last - E_j), gap being
    the report's gap_estimate (first Ritz value above the roots minus the highest root); None for
    every root when no gap was recorded."""
    gap = float(report.get("gap_estimate", 0.0) or 0.0)
    if not gap > 0.0:
        return [None] * len(energies)
    last = float(energies[-1])
    return [float(r) ** 2 / (gap + last - float(e)) for e, r in zip(energies, residuals)]


def max_over_ranks(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def workload_config(wl, precision):
    return {"workload": f"{wl.name}: norb={wl.norb}, nalpha=nbeta={wl.nalpha}, |A|=|B|={wl.A.size:,} "
                        f"Gumbel-top-k strings, {wl.ndets:.2e} determinants, {wl.nroots} root, "
                        f"{precision} sigma + FP64-accurate defect correction, residual <= {wl.tol:g}",
            "norb": wl.norb, "nalpha": wl.nalpha, "nbeta": wl.nbeta, "nA": int(wl.A.size), "nB": int(wl.B.size),
            "ndets": int(wl.ndets), "nroots": wl.nroots, "tol": wl.tol, "precision": precision,
            "step": "sbd_create + sbd_davidson + sbd_destroy (one full solve)",
            "l2": "inputs larger than L2 (C is 0.4-0.8 GB per vector, L2 129 MB)"}


# ---------------------------------------------------------------------------
# CPU oracle timing (tests-only code; timed here as the reported baseline)


def oracle_rows_rate(wl, budget_s: float, seed: int = 0):
    from oracle import oracle as O

    O.build()
    o = O.Oracle.from_workload(wl)
    x = np.random.default_rng([seed, 7]).normal(size=(1, o.N))
    x /= np.linalg.norm(x)
    rng = np.random.default_rng(seed)
    threads = O.num_threads()
    # batches of uniformly drawn rows, each about twice the last, until the budget is spent
    nrows, dt, batch = 0, 0.0, max(64, 8 * threads)
    while dt < budget_s:
        rows = rng.integers(0, o.N, size=batch)
        t0 = time.perf_counter()
        o.sigma_rows(x, rows)
        step = time.perf_counter() - t0
        nrows += batch
        dt += step
        left = budget_s - dt
        batch = int(min(2 * batch, max(64, batch * left / max(step, 1e-9))))
    o.close()
    return nrows / dt, nrows, dt, threads


def oracle_extras(cfg3_rate: float, cfg3_ndets: int, cfg2_sigma_count: int | None = None,
                  full_cfg2: bool = False, cfg2_seconds: float = 5.0) -> dict:
    """Oracle timings on the host cores beside the bounded sample: one full sigma and the full
    Davidson on the full-space norb=8 instance (cfg1); on the 4.0e6-determinant instance (cfg2) one
    full sigma when full_cfg2 (minutes of CPU time), else sigma rows sampled for cfg2_seconds and
    extrapolated to one sigma.  The oracle Davidson on cfg2 (hundreds of sigma products, about a day
    of CPU time) and one sigma on the 1.0e8-determinant instance are not run: they are extrapolated
    from the sigma time and the sampled row rate, and labelled as such."""
    from oracle import oracle as O
    from paper_2601_16637_gb300 import workloads as W

    O.build()
    out = {"threads": O.num_threads()}
    for name in ("cfg1", "cfg2"):
        wl = W.config(name)
        if name == "cfg2" and not full_cfg2:
            rate, nrows, dt, _ = oracle_rows_rate(wl, cfg2_seconds)
            ts = wl.ndets / rate
            out[name] = {"ndets": int(wl.ndets), "sigma_s_extrapolated": ts, "sigma_dets_per_s": rate,
                         "note": f"extrapolated, not run: {nrows} sampled sigma rows in {dt:.1f} s"}
            if cfg2_sigma_count:
                out[name]["davidson_s_extrapolated"] = ts * cfg2_sigma_count
                out[name]["davidson_note"] = (f"extrapolated, not run: sigma time x {cfg2_sigma_count} sigma "
                                              f"products (the GPU FP64 solve of this instance)")
            continue
        o = O.Oracle.from_workload(wl)
        x = W.random_vector(o.N, 100)
        t0 = time.perf_counter()
        o.sigma(x)
        ts = time.perf_counter() - t0
        out[name] = {"ndets": int(wl.ndets), "sigma_s": ts, "sigma_dets_per_s": wl.ndets / ts}
        if name == "cfg1":
            t0 = time.perf_counter()
            e, _, r, it = o.davidson(nroots=wl.nroots, tol=wl.tol)
            out[name]["davidson_s"] = time.perf_counter() - t0
            out[name]["davidson_iterations"] = int(it)
            out[name]["davidson_energy_Ha"] = float(e[0])
        elif cfg2_sigma_count:
            out[name]["davidson_s_extrapolated"] = ts * cfg2_sigma_count
            out[name]["davidson_note"] = (f"extrapolated, not run: measured sigma time x {cfg2_sigma_count} sigma "
                                          f"products (the GPU FP64 solve of this instance)")
        o.close()
    out["cfg3"] = {"ndets": int(cfg3_ndets), "sigma_s_extrapolated": cfg3_ndets / cfg3_rate,
                   "note": "extrapolated, not run: determinants / the sampled sigma-row rate"}
    return out


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return 0
    from paper_2601_16637_gb300 import workloads as W

    wl = W.config(args.workload)
    precision = wl.precision
    budget = args.ref_step_seconds
    for _ in range(args.warmup):
        oracle_rows_rate(wl, min(2.0, budget), seed=1)
    vals, rows_total, t_total, threads = [], 0, 0.0, 1
    for k in range(args.steps):
        v, nrows, dt, threads = oracle_rows_rate(wl, budget, seed=100 + k)
        vals.append(v)
        rows_total += nrows
        t_total += dt
    value = rows_total / t_total
    sample = (f"{args.steps} steps x ~{budget:g} s: {rows_total} sigma rows sampled uniformly from the "
              f"{wl.ndets:.1e} determinants (each row = one determinant's sigma element)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(wl, precision),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm


def kernel_source_digest() -> str:
    """sha256 prefix of the mixed alpha-beta pass's source (the column-stationary kernel: its chunk,
    table and row device functions) and of the four kernels that lay out the source-major singles it
    walks (the item order decides which rows of C it reads when)."""
    csrc = os.path.join(ROOT, "paper_2601_16637_gb300", "csrc")
    src = open(os.path.join(csrc, "sigma.cu")).read()
    start = src.index("template <int KC, int RS>\n__device__ __forceinline__ void src_chunk(")
    end = src.index("\n}\n", src.index("__global__ void __launch_bounds__(kSrcThreads, 1) ab_src_kernel(")) + 3
    tab = open(os.path.join(csrc, "tables.cu")).read()
    parts = []
    for name in ("src_count_kernel(", "src_fill_kernel(", "src_slice_order_kernel(", "src_entry_order_kernel("):
        t0 = tab.index("__global__ void " + name)
        parts.append(tab[t0:tab.index("\n}\n", t0) + 3])
    return hashlib.sha256((src[start:end] + "".join(parts)).encode()).hexdigest()[:16]


def traffic_record(kernel: str):
    """dram bytes per launch from the committed ncu summary, if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    digest = kernel_source_digest()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel and parts[1] == digest:
            return float(parts[2])
    return None


# ---------------------------------------------------------------------------
# batched and served solves (the engine)


def serial_fp64(B, wl, stream):
    """The plain per-instance path: sbd_create + FP64 sbd_davidson + sbd_destroy, same stopping rule."""
    import torch

    t0 = time.perf_counter()
    with B.SBD.from_workload(wl, tol_energy=wl.extra.get("tol_energy", 0.0), stream=stream) as g:
        s = g.davidson(1, wl.tol, "fp64", vectors=None)
    torch.cuda.synchronize()
    return time.perf_counter() - t0, float(s.energies[0]), int(s.status), s.report


def engine_line(args, metric_value, elapsed, n_jobs, stats, extra, clk, config):
    return {"metric": METRIC, "value": metric_value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": config,
            "solves_per_s": n_jobs / elapsed, "gpu_launches": int(stats["kernel_launches"]),
            "graph_launches": int(stats["graph_launches"]), "engine": stats, "clocks": clk, **extra}


def batch_measure(B, insts, subspace: int, warmup: int, steps: int, schedule: str = "lockstep") -> dict:
    """One engine run over `insts` (persistent launches, CUDA graphs), `steps` times after `warmup`
    untimed runs on the two smallest instances, against the serial FP64 per-instance path on the
    same instances and stopping rule.  solves/s count converged jobs only (status 0)."""
    import torch

    opts = dict(max_slots=len(insts), max_subspace=subspace, max_norb=max(w.norb for w in insts),
                max_strings=max(max(w.A.size, w.B.size) for w in insts), max_iter=400, schedule=schedule)
    small = sorted(insts, key=lambda w: w.ndets)[:2]
    for _ in range(warmup):
        with B.Engine(**opts) as e:
            for w in small:
                e.submit(w, tol=w.tol, tol_energy=w.extra["tol_energy"])
            e.run()
    torch.cuda.synchronize()
    elapsed, dets_sigma, results, stats = 0.0, 0.0, [], None
    for _ in range(steps):
        t0 = time.perf_counter()
        with B.Engine(**opts) as e:
            ids = [e.submit(w, tol=w.tol, tol_energy=w.extra["tol_energy"]) for w in insts]
            e.run()
            torch.cuda.synchronize()
            elapsed += time.perf_counter() - t0
            results = [e.result(j) for j in ids]
            stats = e.stats()
        dets_sigma += sum(r["ndets"] * (r["sigma_mixed"] + r["sigma_fp64"]) for r in results)
    stream = torch.cuda.current_stream()
    serial_t, dE, serial_status, serial_it = 0.0, 0.0, [], []
    for w, r in zip(insts, results):
        t, e64, st, rep = serial_fp64(B, w, stream)
        serial_t += t
        serial_status.append(st)
        serial_it.append(rep["iterations"])
        if st == 0 and r["status"] == 0:
            dE = max(dE, abs(e64 - r["energy"]))
    per_run = elapsed / steps
    conv = sum(1 for r in results if r["status"] == 0)
    conv64 = sum(1 for x in serial_status if x == 0)
    its = [r["iterations"] for r in results]
    return {"elapsed": elapsed, "dets_sigma": dets_sigma, "stats": stats, "per_run": per_run,
            "summary": {"instances": len(insts), "total_dets": int(sum(w.ndets for w in insts)),
                        "converged": conv, "solves_per_s": conv / per_run, "seconds_per_batch": per_run,
                        "status_counts": {str(k): sum(1 for r in results if r["status"] == k)
                                          for k in sorted({r["status"] for r in results})},
                        "iterations_min_median_max": [int(np.min(its)), float(np.median(its)), int(np.max(its))],
                        "max_subspace": subspace, "rows_per_item": stats["rows_per_item"], "schedule": schedule},
            "vs_serial_fp64": {"seconds": serial_t, "converged": conv64, "solves_per_s": conv64 / serial_t,
                               "iterations_min_median_max": [int(np.min(serial_it)), float(np.median(serial_it)),
                                                             int(np.max(serial_it))],
                               "speedup": serial_t / per_run, "max_abs_dE_Ha": dE,
                               "statuses": {str(k): serial_status.count(k) for k in sorted(set(serial_status))}}}


def run_batch(args):
    """64 independent instances in one engine (persistent launches, CUDA graphs), against the
    serial FP64 per-instance path on the same instances and stopping rule."""
    from paper_2601_16637_gb300 import binding as B
    from paper_2601_16637_gb300 import workloads as W

    B.load(build_if_missing=True)
    insts = W.batch_instances(args.batch_n)
    clocks = ClockSampler(0)
    clocks.start()
    m = batch_measure(B, insts, args.engine_subspace, args.warmup, args.steps, args.batch_schedule)
    clk = clocks.stop()
    extra = {"batch": m["summary"], "vs_serial_fp64": m["vs_serial_fp64"]}
    config = {"workload": f"batch{len(insts)}: {len(insts)} instances, norb in {{16,20,24,26}}, "
                          f"nalpha=nbeta=round(norb/3), |A|,|B| uniform in [500,5000], own integrals each; "
                          f"1 root, mixed sigma, residual <= {insts[0].tol:g} and Ritz-value change <= 1e-6 Ha",
              "step": "one engine run over all instances (admission, tables, Davidson, FP64 check)",
              "max_subspace": args.engine_subspace, "rows_per_item": m["stats"]["rows_per_item"],
              "l2": "inputs larger than L2 (vectors of all instances ~4 GB)"}
    print(json.dumps(engine_line(args, m["dets_sigma"] / m["elapsed"], m["elapsed"],
                                 m["summary"]["converged"] * args.steps, m["stats"], extra, clk, config)), flush=True)
    return 0


def serve_once(B, opts, jobs):
    """One engine serving the (arrival time, job) trace; returns results, base clock, stats."""
    with B.Engine(**opts) as e:
        base = e.clock()
        ids, i, n = [], 0, len(jobs)
        remaining = 0
        while i < n or remaining > 0:
            now = e.clock() - base
            while i < n and jobs[i][0] <= now:
                w = jobs[i][1]
                ids.append(e.submit(w, tol=w.tol, tol_energy=w.extra["tol_energy"]))
                i += 1
            st = e.stats()
            if st["active"] + st["pending"] > 0:
                remaining = e.step()
            else:
                remaining = 0
                if i < n:
                    time.sleep(max(0.0, min(0.01, jobs[i][0] - (e.clock() - base))))
        results = [e.result(j) for j in ids]
        return results, base, e.stats()


def serve_measure(B, built, traces, rates, subspace: int, budget_bytes: int, max_strings: int, warmup: int,
                  schedule: str = "fair") -> dict:
    """Serves the jobs `built` (arrival times traces[rate]) with one engine per rate (continuous
    batching under a memory budget), and a FIFO queue served one job at a time by the serial FP64
    path on the same arrivals (measured service time per job).  Latencies count from arrival."""
    import torch

    scheds = [x for x in str(schedule).split(",") if x]  # engine runs per schedule, one serial baseline
    opts = dict(max_slots=64, max_subspace=subspace, max_norb=max(w.norb for w in built), max_strings=max_strings,
                max_iter=400, hbm_budget_bytes=int(budget_bytes), schedule=scheds[0])
    small = sorted(built, key=lambda w: w.ndets)[:2]
    for _ in range(warmup):
        with B.Engine(**opts) as e:
            for w in small:
                e.submit(w, tol=w.tol, tol_energy=w.extra["tol_energy"])
            e.run()
    torch.cuda.synchronize()
    runs = []
    for sc in scheds:
        for r in rates:
            jobs = [(t, w) for (t, _, _), w in zip(traces[r], built)]
            results, base, stats = serve_once(B, {**opts, "schedule": sc}, jobs)
            arrivals = np.array([t for t, _ in jobs])
            done = np.array([x["t_done"] - base for x in results])
            runs.append((r, arrivals, done, results, stats, sc))
    stream = torch.cuda.current_stream()
    service, dE, st64 = [], 0.0, []
    for w, res in zip(built, runs[0][3]):
        ts, e64, st, _ = serial_fp64(B, w, stream)
        service.append(ts)
        st64.append(st)
        if st == 0 and res["status"] == 0:
            dE = max(dE, abs(e64 - res["energy"]))
    sweep = []
    n = len(built)
    for r, arrivals, done, results, stats, sc in runs:
        lat = done - arrivals
        span = float(done.max() - arrivals.min())
        conv = sum(1 for x in results if x["status"] == 0)
        fin, tcur = [], 0.0
        for a, sv in zip(arrivals, service):
            tcur = max(tcur, a) + sv
            fin.append(tcur)
        lat64 = np.array(fin) - arrivals
        span64 = float(fin[-1] - arrivals.min())
        conv64 = sum(1 for x in st64 if x == 0)
        sweep.append({"rate_per_s": r, "schedule": sc, "p50_s": float(np.percentile(lat, 50)),
                      "p99_s": float(np.percentile(lat, 99)),
                      "makespan_s": span, "converged": conv, "solves_per_s": conv / span,
                      "bytes_peak": stats["bytes_peak"], "requeued": stats.get("requeued", 0),
                      "status_counts": {str(k): sum(1 for x in results if x["status"] == k)
                                        for k in sorted({x["status"] for x in results})},
                      "serial_fp64": {"p50_s": float(np.percentile(lat64, 50)), "p99_s": float(np.percentile(lat64, 99)),
                                      "makespan_s": span64, "converged": conv64, "solves_per_s": conv64 / span64}})
    r0, arrivals, done, results, stats, _ = runs[0]
    span = float(done.max() - arrivals.min())
    dets_sigma = sum(x["ndets"] * (x["sigma_mixed"] + x["sigma_fp64"]) for x in results)
    return {"span": span, "dets_sigma": dets_sigma, "stats": stats, "n": n,
            "serving": {"requests": n, "rate_per_s": r0, "p50_s": sweep[0]["p50_s"], "p99_s": sweep[0]["p99_s"],
                        "makespan_s": span, "converged": sweep[0]["converged"],
                        "solves_per_s": sweep[0]["solves_per_s"], "status_counts": sweep[0]["status_counts"],
                        "bytes_peak": stats["bytes_peak"], "budget_bytes": opts["hbm_budget_bytes"],
                        "largest_job_dets": int(max(w.ndets for w in built)),
                        "largest_norb": int(max(w.norb for w in built)), "schedule": scheds[0], "sweep": sweep},
            "vs_serial_fp64": {**sweep[0]["serial_fp64"], "service_s_total": float(sum(service)),
                               "max_abs_dE_Ha": dE, "statuses": {str(k): st64.count(k) for k in sorted(set(st64))}}}


def serve_jobs(requests: int, rates, max_strings: int, big: int = 0, big_strings: int = 15000, big_norb: int = 58):
    """The serving trace (seeded Poisson arrivals, workloads.serving_trace) for each rate, its jobs
    built once; `big` extra jobs at the top of the configuration's range (norb big_norb,
    |A| = |B| = big_strings) replace the last ones of the trace, keeping their arrival times."""
    from paper_2601_16637_gb300 import workloads as W

    traces = {r: W.serving_trace(n=requests, rate=r, max_strings=max_strings) for r in rates}
    specs = [dict(spec) for _, spec, _ in traces[rates[0]]]
    for i in range(big):
        sp = specs[requests - 1 - i]
        nel = int(round(big_norb / 3))
        sp.update(name=f"serve-big-{i}", norb=big_norb, nalpha=nel, nbeta=nel, nA=big_strings, nB=big_strings)
    t0 = time.perf_counter()
    built = [W.make_job(sp, te) for sp, (_, _, te) in zip(specs, traces[rates[0]])]
    return traces, built, time.perf_counter() - t0


def run_serve(args):
    """A finite Poisson stream of jobs served by one engine (continuous batching under a memory
    budget), against a FIFO queue served one job at a time by the serial FP64 path, for each of the
    arrival rates given (the same jobs; only the arrival times scale with the rate)."""
    from paper_2601_16637_gb300 import binding as B

    B.load(build_if_missing=True)
    rates = [float(r) for r in str(args.rates).split(",")] if args.rates else [args.rate]
    traces, built, t_build = serve_jobs(args.requests, rates, args.max_strings, big=args.serve_big)
    clocks = ClockSampler(0)
    clocks.start()
    m = serve_measure(B, built, traces, rates, args.engine_subspace, int(args.budget_gb * 1e9),
                      max(args.max_strings, 15000 if args.serve_big else 0), args.warmup, args.serve_schedule)
    clk = clocks.stop()
    m["serving"]["job_build_s"] = t_build
    extra = {"serving": m["serving"], "vs_serial_fp64": m["vs_serial_fp64"]}
    n = m["n"]
    config = {"workload": f"serve: {n} Poisson arrivals at {rates[0]:g}/s, norb in {{24,32,40,48,58}}, "
                          f"nalpha=nbeta=round(norb/3), |A|=|B| log-uniform in [300,{args.max_strings}]"
                          + (f" with the last {args.serve_big} jobs at norb 58, |A|=|B|=15,000" if args.serve_big else "")
                          + f", own integrals each; 1 root, mixed sigma, residual <= {built[0].tol:g} and Ritz-value "
                          f"change <= 1e-6 Ha; admission budget {args.budget_gb:g} GB",
              "step": "the whole trace (arrival of the first job to completion of the last)",
              "l2": "inputs larger than L2"}
    args.steps = 1
    print(json.dumps(engine_line(args, m["dets_sigma"] / m["span"], m["span"], m["serving"]["converged"], m["stats"],
                                 extra, clk, config)), flush=True)
    return 0


def run_shard(args):
    """One instance alpha-row-sharded over the ranks (paper Sec. III): every rank holds the tables
    and its rows of every vector; sigma passes the C blocks around the ring of ranks
    (shard.DistRing: NCCL point-to-point into the library's receive buffers, double buffered), and
    the Davidson dot products are summed over the group.  Total work is fixed as the rank count
    grows ("scaling": "strong"); at one rank it is the sharded code path with a single block."""
    import torch

    from paper_2601_16637_gb300 import binding as B
    from paper_2601_16637_gb300 import shard as S
    from paper_2601_16637_gb300 import workloads as W

    rank, local_rank, world = env_rank()
    world = max(world, 1)
    torch.cuda.set_device(local_rank)
    import torch.distributed as dist

    if world == 1:  # a single rank started without torchrun
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if "MASTER_PORT" not in os.environ:
            import socket

            with socket.socket() as so:
                so.bind(("127.0.0.1", 0))
                os.environ["MASTER_PORT"] = str(so.getsockname()[1])
        os.environ.setdefault("RANK", "0")
        os.environ.setdefault("WORLD_SIZE", "1")
    dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank), init_method="env://")
    B.load(build_if_missing=True)
    wl = W.config(args.workload)
    prec = wl.precision
    stream = torch.cuda.current_stream()
    alloc = B._TorchAllocator()
    h_d = torch.from_numpy(wl.h).cuda()
    eri_d = torch.from_numpy(wl.eri).cuda()
    A_d = torch.from_numpy(wl.A.view(np.int64)).cuda()
    B_d = torch.from_numpy(wl.B.view(np.int64)).cuda()
    ring = S.DistRing()
    comm = ring.comm()

    def step():
        o = B.sbd_default_options()
        o.max_subspace = wl.max_subspace
        o.alloc, o.free = alloc.alloc, alloc.free
        handle = B.sbd_create(wl.norb, wl.nalpha, wl.nbeta, h_d, eri_d, A_d, B_d, o, stream)
        nA, nB = B.sbd_dims(handle)
        bounds = S.row_blocks(nA, world)
        rows = (bounds[rank + 1] - bounds[rank]) * nB
        vec = torch.empty((wl.nroots, rows), dtype=torch.float64, device="cuda")
        e = np.empty(wl.nroots)
        r = np.empty(wl.nroots)
        rc, rep = B.sbd_davidson_sharded(handle, bounds, comm, wl.nroots, wl.tol, prec, e, vec, r)
        B.sbd_destroy(handle)
        return e, r, rep.as_dict()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    launches0 = B.sbd_launch_count()
    clocks = ClockSampler(local_rank)
    clocks.start()
    t0 = time.perf_counter()
    reports, energies, resid = [], None, None
    for _ in range(args.steps):
        energies, resid, rep = step()
        reports.append(rep)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    elapsed = max_over_ranks(time.perf_counter() - t0, world)
    clk = clocks.stop()
    n_sigma = sum(r["sigma_fp64"] + r["sigma_mixed"] for r in reports)
    value = float(wl.ndets) * n_sigma / elapsed
    if rank == 0:
        cfg = workload_config(wl, prec)
        cfg["step"] = "sbd_create + sbd_davidson_sharded + sbd_destroy (one solve, alpha rows sharded over the ranks)"
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None,
                "dtype": "f32+f32x2+f64" if prec == "mixed" else "f64", "data": "synthetic", "config": cfg,
                "parallelism": f"alpha-row sharding over {world} rank(s), ring exchange of C blocks",
                "solves_per_s": args.steps / elapsed, "energy_Ha": float(energies[0]), "residual": float(resid[0]),
                "gpu_launches": int(B.sbd_launch_count() - launches0), "clocks": clk, "last_report": reports[-1]}
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg3")
    ap.add_argument("--mode", default="replicas", choices=["replicas", "shard"],
                    help="replicas: each GPU solves its own instance; shard: one instance over all ranks")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="oracle sample budget for cpu_baseline")
    ap.add_argument("--ref-step-seconds", type=float, default=8.0)
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3, help="solves timed end to end (at most --steps)")
    ap.add_argument("--no-oracle-extras", action="store_true", help="skip the oracle sigma/Davidson timings")
    ap.add_argument("--oracle-full", action="store_true", help="time one full oracle sigma of cfg2 (minutes)")
    ap.add_argument("--batch-n", type=int, default=64, help="instances of the batch64 workload")
    ap.add_argument("--requests", type=int, default=40, help="jobs of the serve workload")
    ap.add_argument("--rate", type=float, default=20.0, help="arrivals per second of the serve workload")
    ap.add_argument("--rates", default="", help="comma-separated arrival rates for a serve sweep (first one reported)")
    ap.add_argument("--max-strings", type=int, default=5000, help="largest |A| = |B| of the serve workload")
    ap.add_argument("--budget-gb", type=float, default=160.0, help="engine admission budget of the serve workload")
    ap.add_argument("--engine-subspace", type=int, default=20, help="Davidson basis per job in the engine")
    ap.add_argument("--engine-schedule", default="",
                    help="engine iterations: jobs share the device by cost (fair; default for serving, where "
                         "latency counts) or all jobs every iteration (lockstep; default for the batched "
                         "workload, submitted at once); the serve workload takes a comma-separated list")
    ap.add_argument("--serve-big", type=int, default=0,
                    help="serve workload: the last N jobs at norb 58, |A|=|B|=15,000 (the top of its range)")
    ap.add_argument("--legs", default="batch,serve",
                    help="default line: engine legs to add (comma-separated: batch, serve; empty for none)")
    ap.add_argument("--leg-batch-n", type=int, default=16, help="instances of the batched leg")
    ap.add_argument("--leg-requests", type=int, default=24, help="jobs of the served leg")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    scheds = [x for x in args.engine_schedule.split(",") if x]
    if any(x not in ("fair", "lockstep") for x in scheds) or (len(scheds) > 1 and args.workload != "serve"):
        ap.error("--engine-schedule: fair or lockstep (a comma-separated list only for --workload serve)")
    args.batch_schedule = args.engine_schedule or "lockstep"
    args.serve_schedule = args.engine_schedule or "fair"
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.mode == "shard":
        return run_shard(args)

    import torch

    from paper_2601_16637_gb300 import binding as B
    from paper_2601_16637_gb300 import workloads as W

    rank, local_rank, world = env_rank()
    if world != args.gpus:
        world = max(world, 1)
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    B.load(build_if_missing=True)
    wl = W.config(args.workload)
    prec = wl.precision
    peaks, peak_src = load_peaks()
    stream = torch.cuda.current_stream()

    # inputs resident in HBM
    h_d = torch.from_numpy(wl.h).cuda()
    eri_d = torch.from_numpy(wl.eri).cuda()
    A_d = torch.from_numpy(wl.A.view(np.int64)).cuda()
    B_d = torch.from_numpy(wl.B.view(np.int64)).cuda()
    vec_d = torch.empty((wl.nroots, wl.ndets), dtype=torch.float64, device="cuda")
    alloc = B._TorchAllocator()

    def options(timing=True, refine=None):
        o = B.sbd_default_options()
        o.max_subspace = wl.max_subspace
        o.timing = int(timing)
        o.alloc, o.free = alloc.alloc, alloc.free
        if refine is not None:
            o.refine_precision = B.PRECISION[refine]
        return o

    def step(h, eri, A, Bs, vec, precision=prec, refine=None):
        handle = B.sbd_create(wl.norb, wl.nalpha, wl.nbeta, h, eri, A, Bs, options(refine=refine), stream)
        e = np.empty(wl.nroots)
        r = np.empty(wl.nroots)
        rc, rep = B.sbd_davidson(handle, wl.nroots, wl.tol, precision, e, vec, r)
        ms, n = B.sbd_kernel_times(handle)
        B.sbd_destroy(handle)
        return e, r, rep.as_dict(), ms, n

    for _ in range(args.warmup):
        step(h_d, eri_d, A_d, B_d, vec_d)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = B.sbd_launch_count()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reports, kms, kn, energies, resid = [], None, None, None, None
    for _ in range(args.steps):
        energies, resid, rep, ms, n = step(h_d, eri_d, A_d, B_d, vec_d)
        reports.append(rep)
        if kms is None:
            kms, kn = ms, n
        else:
            for p in ms:
                for k in ms[p]:
                    kms[p][k] += ms[p][k]
                    kn[p][k] += n[p][k]
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = B.sbd_launch_count() - launches0
    elapsed = ev0.elapsed_time(ev1) / 1e3
    elapsed_max = max_over_ranks(elapsed, world)
    n_sigma = sum(r["sigma_fp64"] + r["sigma_mixed"] for r in reports)
    dets_all = sum_over_ranks(float(wl.ndets) * n_sigma, world)
    value = dets_all / elapsed_max
    solves_per_s = sum_over_ranks(float(args.steps), world) / elapsed_max

    # per-kernel device times of the sigma kernels (events on the launch stream)
    p_main = "mixed" if prec == "mixed" else "fp64"
    kern = {p: {k: {"ms_total": kms[p][k], "launches": kn[p][k],
                    "ms_per_launch": (kms[p][k] / kn[p][k]) if kn[p][k] else None} for k in kms[p]} for p in kms}
    dominant = max(kms[p_main], key=lambda k: kms[p_main][k])
    # algorithmic work per launch (multiply-adds of the sparse contraction, 2 FLOP each)
    handle = B.sbd_create(wl.norb, wl.nalpha, wl.nbeta, h_d, eri_d, A_d, B_d, options(False), stream)
    nsA, ndA = B.sbd_table_size(handle, 0, 1), B.sbd_table_size(handle, 0, 2)
    nsB, ndB = B.sbd_table_size(handle, 1, 1), B.sbd_table_size(handle, 1, 2)
    nA, nB = B.sbd_dims(handle)
    elem = 4 if p_main == "mixed" else 8
    flops = {"ab_pass": 2.0 * nsA * nsB,
             "beta_pass": 2.0 * nA * (2 * nsB + ndB) + 2.0 * nA * nB,
             "alpha_pass": 2.0 * nB * (2 * nsA + ndA)}
    bytes_per_launch = {"transpose": 2.0 * nA * nB * elem}
    ms_dom = kern[p_main][dominant]["ms_per_launch"]
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    if dominant == "transpose":
        achieved = bytes_per_launch["transpose"] / (ms_dom * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s"}
    else:
        if p_main == "mixed":
            peak_tf = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        else:
            peak_tf = FP64_NOMINAL_TFLOPS
        achieved = flops[dominant] / (ms_dom * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if roof["bound"] == "alu":
        if dominant == "ab_pass" and p_main == "mixed":
            # column-stationary pass: the amplitudes sit in registers and each multiply-add gathers
            # one 4-byte integral, so one 128-byte shared-memory wavefront per SM clock feeds 32 FMA
            # (the 64-bit shared-memory adds of the dot products come on top of that)
            ceil_tf = NUM_SMS * 32 * 2 * sm_max * 1e6 / 1e12
            basis = ("one 128-byte shared-memory wavefront per SM clock = 32 FMA with one gathered 4-byte "
                     "operand (amplitudes in registers)")
        else:
            # both FMA operands gathered from shared memory: 128 / (2 * elem) multiply-adds per wavefront
            ceil_tf = NUM_SMS * (128 // (2 * elem)) * 2 * sm_max * 1e6 / 1e12
            basis = (f"one 128-byte shared-memory wavefront per SM clock = {128 // (2 * elem)} FMA with two "
                     f"{elem}-byte operands")
        roof["smem_ceiling"] = {"peak": ceil_tf, "unit": "TFLOP/s", "frac": roof["achieved"] / ceil_tf,
                                "basis": basis}
        if dominant == "ab_pass" and p_main == "mixed":
            two_op = NUM_SMS * 16 * 2 * sm_max * 1e6 / 1e12
            roof["smem_ceiling"]["two_operand_design"] = {
                "peak": two_op, "frac": roof["achieved"] / two_op,
                "basis": "the same wavefront rate when both operands are gathered (16 FMA per wavefront)"}
    roof["kernel"] = f"{dominant} ({p_main})"
    roof["peak_source"] = (f"{peak_src} HBM copy" if roof["bound"] == "hbm" else
                           ("FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x max SM clock" if p_main == "mixed"
                            else "nominal FP64 1.25 TFLOP/s"))
    tr = traffic_record(f"{dominant}_{p_main}")
    roof["traffic"] = tr
    # HBM view of the same launch: compulsory bytes (read C, read and write sigma) and, when the
    # ncu record matches the kernel source, the measured DRAM bytes, against the measured copy peak
    comp = wl.ndets * (elem + 16.0)
    roof["hbm"] = {"compulsory_GBs": comp / (ms_dom * 1e-3) / 1e9,
                   "measured_GBs": (tr / (ms_dom * 1e-3) / 1e9) if tr else None,
                   "peak_GBs": float(peaks["hbm_gbs"]),
                   "frac_compulsory": comp / (ms_dom * 1e-3) / 1e9 / float(peaks["hbm_gbs"])}

    # sigma-only throughput by precision (sum of the four sigma kernels per vector)
    sigma_rate = {}
    for p in ("fp64", "mixed", "f32x2"):
        tot = sum(kms[p].values())
        nv = kn[p]["ab_pass"]
        if nv:
            sigma_rate[p] = wl.ndets * nv / (tot * 1e-3)

    # FP64 comparison solve (outside the timed region)
    mixed_vs_fp64 = None
    if not args.no_fp64_compare and prec == "mixed":
        e64, r64, rep64, ms64, n64 = step(h_d, eri_d, A_d, B_d, vec_d, precision="fp64")
        sigma_rate.setdefault("fp64", wl.ndets * n64["fp64"]["ab_pass"] / (sum(ms64["fp64"].values()) * 1e-3))
        mixed_vs_fp64 = {"E_mixed": float(energies[0]), "E_fp64": float(e64[0]),
                         "abs_diff_Ha": float(abs(energies[0] - e64[0])),
                         "solve_s_mixed": reports[-1]["seconds_total"], "solve_s_fp64": rep64["seconds_total"],
                         "speedup": rep64["seconds_total"] / reports[-1]["seconds_total"]}
        # the literal reading of the precision statement: the defect corrections (and the Ritz
        # combinations of the refined solve) in IEEE FP64 instead of FP32 pairs
        el, rl, repl, _, _ = step(h_d, eri_d, A_d, B_d, vec_d, refine="fp64")
        mixed_vs_fp64["refine_fp64"] = {"E": float(el[0]), "abs_diff_Ha": float(abs(el[0] - e64[0])),
                                        "residual": float(rl[0]), "solve_s": repl["seconds_total"],
                                        "sigma_mixed": repl["sigma_mixed"], "sigma_fp64": repl["sigma_fp64"],
                                        "iterations": repl["iterations"]}
        mixed_vs_fp64["refine_f32x2"] = {"solve_s": reports[-1]["seconds_total"],
                                         "sigma_mixed": reports[-1]["sigma_mixed"],
                                         "sigma_fp64": reports[-1]["sigma_fp64"],
                                         "iterations": reports[-1]["iterations"]}
    B.sbd_destroy(handle)

    # end to end: pinned host inputs, eigenvector back to pinned host memory
    e2e = None
    if not args.no_e2e:
        h_h = torch.from_numpy(wl.h).pin_memory()
        eri_h = torch.from_numpy(wl.eri).pin_memory()
        A_h = torch.from_numpy(wl.A.view(np.int64)).pin_memory()
        B_h = torch.from_numpy(wl.B.view(np.int64)).pin_memory()
        vec_h = torch.empty((wl.nroots, wl.ndets), dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        n_sig_e2e = 0
        for _ in range(min(args.steps, args.e2e_steps)):
            _, _, rep, _, _ = step(h_h, eri_h, A_h, B_h, vec_h)
            n_sig_e2e += rep["sigma_fp64"] + rep["sigma_mixed"]
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, world)
        h2d = wl.h.nbytes + wl.eri.nbytes + wl.A.nbytes + wl.B.nbytes
        d2h = vec_h.numel() * 8 + wl.nroots * 8 * 2
        e2e = {"value": sum_over_ranks(float(wl.ndets) * n_sig_e2e, world) / te, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": min(args.steps, args.e2e_steps)}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        rate, nrows, dt, threads = oracle_rows_rate(wl, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{nrows} sigma rows sampled uniformly from the {wl.ndets:.1e} determinants "
                         f"({dt:.1f} s); each row is one determinant's sigma element"}
        if not args.no_oracle_extras:
            cpu["extras"] = oracle_extras(rate, wl.ndets, cfg2_sigma_count=CFG2_FP64_SIGMA_COUNT,
                                          full_cfg2=args.oracle_full)

    # the batched and served forms (the engine) against the serial FP64 per-instance path, one GPU
    legs = {}
    if rank == 0 and world == 1 and args.legs:
        want = {x.strip() for x in args.legs.split(",") if x.strip()}
        if "batch" in want:
            insts = W.batch_instances(64)[: args.leg_batch_n]
            m = batch_measure(B, insts, args.engine_subspace, warmup=1, steps=1, schedule=args.batch_schedule)
            legs["batch"] = {"workload": f"the first {len(insts)} of the 64 batched instances (norb in "
                                         f"{{16,20,24,26}}, |A|,|B| in [500,5000])",
                             "engine_mixed": m["summary"], "serial_fp64": m["vs_serial_fp64"],
                             "gpu_launches": int(m["stats"]["kernel_launches"])}
        if "serve" in want:
            traces, built, _ = serve_jobs(args.leg_requests, [args.rate], 5000)
            m = serve_measure(B, built, traces, [args.rate], args.engine_subspace, int(args.budget_gb * 1e9), 5000,
                              warmup=1, schedule=args.serve_schedule)
            legs["serve"] = {"workload": f"{args.leg_requests} Poisson arrivals at {args.rate:g}/s, norb in "
                                         f"{{24,32,40,48,58}}, |A|=|B| log-uniform in [300,5000], "
                                         f"{args.budget_gb:g} GB budget",
                             "engine_mixed": m["serving"], "serial_fp64": m["vs_serial_fp64"],
                             "gpu_launches": int(m["stats"]["kernel_launches"])}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                # mixed: FP32 sigma, FP32-pair (FP64-accurate) sigma for the defect corrections, FP64 Davidson
                "dtype": "f32+f32x2+f64" if prec == "mixed" else "f64",
                "data": "synthetic", "config": workload_config(wl, prec),
                "parallelism": "replicas" if world > 1 else "single GPU",
                "solves_per_s": solves_per_s, "sigma_applications_per_step": n_sigma / args.steps,
                "sigma_only_dets_per_s": sigma_rate, "energy_Ha": float(energies[0]),
                "residual": float(resid[0]),
                # Kato-Temple-form estimate of the energy error: residual^2 / (next Ritz value - energy)
                "energy_error_estimate_Ha": energy_error_estimates(energies, resid, reports[-1])[0],
                "kernels": kern, "mixed_vs_fp64": mixed_vs_fp64, "engine_legs": legs or None,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk, "last_report": reports[-1]}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
