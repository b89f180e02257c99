"""Host-side helpers of bench.py (no GPU): the nvidia-smi clock-sample parser that decides whether a
run saw throttling, and the lookup of committed DRAM-traffic records by kernel source digest."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_samples_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "garbage line\n",
        "0, N/A, 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
    ]
    out = bench.parse_clock_samples(lines)
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    hot = bench.parse_clock_samples(["0, 1500, 2070, 1400, 0x48, Active, Active, Not Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    empty = bench.parse_clock_samples([])
    assert empty["sm_mhz"] is None and empty["samples"] == 0


def test_traffic_record_matches_only_the_current_kernel_source():
    digest = bench.kernel_source_digest()
    assert len(digest) == 16 and all(c in "0123456789abcdef" for c in digest)
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    recorded = {}
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#"):
            recorded[(parts[0], parts[1])] = float(parts[2])
    got = bench.traffic_record("ab_pass_mixed")
    if ("ab_pass_mixed", digest) in recorded:
        assert got == recorded[("ab_pass_mixed", digest)]
    else:
        assert got is None  # a record taken on other kernel source is not reported
    assert bench.traffic_record("no_such_kernel") is None


def test_nvidia_smi_is_given_the_device_this_process_uses():
    import uuid

    class Props:
        pass

    p = Props()
    # CUDA_VISIBLE_DEVICES remaps: CUDA device 1 of this process is physical GPU 5
    assert bench.nvsmi_gpu_id(1, props=p, visible="3,5") == "5"
    assert bench.nvsmi_gpu_id(0, props=p, visible="GPU-aaaa,GPU-bbbb") == "GPU-aaaa"
    assert bench.nvsmi_gpu_id(0, props=p, visible="") == "0"
    # with a UUID the device is named by it, whatever CUDA_VISIBLE_DEVICES says
    u = uuid.UUID("12345678-1234-5678-1234-567812345678")
    p.uuid = u
    assert bench.nvsmi_gpu_id(1, props=p, visible="3,5") == "GPU-" + str(u)


def test_energy_error_estimate_uses_the_distance_to_the_next_ritz_value():
    # three roots; the first Ritz value above them lies gap = 0.5 above the third
    e = [-2.0, -1.5, -1.25]
    r = [1e-4, 2e-4, 3e-4]
    est = bench.energy_error_estimates(e, r, {"gap_estimate": 0.5})
    assert abs(est[0] - 1e-8 / (0.5 + 0.75)) < 1e-20
    assert abs(est[1] - 4e-8 / (0.5 + 0.25)) < 1e-20
    assert abs(est[2] - 9e-8 / 0.5) < 1e-20
    assert bench.energy_error_estimates(e, r, {"gap_estimate": 0.0}) == [None, None, None]


def test_engine_schedule_option_is_checked_before_any_gpu_work():
    import subprocess

    def run(*extra):
        return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *extra], cwd=ROOT,
                              capture_output=True, text=True, timeout=120)

    r = run("--engine-schedule", "round-robin")
    assert r.returncode == 2 and "--engine-schedule" in r.stderr
    # a list of schedules is only for the serve workload (one engine run each)
    r = run("--engine-schedule", "fair,lockstep")
    assert r.returncode == 2 and "--engine-schedule" in r.stderr


def test_serve_trace_with_jobs_from_the_top_of_the_range():
    # --serve-big n replaces the last n jobs of the seeded trace by jobs of the top of the range, at
    # the same arrival times; the others are the trace's own jobs
    traces, built, _ = bench.serve_jobs(6, [20.0], 400, big=2, big_strings=300, big_norb=20)
    plain, built0, _ = bench.serve_jobs(6, [20.0], 400)
    assert [t for t, _, _ in traces[20.0]] == [t for t, _, _ in plain[20.0]]
    for w, w0 in zip(built[:4], built0[:4]):
        assert (w.norb, w.A.size, w.B.size) == (w0.norb, w0.A.size, w0.B.size)
    for w in built[4:]:
        assert w.norb == 20 and w.nalpha == w.nbeta == 7 and w.A.size == w.B.size == 300
