"""Batched sigma and the batched / served engine, through the C ABI.

* sbd_sigma_batched computes every instance's sigma with the same arithmetic
  as sbd_sigma (bitwise equal when the rows staged per work item agree) and
  within FP64 rounding of the oracle.
* Engine solves agree with the single-instance FP64 solver and with dense
  diagonalisation; a job's result is bitwise the same alone and in a mix of
  jobs, with admission limited by the memory budget and jobs joining while
  others run; a failing job leaves the others untouched.
"""
import numpy as np
import pytest

from gpu_common import SIGMA_FP64_RTOL, medium, rel_maxnorm
from paper_2601_16637_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_16637_gb300 import build

    build.build()
    return t


@pytest.fixture(scope="module")
def B(torch):
    from paper_2601_16637_gb300 import binding

    binding.load()
    return binding


def _instances():
    # ragged sizes, unequal electron counts, a full space with A == B (shared tables), norb 8..26
    return [medium(), W.make("b1", 12, 3, 4, 150, 97, 0.2, 11), W.config("cfg1"),
            W.make("b3", 20, 7, 7, 900, 900, 0.35, 13), W.make("b4", 26, 9, 9, 700, 400, 0.35, 14)]


@pytest.fixture(scope="module")
def handles(B):
    insts = _instances()
    gs = [B.SBD.from_workload(w) for w in insts]
    yield insts, gs
    for g in gs:
        g.close()


def _vectors(torch, gs, dtype, seed):
    return [torch.from_numpy(W.random_vector(g.N, seed + i)[0]).to("cuda", dtype) for i, g in enumerate(gs)]


@pytest.mark.parametrize("prec", ["mixed", "fp64", "f32x2"])
def test_sigma_batched_is_bitwise_the_single_instance_sigma(torch, B, handles, prec):
    insts, gs = handles
    dt = torch.float32 if prec == "mixed" else torch.float64
    xs = _vectors(torch, gs, dt, 40)
    ref = [g.sigma(x, prec) for g, x in zip(gs, xs)]
    outs = [torch.full((g.N,), float("nan"), dtype=torch.float64, device="cuda") for g in gs]
    B.sbd_sigma_batched([g.handle for g in gs], xs, outs, prec)
    torch.cuda.synchronize()
    for r, o in zip(ref, outs):
        assert torch.equal(r, o)
    # one row per work item: the alpha-beta pass groups its FP32 sums differently, nothing else changes
    outs1 = [torch.empty(g.N, dtype=torch.float64, device="cuda") for g in gs]
    B.sbd_sigma_batched([g.handle for g in gs], xs, outs1, prec, rows_per_item=1)
    for r, o in zip(ref, outs1):
        assert rel_maxnorm(o.cpu().numpy(), r.cpu().numpy()) < {"mixed": 2e-6, "fp64": 1e-14, "f32x2": 1e-13}[prec]


def test_sigma_batched_fp64_matches_the_oracle(torch, B, handles, oracle_mod):
    insts, gs = handles
    pick = [0, 1, 2]
    xs = _vectors(torch, [gs[i] for i in pick], torch.float64, 70)
    outs = [torch.empty(gs[i].N, dtype=torch.float64, device="cuda") for i in pick]
    B.sbd_sigma_batched([gs[i].handle for i in pick], xs, outs, "fp64")
    for i, x, o in zip(pick, xs, outs):
        orc = oracle_mod.Oracle.from_workload(insts[i])
        ref = orc.sigma(x.cpu().numpy()[None, :])[0]
        orc.close()
        assert rel_maxnorm(o.cpu().numpy(), ref) <= SIGMA_FP64_RTOL


def _small_jobs():
    return [W.config("cfg1"), W.make("e1", 12, 4, 4, 220, 180, 0.25, 21), W.make("e2", 14, 5, 4, 300, 250, 0.3, 22),
            W.make("e3", 16, 5, 5, 400, 350, 0.35, 23)]


def _engine(B, **kw):
    opts = dict(max_slots=8, max_subspace=12, max_norb=32, max_strings=2000, rows_per_item=4)
    opts.update(kw)
    return B.Engine(**opts)


def _run_alone(B, wl, tol, tol_energy):
    with _engine(B) as e:
        j = e.submit(wl, tol=tol, tol_energy=tol_energy, keep_vector=True)
        e.run()
        r = e.result(j)
        return r, e.vector(j, r["ndets"])


TOL, TOL_E = 1e-5, 1e-10


@pytest.fixture(scope="module")
def alone(B):
    return [_run_alone(B, wl, TOL, TOL_E) for wl in _small_jobs()]


def test_engine_matches_fp64_solver_and_dense(torch, B, alone, oracle_mod):
    jobs = _small_jobs()
    for wl, (r, v) in zip(jobs, alone):
        assert r["status"] == 0, r
        assert r["residual"] <= TOL
        with B.SBD.from_workload(wl) as g:
            s = g.davidson(1, 1e-9, "fp64")
            assert s.status == 0
            # residual 1e-5 and a converged Ritz value: the energy error is ~ r^2 / gap
            assert abs(r["energy"] - s.energies[0]) < 1e-7
            u = s.vectors[0].cpu().numpy()
            assert abs(float(np.dot(u, v))) > 1 - 1e-6
            assert abs(v[np.argmax(np.abs(v))]) == v[np.argmax(np.abs(v))]  # sign convention
    # the full space against dense diagonalisation of the oracle's matrix
    orc = oracle_mod.Oracle.from_workload(jobs[0])
    e0 = np.linalg.eigvalsh(orc.dense())[0]
    orc.close()
    assert abs(alone[0][0]["energy"] - e0) < 1e-7


def test_engine_results_are_bitwise_the_same_alone_and_in_a_mix(B, alone):
    jobs = _small_jobs()
    with _engine(B) as e:
        ids = [e.submit(wl, tol=TOL, tol_energy=TOL_E, keep_vector=True) for wl in jobs]
        e.run()
        st = e.stats()
        assert st["done"] == len(jobs) and st["active"] == 0 and st["pending"] == 0
        assert st["graph_launches"] > 0 and st["kernel_launches"] > st["graph_launches"]
        for j, (ra, va) in zip(ids, alone):
            r = e.result(j)
            for key in ("status", "iterations", "sigma_mixed", "sigma_fp64", "restarts", "energy", "residual",
                        "energy_mixed"):
                assert r[key] == ra[key], key
            assert np.array_equal(e.vector(j, r["ndets"]), va)


def test_engine_schedules_give_the_same_results(B, alone):
    # fair (by cost) and lockstep schedules differ only in which jobs take part in an iteration:
    # every job's results are bitwise those of its solve alone; the fair schedule runs more, smaller
    # iterations, and its smallest job is done no later than its largest
    jobs = _small_jobs()
    out = {}
    for sched in ("fair", "lockstep"):
        with _engine(B, schedule=sched) as e:
            ids = [e.submit(wl, tol=TOL, tol_energy=TOL_E, keep_vector=True) for wl in jobs]
            e.run()
            res = [e.result(j) for j in ids]
            for j, r, (ra, va) in zip(ids, res, alone):
                for key in ("status", "iterations", "sigma_mixed", "sigma_fp64", "restarts", "energy", "residual"):
                    assert r[key] == ra[key], (sched, key)
                assert np.array_equal(e.vector(j, r["ndets"]), va)
            out[sched] = (e.stats()["steps"], res)
    assert out["fair"][0] > out["lockstep"][0]
    done = [r["t_done"] for r in out["fair"][1]]
    assert done[0] <= done[-1]
    with pytest.raises(ValueError):
        _engine(B, schedule="round-robin")


def _estimate(wl, max_sub=12):
    # the engine's admission estimate: basis and vectors, diagonal + work vector, table reserve
    return wl.ndets * (8 * (2 * max_sub + 3) + 4 + 16) + 16384 * (wl.A.size + wl.B.size)


def test_engine_budget_admission_and_jobs_joining_a_running_batch(B, alone):
    jobs = _small_jobs()
    # room for the largest job, but not for the two largest together
    budget = int(1.3 * _estimate(jobs[3]))
    assert _estimate(jobs[2]) + _estimate(jobs[3]) > budget
    with _engine(B, hbm_budget_bytes=budget) as e:
        ids = [e.submit(wl, tol=TOL, tol_energy=TOL_E, keep_vector=True) for wl in jobs[:2]]
        for _ in range(3):
            e.step()
        assert e.stats()["active"] >= 1
        # two more jobs join the running ones
        ids += [e.submit(wl, tol=TOL, tol_energy=TOL_E, keep_vector=True) for wl in jobs[2:]]
        while e.step() > 0:
            pass
        st = e.stats()
        assert st["bytes_peak"] <= budget and st["done"] == len(jobs)
        res = [e.result(j) for j in ids]
        for r, (ra, va), j in zip(res, alone, ids):
            assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
            assert r["energy"] == ra["energy"] and r["iterations"] == ra["iterations"]
            assert np.array_equal(e.vector(j, r["ndets"]), va)
        # the two largest jobs never held memory at the same time
        a, b = res[2], res[3]
        assert a["t_done"] <= b["t_admit"] or b["t_done"] <= a["t_admit"]


def _basis(wl, max_sub=12):
    # the engine's per-job vectors: V, W [max_sub][N], U, HU, TC in FP64, an FP32 copy, descriptors
    return wl.ndets * (8 * (2 * max_sub + 3) + 4) + 256 * 6 + 8 * 3 * 32 * 32


def test_engine_holds_the_budget_when_the_table_estimate_is_too_low(B, alone):
    # An admission estimate of one byte per string lets the second job be tried while the first one
    # runs; its handle is then created under the budget that is really left, fails, and the job waits
    # at the head of the queue until the first job has freed its memory.
    jobs = _small_jobs()
    real = {}
    for i in (2, 3):
        with B.SBD.from_workload(jobs[i]) as g:
            real[i] = _basis(jobs[i]) + g.memory()
    low2 = _basis(jobs[2]) + 16 * jobs[2].ndets + (jobs[2].A.size + jobs[2].B.size)
    assert low2 < real[2]
    budget = int(real[3] + low2 + 0.5 * (real[2] - low2))
    assert budget < real[2] + real[3]
    with _engine(B, hbm_budget_bytes=budget, table_bytes_per_string=1) as e:
        j3 = e.submit(jobs[3], tol=TOL, tol_energy=TOL_E, keep_vector=True)
        j2 = e.submit(jobs[2], tol=TOL, tol_energy=TOL_E, keep_vector=True)
        e.run()
        st = e.stats()
        assert st["requeued"] >= 1 and st["done"] == 2
        assert st["bytes_peak"] <= budget
        r2, r3 = e.result(j2), e.result(j3)
        assert r2["status"] == 0 and r3["status"] == 0
        assert r3["t_done"] <= r2["t_admit"]
        assert r2["energy"] == alone[2][0]["energy"] and r3["energy"] == alone[3][0]["energy"]
        assert np.array_equal(e.vector(j2, r2["ndets"]), alone[2][1])


def test_engine_reports_a_failing_job_and_finishes_the_others(B, alone):
    jobs = _small_jobs()
    bad = W.make("dup", 12, 4, 4, 220, 180, 0.25, 21)
    bad.A[5] = bad.A[7]
    with _engine(B) as e:
        j0 = e.submit(jobs[1], tol=TOL, tol_energy=TOL_E)
        jb = e.submit(bad, tol=TOL)
        j1 = e.submit(jobs[2], tol=TOL, tol_energy=TOL_E)
        e.run()
        assert e.result(jb)["status"] == -3
        assert e.result(j0)["energy"] == alone[1][0]["energy"]
        assert e.result(j1)["energy"] == alone[2][0]["energy"]
        with pytest.raises(B.SbdError):
            e.vector(jb, 1)
        e.release(jb)
        with pytest.raises(B.SbdError):
            e.result(jb)


def test_engine_norb58_job_alone_and_in_a_mix(B, oracle_mod):
    # the top of the serving configuration's orbital range (norb 58, 19+19 electrons) with small
    # string sets: same result alone and beside other jobs, equal to the single-instance FP64 solve,
    # and an eigenvector whose residual is small on rows of the oracle's sigma
    big = W.make("n58", 58, 19, 19, 300, 260, 0.35, seed=58)
    others = _small_jobs()[1:3]
    opts = dict(max_slots=4, max_subspace=12, max_norb=64, max_strings=2000)
    with B.Engine(**opts) as e:
        j = e.submit(big, tol=TOL, tol_energy=TOL_E, keep_vector=True)
        e.run()
        ra = e.result(j)
        va = e.vector(j, ra["ndets"])
    assert ra["status"] == 0, ra
    with B.Engine(**opts) as e:
        ids = [e.submit(w, tol=TOL, tol_energy=TOL_E) for w in others]
        j = e.submit(big, tol=TOL, tol_energy=TOL_E, keep_vector=True)
        e.run()
        rm = e.result(j)
        assert all(e.result(i)["status"] == 0 for i in ids)
        assert rm["energy"] == ra["energy"] and rm["iterations"] == ra["iterations"]
        assert np.array_equal(e.vector(j, rm["ndets"]), va)
    with B.SBD.from_workload(big) as g:
        s = g.davidson(1, 1e-9, "fp64")
        assert s.status == 0
        assert abs(ra["energy"] - s.energies[0]) < 1e-7
        assert abs(float(np.dot(s.vectors[0].cpu().numpy(), va))) > 1 - 1e-6
    o = oracle_mod.Oracle.from_workload(big)
    rows = np.random.default_rng(58).choice(big.ndets, 40, replace=False)
    hv = o.sigma_rows(va[None, :], rows)[0]
    r = hv - ra["energy"] * va[rows]
    o.close()
    # |r_i| <= ||r|| <= TOL for every row of the exact residual vector
    assert np.abs(r).max() <= 2 * TOL
