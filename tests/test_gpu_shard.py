"""Row-block sigma for alpha-row sharding, through the C ABI on one GPU.

For a partition of the alpha rows into P blocks, the contributions of all source blocks to each
rank's rows (sbd_sigma_block through one block plan per source block) must add up to that rank's
rows of the full sigma: within FP64 rounding for SBD_FP64 and SBD_F32X2 (and against the oracle),
within FP32 grouping for SBD_MIXED.  The ranks are emulated one after another in one process;
nothing waits on anything else.
"""
import numpy as np
import pytest

from gpu_common import SIGMA_FP64_RTOL, medium, rel_maxnorm
from paper_2601_16637_gb300 import shard
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


def _rank_rows(torch, B, g, x, prec, parts, r):
    bounds = shard.row_blocks(g.nA, parts)
    r0, r1 = bounds[r], bounds[r + 1]
    out = torch.zeros((r1 - r0) * g.nB, dtype=torch.float64, device="cuda")
    fn, close = shard.device_block_sigma(g.handle, bounds, r, prec)
    try:
        for b in range(parts):
            fn(b, x[bounds[b] * g.nB: bounds[b + 1] * g.nB], out)
    finally:
        close()
    return out, r0, r1


@pytest.mark.parametrize("prec", ["fp64", "f32x2", "mixed"])
@pytest.mark.parametrize("wl", [medium(), medium(norb=11, n=4, nb=3, nA=197, nB=133, seed=12)], ids=["med", "uneq"])
def test_block_sigma_adds_up_to_the_full_sigma(torch, B, prec, wl):
    tol = {"fp64": 1e-13, "f32x2": 1e-13, "mixed": 2e-6}[prec]
    dt = torch.float32 if prec == "mixed" else torch.float64
    with B.SBD.from_workload(wl) as g:
        x = torch.from_numpy(W.random_vector(g.N, 41)[0]).to("cuda", dt)
        full = g.sigma(x, prec).cpu().numpy()
        for parts in (1, 2, 3):
            for r in range(parts):
                out, r0, r1 = _rank_rows(torch, B, g, x, prec, parts, r)
                ref = full[r0 * g.nB: r1 * g.nB]
                assert rel_maxnorm(out.cpu().numpy(), ref) <= tol, (parts, r)


def test_block_sigma_against_the_oracle_and_a_shared_table_instance(torch, B, oracle_mod):
    # cfg1: A == B, so the two spins share their tables
    for wl in (W.config("cfg1"), medium()):
        with B.SBD.from_workload(wl) as g:
            o = oracle_mod.Oracle.from_workload(wl)
            xn = W.random_vector(g.N, 42)[0]
            ref = o.sigma(xn[None, :])[0]
            x = torch.from_numpy(xn).cuda()
            parts = 4
            got = np.concatenate([_rank_rows(torch, B, g, x, "fp64", parts, r)[0].cpu().numpy() for r in range(parts)])
            assert rel_maxnorm(got, ref) <= SIGMA_FP64_RTOL
            o.close()


def test_ring_driver_on_one_rank_and_plan_errors(torch, B):
    wl = medium()
    with B.SBD.from_workload(wl) as g:
        x = torch.from_numpy(W.random_vector(g.N, 43)[0]).cuda()
        bounds = shard.row_blocks(g.nA, 1)
        fn, close = shard.device_block_sigma(g.handle, bounds, 0, "fp64")
        ring = shard.RingSigma(fn, bounds, 0, 1, g.nB)
        out = torch.empty(g.N, dtype=torch.float64, device="cuda")
        ring(x, out)
        close()
        ref = g.sigma(x, "fp64").cpu().numpy()
        assert rel_maxnorm(out.cpu().numpy(), ref) <= 1e-15
        # products on a side stream: ordered after the ring's zeroing on the current stream, and the
        # current stream waits for them (the output is read there right after)
        side = torch.cuda.Stream()
        fn, close = shard.device_block_sigma(g.handle, bounds, 0, "fp64", stream=side)
        out.fill_(float("nan"))
        shard.RingSigma(fn, bounds, 0, 1, g.nB)(x, out)
        close()
        assert rel_maxnorm(out.cpu().numpy(), ref) <= 1e-15
        for r0, r1, j0, j1 in [(5, 5, 0, 3), (0, g.nA + 1, 0, 3), (0, 3, -1, 2), (0, 3, 2, 1)]:
            with pytest.raises(B.SbdError):
                B.sbd_block_plan_create(g.handle, r0, r1, j0, j1)


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sharded_davidson_matches_the_single_solve(torch, B, world, prec):
    # ranks emulated as threads on one GPU; every host decision uses the summed (global) values,
    # so all ranks must report identical energies, and the solve must match the single-handle one
    import threading

    wl = medium()
    tol = 1e-8 if prec == "fp64" else 1e-7
    with B.SBD.from_workload(wl) as g:
        ref = g.davidson(nroots=2, tol=tol, precision=prec)
        assert ref.status == 0
        vref = ref.vectors.cpu().numpy()
        nA, nB = g.nA, g.nB
    bounds = shard.row_blocks(nA, world)
    ring = shard.ThreadRing(world, timeout=300)
    out = [None] * world

    def rank(r):
        try:
            with B.SBD.from_workload(wl) as h:
                rows = (bounds[r + 1] - bounds[r]) * nB
                e = np.empty(2)
                res = np.empty(2)
                v = torch.empty((2, rows), dtype=torch.float64, device="cuda")
                rc, rep = B.sbd_davidson_sharded(h.handle, bounds, ring.comm(r), 2, tol, prec, e, v, res)
                torch.cuda.synchronize()
                out[r] = (rc, e, res, v.cpu().numpy(), rep.as_dict())
        except Exception as ex:  # reported below
            out[r] = ex

    ts = [threading.Thread(target=rank, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=600)
    for o in out:
        assert not isinstance(o, Exception) and o is not None, o
    e0 = out[0][1]
    for rc, e, res, v, rep in out:
        assert rc == 0 and np.array_equal(e, e0) and np.all(res <= tol)
    assert np.abs(e0 - ref.energies).max() <= (1e-8 if prec == "fp64" else 1e-6)
    vfull = np.concatenate([o[3] for o in out], axis=1)
    for j in range(2):
        assert abs(abs(float(vfull[j] @ vref[j])) - 1.0) <= 1e-6
        assert vfull[j][np.argmax(np.abs(vfull[j]))] > 0
