"""Alpha-row sharding of sigma over ranks (paper Sec. III): row partition, ring schedule, and the
ring exchange with two and three gloo ranks on CPU.  The block products come from the CPU oracle
(sigma of the vector restricted to the block's rows, by linearity), so the test checks the
partition and the exchange: every rank must end with exactly its rows of the full sigma."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2601_16637_gb300 import shard  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_row_blocks_and_ring_schedule():
    assert shard.row_blocks(10, 3) == [0, 4, 7, 10]
    assert shard.row_blocks(6, 6) == [0, 1, 2, 3, 4, 5, 6]
    assert shard.row_blocks(5, 1) == [0, 5]
    with pytest.raises(ValueError):
        shard.row_blocks(2, 3)
    for world in (1, 2, 3, 5):
        for r in range(world):
            s = shard.ring_schedule(r, world)
            assert s[0] == r and sorted(s) == list(range(world))
            # at every step, the block a rank holds is the one its left neighbour held the step before
            if world > 1:
                left = shard.ring_schedule((r - 1) % world, world)
                assert all(s[k + 1] == left[k] for k in range(world - 1))


def _ring_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_2601_16637_gb300 import shard as S
    from paper_2601_16637_gb300 import workloads as W

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    wl = W.make("ring", 10, 3, 4, 61, 45, 0.2, seed=31)
    o = O.Oracle.from_workload(wl)
    nA, nB, N = o.nA, o.nB, o.N
    x = W.random_vector(N, 5)[0]
    bounds = S.row_blocks(nA, world)
    r0, r1 = bounds[rank], bounds[rank + 1]
    rows = np.arange(r0 * nB, r1 * nB)

    def block_sigma(b, c_block, out_rows):
        xf = np.zeros(N)
        xf[bounds[b] * nB: bounds[b + 1] * nB] = c_block.numpy()
        out_rows += torch.from_numpy(o.sigma_rows(xf[None, :], rows)[0])

    ring = S.RingSigma(block_sigma, bounds, rank, world, nB)
    out = torch.empty((r1 - r0) * nB, dtype=torch.float64)
    ring(torch.from_numpy(x[r0 * nB: r1 * nB].copy()), out)
    ref = o.sigma(x[None, :])[0][r0 * nB: r1 * nB]
    err = float(np.abs(out.numpy() - ref).max() / np.abs(ref).max())
    q.put((rank, err, [b for _, b in ring.steps]))
    dist.barrier()
    dist.destroy_process_group()
    o.close()


@pytest.mark.parametrize("world", [2, 3])
def test_ring_sigma_over_gloo_ranks(world, oracle_mod):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_ring_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, err, blocks in res:
        assert err <= 1e-13
        assert blocks == shard.ring_schedule(rank, world)


def test_thread_ring_allreduce_is_identical_on_every_rank():
    # the host side of the in-process communicator: sums in rank order, the same bits everywhere
    import ctypes
    import threading

    from paper_2601_16637_gb300 import binding as B  # noqa: F401  (callback types)

    world = 3
    ring = shard.ThreadRing(world, timeout=30)
    vals = [np.array([1e16, 1.0, -1e16 + r, 0.1 * r]) for r in range(world)]
    got = [None] * world

    def run(r):
        c = ring.comm(r)
        buf = (ctypes.c_double * 4)(*vals[r])
        assert c.allreduce_sum(None, buf, 4) == 0
        got[r] = np.array(buf[:])

    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=60)
    expect = vals[0] + vals[1] + vals[2]
    for g in got:
        assert np.array_equal(g, got[0]) and np.array_equal(g, expect)


def _distring_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import ctypes

    import torch.distributed as dist

    from paper_2601_16637_gb300 import shard as S

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    comm = S.DistRing().comm()
    vals = [1.0 + rank, -2.5 * rank, 1e-3 * (rank + 1), 7.0]
    buf = (ctypes.c_double * 4)(*vals)
    rc = comm.allreduce_sum(None, buf, 4)
    q.put((rank, rc, comm.rank, comm.world, list(buf[:])))
    dist.barrier()
    dist.destroy_process_group()


def test_dist_ring_allreduce_callback_over_gloo_ranks():
    # the host side of the torch.distributed communicator handed to sbd_davidson_sharded: the
    # allreduce callback sums host doubles over the group (gloo: on CPU tensors)
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_distring_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    expect = [sum(1.0 + r for r in range(world)), sum(-2.5 * r for r in range(world)),
              sum(1e-3 * (r + 1) for r in range(world)), 7.0 * world]
    for rank, rc, crank, cworld, got in res:
        assert rc == 0 and crank == rank and cworld == world
        assert np.allclose(got, expect, rtol=1e-15, atol=0)
        assert got == res[0][4]  # every rank holds the same bits


def _dist_ring_exchange_worker(rank, world, port, q):
    import ctypes

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from paper_2601_16637_gb300 import shard as S

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    comm = S.DistRing(buffers="host").comm()
    # blocks of unequal size, as row_blocks gives when the rows do not divide evenly
    sizes = [40 + 8 * r for r in range(world)]
    send = np.arange(sizes[rank], dtype=np.uint8) * 3 + rank
    recv = np.zeros(sizes[(rank - 1) % world], dtype=np.uint8)
    rc = comm.ring_exchange(None, ctypes.c_void_p(send.ctypes.data), send.nbytes,
                            ctypes.c_void_p(recv.ctypes.data), recv.nbytes, None)
    q.put((rank, rc, recv.tolist()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_dist_ring_exchange_callback_over_gloo_ranks(world):
    # the ring callback handed to sbd_davidson_sharded, on host buffers over gloo: every rank
    # receives exactly the block of the rank before it (blocks of different sizes)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dist_ring_exchange_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    sizes = [40 + 8 * r for r in range(world)]
    for rank, rc, got in res:
        prv = (rank - 1) % world
        assert rc == 0
        assert got == (np.arange(sizes[prv], dtype=np.uint8) * 3 + prv).tolist()
