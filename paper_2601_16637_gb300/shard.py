"""Alpha-row sharding of the sigma product over ranks (paper Sec. III, the distributed product).

Rank r owns the alpha rows [bounds[r], bounds[r+1]) of C and of sigma.  The C blocks travel around
the ring of ranks: at step s rank r holds block (r - s) mod P, adds that block's contribution to its
own rows, and meanwhile sends the block on to rank r+1 and receives the next one from rank r-1
(two buffers, so the transfer overlaps the products).  After P steps every rank has met every
block once, and its rows of sigma are complete.

This module is host logic only.  The block products come from a callable
`block_sigma(b, c_block, out_rows)` that adds block b's contribution to the rank's rows; on a GPU
that is sbd_sigma_block through one block plan per source block (`device_block_sigma`).
"""
from __future__ import annotations

from typing import Callable, Sequence


def row_blocks(n: int, parts: int) -> list[int]:
    """Boundaries of `parts` contiguous blocks of [0, n) whose sizes differ by at most one."""
    if parts < 1 or n < parts:
        raise ValueError("need 1 <= parts <= n")
    q, r = divmod(n, parts)
    out = [0]
    for p in range(parts):
        out.append(out[-1] + q + (1 if p < r else 0))
    return out


def ring_schedule(rank: int, world: int) -> list[int]:
    """The source blocks rank `rank` holds at steps 0..world-1 (its own block first)."""
    return [(rank - s) % world for s in range(world)]


class RingSigma:
    """sigma rows of this rank from its own C rows, with the other ranks' blocks passed around a
    ring.  bounds: row_blocks(nA, world); row_len: elements per alpha row (nB)."""

    def __init__(self, block_sigma: Callable, bounds: Sequence[int], rank: int, world: int, row_len: int,
                 group=None):
        if len(bounds) != world + 1:
            raise ValueError("bounds must have world + 1 entries")
        self.block_sigma = block_sigma
        self.bounds = list(bounds)
        self.rank, self.world, self.row_len, self.group = rank, world, row_len, group
        self.steps = []  # (step, block) as processed, for inspection

    def rows(self, b: int) -> int:
        return self.bounds[b + 1] - self.bounds[b]

    def __call__(self, c_own, out_rows):
        import torch
        import torch.distributed as dist

        out_rows.zero_()
        self.steps = []
        P, r = self.world, self.rank
        if P == 1:
            self.block_sigma(0, c_own, out_rows)
            self.steps.append((0, 0))
            return out_rows
        nmax = max(self.rows(b) for b in range(P)) * self.row_len
        bufs = [torch.empty(nmax, dtype=c_own.dtype, device=c_own.device) for _ in range(2)]
        cur, cur_b = c_own, r
        sched = ring_schedule(r, P)
        for s in range(P):
            reqs = []
            if s < P - 1:
                nxt_b = sched[s + 1]
                nxt = bufs[s % 2][: self.rows(nxt_b) * self.row_len]
                reqs = [dist.isend(cur.contiguous(), (r + 1) % P, group=self.group),
                        dist.irecv(nxt, (r - 1) % P, group=self.group)]
            self.block_sigma(cur_b, cur, out_rows)
            self.steps.append((s, cur_b))
            for q in reqs:
                q.wait()
            if s < P - 1:
                cur, cur_b = nxt, nxt_b
        return out_rows


def device_block_sigma(handle, bounds: Sequence[int], rank: int, precision, stream=None):
    """block_sigma for RingSigma on a GPU: one block plan per source block (sbd_block_plan_create),
    products by sbd_sigma_block.  Returns (callable, close).

    RingSigma orders its own device work (zeroing the rows, the NCCL receives it waits for) on
    torch's current stream.  With stream=None the products run there too.  A torch.cuda.Stream
    given here first waits for everything queued on the current stream, and the current stream
    then waits for the product, so a block is never read before it has arrived, rows are never
    added to before they are zeroed, and a receive buffer is not overwritten while a product still
    reads it."""
    from . import binding as B

    r0, r1 = bounds[rank], bounds[rank + 1]
    plans = [B.sbd_block_plan_create(handle, r0, r1, bounds[b], bounds[b + 1]) for b in range(len(bounds) - 1)]

    def block_sigma(b, c_block, out_rows):
        import torch

        cur = torch.cuda.current_stream()
        if stream is None or stream == cur:
            B.sbd_sigma_block(plans[b], c_block, out_rows, precision, cur)
            return
        stream.wait_stream(cur)
        B.sbd_sigma_block(plans[b], c_block, out_rows, precision, stream)
        cur.wait_stream(stream)

    def close():
        for p in plans:
            B.sbd_block_plan_destroy(p)
        plans.clear()

    return block_sigma, close


# ---------------------------------------------------------------------------
# communicators for sbd_davidson_sharded


class _DevBytes:
    """A raw device pointer seen as a uint8 array through the CUDA array interface (for torch)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 2}


def device_view(ptr: int, nbytes: int):
    import torch

    return torch.as_tensor(_DevBytes(ptr, nbytes), device="cuda")


class ThreadRing:
    """Communicator for `world` ranks run as threads of one process on one device: sums in rank
    order (so every rank sees the same bits) and ring exchanges as device-to-device copies.  Each
    rank's thread calls `comm(rank)` once and passes the result to sbd_davidson_sharded."""

    def __init__(self, world: int, timeout: float = 300.0):
        import threading

        self.world = world
        self.barrier = threading.Barrier(world, timeout=timeout)
        self.slots = [None] * world
        self._keep = []

    def comm(self, rank: int):
        from . import binding as B

        def allreduce(ctx, buf, n):
            try:
                import numpy as np

                self.slots[rank] = np.ctypeslib.as_array(buf, shape=(n,)).copy()
                self.barrier.wait()
                total = self.slots[0].copy()
                for r in range(1, self.world):
                    total = total + self.slots[r]
                self.barrier.wait()
                np.ctypeslib.as_array(buf, shape=(n,))[:] = total
                return 0
            except Exception:
                self.barrier.abort()
                return 1

        def ring(ctx, send, send_bytes, recv, recv_bytes, stream):
            try:
                import torch

                self.slots[rank] = (int(send or 0), int(send_bytes))
                self.barrier.wait()
                src, nb = self.slots[(rank - 1) % self.world]
                if nb != recv_bytes:
                    raise ValueError("ring exchange sizes disagree")
                device_view(recv, recv_bytes).copy_(device_view(src, nb))
                torch.cuda.synchronize()
                self.barrier.wait()
                return 0
            except Exception:
                self.barrier.abort()
                return 1

        a, r = B.ALLREDUCE_FN(allreduce), B.RING_FN(ring)
        self._keep += [a, r]
        return B.sbd_comm(rank, self.world, None, a, r)


class DistRing:
    """Communicator over a torch.distributed process group (one process per GPU): allreduce of
    host doubles through a tensor of the group's device, ring exchange of the library's buffers.

    buffers="device" (what sbd_davidson_sharded passes): with NCCL the device buffers are sent and
    received in place (isend/irecv); with gloo they are staged through host memory.  buffers="host":
    the pointers are host memory and travel as CPU tensors (gloo)."""

    def __init__(self, group=None, buffers: str = "device"):
        import torch.distributed as dist

        if buffers not in ("device", "host"):
            raise ValueError("buffers must be 'device' or 'host'")
        self.group = group
        self.buffers = buffers
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self._keep = []

    def comm(self):
        import ctypes

        import numpy as np
        import torch
        import torch.distributed as dist

        from . import binding as B

        nccl = dist.get_backend(self.group) == "nccl"
        dev = "cuda" if nccl else "cpu"
        nxt, prv = (self.rank + 1) % self.world, (self.rank - 1) % self.world

        def host_view(ptr, nbytes):
            return torch.from_numpy(np.ctypeslib.as_array((ctypes.c_uint8 * int(nbytes)).from_address(int(ptr))))

        def allreduce(ctx, buf, n):
            try:
                h = np.ctypeslib.as_array(buf, shape=(n,))
                t = torch.from_numpy(h.copy()).to(dev)
                dist.all_reduce(t, group=self.group)
                h[:] = t.cpu().numpy()
                return 0
            except Exception:
                return 1

        def ring(ctx, send, send_bytes, recv, recv_bytes, stream):
            try:
                if self.buffers == "host":
                    s_t, r_t = host_view(send, send_bytes), host_view(recv, recv_bytes)
                elif nccl:
                    s_t, r_t = device_view(send, send_bytes), device_view(recv, recv_bytes)
                else:  # gloo: stage the device buffers through host memory
                    torch.cuda.synchronize()
                    s_t = device_view(send, send_bytes).cpu()
                    r_t = torch.empty(int(recv_bytes), dtype=torch.uint8)
                reqs = [dist.isend(s_t, nxt, group=self.group), dist.irecv(r_t, prv, group=self.group)]
                for q in reqs:
                    q.wait()
                if self.buffers == "device":
                    if not nccl:
                        device_view(recv, recv_bytes).copy_(r_t)
                    torch.cuda.synchronize()
                return 0
            except Exception:
                return 1

        a, r = B.ALLREDUCE_FN(allreduce), B.RING_FN(ring)
        self._keep += [a, r]
        return B.sbd_comm(self.rank, self.world, None, a, r)
