"""Python binding of the C ABI in include/sbd.h (argument marshalling only).

Every computation runs in libsbd.so on the GPU; this module converts Python
objects (numpy arrays, torch tensors) to pointers, sizes and streams, calls
the entry point of the same name and raises SbdError on a negative status.
There is no fallback: if the library is missing, loading fails loudly.

Device memory for vectors is caller-owned torch tensors; the handle's own
tables live in memory obtained through PyTorch's CUDA caching allocator (the
allocator hooks of sbd_options), unless allocator="cuda" is requested.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

SBD_FP64 = 0
SBD_MIXED = 1
SBD_F32X2 = 2
PRECISION = {"fp64": SBD_FP64, "mixed": SBD_MIXED, "f32x2": SBD_F32X2, SBD_FP64: SBD_FP64, SBD_MIXED: SBD_MIXED,
             SBD_F32X2: SBD_F32X2}

STATUS = {
    0: "SBD_OK", 1: "SBD_NOT_CONVERGED", -1: "SBD_ERR_INVALID_ARG", -2: "SBD_ERR_BAD_STRING",
    -3: "SBD_ERR_DUPLICATE_STRING", -4: "SBD_ERR_NORB", -5: "SBD_ERR_OUT_OF_MEMORY", -6: "SBD_ERR_OVER_BUDGET",
    -7: "SBD_ERR_CUDA", -8: "SBD_ERR_NONFINITE", -9: "SBD_ERR_BREAKDOWN", -10: "SBD_ERR_UNSUPPORTED",
}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class sbd_options(C.Structure):
    _fields_ = [("delta", C.c_double), ("max_subspace", C.c_int), ("max_iter", C.c_int),
                ("hbm_budget_bytes", C.c_size_t), ("ecore", C.c_double), ("table_algo", C.c_int),
                ("verbose", C.c_int), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
                ("timing", C.c_int), ("tol_energy", C.c_double), ("refine_precision", C.c_int),
                ("restart_keep", C.c_int)]


class sbd_report(C.Structure):
    _fields_ = [("iterations", C.c_int), ("sigma_fp64", C.c_int), ("sigma_mixed", C.c_int),
                ("restarts", C.c_int), ("refinements", C.c_int), ("reorthogonalisations", C.c_int),
                ("status", C.c_int),
                ("max_residual", C.c_double), ("seconds_total", C.c_double), ("seconds_sigma", C.c_double),
                ("gap_estimate", C.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class sbd_engine_options(C.Structure):
    _fields_ = [("max_slots", C.c_int), ("max_subspace", C.c_int), ("max_iter", C.c_int),
                ("max_norb", C.c_int), ("max_strings", C.c_int), ("rows_per_item", C.c_int),
                ("delta", C.c_double), ("hbm_budget_bytes", C.c_size_t), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("table_bytes_per_string", C.c_size_t), ("schedule", C.c_int)]


SCHEDULE = {"fair": 0, "lockstep": 1}


class sbd_job_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("sigma_mixed", C.c_int), ("sigma_fp64", C.c_int),
                ("restarts", C.c_int), ("energy", C.c_double), ("residual", C.c_double),
                ("energy_mixed", C.c_double), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("ndets", C.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class sbd_engine_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("graph_launches", C.c_int64), ("kernel_launches", C.c_int64),
                ("rows_per_item", C.c_int), ("tune_ms", C.c_double * 4), ("bytes_in_use", C.c_size_t),
                ("bytes_peak", C.c_size_t), ("active", C.c_int), ("pending", C.c_int), ("done", C.c_int),
                ("requeued", C.c_int64)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["tune_ms"] = list(self.tune_ms)
        return d


ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_double), C.c_int)
RING_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p)


class sbd_comm(C.Structure):
    _fields_ = [("rank", C.c_int), ("world", C.c_int), ("ctx", C.c_void_p), ("allreduce_sum", ALLREDUCE_FN),
                ("ring_exchange", RING_FN)]


class SbdError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{STATUS.get(code, code)}: {message}")
        self.code = code
        self.message = message


_lib = None
_lock = threading.Lock()
_vp, _i64, _i32, _int, _dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_int, C.c_double

_SIGNATURES = {
    "sbd_default_options": (None, [C.POINTER(sbd_options)]),
    "sbd_status_string": (C.c_char_p, [_int]),
    "sbd_create": (_int, [C.POINTER(_vp), _int, _int, _int, _vp, _vp, _vp, _i64, _vp, _i64,
                          C.POINTER(sbd_options), _vp]),
    "sbd_destroy": (_int, [_vp]),
    "sbd_dims": (_int, [_vp, C.POINTER(_i64), C.POINTER(_i64)]),
    "sbd_memory": (_int, [_vp, C.POINTER(C.c_size_t)]),
    "sbd_sorted_strings": (_int, [_vp, _int, _vp]),
    "sbd_table_size": (_int, [_vp, _int, _int, C.POINTER(_i64)]),
    "sbd_tables": (_int, [_vp, _int, _int, _vp, _vp, _vp, _vp]),
    "sbd_string_elements": (_int, [_vp, _int, _int, _vp]),
    "sbd_diagonal": (_int, [_vp, _vp, _vp]),
    "sbd_lookup": (_int, [_vp, _int, _vp, _i64, _vp, _vp]),
    "sbd_sigma": (_int, [_vp, _vp, _vp, _int, _int, _vp]),
    "sbd_davidson": (_int, [_vp, _int, _dbl, _int, _vp, _vp, _vp, C.POINTER(sbd_report)]),
    "sbd_last_error": (C.c_char_p, [_vp]),
    "sbd_kernel_times": (_int, [_vp, _vp, _vp, _int]),
    "sbd_launch_count": (_i64, []),
    "sbd_sort_strings_noalloc": (_int, [_vp, _i64, _int, _int, _vp, C.POINTER(_i64), _vp]),
    "sbd_sigma_batched": (_int, [_int, _vp, _vp, _vp, _int, _int, _vp]),
    "sbd_davidson_sharded": (_int, [_vp, _vp, C.POINTER(sbd_comm), _int, _dbl, _int, _vp, _vp, _vp,
                                    C.POINTER(sbd_report)]),
    "sbd_block_plan_create": (_int, [_vp, _i64, _i64, _i64, _i64, C.POINTER(_vp)]),
    "sbd_sigma_block": (_int, [_vp, _vp, _vp, _int, _vp]),
    "sbd_block_plan_destroy": (_int, [_vp]),
    "sbd_engine_default_options": (None, [C.POINTER(sbd_engine_options)]),
    "sbd_engine_create": (_int, [C.POINTER(_vp), C.POINTER(sbd_engine_options), _vp]),
    "sbd_engine_destroy": (_int, [_vp]),
    "sbd_engine_submit": (_int, [_vp, _int, _int, _int, _vp, _vp, _vp, _i64, _vp, _i64, _dbl, _dbl, _dbl, _int,
                                 C.POINTER(_i64)]),
    "sbd_engine_step": (_int, [_vp, C.POINTER(_int)]),
    "sbd_engine_run": (_int, [_vp]),
    "sbd_engine_result": (_int, [_vp, _i64, C.POINTER(sbd_job_result)]),
    "sbd_engine_vector": (_int, [_vp, _i64, _vp, _i64]),
    "sbd_engine_release": (_int, [_vp, _i64]),
    "sbd_engine_get_stats": (_int, [_vp, C.POINTER(sbd_engine_stats)]),
    "sbd_engine_clock": (_dbl, [_vp]),
}

SBD_PENDING = 2

SBD_NOALLOC_MAX_STRINGS = 65536

KERNEL_SLOTS = ["transpose", "beta_pass", "alpha_pass", "ab_pass"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Loads libsbd.so (building it first only when asked)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2601_16637_gb300.build.build()")
        lib = C.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc: int, handle=None) -> int:
    if rc < 0:
        msg = load().sbd_last_error(handle)
        raise SbdError(rc, msg.decode() if msg else "")
    return rc


def _ptr(x) -> int:
    """Address of a contiguous numpy array or torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class _TorchAllocator:
    """Routes the library's device allocations to PyTorch's caching allocator."""

    def __init__(self):
        import torch

        self.torch = torch
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, ctx, nbytes, stream):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _free(self, ctx, ptr, stream):
        self.torch.cuda.caching_allocator_delete(int(ptr))


def sbd_default_options() -> sbd_options:
    o = sbd_options()
    load().sbd_default_options(C.byref(o))
    return o


def sbd_create(norb, nalpha, nbeta, h, eri, A, B, options: sbd_options | None = None, stream=None) -> int:
    """Returns the opaque handle (an int).  h, eri, A, B: host or device buffers."""
    lib = load()
    out = C.c_void_p()
    A = A.view(np.uint64) if isinstance(A, np.ndarray) else A
    B = B.view(np.uint64) if isinstance(B, np.ndarray) else B
    rc = lib.sbd_create(C.byref(out), int(norb), int(nalpha), int(nbeta), _ptr(h), _ptr(eri), _ptr(A),
                        int(A.numel() if hasattr(A, "numel") else A.size), _ptr(B),
                        int(B.numel() if hasattr(B, "numel") else B.size),
                        C.byref(options) if options is not None else None, _stream(stream))
    _check(rc)
    return out.value


def sbd_destroy(handle) -> None:
    _check(load().sbd_destroy(handle))


def sbd_dims(handle) -> tuple[int, int]:
    a, b = C.c_int64(), C.c_int64()
    _check(load().sbd_dims(handle, C.byref(a), C.byref(b)), handle)
    return a.value, b.value


def sbd_memory(handle) -> int:
    v = C.c_size_t()
    _check(load().sbd_memory(handle, C.byref(v)), handle)
    return v.value


def sbd_sorted_strings(handle, spin: int) -> np.ndarray:
    nA, nB = sbd_dims(handle)
    out = np.empty(nA if spin == 0 else nB, dtype=np.uint64)
    _check(load().sbd_sorted_strings(handle, spin, _ptr(out)), handle)
    return out


def sbd_table_size(handle, spin: int, kind: int) -> int:
    v = C.c_int64()
    _check(load().sbd_table_size(handle, spin, kind, C.byref(v)), handle)
    return v.value


def sbd_tables(handle, spin: int, kind: int):
    """(ptr[int64 n+1], target[int32 m], orbs[uint8 (m,4)], sign[int8 m]) in canonical CSR order."""
    nA, nB = sbd_dims(handle)
    n = nA if spin == 0 else nB
    m = sbd_table_size(handle, spin, kind)
    ptr = np.empty(n + 1, dtype=np.int64)
    tgt = np.empty(max(m, 1), dtype=np.int32)
    orbs = np.empty(max(4 * m, 4), dtype=np.uint8)
    sign = np.empty(max(m, 1), dtype=np.int8)
    _check(load().sbd_tables(handle, spin, kind, _ptr(ptr), _ptr(tgt), _ptr(orbs), _ptr(sign)), handle)
    return ptr, tgt[:m], orbs[:4 * m].reshape(m, 4), sign[:m]


def sbd_string_elements(handle, spin: int, kind: int) -> np.ndarray:
    nA, nB = sbd_dims(handle)
    n = (nA if spin == 0 else nB) if kind == 0 else sbd_table_size(handle, spin, kind)
    out = np.empty(max(n, 1), dtype=np.float64)
    _check(load().sbd_string_elements(handle, spin, kind, _ptr(out)), handle)
    return out[:n]


def sbd_diagonal(handle, out, stream=None) -> None:
    _check(load().sbd_diagonal(handle, _ptr(out), _stream(stream)), handle)


def sbd_lookup(handle, spin: int, keys, idx, stream=None) -> None:
    """keys: device int64/uint64 tensor of strings; idx: device int64 tensor (written)."""
    _check(load().sbd_lookup(handle, spin, _ptr(keys), int(keys.numel()), _ptr(idx), _stream(stream)), handle)


def sbd_sigma(handle, c, sigma, nvec: int, precision, stream=None) -> None:
    _check(load().sbd_sigma(handle, _ptr(c), _ptr(sigma), int(nvec), PRECISION[precision], _stream(stream)), handle)


def sbd_davidson(handle, nroots: int, tol: float, precision, energies: np.ndarray, vecs=None,
                 residuals: np.ndarray | None = None) -> tuple[int, sbd_report]:
    rep = sbd_report()
    rc = load().sbd_davidson(handle, int(nroots), float(tol), PRECISION[precision], _ptr(energies),
                             _ptr(vecs) if vecs is not None else None,
                             _ptr(residuals) if residuals is not None else None, C.byref(rep))
    _check(rc, handle)
    return rc, rep


def sbd_kernel_times(handle, reset: bool = False):
    """({'fp64': {...}, 'mixed': {...}, 'f32x2': {...}} per-kernel milliseconds, same for launch counts)."""
    ms = np.zeros(12)
    n = np.zeros(12, dtype=np.int64)
    _check(load().sbd_kernel_times(handle, _ptr(ms), _ptr(n), int(bool(reset))), handle)
    out_ms, out_n = {}, {}
    for p, off in (("fp64", 0), ("mixed", 4), ("f32x2", 8)):
        out_ms[p] = {k: float(ms[off + i]) for i, k in enumerate(KERNEL_SLOTS)}
        out_n[p] = {k: int(n[off + i]) for i, k in enumerate(KERNEL_SLOTS)}
    return out_ms, out_n


def sbd_launch_count() -> int:
    return int(load().sbd_launch_count())


def sbd_sort_strings_noalloc(keys, norb: int, nel: int, out, stream=None) -> tuple[int, int]:
    """Validates and sorts device strings `keys` into device buffer `out` without any device
    allocation.  Returns (status, bad_index); raises SbdError on errors other than
    SBD_ERR_BAD_STRING / SBD_ERR_DUPLICATE_STRING, which are returned with their index."""
    bad = C.c_int64(-1)
    rc = load().sbd_sort_strings_noalloc(_ptr(keys), int(keys.numel()), int(norb), int(nel), _ptr(out),
                                         C.byref(bad), _stream(stream))
    if rc < 0 and rc not in (-2, -3):
        _check(rc)
    return rc, bad.value


def sbd_sigma_batched(handles, cs, sigmas, precision, rows_per_item: int = 0, stream=None) -> None:
    """sigma of several instances in one batched launch sequence; handles, cs, sigmas: equal-length lists."""
    n = len(handles)
    if not (len(cs) == len(sigmas) == n):
        raise ValueError("handles, cs and sigmas must have the same length")
    hs = (C.c_void_p * max(n, 1))(*handles)
    xs = (C.c_void_p * max(n, 1))(*[_ptr(x) for x in cs])
    ys = (C.c_void_p * max(n, 1))(*[_ptr(y) for y in sigmas])
    _check(load().sbd_sigma_batched(n, hs, xs, ys, PRECISION[precision], int(rows_per_item), _stream(stream)))


def sbd_davidson_sharded(handle, bounds, comm: "sbd_comm", nroots: int, tol: float, precision, energies,
                         vecs_rows=None, residuals=None) -> tuple[int, sbd_report]:
    """One rank of an alpha-row-sharded solve; comm carries rank, world and the callbacks."""
    b = np.ascontiguousarray(bounds, dtype=np.int64)
    rep = sbd_report()
    rc = load().sbd_davidson_sharded(handle, _ptr(b), C.byref(comm), int(nroots), float(tol), PRECISION[precision],
                                     _ptr(energies), _ptr(vecs_rows) if vecs_rows is not None else None,
                                     _ptr(residuals) if residuals is not None else None, C.byref(rep))
    _check(rc, handle)
    return rc, rep


def sbd_block_plan_create(handle, r0, r1, j0, j1) -> int:
    out = C.c_void_p()
    _check(load().sbd_block_plan_create(handle, int(r0), int(r1), int(j0), int(j1), C.byref(out)), handle)
    return out.value


def sbd_sigma_block(plan, c_block, sigma_rows, precision, stream=None) -> None:
    _check(load().sbd_sigma_block(plan, _ptr(c_block), _ptr(sigma_rows), PRECISION[precision], _stream(stream)))


def sbd_block_plan_destroy(plan) -> None:
    _check(load().sbd_block_plan_destroy(plan))


def sbd_engine_default_options() -> sbd_engine_options:
    o = sbd_engine_options()
    load().sbd_engine_default_options(C.byref(o))
    return o


def sbd_engine_create(options: sbd_engine_options | None = None, stream=None) -> int:
    out = C.c_void_p()
    _check(load().sbd_engine_create(C.byref(out), C.byref(options) if options is not None else None,
                                    _stream(stream)))
    return out.value


def sbd_engine_destroy(engine) -> None:
    _check(load().sbd_engine_destroy(engine))


def sbd_engine_submit(engine, norb, nalpha, nbeta, h, eri, A, B, ecore=0.0, tol=1e-6, tol_energy=0.0,
                      keep_vector=False) -> int:
    A = np.ascontiguousarray(A, dtype=np.uint64)
    B = np.ascontiguousarray(B, dtype=np.uint64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    job = C.c_int64()
    _check(load().sbd_engine_submit(engine, int(norb), int(nalpha), int(nbeta), _ptr(h), _ptr(eri), _ptr(A),
                                    int(A.size), _ptr(B), int(B.size), float(ecore), float(tol),
                                    float(tol_energy), int(bool(keep_vector)), C.byref(job)))
    return job.value


def sbd_engine_step(engine) -> int:
    rem = C.c_int()
    _check(load().sbd_engine_step(engine, C.byref(rem)))
    return rem.value


def sbd_engine_run(engine) -> None:
    _check(load().sbd_engine_run(engine))


def sbd_engine_result(engine, job) -> tuple[int, sbd_job_result]:
    r = sbd_job_result()
    rc = load().sbd_engine_result(engine, int(job), C.byref(r))
    _check(rc)
    return rc, r


def sbd_engine_vector(engine, job, out) -> None:
    _check(load().sbd_engine_vector(engine, int(job), _ptr(out), int(out.size if isinstance(out, np.ndarray)
                                                                      else out.numel())))


def sbd_engine_release(engine, job) -> None:
    _check(load().sbd_engine_release(engine, int(job)))


def sbd_engine_get_stats(engine) -> sbd_engine_stats:
    st = sbd_engine_stats()
    _check(load().sbd_engine_get_stats(engine, C.byref(st)))
    return st


def sbd_engine_clock(engine) -> float:
    return float(load().sbd_engine_clock(engine))


def sbd_last_error(handle=None) -> str:
    m = load().sbd_last_error(handle)
    return m.decode() if m else ""


def sbd_status_string(code: int) -> str:
    return load().sbd_status_string(int(code)).decode()


# ---------------------------------------------------------------------------
# convenience wrapper (still marshalling only)


@dataclass
class SolveResult:
    energies: np.ndarray
    residuals: np.ndarray
    vectors: object  # torch tensor [nroots, N] or None
    status: int
    report: dict


class SBD:
    """One selected-space instance on the current CUDA device."""

    def __init__(self, norb, nalpha, nbeta, h, eri, A, B, *, stream=None, allocator: str = "torch",
                 delta: float = 1e-4, max_subspace: int = 0, max_iter: int = 200, hbm_budget_bytes: int = 0,
                 ecore: float = 0.0, table_algo: int = 0, verbose: int = 0, timing: bool = False,
                 tol_energy: float = 0.0, refine_precision: str = "f32x2", restart_keep: int = 0):
        self._opts = sbd_default_options()
        self._opts.delta = delta
        self._opts.max_subspace = max_subspace
        self._opts.max_iter = max_iter
        self._opts.hbm_budget_bytes = hbm_budget_bytes
        self._opts.ecore = ecore
        self._opts.table_algo = table_algo
        self._opts.verbose = verbose
        self._opts.timing = int(bool(timing))
        self._opts.tol_energy = float(tol_energy)
        self._opts.refine_precision = PRECISION[refine_precision]
        self._opts.restart_keep = int(restart_keep)
        self._alloc = None
        if allocator == "torch":
            self._alloc = _TorchAllocator()
            self._opts.alloc = self._alloc.alloc
            self._opts.free = self._alloc.free
        elif allocator != "cuda":
            raise ValueError("allocator must be 'torch' or 'cuda'")
        self.stream = stream
        hh = np.ascontiguousarray(h, dtype=np.float64) if isinstance(h, np.ndarray) else h
        ee = np.ascontiguousarray(eri, dtype=np.float64) if isinstance(eri, np.ndarray) else eri
        AA = np.ascontiguousarray(A, dtype=np.uint64) if isinstance(A, np.ndarray) else A
        BB = np.ascontiguousarray(B, dtype=np.uint64) if isinstance(B, np.ndarray) else B
        self.handle = None
        self.handle = sbd_create(norb, nalpha, nbeta, hh, ee, AA, BB, self._opts, stream)
        self.norb, self.nalpha, self.nbeta = norb, nalpha, nbeta
        self.nA, self.nB = sbd_dims(self.handle)
        self.N = self.nA * self.nB

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(wl.norb, wl.nalpha, wl.nbeta, wl.h, wl.eri, wl.A, wl.B, **kw)

    def close(self):
        if self.handle:
            sbd_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sorted_strings(self, spin: int) -> np.ndarray:
        return sbd_sorted_strings(self.handle, spin)

    def tables(self, spin: int, kind: int):
        return sbd_tables(self.handle, spin, kind)

    def string_elements(self, spin: int, kind: int) -> np.ndarray:
        return sbd_string_elements(self.handle, spin, kind)

    def memory(self) -> int:
        return sbd_memory(self.handle)

    def kernel_times(self, reset: bool = False):
        return sbd_kernel_times(self.handle, reset)

    def diagonal(self):
        import torch
        out = torch.empty(self.N, dtype=torch.float64, device="cuda")
        sbd_diagonal(self.handle, out, self.stream)
        return out

    def lookup(self, spin: int, keys):
        import torch
        idx = torch.empty(keys.numel(), dtype=torch.int64, device=keys.device)
        sbd_lookup(self.handle, spin, keys, idx, self.stream)
        return idx

    def sigma(self, c, precision="fp64", out=None):
        """c: device tensor [N] or [nvec, N] (float64 for fp64, float32 for mixed)."""
        import torch
        want = torch.float32 if PRECISION[precision] == SBD_MIXED else torch.float64
        if c.dtype != want or not c.is_cuda:
            raise TypeError(f"c must be a CUDA {want} tensor")
        c = c.contiguous()
        nvec = 1 if c.dim() == 1 else c.shape[0]
        if c.numel() != nvec * self.N:
            raise ValueError("c has the wrong size")
        if out is None:
            out = torch.empty(c.shape, dtype=torch.float64, device=c.device)
        sbd_sigma(self.handle, c, out, nvec, precision, self.stream)
        return out

    def davidson(self, nroots=1, tol=1e-8, precision="fp64", vectors: str | None = "device") -> SolveResult:
        import torch
        e = np.empty(nroots)
        r = np.empty(nroots)
        v = None
        if vectors == "device":
            v = torch.empty((nroots, self.N), dtype=torch.float64, device="cuda")
        elif vectors == "host":
            v = torch.empty((nroots, self.N), dtype=torch.float64, pin_memory=True)
        rc, rep = sbd_davidson(self.handle, nroots, tol, precision, e, v, r)
        return SolveResult(e, r, v, rc, rep.as_dict())


class Engine:
    """Batched / served solver: jobs submitted here iterate together on the device."""

    def __init__(self, *, max_slots=64, max_subspace=12, max_iter=200, max_norb=64, max_strings=20000,
                 rows_per_item=0, delta=1e-4, hbm_budget_bytes=0, table_bytes_per_string=None,
                 schedule: str = "fair", allocator: str = "torch", stream=None):
        o = sbd_engine_default_options()
        o.max_slots, o.max_subspace, o.max_iter = max_slots, max_subspace, max_iter
        o.max_norb, o.max_strings, o.rows_per_item = max_norb, max_strings, rows_per_item
        o.delta, o.hbm_budget_bytes = delta, hbm_budget_bytes
        if table_bytes_per_string is not None:
            o.table_bytes_per_string = table_bytes_per_string
        if schedule not in SCHEDULE:
            raise ValueError("schedule must be 'fair' or 'lockstep'")
        o.schedule = SCHEDULE[schedule]
        self._alloc = None
        if allocator == "torch":
            self._alloc = _TorchAllocator()
            o.alloc, o.free = self._alloc.alloc, self._alloc.free
        elif allocator != "cuda":
            raise ValueError("allocator must be 'torch' or 'cuda'")
        self._opts = o
        self.engine = None
        self.engine = sbd_engine_create(o, stream)

    def submit(self, wl_or_norb, *args, tol=1e-6, tol_energy=0.0, keep_vector=False, ecore=0.0) -> int:
        """submit(workload) or submit(norb, nalpha, nbeta, h, eri, A, B)."""
        if args:
            norb, (nalpha, nbeta, h, eri, A, B) = wl_or_norb, args
        else:
            w = wl_or_norb
            norb, nalpha, nbeta, h, eri, A, B = w.norb, w.nalpha, w.nbeta, w.h, w.eri, w.A, w.B
        return sbd_engine_submit(self.engine, norb, nalpha, nbeta, h, eri, A, B, ecore, tol, tol_energy, keep_vector)

    def step(self) -> int:
        return sbd_engine_step(self.engine)

    def run(self) -> None:
        sbd_engine_run(self.engine)

    def result(self, job) -> dict | None:
        rc, r = sbd_engine_result(self.engine, job)
        return None if rc == SBD_PENDING else r.as_dict()

    def vector(self, job, n) -> np.ndarray:
        out = np.empty(int(n), dtype=np.float64)
        sbd_engine_vector(self.engine, job, out)
        return out

    def release(self, job) -> None:
        sbd_engine_release(self.engine, job)

    def stats(self) -> dict:
        return sbd_engine_get_stats(self.engine).as_dict()

    def clock(self) -> float:
        return sbd_engine_clock(self.engine)

    def close(self):
        if self.engine:
            sbd_engine_destroy(self.engine)
            self.engine = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
