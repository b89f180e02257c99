"""Python access to the CPU FP64 oracle (sbd_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and the benchmark's
CPU-baseline leg use this module.  The CUDA library never imports it.

build() compiles sbd_oracle.c with gcc (OpenMP) into oracle/_lib/; a planted
mistake can be compiled in with `mutation=k` (used only by the pin-strength
test).  Every function cites the part of the paper it follows in
sbd_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbd_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_lock = threading.Lock()
_libs: dict[int, C.CDLL] = {}

_p = C.c_void_p
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")


def lib_path(mutation: int = 0) -> str:
    return os.path.join(_LIBDIR, f"libsbd_oracle{'' if mutation == 0 else f'_m{mutation}'}.so")


def build(mutation: int = 0, force: bool = False) -> str:
    """Compile the oracle (portable C, no architecture-specific flags)."""
    out = lib_path(mutation)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", f"-DORACLE_MUTATION={mutation}",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load(mutation: int = 0) -> C.CDLL:
    with _lock:
        if mutation in _libs:
            return _libs[mutation]
        lib = C.CDLL(build(mutation))
        lib.oracle_create.argtypes = [C.c_int, C.c_int, C.c_int, _f64p, _f64p, _u64p, C.c_int64, _u64p,
                                      C.c_int64, C.POINTER(_p)]
        lib.oracle_create.restype = C.c_int
        lib.oracle_destroy.argtypes = [_p]
        lib.oracle_ndets.argtypes = [_p]
        lib.oracle_ndets.restype = C.c_int64
        lib.oracle_sorted.argtypes = [_p, C.c_int, _u64p]
        lib.oracle_hij.argtypes = [_p, C.c_int64, C.c_int64]
        lib.oracle_hij.restype = C.c_double
        lib.oracle_diag.argtypes = [_p, _f64p]
        lib.oracle_dense.argtypes = [_p, _f64p]
        lib.oracle_sigma_rows.argtypes = [_p, _f64p, C.c_int, _i64p, C.c_int64, _f64p]
        lib.oracle_sigma.argtypes = [_p, _f64p, C.c_int, _f64p]
        lib.oracle_table_count.argtypes = [_u64p, C.c_int64, C.c_int]
        lib.oracle_table_count.restype = C.c_int64
        lib.oracle_table_fill.argtypes = [_u64p, C.c_int64, C.c_int, C.c_int, _i64p, _i32p, _u8p, _i8p]
        lib.oracle_string_element.argtypes = [C.c_int, _f64p, _f64p, C.c_uint64, C.c_uint64]
        lib.oracle_string_element.restype = C.c_double
        lib.oracle_jacobi.argtypes = [C.c_int, _f64p, _f64p, _f64p]
        lib.oracle_jacobi.restype = C.c_int
        lib.oracle_davidson.argtypes = [_p, C.c_int, C.c_double, C.c_int, C.c_int, C.c_double, _f64p,
                                        _f64p, _f64p]
        lib.oracle_davidson.restype = C.c_int
        lib.oracle_num_threads.restype = C.c_int
        lib.oracle_csr_counts.argtypes = [_p, _i64p]
        lib.oracle_csr_fill.argtypes = [_p, _i64p, _i64p, _f64p]
        _libs[mutation] = lib
        return lib


class OracleError(RuntimeError):
    pass


class Oracle:
    """The selected space A x B with its Hamiltonian, evaluated plainly on the CPU."""

    def __init__(self, norb, nalpha, nbeta, h, eri, A, B, mutation: int = 0):
        self.lib = load(mutation)
        self.norb, self.nalpha, self.nbeta = int(norb), int(nalpha), int(nbeta)
        self.h = np.ascontiguousarray(h, dtype=np.float64)
        self.eri = np.ascontiguousarray(eri, dtype=np.float64).reshape(-1)
        A = np.ascontiguousarray(A, dtype=np.uint64)
        B = np.ascontiguousarray(B, dtype=np.uint64)
        self._h = _p()
        rc = self.lib.oracle_create(self.norb, self.nalpha, self.nbeta, self.h.reshape(-1), self.eri, A,
                                    A.size, B, B.size, C.byref(self._h))
        if rc != 0:
            if self._h:
                self.lib.oracle_destroy(self._h)
                self._h = _p()
            raise OracleError({-1: "bad argument", -2: "bad string", -3: "duplicate string"}.get(rc, rc))
        self.nA, self.nB = A.size, B.size
        self.N = self.nA * self.nB

    @classmethod
    def from_workload(cls, wl, mutation: int = 0):
        return cls(wl.norb, wl.nalpha, wl.nbeta, wl.h, wl.eri, wl.A, wl.B, mutation=mutation)

    def close(self):
        if self._h:
            self.lib.oracle_destroy(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sorted_strings(self, spin: int) -> np.ndarray:
        out = np.empty(self.nA if spin == 0 else self.nB, dtype=np.uint64)
        self.lib.oracle_sorted(self._h, spin, out)
        return out

    def hij(self, i: int, j: int) -> float:
        return self.lib.oracle_hij(self._h, int(i), int(j))

    def diag(self) -> np.ndarray:
        out = np.empty(self.N)
        self.lib.oracle_diag(self._h, out)
        return out

    def dense(self) -> np.ndarray:
        if self.N > 6000:
            raise OracleError("dense H only for N <= 6000")
        out = np.empty(self.N * self.N)
        self.lib.oracle_dense(self._h, out)
        return out.reshape(self.N, self.N)

    def csr(self):
        """The Hamiltonian as a scipy CSR matrix (every H_ij of the space within two differences)."""
        import scipy.sparse as sp

        counts = np.empty(self.N, dtype=np.int64)
        self.lib.oracle_csr_counts(self._h, counts)
        ptr = np.zeros(self.N + 1, dtype=np.int64)
        np.cumsum(counts, out=ptr[1:])
        cols = np.empty(ptr[-1], dtype=np.int64)
        vals = np.empty(ptr[-1])
        self.lib.oracle_csr_fill(self._h, ptr, cols, vals)
        return sp.csr_matrix((vals, cols, ptr), shape=(self.N, self.N))

    def sigma(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
        out = np.empty_like(x)
        self.lib.oracle_sigma(self._h, x.reshape(-1), x.shape[0], out.reshape(-1))
        return out

    def sigma_rows(self, x: np.ndarray, rows) -> np.ndarray:
        x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.empty((x.shape[0], rows.size))
        self.lib.oracle_sigma_rows(self._h, x.reshape(-1), x.shape[0], rows, rows.size, out.reshape(-1))
        return out

    def davidson(self, nroots=1, tol=1e-8, max_iter=200, max_sub=0, delta=1e-4):
        if max_sub <= 0:
            max_sub = max(24, 8 * nroots)
        e = np.empty(nroots)
        r = np.empty(nroots)
        v = np.empty(nroots * self.N)
        it = self.lib.oracle_davidson(self._h, nroots, tol, max_iter, max_sub, delta, e, v, r)
        return e, v.reshape(nroots, self.N), r, it


def string_table(S: np.ndarray, norb: int, kind: int, mutation: int = 0):
    """Canonical CSR excitation table of one sorted string set.

    Returns (ptr[int64 n+1], target[int32], orbs[uint8 (m,4)], sign[int8]).
    kind 1 = singles, kind 2 = doubles.
    """
    lib = load(mutation)
    S = np.ascontiguousarray(S, dtype=np.uint64)
    m = lib.oracle_table_count(S, S.size, kind)
    ptr = np.empty(S.size + 1, dtype=np.int64)
    tgt = np.empty(m, dtype=np.int32)
    orbs = np.empty(4 * m, dtype=np.uint8)
    sign = np.empty(m, dtype=np.int8)
    lib.oracle_table_fill(S, S.size, norb, kind, ptr, tgt, orbs, sign)
    return ptr, tgt, orbs.reshape(m, 4), sign


def string_element(norb, h, eri, si: int, sj: int, mutation: int = 0) -> float:
    """<si|H|sj> for one spin species alone (the other spin empty)."""
    lib = load(mutation)
    return lib.oracle_string_element(int(norb), np.ascontiguousarray(h, dtype=np.float64).reshape(-1),
                                     np.ascontiguousarray(eri, dtype=np.float64).reshape(-1),
                                     int(si), int(sj))


def jacobi(T: np.ndarray, mutation: int = 0):
    """Eigenpairs of a small symmetric matrix by cyclic Jacobi (ascending)."""
    lib = load(mutation)
    k = T.shape[0]
    a = np.ascontiguousarray(T, dtype=np.float64).copy().reshape(-1)
    ev = np.empty(k)
    vec = np.empty(k * k)
    lib.oracle_jacobi(k, a, ev, vec)
    return ev, vec.reshape(k, k)


def num_threads() -> int:
    return int(load().oracle_num_threads())
