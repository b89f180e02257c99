"""Literal second quantisation on the full Fock space (test helper).

Builds the fermionic operators of 2*norb modes as Jordan-Wigner Kronecker
products (mode 0 the least significant bit of the basis index; alpha modes
0..norb-1, beta modes norb..2norb-1) and assembles the Hamiltonian of the
paper's Eq. 3 term by term from operator products:

    H = sum_{pq,s} h_pq a+_{ps} a_{qs}
      + 1/2 sum_{pqrs} sum_{s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}.

No Slater-Condon rule, phase formula or string factorisation is used: the
signs come only from the Z strings of the Jordan-Wigner matrices.  This is
the brute-force pin the oracle is checked against on tiny spaces.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_SM = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))  # |1> -> |0>
_Z = sp.csr_matrix(np.diag([1.0, -1.0]))
_I = sp.identity(2, format="csr")


def annihilators(nmodes: int) -> list[sp.csr_matrix]:
    """a_m for m < nmodes; basis index x = sum_m n_m 2^m."""
    ops = []
    for m in range(nmodes):
        op = sp.identity(1, format="csr")
        # Kronecker factors from the most significant mode (nmodes-1) down to mode 0
        for k in range(nmodes - 1, -1, -1):
            f = _I if k > m else (_SM if k == m else _Z)
            op = sp.kron(op, f, format="csr")
        ops.append(op)
    return ops


def fock_hamiltonian(h: np.ndarray, eri: np.ndarray, tol: float = 0.0) -> sp.csr_matrix:
    norb = h.shape[0]
    a = annihilators(2 * norb)
    ad = [x.T.tocsr() for x in a]
    dim = 1 << (2 * norb)
    H = sp.csr_matrix((dim, dim))
    for s in range(2):
        for p in range(norb):
            for q in range(norb):
                if h[p, q] != 0.0:
                    H = H + h[p, q] * (ad[p + s * norb] @ a[q + s * norb])
    for s in range(2):
        for t in range(2):
            for p in range(norb):
                for r in range(norb):
                    left = ad[p + s * norb] @ ad[r + t * norb]
                    for q in range(norb):
                        for ss in range(norb):
                            v = eri[p, q, r, ss]
                            if v == 0.0:
                                continue
                            H = H + (0.5 * v) * (left @ (a[ss + t * norb] @ a[q + s * norb]))
    return H.tocsr()


def selected_block(H: sp.csr_matrix, norb: int, A_sorted, B_sorted) -> np.ndarray:
    """Rows/columns of the determinants (a, b) in a-major, b-minor order."""
    idx = np.array([int(a) | (int(b) << norb) for a in A_sorted for b in B_sorted], dtype=np.int64)
    return H[idx][:, idx].toarray()


def string_operator(norb: int, creators, annihilators_, si: int, sj: int) -> float:
    """<si| prod(a+ creators) prod(a annihilators) |sj> on one spin's norb modes.

    creators are applied left to right as written (a+_c0 a+_c1 ...), then the
    annihilators (a_d0 a_d1 ...), i.e. the operator string
    a+_{c0} a+_{c1} ... a_{d0} a_{d1} ... acting on |sj>.
    """
    a = annihilators(norb)
    op = sp.identity(1 << norb, format="csr")
    for c in creators:
        op = op @ a[c].T
    for d in annihilators_:
        op = op @ a[d]
    return float(op[si, sj])
