"""Pins of the CPU oracle against things other than itself (no GPU).

Each check below is fixed by mathematics independent of the oracle's code:
literal second quantisation (Jordan-Wigner matrices), closed forms,
invariants, dense brute force and a library eigensolver.  The last test
plants known mistakes in the oracle and checks that some pin catches each.
"""
import math

import numpy as np
import pytest

import secondq
from paper_2601_16637_gb300 import workloads as W


def _subset(strings, k, seed):
    rng = np.random.default_rng(seed)
    return strings[rng.choice(strings.size, size=k, replace=False)]


def _random_instance(norb, na, nb, nA=None, nB=None, seed=0):
    h = W.one_electron(norb, seed)
    eri = W.two_electron(norb, seed)
    SA = W.all_strings(norb, na)
    SB = W.all_strings(norb, nb)
    A = SA if nA is None else _subset(SA, nA, seed + 11)
    B = SB if nB is None else _subset(SB, nB, seed + 12)
    return h, eri, A, B


# ---------------------------------------------------------------------------
# the brute-force tool itself


def test_jordan_wigner_anticommutation():
    a = secondq.annihilators(4)
    dim = 16
    for m in range(4):
        for n in range(4):
            acomm = (a[m] @ a[n].T + a[n].T @ a[m]).toarray()
            expect = np.eye(dim) if m == n else np.zeros((dim, dim))
            assert np.array_equal(acomm, expect)
            assert not np.any((a[m] @ a[n] + a[n] @ a[m]).toarray())


# ---------------------------------------------------------------------------
# matrix elements against literal second quantisation (Eq. 3 read in chemists' order)


@pytest.mark.parametrize("norb,na,nb,nA,nB,seed", [
    (4, 2, 2, None, None, 0),   # full space, 36 determinants
    (4, 3, 1, None, None, 1),   # unequal electron counts
    (5, 2, 3, 7, 6, 2),         # selected subsets of A and B
    (5, 1, 1, None, None, 3),
])
def test_oracle_equals_second_quantisation(oracle_mod, norb, na, nb, nA, nB, seed):
    h, eri, A, B = _random_instance(norb, na, nb, nA, nB, seed)
    o = oracle_mod.Oracle(norb, na, nb, h, eri, A, B)
    Hf = secondq.fock_hamiltonian(h, eri)
    ref = secondq.selected_block(Hf, norb, o.sorted_strings(0), o.sorted_strings(1))
    got = o.dense()
    assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
    # the diagonal entry point (used for the preconditioner, Sec. II-E) on its own
    d = o.diag()
    assert np.abs(d - np.diag(ref)).max() <= 1e-13 * max(1.0, np.abs(ref).max())
    assert np.array_equal(d, np.diag(got))


def test_string_tables_signs_against_jordan_wigner(oracle_mod):
    norb = 6
    S = np.sort(W.all_strings(norb, 3))
    for kind in (1, 2):
        ptr, tgt, orbs, sign = oracle_mod.string_table(S, norb, kind)
        # completeness and canonical order
        for i in range(S.size):
            js = [j for j in range(S.size) if bin(int(S[i]) ^ int(S[j])).count("1") == 2 * kind]
            assert list(tgt[ptr[i]:ptr[i + 1]]) == js
        for i in range(S.size):
            for e in range(ptr[i], ptr[i + 1]):
                j = tgt[e]
                p1, p2, q1, q2 = (int(v) for v in orbs[e])
                if kind == 1:
                    ref = secondq.string_operator(norb, [p1], [q1], int(S[i]), int(S[j]))
                else:
                    ref = secondq.string_operator(norb, [p1, p2], [q2, q1], int(S[i]), int(S[j]))
                assert ref == sign[e] and abs(ref) == 1.0


def test_string_element_against_second_quantisation(oracle_mod):
    norb = 4
    h, eri, _, _ = _random_instance(norb, 2, 2)
    Hf = secondq.fock_hamiltonian(h, eri)
    S = W.all_strings(norb, 2)
    for si in S:
        for sj in S:
            got = oracle_mod.string_element(norb, h, eri, int(si), int(sj))
            assert abs(got - Hf[int(si), int(sj)]) <= 1e-13


# ---------------------------------------------------------------------------
# closed forms


def test_one_alpha_one_beta_closed_form(oracle_mod):
    # n_alpha = n_beta = 1: H_{(p,r),(q,s)} = h_pq d_rs + d_pq h_rs + (pq|rs)
    norb = 4
    h, eri, A, B = _random_instance(norb, 1, 1)
    o = oracle_mod.Oracle(norb, 1, 1, h, eri, A, B)
    H = o.dense()
    I = np.eye(norb)
    ref = (np.einsum("pq,rs->prqs", h, I) + np.einsum("pq,rs->prqs", I, h)
           + np.einsum("pqrs->prqs", eri)).reshape(norb * norb, norb * norb)
    assert np.abs(H - ref).max() <= 1e-14


def test_hubbard_dimer(oracle_mod):
    # two sites, one alpha and one beta electron: E0 = (U - sqrt(U^2 + 16 t^2)) / 2
    for t, U in [(1.0, 4.0), (0.5, 1.0), (1.0, 0.0)]:
        h = np.array([[0.0, -t], [-t, 0.0]])
        eri = np.zeros((2, 2, 2, 2))
        eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
        A = np.array([1, 2], dtype=np.uint64)
        o = oracle_mod.Oracle(2, 1, 1, h, eri, A, A)
        e0 = np.linalg.eigvalsh(o.dense())[0]
        assert abs(e0 - (U - math.sqrt(U * U + 16 * t * t)) / 2) <= 1e-13


def test_closed_shell_hartree_fock_diagonal(oracle_mod):
    norb, n = 7, 3
    h, eri, A, B = _random_instance(norb, n, n, 10, 10, seed=5)
    hf = np.uint64((1 << n) - 1)
    if hf not in A:
        A[0] = hf
    if hf not in B:
        B[0] = hf
    o = oracle_mod.Oracle(norb, n, n, h, eri, A, B)
    ia = int(np.searchsorted(o.sorted_strings(0), hf))
    ib = int(np.searchsorted(o.sorted_strings(1), hf))
    occ = range(n)
    ref = 2 * sum(h[i, i] for i in occ) + sum(2 * eri[i, i, j, j] - eri[i, j, j, i] for i in occ for j in occ)
    got = o.hij(ia * o.nB + ib, ia * o.nB + ib)
    assert abs(got - ref) <= 1e-13 * abs(ref)


def test_zero_eri_diagonal_h_is_sum_of_orbital_energies(oracle_mod):
    norb, na, nb = 8, 3, 2
    eps = np.sort(np.random.default_rng(1).normal(size=norb))[::-1].copy()  # unsorted w.r.t. index
    h = np.diag(eps)
    eri = np.zeros((norb,) * 4)
    A, B = W.all_strings(norb, na), W.all_strings(norb, nb)
    o = oracle_mod.Oracle(norb, na, nb, h, eri, A, B)
    H = o.dense()
    assert np.abs(H - np.diag(np.diag(H))).max() == 0.0
    e0 = np.linalg.eigvalsh(H)[0]
    ref = np.sort(eps)[:na].sum() + np.sort(eps)[:nb].sum()
    assert abs(e0 - ref) <= 1e-13
    # selected subset: the minimum over the selected (a, b) pairs
    As, Bs = _subset(A, 9, 3), _subset(B, 7, 4)
    o2 = oracle_mod.Oracle(norb, na, nb, h, eri, As, Bs)
    ref2 = min(sum(eps[p] for p in range(norb) if int(a) >> p & 1) for a in As) + \
        min(sum(eps[p] for p in range(norb) if int(b) >> p & 1) for b in Bs)
    assert abs(np.linalg.eigvalsh(o2.dense())[0] - ref2) <= 1e-13


def test_zero_eri_general_h_full_space(oracle_mod):
    norb, na, nb = 6, 2, 3
    h, _, A, B = _random_instance(norb, na, nb, seed=7)
    h = h + np.random.default_rng(0).normal(scale=0.3, size=h.shape)
    h = 0.5 * (h + h.T)
    eri = np.zeros((norb,) * 4)
    o = oracle_mod.Oracle(norb, na, nb, h, eri, A, B)
    w = np.linalg.eigvalsh(h)
    assert abs(np.linalg.eigvalsh(o.dense())[0] - (w[:na].sum() + w[:nb].sum())) <= 1e-12


# ---------------------------------------------------------------------------
# invariants


def test_orbital_rotation_invariance_full_space(oracle_mod):
    norb, na, nb = 5, 2, 2
    h, eri, A, B = _random_instance(norb, na, nb, seed=4)
    Q, _ = np.linalg.qr(np.random.default_rng(9).normal(size=(norb, norb)))
    h2 = Q.T @ h @ Q
    eri2 = np.einsum("ap,bq,cr,ds,abcd->pqrs", Q, Q, Q, Q, eri, optimize=True)
    e1 = np.linalg.eigvalsh(oracle_mod.Oracle(norb, na, nb, h, eri, A, B).dense())
    e2 = np.linalg.eigvalsh(oracle_mod.Oracle(norb, na, nb, h2, eri2, A, B).dense())
    assert np.abs(e1 - e2).max() <= 1e-10


def test_sigma_equals_dense_product_and_is_hermitian(oracle_mod):
    norb, na, nb = 10, 3, 3
    h, eri, A, B = _random_instance(norb, na, nb, 60, 55, seed=8)
    o = oracle_mod.Oracle(norb, na, nb, h, eri, A, B)
    H = o.dense()
    assert np.abs(H - H.T).max() <= 1e-14 * np.abs(H).max()
    x = W.random_vector(o.N, 1, nvec=2)
    s = o.sigma(x)
    assert np.abs(s - x @ H.T).max() <= 1e-13 * np.abs(s).max()
    lhs, rhs = x[0] @ s[1], s[0] @ x[1]
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_explicit_csr_equals_dense(oracle_mod):
    # the assembled matrix (Sec. II-A, explicit) holds exactly the dense H's nonzeros
    wl = W.make("t", 10, 3, 3, 45, 40, 0.3, seed=4)
    o = oracle_mod.Oracle.from_workload(wl)
    H = o.dense()
    Hs = o.csr().toarray()
    assert np.array_equal(Hs, H)


def test_sigma_rows_match_full_sigma(oracle_mod):
    wl = W.make("t", 12, 4, 4, 150, 140, 0.3, seed=3)
    o = oracle_mod.Oracle.from_workload(wl)
    x = W.random_vector(o.N, 2)
    full = o.sigma(x)
    rows = np.array([0, 5, o.N - 1, o.N // 2, 1234], dtype=np.int64)
    assert np.array_equal(o.sigma_rows(x, rows), full[:, rows])


def test_alpha_beta_transpose_symmetry(oracle_mod):
    # A = B and n_alpha = n_beta: sigma(C^T) = sigma(C)^T
    norb, n = 9, 3
    h, eri, A, _ = _random_instance(norb, n, n, 40, 40, seed=6)
    o = oracle_mod.Oracle(norb, n, n, h, eri, A, A)
    c = np.random.default_rng(2).normal(size=(40, 40))
    s = o.sigma(c.reshape(1, -1)).reshape(40, 40)
    sT = o.sigma(c.T.copy().reshape(1, -1)).reshape(40, 40)
    assert np.abs(sT - s.T).max() <= 1e-13 * np.abs(s).max()


# ---------------------------------------------------------------------------
# eigensolvers


def test_jacobi_against_library_eigh(oracle_mod):
    rng = np.random.default_rng(0)
    for k in (1, 2, 5, 24, 48):
        M = rng.normal(size=(k, k))
        M = M + M.T
        ev, vec = oracle_mod.jacobi(M)
        ref = np.linalg.eigvalsh(M)
        assert np.abs(ev - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
        assert np.abs(vec.T @ vec - np.eye(k)).max() <= 1e-12
        assert np.abs(M @ vec - vec * ev).max() <= 1e-11 * max(1.0, np.abs(ref).max())


def test_davidson_matches_dense_diagonalisation_cfg1(oracle_mod):
    wl = W.config("cfg1")
    o = oracle_mod.Oracle.from_workload(wl)
    ref = np.linalg.eigvalsh(o.dense())
    e, v, r, it = o.davidson(nroots=1, tol=1e-10)
    assert it > 0 and r[0] <= 1e-10
    assert abs(e[0] - ref[0]) <= 1e-10


def test_block_davidson_three_roots(oracle_mod):
    wl = W.make("t", 12, 4, 4, 70, 64, 0.35, seed=1)
    o = oracle_mod.Oracle.from_workload(wl)
    ref = np.linalg.eigvalsh(o.dense())[:3]
    e, v, r, it = o.davidson(nroots=3, tol=1e-8)
    assert it > 0
    assert np.abs(e - ref).max() <= 1e-10
    # Ritz vectors are orthonormal eigenvectors
    assert np.abs(v @ v.T - np.eye(3)).max() <= 1e-9


# ---------------------------------------------------------------------------
# pin strength: each planted mistake must be caught by at least one pin

_MUTATIONS = {
    1: "exchange term dropped from the antisymmetrised integral",
    2: "double-excitation phase negated",
    3: "chemists'/physicists' index order swapped",
    4: "one-electron term dropped from single excitations",
    5: "factor 1/2 dropped from the diagonal two-electron sum",
}


def _pins_pass(oracle_mod, mutation):
    ok = True
    norb, na, nb = 4, 2, 2
    h, eri, A, B = _random_instance(norb, na, nb, seed=0)
    o = oracle_mod.Oracle(norb, na, nb, h, eri, A, B, mutation=mutation)
    ref = secondq.selected_block(secondq.fock_hamiltonian(h, eri), norb, o.sorted_strings(0),
                                 o.sorted_strings(1))
    ok &= np.abs(o.dense() - ref).max() <= 1e-13 * np.abs(ref).max()
    h1, eri1, A1, B1 = _random_instance(4, 1, 1)
    o1 = oracle_mod.Oracle(4, 1, 1, h1, eri1, A1, B1, mutation=mutation)
    I = np.eye(4)
    ref1 = (np.einsum("pq,rs->prqs", h1, I) + np.einsum("pq,rs->prqs", I, h1)
            + np.einsum("pqrs->prqs", eri1)).reshape(16, 16)
    ok &= np.abs(o1.dense() - ref1).max() <= 1e-14
    return bool(ok)


def test_pins_pass_on_the_real_oracle(oracle_mod):
    assert _pins_pass(oracle_mod, 0)


@pytest.mark.parametrize("mutation", sorted(_MUTATIONS))
def test_planted_mistake_is_caught(oracle_mod, mutation):
    oracle_mod.build(mutation)
    assert not _pins_pass(oracle_mod, mutation), _MUTATIONS[mutation]


# ---------------------------------------------------------------------------
# a published worked example


def load_h2_golden():
    """The minimal-basis H2 full CI of the golden fixture: integrals expanded to all index
    permutations of real orbitals, (pq|rs) = (qp|rs) = (pq|sr) = (rs|pq), and the printed values."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "h2_minimal_basis.txt")
    vals, h, eri = {}, None, None
    for line in open(path):
        f = line.split("#")[0].split()
        if not f:
            continue
        if f[0] == "h":
            h[int(f[1]), int(f[2])] = h[int(f[2]), int(f[1])] = float(f[3])
        elif f[0] == "eri":
            p, q, r, s = map(int, f[1:5])
            for a, b, c, d in [(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r)]:
                eri[a, b, c, d] = eri[c, d, a, b] = float(f[5])
        else:
            vals[f[0]] = float(f[1])
            if f[0] == "norb":
                n = int(vals["norb"])
                h, eri = np.zeros((n, n)), np.zeros((n, n, n, n))
    return vals, h, eri


def _h2_pin_passes(oracle_mod, mutation=0):
    # the full space of one alpha and one beta electron in two orbitals: the Hartree-Fock
    # determinant, two singles (decoupled by g/u symmetry) and the double excitation
    vals, h, eri = load_h2_golden()
    A = np.array([1, 2], dtype=np.uint64)
    H = oracle_mod.Oracle(2, 1, 1, h, eri, A, A, mutation=mutation).dense()
    hf, dbl = 0, 3  # (alpha, beta) = (orbital 0, orbital 0) and (1, 1)
    e0 = np.linalg.eigvalsh(H)[0]
    return bool(abs(H[hf, hf] - vals["E_hf_electronic"]) <= 1e-12  # 2 h11 + J11, exact in the printed digits
                and abs(H[hf, dbl] - vals["coupling_hf_double"]) <= 1e-12  # K12
                and abs(H[hf, 1]) <= 1e-15 and abs(H[hf, 2]) <= 1e-15  # Brillouin / symmetry
                # printed to four decimals from integrals rounded to four decimals
                and abs((e0 - H[hf, hf]) - vals["E_corr"]) <= 1.5e-4
                and abs(e0 + 1.0 / vals["R_bohr"] - vals["E_total_fci"]) <= 1.5e-4)


def test_h2_minimal_basis_full_ci_against_the_textbook(oracle_mod):
    assert _h2_pin_passes(oracle_mod)


@pytest.mark.parametrize("mutation", [1, 3, 5])
def test_h2_pin_catches_planted_mistakes(oracle_mod, mutation):
    oracle_mod.build(mutation)
    assert not _h2_pin_passes(oracle_mod, mutation), _MUTATIONS[mutation]
