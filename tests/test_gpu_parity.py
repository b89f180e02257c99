"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Strings, lookups and excitation tables are compared bit-exactly; string
matrix elements and the diagonal to FP64 rounding; FP64 sigma to 1e-12
relative max-norm; eigenvalues to 1e-8 Ha (FP64) and 1e-6 Ha (mixed).
"""
import numpy as np
import pytest

from gpu_common import (EIG_FP64_ATOL, EIG_MIXED_ATOL, SIGMA_FP64_RTOL, SIGMA_MIXED_RTOL, medium,
                        rel_maxnorm)
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
def B():
    from paper_2601_16637_gb300 import binding

    binding.load()
    return binding


@pytest.fixture(scope="module")
def cfg2():
    return W.config("cfg2")


@pytest.fixture(scope="module")
def cfg2_pair(torch, B, cfg2, oracle_mod):
    g = B.SBD.from_workload(cfg2)
    o = oracle_mod.Oracle.from_workload(cfg2)
    yield g, o
    g.close()
    o.close()


@pytest.fixture(scope="module")
def med_pair(torch, B, oracle_mod):
    wl = medium()
    g = B.SBD.from_workload(wl)
    o = oracle_mod.Oracle.from_workload(wl)
    yield wl, g, o
    g.close()
    o.close()


# ---------------------------------------------------------------------------
# strings, lookup, tables


@pytest.mark.parametrize("name", ["cfg1", "cfg2"])
def test_sorted_strings_bit_exact(torch, B, oracle_mod, name):
    wl = W.config(name)
    with B.SBD.from_workload(wl) as g:
        o = oracle_mod.Oracle.from_workload(wl)
        for spin in (0, 1):
            assert np.array_equal(g.sorted_strings(spin), o.sorted_strings(spin))


def test_sort_large_random_set(torch, B):
    # 60,000 distinct strings of 40 orbitals: several sort tiles, 5 radix digits
    rng = np.random.default_rng(3)
    s = W.gumbel_top_k(40, 13, 60000, 0.1, rng)
    with B.SBD(40, 13, 1, np.zeros((40, 40)), np.zeros((40,) * 4), s, np.array([1], dtype=np.uint64),
               allocator="cuda") as g:
        assert np.array_equal(g.sorted_strings(0), np.sort(s))


def test_lookup_hits_and_misses(torch, B, cfg2_pair):
    g, o = cfg2_pair
    S = g.sorted_strings(1)
    rng = np.random.default_rng(0)
    pick = rng.integers(0, S.size, size=5000)
    absent = W.gumbel_top_k(16, 5, 3000, 0.0, rng)
    absent = absent[~np.isin(absent, S)]
    keys = np.concatenate([S[pick], absent, S[[0, S.size - 1]]])
    expect = np.concatenate([pick, -np.ones(absent.size, dtype=np.int64), [0, S.size - 1]])
    kt = torch.from_numpy(keys.view(np.int64)).cuda()
    idx = g.lookup(1, kt).cpu().numpy()
    assert np.array_equal(idx, expect)


@pytest.mark.parametrize("algo", [1, 2])
def test_tables_bit_exact_against_oracle(torch, B, oracle_mod, cfg2, algo):
    with B.SBD.from_workload(cfg2, table_algo=algo) as g:
        for spin in (0, 1):
            S = g.sorted_strings(spin)
            for kind in (1, 2):
                ptr, tgt, orbs, sign = g.tables(spin, kind)
                optr, otgt, oorbs, osign = oracle_mod.string_table(S, cfg2.norb, kind)
                assert np.array_equal(ptr, optr)
                assert np.array_equal(tgt, otgt)
                assert np.array_equal(orbs, oorbs)
                assert np.array_equal(sign, osign)


def test_table_builders_agree_on_a_sparse_large_set(torch, B):
    wl = W.make("t", 24, 8, 8, 6000, 5000, 0.35, seed=9)
    outs = []
    for algo in (1, 2):
        with B.SBD.from_workload(wl, table_algo=algo) as g:
            outs.append([g.tables(s, k) for s in (0, 1) for k in (1, 2)])
    for a, b in zip(*outs):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_string_elements_against_oracle(torch, B, oracle_mod, cfg2_pair):
    g, _ = cfg2_pair
    wl = W.config("cfg2")
    rng = np.random.default_rng(1)
    for spin in (0, 1):
        S = g.sorted_strings(spin)
        dg = g.string_elements(spin, 0)
        for i in rng.integers(0, S.size, 300):
            ref = oracle_mod.string_element(wl.norb, wl.h, wl.eri, int(S[i]), int(S[i]))
            assert abs(dg[i] - ref) <= 1e-12 * max(1.0, abs(ref))
        for kind in (1, 2):
            ptr, tgt, _, _ = g.tables(spin, kind)
            val = g.string_elements(spin, kind)
            src = np.repeat(np.arange(S.size), np.diff(ptr))
            for e in rng.integers(0, tgt.size, 3000):
                ref = oracle_mod.string_element(wl.norb, wl.h, wl.eri, int(S[src[e]]), int(S[tgt[e]]))
                assert abs(val[e] - ref) <= 1e-13 * max(1.0, abs(ref))


def test_diagonal_against_oracle(torch, B, med_pair):
    wl, g, o = med_pair
    hd = g.diagonal().cpu().numpy()
    assert rel_maxnorm(hd, o.diag()) <= 1e-13


# ---------------------------------------------------------------------------
# sigma


@pytest.mark.parametrize("prec", ["fp64", "f32x2"])
def test_sigma_fp64_full_against_oracle(torch, B, med_pair, prec):
    wl, g, o = med_pair
    x = W.random_vector(g.N, 7, nvec=2)
    got = g.sigma(torch.from_numpy(x).cuda(), prec).cpu().numpy()
    ref = o.sigma(x)
    assert rel_maxnorm(got, ref) <= SIGMA_FP64_RTOL


def test_sigma_fp64_unequal_electrons_and_sets(torch, B, oracle_mod):
    wl = medium(norb=11, n=4, nb=3, nA=197, nB=133, seed=12)
    with B.SBD.from_workload(wl) as g:
        o = oracle_mod.Oracle.from_workload(wl)
        x = W.random_vector(g.N, 8)
        ref = o.sigma(x)[0]
        for prec in ("fp64", "f32x2"):
            got = g.sigma(torch.from_numpy(x[0]).cuda(), prec).cpu().numpy()
            assert rel_maxnorm(got, ref) <= SIGMA_FP64_RTOL, prec
        assert rel_maxnorm(_mixed(torch, g, x[0]), ref) <= SIGMA_MIXED_RTOL


def _mixed(torch, g, x):
    return g.sigma(torch.from_numpy(np.asarray(x)).float().cuda(), "mixed").cpu().numpy()


def test_sigma_pair_split_edge_values(torch, B, med_pair):
    # the FP32-pair sigma splits every amplitude into hi + lo on the integer pipe: exact zeros,
    # magnitudes below the FP32 normal range (flushed to signed zeros: at most 2^-126 each) and
    # large ones must give the FP64 sigma to FP64 accuracy; NaN amplitudes must give NaN
    wl, g, o = med_pair
    x = W.random_vector(g.N, 21)[0]
    rng = np.random.default_rng(4)
    idx = rng.permutation(g.N)
    x[idx[:5000]] = 0.0
    x[idx[5000:5100]] *= 1e-300
    x[idx[5100:5200]] = np.copysign(1e-40, x[idx[5100:5200]])
    x[idx[5200:5300]] *= 1e30
    s64 = g.sigma(torch.from_numpy(x).cuda(), "fp64").cpu().numpy()
    s2 = g.sigma(torch.from_numpy(x).cuda(), "f32x2").cpu().numpy()
    assert rel_maxnorm(s2, s64) <= SIGMA_FP64_RTOL
    # a vector of small values only (pair parts and cross products stay FP32-normal): same accuracy
    y = W.random_vector(g.N, 22)[0] * 1e-20
    assert rel_maxnorm(g.sigma(torch.from_numpy(y).cuda(), "f32x2").cpu().numpy(),
                       g.sigma(torch.from_numpy(y).cuda(), "fp64").cpu().numpy()) <= SIGMA_FP64_RTOL
    z = W.random_vector(g.N, 23)[0]
    z[idx[7]] = np.nan
    assert np.isnan(g.sigma(torch.from_numpy(z).cuda(), "f32x2").cpu().numpy()[idx[7]])


def test_sigma_mixed_against_fp64(torch, B, med_pair):
    wl, g, o = med_pair
    x = W.random_vector(g.N, 9)[0]
    s64 = g.sigma(torch.from_numpy(x).cuda(), "fp64")
    s32 = g.sigma(torch.from_numpy(x).float().cuda(), "mixed")
    assert rel_maxnorm(s32.cpu().numpy(), s64.cpu().numpy()) <= SIGMA_MIXED_RTOL


def test_sigma_is_deterministic(torch, B, med_pair):
    wl, g, o = med_pair
    x = torch.from_numpy(W.random_vector(g.N, 10)[0]).cuda()
    a = g.sigma(x, "fp64")
    b = g.sigma(x, "fp64")
    assert torch.equal(a, b)
    # the mixed alpha-beta pass adds through shared-memory atomics, in fixed point: still bitwise
    a = g.sigma(x.float(), "mixed")
    b = g.sigma(x.float(), "mixed")
    assert torch.equal(a, b)


def test_sigma_mixed_several_alpha_chunks(torch, B, oracle_mod):
    # the full norb=13, 5-electron alpha space: every string has 40 in-set singles, taken by the
    # mixed alpha-beta pass as a 32-wide and an 8-wide chunk; a ragged beta set of 61 strings
    A = W.all_strings(13, 5)
    Bs = W.gumbel_top_k(13, 3, 61, 0.2, np.random.default_rng(9))
    h, eri = W.one_electron(13, 9), W.two_electron(13, 9)
    with B.SBD(13, 5, 3, h, eri, A, Bs) as g:
        o = oracle_mod.Oracle(13, 5, 3, h, eri, A, Bs)
        x = W.random_vector(g.N, 12)[0]
        ref = o.sigma(x[None, :])[0]
        assert rel_maxnorm(_mixed(torch, g, x), ref) <= SIGMA_MIXED_RTOL
        assert rel_maxnorm(g.sigma(torch.from_numpy(x).cuda(), "fp64").cpu().numpy(), ref) <= SIGMA_FP64_RTOL
        o.close()


def test_sigma_hermitian_and_transpose_symmetric(torch, B):
    # A = B, n_alpha = n_beta: sigma(C^T) = sigma(C)^T, and <x|Hy> = <Hx|y>
    wl = W.make("t", 13, 4, 4, 250, 250, 0.3, seed=4)
    with B.SBD(wl.norb, 4, 4, wl.h, wl.eri, wl.A, wl.A) as g:
        n = g.nA
        c = torch.from_numpy(np.random.default_rng(2).normal(size=(n, n))).cuda()
        s = g.sigma(c.reshape(-1), "fp64").reshape(n, n)
        sT = g.sigma(c.T.contiguous().reshape(-1), "fp64").reshape(n, n)
        assert rel_maxnorm(sT.cpu().numpy(), s.T.cpu().numpy()) <= 1e-13
        y = torch.from_numpy(np.random.default_rng(3).normal(size=n * n)).cuda()
        sy = g.sigma(y, "fp64")
        lhs = float(torch.dot(c.reshape(-1), sy))
        rhs = float(torch.dot(s.reshape(-1), y))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_sigma_cfg2_full_size_sampled_rows(torch, B, cfg2_pair):
    g, o = cfg2_pair
    x = W.random_vector(g.N, 100)[0]
    got = g.sigma(torch.from_numpy(x).cuda(), "fp64").cpu().numpy()
    rows = np.random.default_rng(5).integers(0, g.N, 400)
    ref = o.sigma_rows(x, rows)[0]
    assert rel_maxnorm(got[rows], ref) <= SIGMA_FP64_RTOL
    # the FP32-pair sigma against the FP64 one on every element, and against the oracle rows
    got2 = g.sigma(torch.from_numpy(x).cuda(), "f32x2").cpu().numpy()
    assert rel_maxnorm(got2, got) <= 1e-13
    assert rel_maxnorm(got2[rows], ref) <= SIGMA_FP64_RTOL


@pytest.mark.parametrize("shape", [(1, 40), (37, 1), (1, 1)])
def test_sigma_degenerate_single_string_sets(torch, B, oracle_mod, shape):
    nA, nB = shape
    wl = W.make("t", 9, 3, 3, nA, nB, 0.2, seed=6)
    with B.SBD.from_workload(wl) as g:
        o = oracle_mod.Oracle.from_workload(wl)
        x = W.random_vector(g.N, 1)
        for prec in ("fp64", "f32x2"):
            got = g.sigma(torch.from_numpy(x[0]).cuda(), prec).cpu().numpy()
            assert rel_maxnorm(got, o.sigma(x)[0]) <= SIGMA_FP64_RTOL, prec
        assert rel_maxnorm(_mixed(torch, g, x[0]), o.sigma(x)[0]) <= SIGMA_MIXED_RTOL


def test_sigma_zero_and_full_shells(torch, B, oracle_mod):
    # no beta electrons (the empty string) and a completely filled alpha shell
    norb = 6
    h, eri = W.one_electron(norb, 1), W.two_electron(norb, 1)
    for na, nb in [(3, 0), (6, 2)]:
        A = W.all_strings(norb, na)
        Bs = W.all_strings(norb, nb)
        with B.SBD(norb, na, nb, h, eri, A, Bs) as g:
            o = oracle_mod.Oracle(norb, na, nb, h, eri, A, Bs)
            x = W.random_vector(g.N, 2)
            for prec in ("fp64", "f32x2"):
                got = g.sigma(torch.from_numpy(x[0]).cuda(), prec).cpu().numpy()
                assert rel_maxnorm(got, o.sigma(x)[0]) <= SIGMA_FP64_RTOL, prec
            assert rel_maxnorm(_mixed(torch, g, x[0]), o.sigma(x)[0]) <= SIGMA_MIXED_RTOL


def test_h2_minimal_basis_golden(torch, B, oracle_mod):
    # the textbook minimal-basis H2 full CI (tests/golden): two orbitals, four determinants
    from test_oracle_pins import load_h2_golden

    vals, h, eri = load_h2_golden()
    A = np.array([1, 2], dtype=np.uint64)
    o = oracle_mod.Oracle(2, 1, 1, h, eri, A, A)
    e_dense = np.linalg.eigvalsh(o.dense())[0]
    with B.SBD(2, 1, 1, h, eri, A, A) as g:
        x = W.random_vector(g.N, 3)
        for prec in ("fp64", "f32x2"):
            got = g.sigma(torch.from_numpy(x[0]).cuda(), prec).cpu().numpy()
            assert rel_maxnorm(got, o.sigma(x)[0]) <= SIGMA_FP64_RTOL, prec
        assert rel_maxnorm(_mixed(torch, g, x[0]), o.sigma(x)[0]) <= SIGMA_MIXED_RTOL
        res = g.davidson(nroots=1, tol=1e-10, precision="fp64")
        assert res.status == 0
        assert abs(res.energies[0] - e_dense) <= 1e-12
        assert abs(res.energies[0] + 1.0 / vals["R_bohr"] - vals["E_total_fci"]) <= 1.5e-4
    o.close()


def test_sigma_norb_64(torch, B, oracle_mod):
    # the largest orbital count: strings using bit 63
    norb, n = 64, 2
    rng = np.random.default_rng(11)
    h = W.one_electron(norb, 3)
    eri = W.two_electron(norb, 3)
    S = set()
    while len(S) < 40:
        p = rng.choice(norb, size=n, replace=False)
        S.add(int(sum(1 << int(q) for q in p)))
    S.add((1 << 63) | (1 << 62))
    S.add((1 << 63) | 1)
    A = np.array(sorted(S), dtype=np.uint64)
    with B.SBD(norb, n, n, h, eri, A, A) as g:
        o = oracle_mod.Oracle(norb, n, n, h, eri, A, A)
        for spin in (0, 1):
            for kind in (1, 2):
                got = g.tables(spin, kind)
                ref = oracle_mod.string_table(A, norb, kind)
                for x, y in zip(got, ref):
                    assert np.array_equal(x, y)
        x = W.random_vector(g.N, 3)
        for prec in ("fp64", "f32x2"):
            got = g.sigma(torch.from_numpy(x[0]).cuda(), prec).cpu().numpy()
            assert rel_maxnorm(got, o.sigma(x)[0]) <= SIGMA_FP64_RTOL, prec
        assert rel_maxnorm(_mixed(torch, g, x[0]), o.sigma(x)[0]) <= SIGMA_MIXED_RTOL


# ---------------------------------------------------------------------------
# Davidson


def test_davidson_cfg1_against_dense(torch, B, oracle_mod):
    wl = W.config("cfg1")
    o = oracle_mod.Oracle.from_workload(wl)
    ref = np.linalg.eigvalsh(o.dense())
    with B.SBD.from_workload(wl) as g:
        res = g.davidson(nroots=1, tol=wl.tol)
        assert res.status == 0
        assert abs(res.energies[0] - ref[0]) <= EIG_FP64_ATOL
        assert res.residuals[0] <= wl.tol
        u = res.vectors[0].cpu().numpy()
        assert abs(np.linalg.norm(u) - 1) <= 1e-12
        # eigenvector: residual against the oracle sigma
        r = o.sigma(u[None, :])[0] - res.energies[0] * u
        assert np.linalg.norm(r) <= 10 * wl.tol
        # the first Ritz value above the root is an upper bound of the second eigenvalue (interlacing)
        assert res.report["gap_estimate"] >= (ref[1] - ref[0]) - 1e-8


@pytest.fixture(scope="module")
def med_lanczos(med_pair):
    # reference eigenvalues: library Lanczos on the oracle's explicit CSR matrix
    import scipy.sparse.linalg as sl

    wl, g, o = med_pair
    H = o.csr()
    ev, vec = sl.eigsh(H, k=3, which="SA", tol=1e-13)
    order = np.argsort(ev)
    return ev[order], vec[:, order].T


@pytest.mark.parametrize("prec", ["fp64", "f32x2"])
def test_davidson_three_roots_against_lanczos(torch, B, med_pair, med_lanczos, prec):
    wl, g, o = med_pair
    e_ref, v_ref = med_lanczos
    res = g.davidson(nroots=3, tol=1e-8, precision=prec)
    assert res.status == 0
    assert np.abs(res.energies - e_ref).max() <= EIG_FP64_ATOL
    V = res.vectors.cpu().numpy()
    assert np.abs(V @ V.T - np.eye(3)).max() <= 1e-9
    for j in range(3):
        assert abs(abs(V[j] @ v_ref[j]) - 1) <= 1e-6
        # sign convention: the largest-magnitude component is positive
        assert V[j][np.argmax(np.abs(V[j]))] > 0


def test_davidson_mixed_matches_fp64(torch, B, med_pair, med_lanczos):
    wl, g, o = med_pair
    e_ref, _ = med_lanczos
    r64 = g.davidson(nroots=1, tol=1e-7, precision="fp64")
    rmx = g.davidson(nroots=1, tol=1e-7, precision="mixed")
    assert r64.status == 0 and rmx.status == 0, (r64.report, rmx.report)
    assert abs(rmx.energies[0] - r64.energies[0]) <= EIG_MIXED_ATOL
    assert abs(rmx.energies[0] - e_ref[0]) <= EIG_MIXED_ATOL
    assert rmx.report["refinements"] >= 1 and rmx.report["sigma_mixed"] > 0
    assert rmx.residuals[0] <= 1e-7
    # the mixed solve needs at most a few FP64 sigma products
    assert rmx.report["sigma_fp64"] <= 10
    # defect corrections with the IEEE FP64 sigma instead of FP32 pairs
    with B.SBD.from_workload(wl, refine_precision="fp64") as g64:
        r2 = g64.davidson(nroots=1, tol=1e-7, precision="mixed")
        assert r2.status == 0 and abs(r2.energies[0] - r64.energies[0]) <= EIG_MIXED_ATOL


def test_davidson_restart_size_option(torch, B, med_pair, med_lanczos):
    # a larger thick-restart basis converges to the same roots
    wl, g, o = med_pair
    e_ref, _ = med_lanczos
    with B.SBD.from_workload(wl, restart_keep=12) as g12:
        res = g12.davidson(nroots=3, tol=1e-8)
        assert res.status == 0 and np.abs(res.energies - e_ref).max() <= EIG_FP64_ATOL


@pytest.mark.parametrize("prec,max_sub", [("f32x2", 32), ("mixed", 32), ("f32x2", 48), ("mixed", 12)])
def test_davidson_one_root_basis_sizes(torch, B, med_pair, med_lanczos, prec, max_sub):
    # one root in FP32 pairs: the Ritz pass also forms the Gram-Schmidt projections (basis of up to
    # 32 vectors), larger bases take the separate projection pass; the pair dot products run in
    # chunks of 8 basis vectors.  Every size must reach the Lanczos root and an FP64-accurate vector.
    wl, g, o = med_pair
    e_ref, v_ref = med_lanczos
    with B.SBD.from_workload(wl, max_subspace=max_sub) as gs:
        res = gs.davidson(nroots=1, tol=1e-8, precision=prec)
        assert res.status == 0, res.report
        assert abs(res.energies[0] - e_ref[0]) <= EIG_FP64_ATOL
        u = res.vectors[0].cpu().numpy()
        assert abs(np.linalg.norm(u) - 1) <= 1e-10
        assert abs(abs(u @ v_ref[0]) - 1) <= 1e-8
        r = o.sigma(u[None, :])[0] - res.energies[0] * u
        assert np.linalg.norm(r) <= 1e-7


def test_davidson_mixed_three_roots(torch, B, med_pair, med_lanczos):
    wl, g, o = med_pair
    e_ref, _ = med_lanczos
    res = g.davidson(nroots=3, tol=1e-8, precision="mixed")
    assert res.status == 0, res.report
    assert np.abs(res.energies - e_ref).max() <= EIG_FP64_ATOL


def test_davidson_cfg2_three_roots_residuals(torch, B, cfg2_pair):
    g, o = cfg2_pair
    res = g.davidson(nroots=3, tol=1e-8)
    assert res.status == 0
    assert np.all(np.diff(res.energies) >= 0)
    u = res.vectors.cpu().numpy()
    rows = np.random.default_rng(8).integers(0, g.N, 200)
    hu = o.sigma_rows(u, rows)
    for j in range(3):
        r = hu[j] - res.energies[j] * u[j, rows]
        # sampled residual entries cannot exceed the full residual norm
        assert np.abs(r).max() <= 10 * 1e-8


# ---------------------------------------------------------------------------
# error paths (the failure is made on the host or in the inputs; no GPU fault)


def test_error_duplicate_bad_string_and_nonfinite(torch, B):
    wl = W.make("t", 10, 3, 3, 30, 30, 0.3, seed=2)
    dup = wl.A.copy()
    dup[5] = dup[6]
    with pytest.raises(B.SbdError) as e:
        B.SBD(wl.norb, 3, 3, wl.h, wl.eri, dup, wl.B)
    assert e.value.code == -3
    bad = wl.B.copy()
    bad[3] = np.uint64(0b1111)
    with pytest.raises(B.SbdError) as e:
        B.SBD(wl.norb, 3, 3, wl.h, wl.eri, wl.A, bad)
    assert e.value.code == -2
    out_of_range = wl.A.copy()
    out_of_range[0] = np.uint64((1 << 10) | 3)
    with pytest.raises(B.SbdError) as e:
        B.SBD(wl.norb, 3, 3, wl.h, wl.eri, out_of_range, wl.B)
    assert e.value.code == -2
    h = wl.h.copy()
    h[1, 2] = np.nan
    with pytest.raises(B.SbdError) as e:
        B.SBD(wl.norb, 3, 3, h, wl.eri, wl.A, wl.B)
    assert e.value.code == -8


def test_error_more_strings_than_the_packed_lists_hold(torch, B):
    # the sigma lists pack a string index in 18 bits: 2^18 strings per spin is one too many
    norb, n = 22, 8
    A = W.all_strings(norb, n)[: 1 << 18]
    Bs = W.all_strings(norb, 1)[:3]
    h, eri = W.one_electron(norb, 3), W.two_electron(norb, 3)
    with pytest.raises(B.SbdError) as e:
        B.SBD(norb, n, 1, h, eri, A, Bs)
    assert e.value.code == -10  # SBD_ERR_UNSUPPORTED


def test_error_budget_and_failing_allocator(torch, B):
    wl = W.make("t", 10, 3, 3, 30, 30, 0.3, seed=2)
    with pytest.raises(B.SbdError) as e:
        B.SBD.from_workload(wl, hbm_budget_bytes=4096)
    assert e.value.code == -6
    # an allocator that fails on its 5th request
    calls = {"n": 0}
    import ctypes

    def alloc(ctx, nbytes, stream):
        calls["n"] += 1
        if calls["n"] >= 5:
            return None
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))

    def free(ctx, ptr, stream):
        torch.cuda.caching_allocator_delete(int(ptr))

    opts = B.sbd_default_options()
    fa, ff = B.ALLOC_FN(alloc), B.FREE_FN(free)
    opts.alloc, opts.free = fa, ff
    with pytest.raises(B.SbdError) as e:
        B.sbd_create(wl.norb, 3, 3, wl.h, wl.eri, wl.A, wl.B, opts, 0)
    assert e.value.code == -5
    torch.cuda.synchronize()


def test_not_converged_returns_estimates(torch, B, med_pair):
    wl, g, o = med_pair
    g2 = B.SBD.from_workload(wl, max_iter=2)
    res = g2.davidson(nroots=1, tol=1e-12)
    assert res.status == 1
    assert np.isfinite(res.energies[0]) and res.residuals[0] > 1e-12
    g2.close()


# ---------------------------------------------------------------------------
# full-size norb=29 workload (1e8 determinants), sampled rows against the oracle


@pytest.fixture(scope="module")
def cfg3_pair(torch, B, oracle_mod):
    wl = W.config("cfg3")
    g = B.SBD.from_workload(wl, max_subspace=wl.max_subspace)
    o = oracle_mod.Oracle.from_workload(wl)
    yield wl, g, o
    g.close()
    o.close()


def test_sigma_cfg3_full_size_sampled_rows(torch, B, cfg3_pair):
    wl, g, o = cfg3_pair
    x = W.random_vector(g.N, 100)[0]
    xt = torch.from_numpy(x).cuda()
    rows = np.random.default_rng(7).integers(0, g.N, 96)
    ref = o.sigma_rows(x, rows)[0]
    s64 = g.sigma(xt, "fp64").cpu().numpy()
    assert rel_maxnorm(s64[rows], ref) <= SIGMA_FP64_RTOL
    s2 = g.sigma(xt, "f32x2").cpu().numpy()
    assert rel_maxnorm(s2[rows], ref) <= SIGMA_FP64_RTOL
    assert rel_maxnorm(s2, s64) <= 1e-13
    s32 = g.sigma(xt.float(), "mixed").cpu().numpy()
    assert rel_maxnorm(s32[rows], ref) <= SIGMA_MIXED_RTOL


def test_solve_cfg3_mixed_residual_on_sampled_rows(torch, B, cfg3_pair):
    wl, g, o = cfg3_pair
    res = g.davidson(nroots=1, tol=wl.tol, precision="mixed")
    assert res.status == 0, res.report
    assert res.residuals[0] <= wl.tol
    u = res.vectors[0].cpu().numpy()
    assert abs(np.linalg.norm(u) - 1.0) <= 1e-10
    rows = np.random.default_rng(9).integers(0, g.N, 64)
    r = o.sigma_rows(u, rows)[0] - res.energies[0] * u[rows]
    # every entry of the residual is bounded by its norm (FP64-evaluated by the solver)
    assert np.abs(r).max() <= 2 * wl.tol
