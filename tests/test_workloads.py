"""The seeded input generator: structure of the drawn integrals and strings (no GPU)."""
import math

import numpy as np

from paper_2601_16637_gb300 import workloads as W


def test_integrals_symmetry_and_psd():
    norb = 7
    h = W.one_electron(norb, 3)
    eri = W.two_electron(norb, 3)
    assert np.array_equal(h, h.T)
    assert np.allclose(np.diag(h), -2.0 + 0.15 * np.arange(norb))
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (1, 0, 3, 2), (3, 2, 1, 0)]:
        assert np.allclose(eri, eri.transpose(perm), atol=1e-15)
    w = np.linalg.eigvalsh(eri.reshape(norb * norb, norb * norb))
    assert w.min() > -1e-12


def test_strings_are_valid_distinct_and_include_aufbau():
    for norb, n, k, lam in [(16, 5, 2000, 0.35), (12, 4, 100, 0.0), (40, 13, 500, 0.35)]:
        rng = np.random.default_rng(0)
        s = W.gumbel_top_k(norb, n, k, lam, rng)
        assert s.size == k and np.unique(s).size == k
        assert all(bin(int(x)).count("1") == n and int(x) >> norb == 0 for x in s)
        assert np.uint64((1 << n) - 1) in s


def test_full_space_enumeration():
    s = W.all_strings(9, 4)
    assert s.size == math.comb(9, 4) and np.unique(s).size == s.size


def test_low_orbital_bias():
    rng = np.random.default_rng(1)
    s = W.gumbel_top_k(16, 5, 300, 0.35, rng)
    mean_occ = np.mean([sum(p for p in range(16) if int(x) >> p & 1) for x in s])
    uniform = 5 * 15 / 2
    assert mean_occ < uniform


def test_deterministic_by_seed():
    a = W.config("cfg1")
    b = W.config("cfg1")
    assert np.array_equal(a.A, b.A) and np.array_equal(a.eri, b.eri)
    c = W.make("x", 16, 5, 5, 100, 100, 0.35, seed=1)
    d = W.make("x", 16, 5, 5, 100, 100, 0.35, seed=2)
    assert not np.array_equal(c.A, d.A)


def test_batched_workload_shapes():
    insts = W.batch_instances(6, seed=4)
    assert len(insts) == 6
    for w in insts:
        assert w.norb in (16, 20, 24, 26) and w.nalpha == w.nbeta == round(w.norb / 3)
        full = math.comb(w.norb, w.nalpha)
        assert 1 <= w.A.size <= min(5000, full) and 1 <= w.B.size <= min(5000, full)
        assert w.A.size >= min(500, full) and w.B.size >= min(500, full)
        assert len(set(w.A.tolist())) == w.A.size
        assert w.tol == 1e-4 and w.extra["tol_energy"] == 1e-6
    # own integrals per instance, reproducible
    same = [(a, b) for i, a in enumerate(insts) for b in insts[i + 1:] if a.norb == b.norb]
    assert all(not np.allclose(a.h, b.h) for a, b in same)
    again = W.batch_instances(6, seed=4)
    assert all(np.array_equal(a.A, b.A) and np.array_equal(a.eri, b.eri) for a, b in zip(insts, again))


def test_serving_trace_scales_arrivals_only():
    slow, fast = W.serving_trace(n=30, rate=1.0), W.serving_trace(n=30, rate=20.0)
    assert [s for _, s, _ in slow] == [s for _, s, _ in fast]
    t1 = np.array([t for t, _, _ in slow])
    t20 = np.array([t for t, _, _ in fast])
    assert np.all(np.diff(t1) > 0) and np.allclose(t1, 20.0 * t20)
    for _, spec, tol_e in fast:
        assert spec["norb"] in (24, 32, 40, 48, 58) and spec["nalpha"] == round(spec["norb"] / 3)
        assert 300 <= spec["nA"] <= 20000 and spec["nA"] == spec["nB"] and tol_e == 1e-6
