"""Seeded synthetic inputs for selected-basis diagonalization (SBD).

This module only draws inputs: one-electron integrals h_pq, two-electron
integrals (pq|rs) in chemists' notation, and the selected alpha/beta string
sets A and B.  It holds none of the Hamiltonian arithmetic, so both the CUDA
path and the CPU oracle can consume its output without sharing any of the
method's code.

The paper's own workload (Sec. IV: Fe4S4, 6,000 quantum-sampled 36-bit
configurations, 3.6e7 determinants) is not available; these generators stand
in for it with the same structure: a low-orbital-biased selected string set of
fixed popcount, dense 8-fold-symmetric integrals and a product space A x B.

Recipe (all numbers below are the workload definitions, not tunables):

* h: symmetric; diagonal eps_p = -2 + 0.15 p; upper triangle off the diagonal
  drawn N(0, (0.05 exp(-|p-q|/4))^2) and mirrored.
* (pq|rs) = sum_{L < 2 norb} B^L_pq B^L_rs with B^L symmetric, its upper
  triangle (diagonal included) iid N(0, 0.12^2) and mirrored.  The result is
  positive semi-definite as a (pq),(rs) matrix and 8-fold symmetric.
* strings: Gumbel-top-k sampling without replacement, the log-weight of a
  string being -lam * sum of its occupied orbital indices.  The draw is exact
  over the enumerated space when C(norb, n) <= 2^26; beyond that each string
  is drawn as a Gumbel-top-n over orbitals (Plackett-Luce) and duplicates are
  rejected, which is an approximation of the same bias.  The aufbau string
  (lowest n orbitals occupied) is always included.  Strings are returned in
  draw order (not sorted), so consumers exercise their own sorting.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

EXACT_ENUMERATION_LIMIT = 1 << 26

# stream tags for np.random.default_rng([seed, tag])
_TAG_H, _TAG_ERI, _TAG_A, _TAG_B = 0, 1, 2, 3


@dataclass
class Workload:
    """One SBD instance: integrals, string sets and solve parameters."""

    name: str
    norb: int
    nalpha: int
    nbeta: int
    h: np.ndarray            # [norb, norb] float64, symmetric
    eri: np.ndarray          # [norb, norb, norb, norb] float64, (pq|rs)
    A: np.ndarray            # [nA] uint64, alpha strings (draw order)
    B: np.ndarray            # [nB] uint64, beta strings (draw order)
    nroots: int = 1
    tol: float = 1e-8
    precision: str = "fp64"
    max_subspace: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def ndets(self) -> int:
        return int(self.A.size) * int(self.B.size)


def one_electron(norb: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, _TAG_H])
    h = np.zeros((norb, norb))
    for p in range(norb):
        h[p, p] = -2.0 + 0.15 * p
    iu = np.triu_indices(norb, k=1)
    sd = 0.05 * np.exp(-np.abs(iu[0] - iu[1]) / 4.0)
    h[iu] = rng.normal(0.0, 1.0, size=sd.size) * sd
    h[(iu[1], iu[0])] = h[iu]
    return h


def two_electron(norb: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, _TAG_ERI])
    nl = 2 * norb
    iu = np.triu_indices(norb)
    Bl = np.zeros((nl, norb, norb))
    for L in range(nl):
        v = rng.normal(0.0, 0.12, size=iu[0].size)
        Bl[L][iu] = v
        Bl[L][(iu[1], iu[0])] = v
    flat = Bl.reshape(nl, norb * norb)
    eri = flat.T @ flat
    return np.ascontiguousarray(eri.reshape(norb, norb, norb, norb))


def all_strings(norb: int, n: int) -> np.ndarray:
    """Every uint64 string with n of the low norb bits set (unsorted)."""
    if not (0 <= n <= norb <= 64):
        raise ValueError("need 0 <= n <= norb <= 64")
    # level[k] = strings over bits [0, m) with k bits set
    level = {0: np.zeros(1, dtype=np.uint64)}
    for m in range(norb):
        bit = np.uint64(1) << np.uint64(m)
        nxt = {}
        lo = max(0, n - (norb - m - 1))
        for k in range(lo, min(n, m + 1) + 1):
            parts = []
            if k in level:
                parts.append(level[k])
            if k - 1 in level:
                parts.append(level[k - 1] | bit)
            if parts:
                nxt[k] = np.concatenate(parts) if len(parts) > 1 else parts[0]
        level = nxt
    return level[n]


def _orbital_sum(strings: np.ndarray, norb: int) -> np.ndarray:
    tot = np.zeros(strings.size, dtype=np.float64)
    for p in range(norb):
        tot += p * ((strings >> np.uint64(p)) & np.uint64(1)).astype(np.float64)
    return tot


def gumbel_top_k(norb: int, n: int, k: int, lam: float, rng: np.random.Generator) -> np.ndarray:
    """k distinct strings, log-weight -lam * sum(occupied indices)."""
    total = math.comb(norb, n)
    aufbau = np.uint64((1 << n) - 1) if n < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    if k >= total:
        s = all_strings(norb, n)
        return s[rng.permutation(s.size)]
    if total <= EXACT_ENUMERATION_LIMIT:
        s = all_strings(norb, n)
        score = -lam * _orbital_sum(s, norb) + rng.gumbel(size=s.size)
        top = np.argpartition(-score, k - 1)[:k]
        top = top[np.argsort(-score[top], kind="stable")]
        out = s[top]
    else:
        seen: dict[int, None] = {}
        logw = -lam * np.arange(norb, dtype=np.float64)
        while len(seen) < k:
            batch = max(1024, 2 * (k - len(seen)))
            g = logw[None, :] + rng.gumbel(size=(batch, norb))
            occ = np.argpartition(-g, n - 1, axis=1)[:, :n]
            bits = (np.uint64(1) << occ.astype(np.uint64))
            strs = np.bitwise_or.reduce(bits, axis=1)
            for x in strs.tolist():
                if x not in seen:
                    seen[x] = None
                    if len(seen) == k:
                        break
        out = np.fromiter(seen.keys(), dtype=np.uint64, count=k)
    if not np.any(out == aufbau):
        out[-1] = aufbau
    return out


def make(name: str, norb: int, nalpha: int, nbeta: int, nA: int | None, nB: int | None,
         lam: float, seed: int, **solve) -> Workload:
    """Build one instance; nA/nB = None selects the full string space."""
    h = one_electron(norb, seed)
    eri = two_electron(norb, seed)
    ra = np.random.default_rng([seed, _TAG_A])
    rb = np.random.default_rng([seed, _TAG_B])
    fullA, fullB = math.comb(norb, nalpha), math.comb(norb, nbeta)
    A = gumbel_top_k(norb, nalpha, fullA if nA is None else nA, lam, ra)
    B = gumbel_top_k(norb, nbeta, fullB if nB is None else nB, lam, rb)
    return Workload(name, norb, nalpha, nbeta, h, eri, A, B, **solve)


# The configurations the library is exercised and measured on.
#   cfg1: full space norb=8, 4+4 electrons (4,900 determinants), 1 root, tol 1e-10
#   cfg2: norb=16, 5+5, |A|=|B|=2,000 (4.0e6 determinants), lam 0.35, 3 roots, tol 1e-8
#   cfg3: norb=29, 10+10, |A|=|B|=10,000 (1.0e8 determinants), lam 0.25, mixed precision,
#         1 root, subspace <= 24
#   cfg3-6000: cfg3 with |A|=|B|=6,000 (3.6e7 determinants)
CONFIGS = {
    "cfg1": dict(norb=8, nalpha=4, nbeta=4, nA=None, nB=None, lam=0.0, seed=0,
                 nroots=1, tol=1e-10, precision="fp64"),
    "cfg2": dict(norb=16, nalpha=5, nbeta=5, nA=2000, nB=2000, lam=0.35, seed=1,
                 nroots=3, tol=1e-8, precision="fp64"),
    "cfg3": dict(norb=29, nalpha=10, nbeta=10, nA=10000, nB=10000, lam=0.25, seed=2,
                 nroots=1, tol=1e-6, precision="mixed", max_subspace=24),
    # the norb=29 workload at |A|=|B|=6,000 (3.6e7 determinants, the paper's determinant count):
    # same kernels and launch shapes, a smaller footprint for profiler captures
    "cfg3-6000": dict(norb=29, nalpha=10, nbeta=10, nA=6000, nB=6000, lam=0.25, seed=2,
                      nroots=1, tol=1e-6, precision="mixed", max_subspace=24),
    # a job from the top of the serving range (norb 58, 19+19 electrons, |A| = |B| = 15,000: 2.25e8
    # determinants), for profiling the large-norb kernels (with --strings for a smaller capture)
    "serve-top": dict(norb=58, nalpha=19, nbeta=19, nA=15000, nB=15000, lam=0.35, seed=77,
                      nroots=1, tol=1e-4, precision="mixed", max_subspace=20),
}


def batch_instances(n: int = 64, seed: int = 4, lam: float = 0.35, tol: float = 1e-4,
                    tol_energy: float = 1e-6) -> list[Workload]:
    """The batched workload: n independent instances, norb uniform in {16, 20, 24, 26},
    nalpha = nbeta = round(norb / 3), |A| and |B| uniform in [500, 5000] (clamped to the full
    string space), each with its own seeded integrals.  tol / tol_energy: the residual and
    Ritz-value-change thresholds that stand for "1e-6 Ha" (a residual of 1e-4 bounds the
    eigenvalue error by about 1e-8 / gap)."""
    rng = np.random.default_rng([seed, 200])
    out = []
    for i in range(n):
        norb = int(rng.choice([16, 20, 24, 26]))
        nel = int(round(norb / 3))
        full = math.comb(norb, nel)
        nA = min(int(rng.integers(500, 5001)), full)
        nB = min(int(rng.integers(500, 5001)), full)
        wl = make(f"batch{n}-{i}", norb, nel, nel, nA, nB, lam, seed=1000 * seed + i, nroots=1, tol=tol,
                  precision="mixed")
        wl.extra["tol_energy"] = tol_energy
        out.append(wl)
    return out


def serving_trace(n: int = 200, rate: float = 20.0, seed: int = 5, lam: float = 0.35, tol: float = 1e-4,
                  tol_energy: float = 1e-6, max_strings: int = 20000, min_strings: int = 300,
                  norbs=(24, 32, 40, 48, 58)) -> list[tuple[float, Workload]]:
    """The serving workload: a finite Poisson stream of n jobs at `rate` per second.  Each job has
    norb uniform in `norbs`, nalpha = nbeta = round(norb / 3), |A| = |B| log-uniform in
    [min_strings, max_strings] and its own seeded integrals.  Returns (arrival time s, job) pairs
    in arrival order; the instances are built lazily by the caller through `make_job`."""
    rng = np.random.default_rng([seed, 300])
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        norb = int(rng.choice(list(norbs)))
        nel = int(round(norb / 3))
        ns = int(round(math.exp(rng.uniform(math.log(min_strings), math.log(max_strings)))))
        ns = min(ns, math.comb(norb, nel))
        spec = dict(name=f"serve-{i}", norb=norb, nalpha=nel, nbeta=nel, nA=ns, nB=ns, lam=lam,
                    seed=1000 * seed + i, nroots=1, tol=tol, precision="mixed")
        out.append((t, spec, tol_energy))
    return out


def make_job(spec: dict, tol_energy: float) -> Workload:
    """Builds one serving job from its spec (see serving_trace)."""
    wl = make(**spec)
    wl.extra["tol_energy"] = tol_energy
    return wl


def config(name: str, **override) -> Workload:
    spec = dict(CONFIGS[name])
    spec.update(override)
    return make(name, **spec)


def random_vector(n: int, seed: int, nvec: int = 1) -> np.ndarray:
    """Normalised N(0,1) test amplitudes, shape [nvec, n] float64."""
    rng = np.random.default_rng([seed, 100])
    x = rng.normal(size=(nvec, n))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x
