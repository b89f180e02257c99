"""Shared helpers of the GPU tests: instances, the oracle, tolerances."""
import numpy as np

from paper_2601_16637_gb300 import workloads as W

# FP64 sigma: relative max-norm error bound (sigma compared on the same inputs)
SIGMA_FP64_RTOL = 1e-12
# FP64 eigenvalues against the oracle / dense diagonalisation, in Hartree
EIG_FP64_ATOL = 1e-8
# mixed-precision solve (FP32 sigma + FP64 defect correction) against FP64, in Hartree
EIG_MIXED_ATOL = 1e-6
# mixed sigma alone: FP32 amplitudes/integrals, FP32 sums per excitation list
SIGMA_MIXED_RTOL = 2e-5


def medium(norb=14, n=4, nA=331, nB=297, lam=0.3, seed=5, nb=None):
    """Several staging tiles and ragged tails in both string sets."""
    return W.make("medium", norb, n, n if nb is None else nb, nA, nB, lam, seed)


def rel_maxnorm(got, ref):
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max() / max(np.abs(np.asarray(ref)).max(), 1e-300))
