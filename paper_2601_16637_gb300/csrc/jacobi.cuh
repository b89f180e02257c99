// Symmetric eigensolver for the small projected matrices of Davidson (paper
// Sec. II-C, Rayleigh-Ritz step), shared by the single-instance solver and the
// batched engine.
#pragma once

namespace sbd {

constexpr int kJacobiMax = 64;  // largest matrix order

// Eigenpairs of the symmetric k x k matrix T (upper and lower parts averaged)
// by parallel-order Jacobi rotations in one CTA.  Each sweep runs k-1 rounds
// of the round-robin (tournament) pairing of the k indices; the k/2 pairs of
// a round are disjoint, so their rotations commute and are applied together:
// first to the columns of A and of the eigenvector matrix V, then to the rows
// of A.  A rotation is skipped when |a_pq| is negligible against both
// diagonal entries; the sweeps stop when a sweep rotates nothing.
// evals ascending; Y[a*ldy + j] is component a of eigenvector j.
// js: 2 k^2 doubles of shared memory supplied by the caller; k <= kJacobiMax.
__device__ inline void jacobi_eig(const double *__restrict__ T, int ldt, int k, double *evals, double *Y, int ldy,
                                  double *js)
{
    double *A = js, *V = js + k * k;
    __shared__ int pos[kJacobiMax + 1];
    __shared__ int pp[kJacobiMax / 2 + 1], qq[kJacobiMax / 2 + 1];
    __shared__ double cc[kJacobiMax / 2 + 1], ss[kJacobiMax / 2 + 1];
    __shared__ int rotated;
    __shared__ int ord[kJacobiMax];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < k * k; t += nt) {
        const int i = t / k, j = t % k;
        A[t] = 0.5 * (T[i * ldt + j] + T[j * ldt + i]);
        V[t] = i == j ? 1.0 : 0.0;
    }
    const int m = (k + 1) & ~1;  // even number of players (index k is a bye when k is odd)
    const int half = m / 2;
    for (int i = tid; i < m; i += nt) pos[i] = i;
    __syncthreads();
    for (int sweep = 0; sweep < 60 && k > 1; ++sweep) {
        if (tid == 0) rotated = 0;
        for (int round = 0; round < m - 1; ++round) {
            if (tid < half) {
                int p = pos[tid], q = pos[m - 1 - tid];
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                double c = 1.0, s = 0.0;
                if (q < k) {
                    const double apq = A[p * k + q], app = A[p * k + p], aqq = A[q * k + q];
                    const double g = 100.0 * fabs(apq);
                    if (apq != 0.0 && !(fabs(app) + g == fabs(app) && fabs(aqq) + g == fabs(aqq))) {
                        const double theta = (aqq - app) / (2.0 * apq);
                        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                        rotated = 1;
                    } else if (apq != 0.0) {
                        A[p * k + q] = 0.0;  // negligible: set to zero, as the sequential method does
                        A[q * k + p] = 0.0;
                    }
                }
                pp[tid] = p;
                qq[tid] = q;
                cc[tid] = c;
                ss[tid] = s;
            }
            __syncthreads();
            // columns p, q of A and V
            for (int w = tid; w < half * k; w += nt) {
                const int t = w / k, r = w % k;
                const int p = pp[t], q = qq[t];
                if (q < k && ss[t] != 0.0) {
                    const double c = cc[t], s = ss[t];
                    const double arp = A[r * k + p], arq = A[r * k + q];
                    A[r * k + p] = c * arp - s * arq;
                    A[r * k + q] = s * arp + c * arq;
                    const double vrp = V[r * k + p], vrq = V[r * k + q];
                    V[r * k + p] = c * vrp - s * vrq;
                    V[r * k + q] = s * vrp + c * vrq;
                }
            }
            __syncthreads();
            // rows p, q of A
            for (int w = tid; w < half * k; w += nt) {
                const int t = w / k, r = w % k;
                const int p = pp[t], q = qq[t];
                if (q < k && ss[t] != 0.0) {
                    const double c = cc[t], s = ss[t];
                    const double apr = A[p * k + r], aqr = A[q * k + r];
                    A[p * k + r] = c * apr - s * aqr;
                    A[q * k + r] = s * apr + c * aqr;
                }
            }
            __syncthreads();
            // next pairing: position 0 stays, the others rotate by one
            if (tid == 0) {
                const int last = pos[m - 1];
                for (int i = m - 1; i > 1; --i) pos[i] = pos[i - 1];
                pos[1] = last;
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();
        if (!any) break;
    }
    if (tid == 0) {
        for (int i = 0; i < k; ++i) ord[i] = i;
        for (int i = 0; i < k; ++i)
            for (int j = i + 1; j < k; ++j)
                if (A[ord[j] * k + ord[j]] < A[ord[i] * k + ord[i]]) {
                    const int t = ord[i];
                    ord[i] = ord[j];
                    ord[j] = t;
                }
    }
    __syncthreads();
    for (int t = tid; t < k * k; t += nt) {
        const int a = t / k, j = t % k;
        Y[a * ldy + j] = V[a * k + ord[j]];
    }
    for (int j = tid; j < k; j += nt) evals[j] = A[ord[j] * k + ord[j]];
}

}  // namespace sbd
