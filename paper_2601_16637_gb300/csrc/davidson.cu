// Block Davidson on the device (paper Sec. II-C, with the damped diagonal
// preconditioner of Sec. II-E and the stopping tests of Sec. II-G).
//
// Per iteration: Rayleigh-Ritz on the projected matrix T = V^T W (parallel
// Jacobi in one CTA), one fused pass for the Ritz vectors U = V Y, HU = W Y,
// the residual norms and the preconditioned corrections
// t = r / (sign(d) max(|d|, delta)), d = Hd - theta (Eq. 7); block classical
// Gram-Schmidt against the basis, with a second pass when the first removed
// more than 1 - 1/sqrt(2) of the norm; and the sigma product of the new basis
// vectors.  A thick restart keeps the lowest Ritz vectors when the basis is
// full.
//
// All vectors, T, the Ritz quantities and every reduction are FP64 (two-stage
// reductions in a fixed order, so results are reproducible).  In mixed mode
// the sigma of new basis vectors uses FP32 amplitudes (SBD_MIXED, with the
// diagonal term taken from the FP64 vector); when the residual computed from
// that sigma stops improving, the Ritz vectors are multiplied by the FP64
// sigma (defect correction): their FP64 Rayleigh quotients and residuals
// decide convergence, the basis keeps the lowest Ritz vectors with exact W
// columns for the targets, and projected-matrix entries that pair an exact
// column with a mixed one use the exact column, so FP32 noise does not couple
// into the converged direction.
//
// The vector kernels are HBM-streaming: every thread keeps kLoad independent
// loads in flight before it consumes them.  On GB300 their FP64 multiply-adds,
// not HBM, set the pace (the FP64 pipe is ~1/64 of the FP32 pipe).  Solves that
// take FP64-accurate arithmetic from FP32 pairs (SBD_F32X2, and mixed solves
// refined that way) therefore form the Ritz combinations in pairs: each loaded
// FP64 value is split once on the integer pipe and feeds one pair product per
// combined vector on the FP32 pipe (48-bit accurate), and each result is
// rounded to FP64 once.  Dot products and axpys use each loaded value in a
// single product, where the split costs more than the FP64 multiply-add it
// replaces, so they stay on the FP64 pipe.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <type_traits>

#include "common.cuh"
#include "jacobi.cuh"
#include "pair.cuh"

namespace sbd {

namespace {

constexpr int kBlas = 256;    // threads per BLAS block
constexpr int kLoad = 8;      // loads each thread issues before using them
constexpr int kDotMax = 32;   // dot products per multi-dot launch
constexpr int kRitzMax = 16;  // vectors combined per launch
constexpr int kMaxSub = 64;   // largest subspace the Jacobi kernel takes
constexpr int kPart = kDotMax + 1;  // partial-sum slots per block (dots + one norm)

int blas_grid(const Ctx &c, int64_t N)
{
    int64_t g = (N + kBlas - 1) / kBlas;
    int64_t cap = (int64_t)4 * (c.num_sms > 0 ? c.num_sms : 152);
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T s = T(0);
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;  // valid in thread 0
}

// partial[b*kPart + a] = sum over block b's elements of X[a][i] y[i] (a < k <= kDotMax);
// with NORM also partial[b*kPart + kDotMax] = sum y[i]^2
template <bool NORM, int KB>
__global__ void __launch_bounds__(kBlas, KB <= 16 ? 4 : 2) mdot_partial(const double *__restrict__ X, int64_t ldx, int k,
                                                      const double *__restrict__ y, int64_t N, double *partial)
{
    __shared__ double red[kBlas / 32];
    double acc[KB];
#pragma unroll
    for (int a = 0; a < KB; ++a) acc[a] = 0.0;
    double an = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kBlas + threadIdx.x; i < N; i += (int64_t)gridDim.x * kBlas) {
        const double yi = y[i];
        if (NORM) an += yi * yi;
#pragma unroll
        for (int a0 = 0; a0 < KB; a0 += kLoad) {
            if (a0 < k) {
                double x[kLoad];
#pragma unroll
                for (int u = 0; u < kLoad; ++u) x[u] = (a0 + u < k) ? X[(a0 + u) * ldx + i] : 0.0;
#pragma unroll
                for (int u = 0; u < kLoad; ++u) acc[a0 + u] += x[u] * yi;
            }
        }
    }
#pragma unroll
    for (int a = 0; a < KB; ++a)
        if (a < k) {  // k is uniform over the block
            const double s = block_sum(acc[a], red);
            if (threadIdx.x == 0) partial[blockIdx.x * kPart + a] = s;
        }
    if (NORM) {
        const double s = block_sum(an, red);
        if (threadIdx.x == 0) partial[blockIdx.x * kPart + kDotMax] = s;
    }
}

// The same sums in FP32 pairs (48-bit operands, FP32 pipe; one FP64 rounding per block sum), for
// the pair-arithmetic solves.  blockIdx.y picks a chunk of kPairChunk basis vectors, so that the
// accumulators stay few (the FP64 form is bound by the FP64 pipe, one multiply-add per element and
// basis vector; this one runs near the HBM rate).  With NORM, chunk 0 also sums y^2 in FP64.
constexpr int kPairChunk = 8;
template <bool NORM>
__global__ void __launch_bounds__(kBlas) mdot_pair_partial(const double *__restrict__ X, int64_t ldx, int k,
                                                           const double *__restrict__ y, int64_t N, double *partial)
{
    __shared__ double red[kBlas / 32];
    const int a0 = blockIdx.y * kPairChunk;
    const int kc = min(kPairChunk, k - a0);
    X += a0 * ldx;
    const bool nrm = NORM && blockIdx.y == 0;
    F2 acc[kPairChunk];
#pragma unroll
    for (int a = 0; a < kPairChunk; ++a) acc[a] = F2(0.f);
    double an = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kBlas + threadIdx.x; i < N; i += (int64_t)gridDim.x * kBlas) {
        const double yi = y[i];
        if (nrm) an += yi * yi;
        const F2 ys = f2_split(yi);
        double x[kPairChunk];
#pragma unroll
        for (int u = 0; u < kPairChunk; ++u) x[u] = u < kc ? X[u * ldx + i] : 0.0;
#pragma unroll
        for (int u = 0; u < kPairChunk; ++u) f2_mac(acc[u], f2_split(x[u]), ys);
    }
#pragma unroll
    for (int a = 0; a < kPairChunk; ++a)
        if (a < kc) {  // kc is uniform over the block
            const double s = block_sum(f2_value(acc[a]), red);
            if (threadIdx.x == 0) partial[blockIdx.x * kPart + a0 + a] = s;
        }
    if (nrm) {
        const double s = block_sum(an, red);
        if (threadIdx.x == 0) partial[blockIdx.x * kPart + kDotMax] = s;
    }
}

// out1[a*st1] (and out2[a*st2] when given) = sum_b partial[b][a] for a < k;
// slot kDotMax (the norm) goes to *norm2 when given.  Fixed summation order.
__global__ void mdot_final(const double *partial, int nblocks, int k, double *out1, int64_t st1, double *out2,
                           int64_t st2, double *norm2)
{
    const int a = threadIdx.x;
    if (a < k) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[b * kPart + a];
        out1[a * st1] = s;
        if (out2) out2[a * st2] = s;
    } else if (a == kDotMax && norm2) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[b * kPart + kDotMax];
        *norm2 = s;
    }
}

// y -= sum_a coef[a] X[a] (a < k <= kMaxSub); with NORM, partial[b*kPart + kDotMax] = sum of the new y^2.
// PAIR: the sum over a in FP32 pairs, subtracted from y in FP64.
template <bool NORM, bool PAIR>
__global__ void __launch_bounds__(kBlas) maxpy_kernel(const double *__restrict__ X, int64_t ldx, int k,
                                                      const double *__restrict__ coef, double *y, int64_t N,
                                                      double *partial)
{
    __shared__ double cs[kMaxSub];
    __shared__ double red[kBlas / 32];
    F2 *cs2 = reinterpret_cast<F2 *>(cs);  // PAIR: the coefficients as pairs (8 bytes each)
    for (int a = threadIdx.x; a < kMaxSub; a += kBlas) {
        const double v = a < k ? coef[a] : 0.0;
        if (PAIR) cs2[a] = f2_split(v);
        else cs[a] = v;
    }
    __syncthreads();
    double an = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kBlas + threadIdx.x; i < N; i += (int64_t)gridDim.x * kBlas) {
        using Acc = typename std::conditional<PAIR, F2, double>::type;
        Acc s = Acc(0.f);
        for (int a0 = 0; a0 < k; a0 += kLoad) {
            double x[kLoad];
#pragma unroll
            for (int u = 0; u < kLoad; ++u) x[u] = (a0 + u < k) ? X[(a0 + u) * ldx + i] : 0.0;
#pragma unroll
            for (int u = 0; u < kLoad; ++u) {
                const int a = min(a0 + u, kMaxSub - 1);
                if constexpr (PAIR) f2_mac(s, cs2[a], f2_split(x[u]));
                else s += cs[a] * x[u];
            }
        }
        double sv;
        if constexpr (PAIR) sv = f2_value(s);
        else sv = s;
        const double yn = y[i] - sv;
        y[i] = yn;
        if (NORM) an += yn * yn;
    }
    if (NORM) {
        const double s = block_sum(an, red);
        if (threadIdx.x == 0) partial[blockIdx.x * kPart + kDotMax] = s;
    }
}

// out[j] = sum_a Y[a*ldy + j] X[a] and hout[j] = sum_a Y[a*ldy + j] H[a] for j < m <= kRitzMax, a < k.
// With RITZ (the Ritz step), also: r = hout - theta[j] out, partial[b*kPart + j] = sum r^2 and the
// preconditioned correction tc[j] = r / (sign(d) max(|d|, delta)), d = hd - theta[j].
// PAIR: the sums over a in FP32 pairs, one FP64 rounding per output element.
template <bool RITZ, int M, bool PAIR>
__global__ void __launch_bounds__(kBlas) combine_kernel(const double *__restrict__ X, const double *__restrict__ H,
                                                        int64_t ldx, int k, const double *__restrict__ Y, int ldy,
                                                        int m, double *out, double *hout, int64_t ldo,
                                                        const double *__restrict__ theta,
                                                        const double *__restrict__ hd, double delta, double *tc,
                                                        double *partial, int64_t N)
{
    __shared__ double ys[kMaxSub * kRitzMax];
    __shared__ double th[kRitzMax];
    __shared__ double red[kBlas / 32];
    F2 *ys2 = reinterpret_cast<F2 *>(ys);  // PAIR: the same coefficients as pairs (8 bytes each)
    for (int t = threadIdx.x; t < k * m; t += kBlas) {
        const double v = Y[(t / m) * ldy + (t % m)];
        if (PAIR) ys2[t] = f2_split(v);
        else ys[t] = v;
    }
    if (RITZ)
        for (int j = threadIdx.x; j < m; j += kBlas) th[j] = theta[j];
    __syncthreads();
    using Acc = typename std::conditional<PAIR, F2, double>::type;
    double racc[M];
#pragma unroll
    for (int j = 0; j < M; ++j) racc[j] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kBlas + threadIdx.x; i < N; i += (int64_t)gridDim.x * kBlas) {
        Acc u[M], hu[M];
#pragma unroll
        for (int j = 0; j < M; ++j) u[j] = hu[j] = Acc(0.f);
        for (int a0 = 0; a0 < k; a0 += kLoad / 2) {
            double x[kLoad / 2], h[kLoad / 2];
#pragma unroll
            for (int q = 0; q < kLoad / 2; ++q) {
                const bool ok = a0 + q < k;
                x[q] = ok ? X[(a0 + q) * ldx + i] : 0.0;
                h[q] = ok ? H[(a0 + q) * ldx + i] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < kLoad / 2; ++q) {
                // coefficient rows a >= k were never written (stale shared memory): skip, do not
                // multiply by the zero-filled x, h (a stale NaN or infinity would survive that)
                if (a0 + q >= k) continue;
                const int a = a0 + q;
                if constexpr (PAIR) {
                    const F2 xs = f2_split(x[q]), hs = f2_split(h[q]);
#pragma unroll
                    for (int j = 0; j < M; ++j)
                        if (j < m) {
                            f2_mac(u[j], ys2[a * m + j], xs);
                            f2_mac(hu[j], ys2[a * m + j], hs);
                        }
                } else {
#pragma unroll
                    for (int j = 0; j < M; ++j)
                        if (j < m) {
                            u[j] += ys[a * m + j] * x[q];
                            hu[j] += ys[a * m + j] * h[q];
                        }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < M; ++j)
            if (j < m) {
                double uj, huj;
                if constexpr (PAIR) {
                    uj = f2_value(u[j]);
                    huj = f2_value(hu[j]);
                } else {
                    uj = u[j];
                    huj = hu[j];
                }
                out[j * ldo + i] = uj;
                hout[j * ldo + i] = huj;
                if (RITZ) {
                    const double r = huj - th[j] * uj;
                    racc[j] += r * r;
                    const double d = hd[i] - th[j];
                    tc[j * ldo + i] = r * precond_factor(d, delta);
                }
            }
    }
    if (RITZ) {
#pragma unroll
        for (int j = 0; j < M; ++j)
            if (j < m) {
                const double s = block_sum(racc[j], red);
                if (threadIdx.x == 0) partial[blockIdx.x * kPart + j] = s;
            }
    }
}

// The Ritz step of one root in FP32 pairs (combine_kernel<true, 1, true>) and, from the same loaded
// and split basis values, the first Gram-Schmidt projections of the new correction:
// partial2[b*kPart + a] = sum over block b of X[a] . tc (a < k <= KB), partial2[b*kPart + kDotMax] =
// tc . tc.  A block works on tiles of kBlas elements: each thread parks its element's split X[a]
// and its split tc in shared memory ([KB + 1][kBlas] pairs, dynamic), then warp w sums the products
// of basis vectors a = w, w + 8, ... over the tile (a few accumulators per thread instead of KB, so
// three blocks fit an SM).  A separate pass would read the basis from HBM again.
template <int KB>
__global__ void __launch_bounds__(kBlas, 3) ritz_dots_kernel(const double *__restrict__ X,
                                                             const double *__restrict__ H, int64_t ldx, int k,
                                                             const double *__restrict__ Y, double *out, double *hout,
                                                             const double *__restrict__ theta,
                                                             const double *__restrict__ hd, double delta, double *tc,
                                                             double *partial, double *partial2, int64_t N)
{
    static_assert(KB % (kBlas / 32) == 0, "basis vectors are dealt to the warps in equal numbers");
    constexpr int kWarps = kBlas / 32, kPerWarp = KB / kWarps;
    extern __shared__ F2 xsh[];  // [KB][kBlas] split basis values, then [kBlas] split corrections
    F2 *tsh = xsh + KB * kBlas;
    __shared__ F2 ys2[KB];
    __shared__ double red[kBlas / 32];
    __shared__ double wsum[KB];
    for (int a = threadIdx.x; a < KB; a += kBlas) ys2[a] = a < k ? f2_split(Y[a * kMaxSub]) : F2(0.f);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double th = theta[0];
    double racc = 0.0, nacc = 0.0;
    F2 dacc[kPerWarp];
#pragma unroll
    for (int j = 0; j < kPerWarp; ++j) dacc[j] = F2(0.f);
    for (int64_t t0 = (int64_t)blockIdx.x * kBlas; t0 < N; t0 += (int64_t)gridDim.x * kBlas) {  // uniform
        const int64_t i = t0 + threadIdx.x;
        const bool valid = i < N;
        F2 u(0.f), hu(0.f);
#pragma unroll 2
        for (int a0 = 0; a0 < k; a0 += kLoad / 2) {
            double x[kLoad / 2], h[kLoad / 2];
#pragma unroll
            for (int q = 0; q < kLoad / 2; ++q) {
                const bool ok = a0 + q < k && valid;
                x[q] = ok ? X[(a0 + q) * ldx + i] : 0.0;
                h[q] = ok ? H[(a0 + q) * ldx + i] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < kLoad / 2; ++q) {
                const int a = a0 + q;
                if (a < k) {
                    const F2 xs = f2_split(x[q]);
                    xsh[a * kBlas + threadIdx.x] = xs;
                    f2_mac(u, ys2[a], xs);
                    f2_mac(hu, ys2[a], f2_split(h[q]));
                }
            }
        }
        F2 ts(0.f);
        if (valid) {
            const double uj = f2_value(u), huj = f2_value(hu);
            out[i] = uj;
            hout[i] = huj;
            const double r = huj - th * uj;
            racc += r * r;
            const double t = r * precond_factor(hd[i] - th, delta);
            tc[i] = t;
            nacc += t * t;
            ts = f2_split(t);
        }
        tsh[threadIdx.x] = ts;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPerWarp; ++j) {
            const int a = warp + kWarps * j;
            if (a < k)
#pragma unroll
                for (int e = lane; e < kBlas; e += 32) f2_mac(dacc[j], xsh[a * kBlas + e], tsh[e]);
        }
        __syncthreads();  // the tile's shared memory is rewritten next
    }
    const double sr = block_sum(racc, red);
    if (threadIdx.x == 0) partial[blockIdx.x * kPart] = sr;
#pragma unroll
    for (int j = 0; j < kPerWarp; ++j) {
        double v = f2_value(dacc[j]);
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) wsum[warp + kWarps * j] = v;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < k; a += kBlas) partial2[blockIdx.x * kPart + a] = wsum[a];
    const double sn = block_sum(nacc, red);
    if (threadIdx.x == 0) partial2[blockIdx.x * kPart + kDotMax] = sn;
}
template <int KB>
constexpr int ritz_dots_smem()
{
    return (KB + 1) * kBlas * (int)sizeof(F2);
}

// partial[b*kPart + j] = sum over block b of (HU[j] - theta[j] U[j])^2, j < m <= kRitzMax
__global__ void __launch_bounds__(kBlas, 4) resid_partial(const double *__restrict__ U, const double *__restrict__ HU,
                                                       int64_t ld, int m, const double *__restrict__ theta,
                                                       int64_t N, double *partial)
{
    __shared__ double red[kBlas / 32];
    double acc[kRitzMax];
#pragma unroll
    for (int j = 0; j < kRitzMax; ++j) acc[j] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kBlas + threadIdx.x; i < N; i += (int64_t)gridDim.x * kBlas) {
#pragma unroll
        for (int j = 0; j < kRitzMax; ++j)
            if (j < m) {
                const double r = HU[j * ld + i] - theta[j] * U[j * ld + i];
                acc[j] += r * r;
            }
    }
#pragma unroll
    for (int j = 0; j < kRitzMax; ++j)
        if (j < m) {
            const double s = block_sum(acc[j], red);
            if (threadIdx.x == 0) partial[blockIdx.x * kPart + j] = s;
        }
}

// t = (hu - theta u) / (sign(d) max(|d|, delta)), d = Hd - theta   (Eq. 7; see precond_factor)
__global__ void precond_kernel(const double *__restrict__ u, const double *__restrict__ hu,
                               const double *__restrict__ hd, const double *__restrict__ theta, double delta,
                               double *t, int64_t N)
{
    const double th = *theta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = hd[i] - th;
        t[i] = (hu[i] - th * u[i]) * precond_factor(d, delta);
    }
}

// dst = src * s (dst may equal src)
__global__ void scale_kernel(const double *src, double *dst, double s, int64_t N)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] * s;
}

__global__ void set_kernel(double *x, int64_t idx, double v) { x[idx] = v; }

// two-stage argmin of x over indices not in excl[0..nexcl); ties -> lower index
__global__ void argmin_partial(const double *__restrict__ x, int64_t N, const int64_t *excl, int nexcl,
                               double *pv, int64_t *pi)
{
    __shared__ double sv[kBlas];
    __shared__ int64_t si[kBlas];
    double bv = INFINITY;
    int64_t bi = -1;
    for (int64_t i = blockIdx.x * (int64_t)kBlas + threadIdx.x; i < N; i += (int64_t)gridDim.x * kBlas) {
        bool skip = false;
        for (int e = 0; e < nexcl; ++e) skip |= excl[e] == i;
        if (skip) continue;
        const double v = x[i];
        if (bi < 0 || v < bv || (v == bv && i < bi)) {
            bv = v;
            bi = i;
        }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = kBlas / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double ov = sv[threadIdx.x + s];
            const int64_t oi = si[threadIdx.x + s];
            if (oi >= 0 && (si[threadIdx.x] < 0 || ov < sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < si[threadIdx.x]))) {
                sv[threadIdx.x] = ov;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = sv[0];
        pi[blockIdx.x] = si[0];
    }
}

// index of the largest |x_i| (ties -> lower index) in pi[blockIdx]
__global__ void argmaxabs_partial(const double *__restrict__ x, int64_t N, double *pv, int64_t *pi)
{
    __shared__ double sv[kBlas];
    __shared__ int64_t si[kBlas];
    double bv = -1.0;
    int64_t bi = -1;
    for (int64_t i = blockIdx.x * (int64_t)kBlas + threadIdx.x; i < N; i += (int64_t)gridDim.x * kBlas) {
        const double v = fabs(x[i]);
        if (v > bv) {
            bv = v;
            bi = i;
        }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = kBlas / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double ov = sv[threadIdx.x + s];
            const int64_t oi = si[threadIdx.x + s];
            if (oi >= 0 && (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < si[threadIdx.x]))) {
                sv[threadIdx.x] = ov;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = sv[0];
        pi[blockIdx.x] = si[0];
    }
}

__global__ void jacobi_kernel(const double *__restrict__ T, int ldt, int k, double *evals, double *Y, int ldy)
{
    extern __shared__ double js[];
    jacobi_eig(T, ldt, k, evals, Y, ldy, js);
}

// ---------------------------------------------------------------------------
// host side

struct Work {
    Ctx &c;
    cudaStream_t s;
    int64_t N;      // local vector length (this rank's rows in a sharded solve)
    int64_t off;    // global index of local element 0
    ShardCtx *sh;   // null: one process holds the whole vectors
    bool pair = false;  // Ritz combinations, basis dot products and updates summed in FP32 pairs
    int grid;
    double *partial = nullptr;  // [grid][kPart]
    double *partial2 = nullptr; // [grid][kPart]: projections from the fused Ritz pass
    double *dscal = nullptr;    // kMaxSub + 1 doubles: local dot products before the sum over ranks
    double *pv = nullptr;
    int64_t *pi = nullptr;
    std::vector<double> hpart;
    Work(Ctx &cc, int64_t n, int64_t o, ShardCtx *shard)
        : c(cc), s(cc.stream), N(n), off(o), sh(shard), grid(blas_grid(cc, n)) {}

    // sum over ranks of n host doubles (no-op without sharding)
    void allreduce(double *h, int n)
    {
        if (!sh || sh->world == 1 || n == 0) return;
        if (sh->comm.allreduce_sum(sh->comm.ctx, h, n) != 0) fail(SBD_ERR_CUDA, "allreduce_sum callback failed");
    }
    // replace n device doubles (stride st) by their sums over the ranks
    void globalize(double *dev, int64_t st, int n)
    {
        if (!sh || sh->world == 1 || n == 0 || !dev) return;
        std::vector<double> h((size_t)n);
        SBD_CUDA(cudaMemcpy2DAsync(h.data(), sizeof(double), dev, st * sizeof(double), sizeof(double), n,
                                   cudaMemcpyDeviceToHost, s));
        SBD_CUDA(cudaStreamSynchronize(s));
        allreduce(h.data(), n);
        SBD_CUDA(cudaMemcpy2DAsync(dev, st * sizeof(double), h.data(), sizeof(double), sizeof(double), n,
                                   cudaMemcpyHostToDevice, s));
    }

    // out1[a*st1] (and out2[a*st2]) = X[a] . y for a < k; with norm2, also y . y.  In a sharded solve
    // the local sums go to a contiguous scratch first, are summed over the ranks, then written out
    // (out1 and out2 may share an entry).
    // With pair, the products are summed in FP32 pairs unless fp64 asks for FP64 arithmetic.
    void dots(const double *X, int64_t ldx, int k, const double *y, double *out1, int64_t st1,
              double *out2 = nullptr, int64_t st2 = 0, double *norm2 = nullptr, bool fp64 = false)
    {
        const bool pr = pair && !fp64;
        if (sh && sh->world > 1) {
            double *tmp = dscal;  // kMaxSub + 1 doubles
            local_dots(X, ldx, k, y, tmp, 1, nullptr, 0, norm2 ? tmp + k : nullptr, pr);
            std::vector<double> h((size_t)k + 1, 0.0);
            const int n = k + (norm2 ? 1 : 0);
            SBD_CUDA(cudaMemcpyAsync(h.data(), tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
            SBD_CUDA(cudaStreamSynchronize(s));
            allreduce(h.data(), n);
            if (k) {
                SBD_CUDA(cudaMemcpy2DAsync(out1, st1 * sizeof(double), h.data(), sizeof(double), sizeof(double), k,
                                           cudaMemcpyHostToDevice, s));
                if (out2)
                    SBD_CUDA(cudaMemcpy2DAsync(out2, st2 * sizeof(double), h.data(), sizeof(double), sizeof(double), k,
                                               cudaMemcpyHostToDevice, s));
            }
            if (norm2) SBD_CUDA(cudaMemcpyAsync(norm2, h.data() + k, sizeof(double), cudaMemcpyHostToDevice, s));
            SBD_CUDA(cudaStreamSynchronize(s));  // h leaves scope
            return;
        }
        local_dots(X, ldx, k, y, out1, st1, out2, st2, norm2, pr);
    }
    template <bool NORM, bool PAIR>
    void launch_mdot(const double *Xa, int64_t ldx, int kb, const double *y)
    {
        if (PAIR) {
            const dim3 g(grid, std::max(1, (kb + kPairChunk - 1) / kPairChunk));
            mdot_pair_partial<NORM><<<g, kBlas, 0, s>>>(Xa, ldx, kb, y, N, partial);
            SBD_LAUNCH("mdot_pair_partial");
            return;
        }
        if (kb <= 8) mdot_partial<NORM, 8><<<grid, kBlas, 0, s>>>(Xa, ldx, kb, y, N, partial);
        else if (kb <= 16) mdot_partial<NORM, 16><<<grid, kBlas, 0, s>>>(Xa, ldx, kb, y, N, partial);
        else mdot_partial<NORM, kDotMax><<<grid, kBlas, 0, s>>>(Xa, ldx, kb, y, N, partial);
        SBD_LAUNCH("mdot_partial");
    }
    void local_dots(const double *X, int64_t ldx, int k, const double *y, double *out1, int64_t st1,
                    double *out2, int64_t st2, double *norm2, bool pr)
    {
        for (int a0 = 0; a0 < k || (a0 == 0 && norm2); a0 += kDotMax) {
            const int kb = std::min(kDotMax, k - a0);
            const bool nrm = norm2 && a0 == 0;
            const double *Xa = X + a0 * ldx;
            if (nrm) {
                if (pr) launch_mdot<true, true>(Xa, ldx, kb, y);
                else launch_mdot<true, false>(Xa, ldx, kb, y);
            } else {
                if (pr) launch_mdot<false, true>(Xa, ldx, kb, y);
                else launch_mdot<false, false>(Xa, ldx, kb, y);
            }
            mdot_final<<<1, kDotMax + 1, 0, s>>>(partial, grid, kb, out1 + a0 * st1, st1,
                                                 out2 ? out2 + a0 * st2 : nullptr, st2, nrm ? norm2 : nullptr);
            SBD_LAUNCH("mdot_final");
            if (k <= a0 + kDotMax) break;
        }
    }
    // y -= X coef; with norm2, also the new y . y
    void axpys(const double *X, int64_t ldx, int k, const double *coef, double *y, double *norm2 = nullptr)
    {
        if (norm2) {
            if (pair) maxpy_kernel<true, true><<<grid, kBlas, 0, s>>>(X, ldx, k, coef, y, N, partial);
            else maxpy_kernel<true, false><<<grid, kBlas, 0, s>>>(X, ldx, k, coef, y, N, partial);
            SBD_LAUNCH("maxpy_kernel");
            mdot_final<<<1, kDotMax + 1, 0, s>>>(partial, grid, 0, nullptr, 0, nullptr, 0, norm2);
            SBD_LAUNCH("mdot_final");
            globalize(norm2, 1, 1);
        } else {
            if (pair) maxpy_kernel<false, true><<<grid, kBlas, 0, s>>>(X, ldx, k, coef, y, N, partial);
            else maxpy_kernel<false, false><<<grid, kBlas, 0, s>>>(X, ldx, k, coef, y, N, partial);
            SBD_LAUNCH("maxpy_kernel");
        }
    }
    template <bool RITZ, bool PAIR>
    void launch_combine_p(const double *X, const double *H, int64_t ldx, int k, const double *Y, int ldy, int m,
                          double *out, double *hout, int64_t ldo, const double *theta, const double *hd, double delta,
                          double *tc)
    {
        if (m <= 1)
            combine_kernel<RITZ, 1, PAIR><<<grid, kBlas, 0, s>>>(X, H, ldx, k, Y, ldy, m, out, hout, ldo, theta, hd,
                                                                 delta, tc, partial, N);
        else if (m <= 4)
            combine_kernel<RITZ, 4, PAIR><<<grid, kBlas, 0, s>>>(X, H, ldx, k, Y, ldy, m, out, hout, ldo, theta, hd,
                                                                 delta, tc, partial, N);
        else if (m <= 8)
            combine_kernel<RITZ, 8, PAIR><<<grid, kBlas, 0, s>>>(X, H, ldx, k, Y, ldy, m, out, hout, ldo, theta, hd,
                                                                 delta, tc, partial, N);
        else
            combine_kernel<RITZ, kRitzMax, PAIR><<<grid, kBlas, 0, s>>>(X, H, ldx, k, Y, ldy, m, out, hout, ldo, theta,
                                                                        hd, delta, tc, partial, N);
        SBD_LAUNCH("combine_kernel");
    }
    template <bool RITZ>
    void launch_combine(const double *X, const double *H, int64_t ldx, int k, const double *Y, int ldy, int m,
                        double *out, double *hout, int64_t ldo, const double *theta, const double *hd, double delta,
                        double *tc)
    {
        if (pair) launch_combine_p<RITZ, true>(X, H, ldx, k, Y, ldy, m, out, hout, ldo, theta, hd, delta, tc);
        else launch_combine_p<RITZ, false>(X, H, ldx, k, Y, ldy, m, out, hout, ldo, theta, hd, delta, tc);
    }
    // out[j] = sum_a Y[a][j] X[a], hout[j] = sum_a Y[a][j] H[a], j < m, a < k
    void combine(const double *X, const double *H, int64_t ldx, int k, const double *Y, int ldy, int m, double *out,
                 double *hout, int64_t ldo)
    {
        for (int j0 = 0; j0 < m; j0 += kRitzMax) {
            const int mb = std::min(kRitzMax, m - j0);
            launch_combine<false>(X, H, ldx, k, Y + j0, ldy, mb, out + j0 * ldo, hout + j0 * ldo, ldo, nullptr,
                                  nullptr, 0.0, nullptr);
        }
    }
    // the Ritz step: U, HU, the corrections tc and the residual norms (host) for j < m <= kRitzMax.
    // With one root, FP32 pairs, one process and k <= kDotMax, the same pass also leaves the first
    // Gram-Schmidt projections V^T tc and tc . tc in partial2 (returns true; see proj_dots).
    bool ritz(const double *V, const double *W, int64_t ld, int k, const double *Y, int ldy, int m, double *U,
              double *HU, const double *theta, const double *hd, double delta, double *tc, double *rn_host)
    {
        const bool fuse = pair && m == 1 && k >= 1 && k <= kDotMax && (!sh || sh->world == 1) && partial2;
        if (!fuse) {
            launch_combine<true>(V, W, ld, k, Y, ldy, m, U, HU, ld, theta, hd, delta, tc);
            reduce_norms(m, rn_host);
            return false;
        }
        // every block of the fused pass resident at once: a grid-strided block left for a second
        // wave would run its whole share at a fraction of the occupancy
        if (k <= 8) launch_ritz_dots<8>(V, W, ld, k, Y, U, HU, theta, hd, delta, tc);
        else if (k <= 16) launch_ritz_dots<16>(V, W, ld, k, Y, U, HU, theta, hd, delta, tc);
        else if (k <= 24) launch_ritz_dots<24>(V, W, ld, k, Y, U, HU, theta, hd, delta, tc);
        else launch_ritz_dots<kDotMax>(V, W, ld, k, Y, U, HU, theta, hd, delta, tc);
        reduce_norms(m, rn_host, rgrid);
        return true;
    }
    int rgrid = 0;  // blocks of the last fused Ritz pass (partial sums in partial, partial2)
    template <int KB>
    void launch_ritz_dots(const double *V, const double *W, int64_t ld, int k, const double *Y, double *U,
                          double *HU, const double *theta, const double *hd, double delta, double *tc)
    {
        int per_sm = 0;
        SBD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ritz_dots_kernel<KB>, kBlas,
                                                               ritz_dots_smem<KB>()));
        rgrid = std::max(1, std::min(grid, per_sm * (c.num_sms > 0 ? c.num_sms : 152)));
        ritz_dots_kernel<KB><<<rgrid, kBlas, ritz_dots_smem<KB>(), s>>>(V, W, ld, k, Y, U, HU, theta, hd, delta, tc,
                                                                         partial, partial2, N);
        SBD_LAUNCH("ritz_dots_kernel");
    }
    // coef[a] = X[a] . tc (a < k) and *norm2 = tc . tc from the sums the fused Ritz pass left in
    // partial2; valid while X, k and tc are those of that pass
    void proj_dots(int k, double *coef, double *norm2)
    {
        mdot_final<<<1, kDotMax + 1, 0, s>>>(partial2, rgrid, k, coef, 1, nullptr, 0, norm2);
        SBD_LAUNCH("mdot_final");
    }
    // nb: blocks that wrote partial (0: the BLAS grid)
    void reduce_norms(int m, double *rn_host, int nb = 0)
    {
        if (nb <= 0) nb = grid;
        hpart.assign((size_t)nb * kPart, 0.0);
        SBD_CUDA(cudaMemcpyAsync(hpart.data(), partial, sizeof(double) * nb * kPart, cudaMemcpyDeviceToHost, s));
        SBD_CUDA(cudaStreamSynchronize(s));
        std::vector<double> acc((size_t)m, 0.0);
        for (int j = 0; j < m; ++j)
            for (int b = 0; b < nb; ++b) acc[j] += hpart[(size_t)b * kPart + j];
        allreduce(acc.data(), m);
        for (int j = 0; j < m; ++j) rn_host[j] = sqrt(acc[j]);
    }
    // residual norms ||HU_j - theta_j U_j||, j < m (theta on device)
    void resid_norms(const double *U, const double *HU, int64_t ld, int m, const double *theta, double *out_host)
    {
        resid_partial<<<grid, kBlas, 0, s>>>(U, HU, ld, m, theta, N, partial);
        SBD_LAUNCH("resid_partial");
        reduce_norms(m, out_host);
    }
    void scale(const double *src, double *dst, double f)
    {
        scale_kernel<<<grid, kBlas, 0, s>>>(src, dst, f, N);
        SBD_LAUNCH("scale_kernel");
    }
    // global index of the smallest entry not in excl (global indices); ties: lowest index
    int64_t argmin(const double *x, const std::vector<int64_t> &excl_global, int64_t *dexcl)
    {
        std::vector<int64_t> excl;
        for (int64_t g : excl_global)
            if (g >= off && g < off + N) excl.push_back(g - off);
        if (!excl.empty())
            SBD_CUDA(cudaMemcpyAsync(dexcl, excl.data(), excl.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        argmin_partial<<<grid, kBlas, 0, s>>>(x, N, dexcl, (int)excl.size(), pv, pi);
        SBD_LAUNCH("argmin_partial");
        std::vector<double> v(grid);
        std::vector<int64_t> id(grid);
        SBD_CUDA(cudaMemcpyAsync(v.data(), pv, sizeof(double) * grid, cudaMemcpyDeviceToHost, s));
        SBD_CUDA(cudaMemcpyAsync(id.data(), pi, sizeof(int64_t) * grid, cudaMemcpyDeviceToHost, s));
        SBD_CUDA(cudaStreamSynchronize(s));
        int64_t bi = -1;
        double bv = INFINITY;
        for (int b = 0; b < grid; ++b)
            if (id[b] >= 0 && (bi < 0 || v[b] < bv || (v[b] == bv && id[b] < bi))) {
                bv = v[b];
                bi = id[b];
            }
        if (bi >= 0) bi += off;
        return pick_global(bv, bi, false);
    }
    // the rank-local candidates (value, global index) of every rank, gathered through a sum over a
    // one-slot-per-rank array; the best by value (smallest, or largest with `largest`), ties by index
    int64_t pick_global(double &val, int64_t idx, bool largest)
    {
        if (!sh || sh->world == 1) return idx;
        const int W = sh->world;
        std::vector<double> buf((size_t)3 * W, 0.0);
        buf[(size_t)3 * sh->rank] = idx >= 0 ? 1.0 : 0.0;
        buf[(size_t)3 * sh->rank + 1] = idx >= 0 ? val : 0.0;
        buf[(size_t)3 * sh->rank + 2] = (double)idx;
        allreduce(buf.data(), 3 * W);
        int64_t bi = -1;
        double bv = 0.0;
        for (int r = 0; r < W; ++r) {
            if (buf[(size_t)3 * r] == 0.0) continue;
            const double v = buf[(size_t)3 * r + 1];
            const int64_t i = (int64_t)buf[(size_t)3 * r + 2];
            const bool better = largest ? v > bv : v < bv;
            if (bi < 0 || better || (v == bv && i < bi)) {
                bv = v;
                bi = i;
            }
        }
        val = bv;
        return bi;
    }
    double value_at_argmaxabs(const double *x)
    {
        argmaxabs_partial<<<grid, kBlas, 0, s>>>(x, N, pv, pi);
        SBD_LAUNCH("argmaxabs_partial");
        std::vector<double> v(grid);
        std::vector<int64_t> id(grid);
        SBD_CUDA(cudaMemcpyAsync(v.data(), pv, sizeof(double) * grid, cudaMemcpyDeviceToHost, s));
        SBD_CUDA(cudaMemcpyAsync(id.data(), pi, sizeof(int64_t) * grid, cudaMemcpyDeviceToHost, s));
        SBD_CUDA(cudaStreamSynchronize(s));
        int64_t bi = -1;
        double bv = -1.0;
        for (int b = 0; b < grid; ++b)
            if (id[b] >= 0 && (v[b] > bv || (v[b] == bv && id[b] < bi))) {
                bv = v[b];
                bi = id[b];
            }
        double val = 0.0;
        if (bi >= 0) {
            SBD_CUDA(cudaMemcpyAsync(&val, x + bi, sizeof(double), cudaMemcpyDeviceToHost, s));
            SBD_CUDA(cudaStreamSynchronize(s));
        }
        if (!sh || sh->world == 1) return val;
        // the signed value at the largest |x| over all ranks
        double a = fabs(val);
        const int64_t g = pick_global(a, bi >= 0 ? bi + off : -1, true);
        std::vector<double> h(1, (bi >= 0 && bi + off == g) ? val : 0.0);
        allreduce(h.data(), 1);
        return h[0];
    }
};

}  // namespace

int davidson(Ctx &c, int nroots, double tol, sbd_precision prec, double *energies, double *vecs, double *resid,
             sbd_report *rep, ShardCtx *shard)
{
    using clock = std::chrono::steady_clock;
    const auto t_start = clock::now();
    // a sharded solve holds only this rank's rows of every vector
    const int64_t N = shard ? shard->rows() * c.nB : c.N;
    const int64_t off = shard ? shard->row0() * c.nB : 0;
    const double *hd = c.hd + off;
    if (nroots < 1 || nroots > kRitzMax || nroots > c.N) fail(SBD_ERR_INVALID_ARG, "nroots must be in 1..min(16, N)");
    if (!(tol > 0.0)) fail(SBD_ERR_INVALID_ARG, "tol must be positive");
    const double delta = c.opt.delta > 0.0 ? c.opt.delta : 1e-4;
    const int max_iter = c.opt.max_iter > 0 ? c.opt.max_iter : 200;
    int max_sub = c.opt.max_subspace > 0 ? c.opt.max_subspace : std::max(24, 8 * nroots);
    max_sub = (int)std::min<int64_t>(std::min(max_sub, kMaxSub), c.N);
    if (max_sub < 2 * nroots && c.N >= 2 * nroots) max_sub = 2 * nroots;
    const bool mixed = prec == SBD_MIXED;
    // the FP64-accurate sigma: the solve's own precision, or for mixed solves the refinement precision
    const sbd_precision exact_prec =
        mixed ? (c.opt.refine_precision == SBD_F32X2 ? SBD_F32X2 : SBD_FP64) : prec;

    // keep the basis inside the budget: V, W, U, HU, corrections (+ FP32 copy)
    auto need = [&](int ms, int nk) {
        return ((size_t)(2 * ms + 2 * nk + nroots)) * (size_t)N * sizeof(double) + (mixed ? (size_t)N * 4 : 0) +
               (1u << 22);
    };
    auto keep_for = [&](int ms) {
        if (c.opt.restart_keep > 0) return std::max(nroots, std::min(ms - nroots, c.opt.restart_keep));
        return std::max(nroots, std::min(ms - nroots, std::max(2 * nroots, ms / 3)));
    };
    int nkeep = keep_for(max_sub);
    if (c.opt.hbm_budget_bytes) {
        while (max_sub > 2 * nroots && c.bytes_held + need(max_sub, nkeep) > c.opt.hbm_budget_bytes) {
            --max_sub;
            nkeep = keep_for(max_sub);
        }
    }
    sbd_report r{};
    r.status = SBD_OK;
    SBD_CUDA(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(2 * sizeof(double) * kMaxSub * kMaxSub)));
    SBD_CUDA(cudaFuncSetAttribute(ritz_dots_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ritz_dots_smem<16>()));
    SBD_CUDA(cudaFuncSetAttribute(ritz_dots_kernel<24>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ritz_dots_smem<24>()));
    SBD_CUDA(cudaFuncSetAttribute(ritz_dots_kernel<kDotMax>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ritz_dots_smem<kDotMax>()));

    Work w(c, N, off, shard);
    w.pair = prec == SBD_F32X2 || (mixed && exact_prec == SBD_F32X2);
    std::vector<void *> owned;
    auto grab = [&](size_t bytes) {
        void *p = dalloc(c, bytes);
        owned.push_back(p);
        return p;
    };
    int status = SBD_OK;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    try {
        double *V = (double *)grab((size_t)max_sub * N * sizeof(double));
        double *W = (double *)grab((size_t)max_sub * N * sizeof(double));
        double *U = (double *)grab((size_t)nkeep * N * sizeof(double));
        double *HU = (double *)grab((size_t)nkeep * N * sizeof(double));
        double *TC = (double *)grab((size_t)nroots * N * sizeof(double));
        float *c32 = mixed ? (float *)grab((size_t)N * sizeof(float)) : nullptr;
        double *T = (double *)grab(sizeof(double) * kMaxSub * kMaxSub);
        double *Y = (double *)grab(sizeof(double) * kMaxSub * kMaxSub);
        double *theta = (double *)grab(sizeof(double) * kMaxSub);
        double *coef = (double *)grab(sizeof(double) * kMaxSub);
        double *dscr = (double *)grab(sizeof(double) * kMaxSub);
        int64_t *dexcl = (int64_t *)grab(sizeof(int64_t) * (kRitzMax + 1));
        w.partial = (double *)grab(sizeof(double) * (size_t)w.grid * kPart);
        w.partial2 = (double *)grab(sizeof(double) * (size_t)w.grid * kPart);
        w.pv = (double *)grab(sizeof(double) * w.grid);
        w.pi = (int64_t *)grab(sizeof(int64_t) * w.grid);
        w.dscal = (double *)grab(sizeof(double) * (kMaxSub + 1));
        const int64_t ld = N;
        SBD_CUDA(cudaEventCreate(&ev0));
        SBD_CUDA(cudaEventCreate(&ev1));
        double sigma_ms = 0.0;

        // exact[a]: W column a came from the FP64 sigma (always, in FP64 mode)
        std::vector<char> exact(kMaxSub, mixed ? 0 : 1);
        auto sigma_cols = [&](int b0, int nb, bool fp64) {
            SBD_CUDA(cudaEventRecord(ev0, w.s));
            for (int b = b0; b < b0 + nb; ++b) {
                if (!fp64) {
                    to_float(V + b * ld, c32, N, w.s);
                    if (shard) ring_sigma(*shard, c, c32, W + b * ld, SBD_MIXED, w.s, V + b * ld);
                    else sigma_apply(c, c32, W + b * ld, SBD_MIXED, w.s, V + b * ld);
                    r.sigma_mixed++;
                } else {
                    if (shard) ring_sigma(*shard, c, V + b * ld, W + b * ld, exact_prec, w.s);
                    else sigma_apply(c, V + b * ld, W + b * ld, exact_prec, w.s);
                    r.sigma_fp64++;
                }
                exact[b] = fp64;
            }
            SBD_CUDA(cudaEventRecord(ev1, w.s));
            SBD_CUDA(cudaEventSynchronize(ev1));
            float ms = 0.f;
            SBD_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
            sigma_ms += ms;
        };
        // column b of T (and its mirror row) against V[0..kk): T[a][b] = V[a].W[b].  Where one of
        // the pair has an FP64-exact W column and the other does not, the exact one is used,
        // T[a][b] = W[a].V[b], so that mixed-precision noise never couples into exact columns.
        auto extend_T = [&](int b, int kk) {
            w.dots(V, ld, kk, W + b * ld, T + b, kMaxSub, T + b * kMaxSub, 1);
            if (!exact[b])
                for (int a = 0; a < kk; ++a)
                    if (exact[a] && a != b)
                        w.dots(W + a * ld, 0, 1, V + b * ld, T + a * kMaxSub + b, 1, T + b * kMaxSub + a, 1);
        };
        auto rebuild_T = [&](int kk) {
            SBD_CUDA(cudaMemsetAsync(T, 0, sizeof(double) * kMaxSub * kMaxSub, w.s));
            for (int b = 0; b < kk; ++b)
                if (!exact[b]) extend_T(b, kk);
            for (int b = 0; b < kk; ++b)
                if (exact[b]) w.dots(V, ld, kk, W + b * ld, T + b, kMaxSub, T + b * kMaxSub, 1);
        };
        // V' = V Y[:, :nk], W' = W Y[:, :nk] through the U/HU staging buffers
        auto compress = [&](int kk, int nk) {
            w.combine(V, W, ld, kk, Y, kMaxSub, nk, U, HU, ld);
            SBD_CUDA(cudaMemcpyAsync(V, U, (size_t)nk * N * sizeof(double), cudaMemcpyDeviceToDevice, w.s));
            SBD_CUDA(cudaMemcpyAsync(W, HU, (size_t)nk * N * sizeof(double), cudaMemcpyDeviceToDevice, w.s));
        };

        // 1. initial vectors: unit vectors on the lowest diagonal entries
        SBD_CUDA(cudaMemsetAsync(V, 0, (size_t)nroots * N * sizeof(double), w.s));
        std::vector<int64_t> chosen;
        for (int j = 0; j < nroots; ++j) {
            const int64_t idx = w.argmin(hd, chosen, dexcl);  // global index
            chosen.push_back(idx);
            if (idx >= off && idx < off + N) {
                set_kernel<<<1, 1, 0, w.s>>>(V + j * ld, idx - off, 1.0);
                SBD_LAUNCH("set_kernel");
            }
        }
        int k = nroots;
        sigma_cols(0, k, !mixed);
        rebuild_T(k);

        std::vector<double> th(kMaxSub), rn(nroots), hist, th_prev;
        int k_ritz = 0;  // th[0..k_ritz) are the Ritz values of the last Rayleigh-Ritz step
        bool converged = false;
        double switch_floor = -1.0;  // mixed: residual level that triggers an FP64 check
        int since_ref = 0;
        int iter = 0;
        while (true) {
            // 2b-2c. Rayleigh-Ritz
            jacobi_kernel<<<1, 256, 2 * sizeof(double) * k * k, w.s>>>(T, kMaxSub, k, theta, Y, kMaxSub);
            SBD_LAUNCH("jacobi_kernel");
            // 2d + 2f. Ritz vectors, residual norms and the preconditioned corrections in one pass
            // proj_ok: V, k and TC still those of the fused pass (cleared by a refinement or a restart)
            bool proj_ok = w.ritz(V, W, ld, k, Y, kMaxSub, nroots, U, HU, theta, hd, delta, TC, rn.data());
            SBD_CUDA(cudaMemcpyAsync(th.data(), theta, sizeof(double) * k, cudaMemcpyDeviceToHost, w.s));
            SBD_CUDA(cudaStreamSynchronize(w.s));
            k_ritz = k;
            harvest_timing(c);
            double rmax = *std::max_element(rn.begin(), rn.end());
            if (c.opt.verbose)
                fprintf(stderr, "[sbd] iter %d k=%d theta0=%.12f rmax=%.3e %s\n", iter, k, th[0] + c.opt.ecore, rmax,
                        mixed ? "mixed" : (prec == SBD_F32X2 ? "f32x2" : "fp64"));
            bool checked = !mixed;
            if (mixed) {
                hist.push_back(rmax);
                ++since_ref;
                double thmax = 0.0;
                for (int j = 0; j < nroots; ++j) thmax = std::max(thmax, fabs(th[j]));
                const double floor_now = switch_floor >= 0.0 ? switch_floor : std::max(tol, 1e-6 * thmax);
                // no halving in 8 iterations, at a level where FP32 noise can matter
                const bool stalled = since_ref > 8 && rmax > 0.5 * hist[hist.size() - 9] && rmax < 1e-4 * thmax;
                if (rmax <= std::max(tol, floor_now) || stalled || iter >= max_iter) {
                    // defect correction: keep the lowest Ritz vectors, replace the target
                    // columns' W by the FP64 sigma, decide convergence on FP64 residuals
                    const int nk = std::min(std::max(nkeep, nroots), k);
                    compress(k, nk);
                    sigma_cols(0, nroots, true);
                    SBD_CUDA(cudaMemcpyAsync(HU, W, (size_t)nroots * N * sizeof(double), cudaMemcpyDeviceToDevice, w.s));
                    for (int j = 0; j < nroots; ++j) {
                        // the Rayleigh quotients that decide convergence: FP64 products
                        w.dots(U + j * ld, 0, 1, HU + j * ld, dscr + 2 * j, 1, nullptr, 0, nullptr, true);
                        w.dots(U + j * ld, 0, 1, U + j * ld, dscr + 2 * j + 1, 1, nullptr, 0, nullptr, true);
                    }
                    std::vector<double> hd2(2 * nroots);
                    SBD_CUDA(cudaMemcpyAsync(hd2.data(), dscr, sizeof(double) * 2 * nroots, cudaMemcpyDeviceToHost, w.s));
                    SBD_CUDA(cudaStreamSynchronize(w.s));
                    for (int j = 0; j < nroots; ++j) th[j] = hd2[2 * j] / hd2[2 * j + 1];
                    SBD_CUDA(cudaMemcpyAsync(theta, th.data(), sizeof(double) * nroots, cudaMemcpyHostToDevice, w.s));
                    w.resid_norms(U, HU, ld, nroots, theta, rn.data());
                    for (int j = 0; j < nroots; ++j) {
                        precond_kernel<<<w.grid, kBlas, 0, w.s>>>(U + j * ld, HU + j * ld, hd, theta + j, delta,
                                                                  TC + j * ld, N);
                        SBD_LAUNCH("precond_kernel");
                    }
                    rmax = *std::max_element(rn.begin(), rn.end());
                    r.refinements++;
                    checked = true;
                    proj_ok = false;
                    if (c.opt.verbose)
                        fprintf(stderr, "[sbd] refine %d theta0=%.12f rmax(fp64)=%.3e k=%d\n", r.refinements,
                                th[0] + c.opt.ecore, rmax, nk);
                    k = nk;
                    for (int a = nroots; a < k; ++a) exact[a] = 0;
                    rebuild_T(k);
                    switch_floor = std::max(0.5 * tol, 1e-3 * rmax);
                    since_ref = 0;
                    hist.clear();
                }
            }
            if (checked) {
                int nconv = 0;
                for (int j = 0; j < nroots; ++j)
                    nconv += rn[j] <= tol && (!(c.opt.tol_energy > 0.0) ||
                                              (j < (int)th_prev.size() && fabs(th[j] - th_prev[j]) <= c.opt.tol_energy));
                if (nconv == nroots) {
                    converged = true;
                    break;
                }
            }
            th_prev.assign(th.begin(), th.begin() + nroots);
            if (iter >= max_iter) break;
            ++iter;
            // 2h. thick restart when the new vectors would not fit
            int nnew = 0;
            for (int j = 0; j < nroots; ++j) nnew += rn[j] > tol;
            if (k + nnew > max_sub) {
                const int nk = std::min(nkeep, k);
                compress(k, nk);
                k = nk;
                proj_ok = false;
                if (mixed)
                    for (int a = 0; a < k; ++a) exact[a] = 0;
                // V' = V Y, W' = W Y with orthonormal Y: the projected matrix is diag(theta)
                std::vector<double> Td((size_t)kMaxSub * kMaxSub, 0.0);
                for (int a = 0; a < k; ++a) Td[(size_t)a * kMaxSub + a] = th[a];
                SBD_CUDA(cudaMemcpyAsync(T, Td.data(), sizeof(double) * Td.size(), cudaMemcpyHostToDevice, w.s));
                SBD_CUDA(cudaStreamSynchronize(w.s));
                r.restarts++;
            }
            // 2g. orthogonalise the corrections against V by classical Gram-Schmidt, with a second
            // pass when the first removed more than 1/sqrt(2) of the norm (the DGKS criterion);
            // normalise and append
            const int k_old = k;
            for (int j = 0; j < nroots; ++j) {
                if (rn[j] <= tol) continue;
                double *t = TC + j * ld;
                if (proj_ok) w.proj_dots(k, coef, dscr + 0);           // from the Ritz pass
                else w.dots(V, ld, k, t, coef, 1, nullptr, 0, dscr + 0); // c = V^T t, |t|^2 before
                w.axpys(V, ld, k, coef, t, dscr + 1);                   // t -= V c, |t|^2 after
                double nn[2];
                SBD_CUDA(cudaMemcpyAsync(nn, dscr, sizeof(nn), cudaMemcpyDeviceToHost, w.s));
                SBD_CUDA(cudaStreamSynchronize(w.s));
                if (!(nn[1] > 0.5 * nn[0])) {
                    w.dots(V, ld, k, t, coef, 1);                       // c = V^T t
                    w.axpys(V, ld, k, coef, t, dscr + 1);               // t -= V c, |t|^2 after
                    SBD_CUDA(cudaMemcpyAsync(nn + 1, dscr + 1, sizeof(double), cudaMemcpyDeviceToHost, w.s));
                    SBD_CUDA(cudaStreamSynchronize(w.s));
                    r.reorthogonalisations++;
                }
                const double n0 = sqrt(nn[0]), n1 = sqrt(nn[1]);
                if (!(n1 > 1e-10 * n0) || !std::isfinite(n1)) continue;
                w.scale(t, V + k * ld, 1.0 / n1);
                ++k;
            }
            if (k == k_old) {
                status = SBD_ERR_BREAKDOWN;
                c.last_error = "Davidson breakdown: no correction survived orthogonalisation";
                break;
            }
            // 2a. sigma of the new basis vectors, then extend T
            sigma_cols(k_old, k - k_old, !mixed);
            for (int b = k_old; b < k; ++b) extend_T(b, b + 1);
        }
        r.iterations = iter;
        r.seconds_sigma = sigma_ms * 1e-3;
        // sign convention: the largest-magnitude component of each vector is positive
        for (int j = 0; j < nroots; ++j) {
            const double v = w.value_at_argmaxabs(U + j * ld);
            if (v < 0.0) w.scale(U + j * ld, U + j * ld, -1.0);
        }
        double rmax = 0.0;
        for (int j = 0; j < nroots; ++j) {
            energies[j] = th[j] + c.opt.ecore;
            if (resid) resid[j] = rn[j];
            rmax = std::max(rmax, rn[j]);
        }
        r.max_residual = rmax;
        // the first Ritz value above the roots bounds the next eigenvalue from above (interlacing)
        r.gap_estimate = k_ritz > nroots ? th[nroots] - th[nroots - 1] : 0.0;
        if (vecs)
            SBD_CUDA(cudaMemcpyAsync(vecs, U, (size_t)nroots * N * sizeof(double), cudaMemcpyDefault, w.s));
        SBD_CUDA(cudaStreamSynchronize(w.s));
        if (status == SBD_OK && !converged) status = SBD_NOT_CONVERGED;
    } catch (...) {
        if (ev0) (void)cudaEventDestroy(ev0);
        if (ev1) (void)cudaEventDestroy(ev1);
        for (void *p : owned) dfree(c, p);
        throw;
    }
    (void)cudaEventDestroy(ev0);
    (void)cudaEventDestroy(ev1);
    for (void *p : owned) dfree(c, p);
    r.status = status;
    r.seconds_total = std::chrono::duration<double>(clock::now() - t_start).count();
    if (rep) *rep = r;
    return status;
}

}  // namespace sbd
