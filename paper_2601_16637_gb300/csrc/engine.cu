// Batched / served Davidson engine: many independent instances ("jobs") iterate
// together on one device.  Each job runs the Davidson method of the paper
// (Sec. II-C; preconditioner of Eq. 7) with the mixed-precision sigma product
// (Sec. II-A/B) and an FP64 sigma check of its converged Ritz vector.
//
// Device layout.  A job occupies a slot: its handle (tables, Hamiltonian
// diagonal, a transposed work vector) plus V, W [max_sub][N], U, HU, TC [N]
// (FP64) and an FP32 copy of the newest basis vector.  Every vector operation
// of an iteration runs over the concatenation of all slots' vectors, cut into
// fixed chunks of kChunk elements that never straddle two slots; a chunk's
// partial sums go to its own row of a partial-sum table, and each slot reduces
// its own rows in a fixed order.  The sigma products of all slots share one
// persistent launch per pass (sigma.cu).  Nothing a job computes depends on
// the other jobs, so its results are bitwise the same alone and in any mix.
//
// One engine iteration = graph A (Rayleigh-Ritz: Jacobi per slot, Ritz vector,
// residual, preconditioned correction) and graph B (thick-restart compression,
// classical Gram-Schmidt of the correction (a second pass where the first removed more than
// half of its squared norm), normalisation, batched
// mixed sigma of the new vector, extension of the projected matrix; and for
// jobs that have converged in mixed precision, the batched FP64 sigma of the
// Ritz vector with its Rayleigh quotient and residual).  Both graphs are
// captured once; per iteration the host writes the slot descriptors into
// pinned memory (copied by the graph's first node), replays, and reads back a
// small status array.  All per-slot decisions (converged, restart, check) are
// taken on the host between the two graphs.
//
// The vector operations of the Davidson steps (Ritz combinations, Gram-Schmidt
// dot products and updates, the projected-matrix column, the restart) sum in
// FP32 pairs (pair.cuh: 48-bit operands on the FP32 pipe; GB300's FP64 pipe
// runs one multiply-add per loaded element below the HBM rate); the FP64 check
// of a converged vector (its Rayleigh quotient and residual) stays FP64.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "jacobi.cuh"
#include "pair.cuh"

namespace sbd {

namespace {

constexpr int kEThreads = 256;           // threads per vector-kernel block
constexpr int64_t kChunk = 1 << 15;      // vector elements per chunk
constexpr int kEMaxSub = 32;             // largest basis per job
constexpr int kEPart = kEMaxSub + 1;     // partial-sum slots per chunk: kEMaxSub dots + one norm
constexpr int kNorm = kEMaxSub;          // index of the norm slot
constexpr int kLoadE = 4;                // vectors loaded together in the multi-vector loops

enum : int { kRitz = 1, kRestart = 2, kGrow = 4, kCheck = 8 };

// per-slot scalars (SlotDev::red)
enum : int {
    kRedResid = 0,   // ||Wy - theta V y||^2 (mixed)
    kRedBefore = 1,  // |t|^2 before Gram-Schmidt
    kRedAfter = 2,   // |t|^2 after
    kRedScale = 3,   // 1/|t| when the correction is kept, else 0
    kRedUH = 4,      // u . H64 u
    kRedUU = 5,      // u . u
    kRedTheta64 = 6, // FP64 Rayleigh quotient
    kRedR64 = 7,     // ||H64 u - theta64 u||^2
    kRedNeed2 = 8,   // 1 when the first Gram-Schmidt pass removed more than half of |t|^2
    kRedCount = 9
};

struct SlotDev {
    int64_t N;
    double *V, *W, *U, *HU, *TC;
    float *c32;
    const double *hd;
    double *T;      // [kEMaxSub][kEMaxSub]
    double *Y;      // [kEMaxSub][kEMaxSub]
    double *theta;  // [kEMaxSub]
    double *coef;   // [kEMaxSub]
    double *red;    // [kRedCount]
    double delta;
    int k;          // basis size entering the iteration
    int kind;       // kRitz | kRestart | kGrow | kCheck for the graph being replayed
    int nk;         // vectors kept by a restart
    int pad;
    int64_t chunk0, chunk1;  // this slot's chunks
};

struct Header {
    int nslot;
    int nchunk;
};

struct Status {
    double theta0, resid2, scale, theta64, r64sq, uu;
};

__device__ __forceinline__ int keff(const SlotDev &d) { return (d.kind & kRestart) ? d.nk : d.k; }

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

// Rayleigh-Ritz on the projected matrix, one CTA per slot
__global__ void e_jacobi_kernel(const Header *hdr, const SlotDev *slots)
{
    extern __shared__ double js[];
    const int s = blockIdx.x;
    if (s >= hdr->nslot) return;
    const SlotDev d = slots[s];
    if (!(d.kind & kRitz) || d.k < 1) return;
    jacobi_eig(d.T, kEMaxSub, d.k, d.theta, d.Y, kEMaxSub, js);
}

// u = V y0, hu = W y0 (y0: the lowest eigenvector of T), r = hu - theta0 u,
// t = r / (sign(dd) max(|dd|, delta)), dd = Hd - theta0  (Eq. 7); partial |r|^2 per chunk
__global__ void __launch_bounds__(kEThreads) e_ritz_kernel(const Header *hdr, const SlotDev *slots,
                                                          const int *chunk_slot, const int64_t *chunk_off,
                                                          double *partial)
{
    __shared__ F2 ys[kEMaxSub];
    __shared__ double red[kEThreads / 32];
    const int nchunk = hdr->nchunk;
    for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
        const int s = chunk_slot[c];
        const SlotDev &d = slots[s];
        if (!(d.kind & kRitz)) continue;
        const int k = d.k;
        __syncthreads();
        for (int a = threadIdx.x; a < kEMaxSub; a += kEThreads) ys[a] = a < k ? f2_split(d.Y[a * kEMaxSub]) : F2(0.f);
        __syncthreads();
        const double th = d.theta[0], delta = d.delta;
        const int64_t e0 = chunk_off[c], e1 = min(e0 + kChunk, d.N);
        double racc = 0.0;
        for (int64_t i = e0 + threadIdx.x; i < e1; i += kEThreads) {
            F2 up(0.f), hup(0.f);
            for (int a0 = 0; a0 < k; a0 += kLoadE) {
                double x[kLoadE], h[kLoadE];
#pragma unroll
                for (int q = 0; q < kLoadE; ++q) {
                    const bool ok = a0 + q < k;
                    x[q] = ok ? d.V[(a0 + q) * d.N + i] : 0.0;
                    h[q] = ok ? d.W[(a0 + q) * d.N + i] : 0.0;
                }
#pragma unroll
                for (int q = 0; q < kLoadE; ++q)
                    if (a0 + q < k) {
                        f2_mac(up, ys[a0 + q], f2_split(x[q]));
                        f2_mac(hup, ys[a0 + q], f2_split(h[q]));
                    }
            }
            const double u = f2_value(up), hu = f2_value(hup);
            const double r = hu - th * u;
            racc += r * r;
            const double dd = d.hd[i] - th;
            d.U[i] = u;
            d.HU[i] = hu;
            d.TC[i] = r * precond_factor(dd, delta);
        }
        const double sum = block_sum(racc, red);
        if (threadIdx.x == 0) partial[(int64_t)c * kEPart + 0] = sum;
    }
}

// Multi-dot over the chunks of participating slots: partial[c][a] = X_a . y for a < cnt and,
// with NORM, partial[c][kNorm] = z . z.  MODE selects the operands:
//   0 (Gram-Schmidt): X = V[0..keff), y = TC, z = TC        slots with kGrow
//   1 (T extension):  X = V[0..keff], y = W[keff]           slots with kGrow
//   2 (FP64 check):   X = U, y = TC (= H64 u), z = U        slots with kCheck
template <int MODE, bool NORM>
__global__ void __launch_bounds__(kEThreads) e_dots_kernel(const Header *hdr, const SlotDev *slots,
                                                          const int *chunk_slot, const int64_t *chunk_off,
                                                          double *partial)
{
    constexpr int G = 8;  // dot products per sweep over the chunk
    __shared__ double red[kEThreads / 32];
    const int nchunk = hdr->nchunk;
    for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
        const SlotDev &d = slots[chunk_slot[c]];
        const int mask = MODE == 2 ? kCheck : kGrow;
        if (!(d.kind & mask)) continue;
        if (MODE == 0 && !NORM && d.red[kRedNeed2] == 0.0) continue;  // second Gram-Schmidt pass not needed
        const int ke = keff(d);
        const int cnt = MODE == 0 ? ke : (MODE == 1 ? ke + 1 : 1);
        const double *X = MODE == 2 ? d.U : d.V;
        const double *y = MODE == 1 ? d.W + (int64_t)ke * d.N : d.TC;
        const double *z = MODE == 2 ? d.U : d.TC;
        const int64_t e0 = chunk_off[c], e1 = min(e0 + kChunk, d.N);
        // sweeps of G vectors (the norm rides on the first sweep); at least one sweep for the norm
        for (int a0 = 0; a0 < cnt || (a0 == 0 && NORM); a0 += G) {
            // MODE 0, 1: pair products; MODE 2 (the FP64 check): FP64
            using Acc = typename std::conditional<MODE == 2, double, F2>::type;
            Acc acc[G];
#pragma unroll
            for (int q = 0; q < G; ++q) acc[q] = Acc(0.f);
            double nacc = 0.0;
            for (int64_t i = e0 + threadIdx.x; i < e1; i += kEThreads) {
                double x[G];
#pragma unroll
                for (int q = 0; q < G; ++q) x[q] = a0 + q < cnt ? X[(int64_t)(a0 + q) * d.N + i] : 0.0;
                const double yi = y[i];
                if (NORM && a0 == 0) {
                    const double zi = z[i];
                    nacc += zi * zi;
                }
                if constexpr (MODE == 2) {
#pragma unroll
                    for (int q = 0; q < G; ++q) acc[q] += x[q] * yi;
                } else {
                    const F2 ys = f2_split(yi);
#pragma unroll
                    for (int q = 0; q < G; ++q) f2_mac(acc[q], f2_split(x[q]), ys);
                }
            }
#pragma unroll
            for (int q = 0; q < G; ++q)
                if (a0 + q < cnt) {
                    double v;
                    if constexpr (MODE == 2) v = acc[q];
                    else v = f2_value(acc[q]);
                    const double sum = block_sum(v, red);
                    if (threadIdx.x == 0) partial[(int64_t)c * kEPart + a0 + q] = sum;
                }
            if (NORM && a0 == 0) {
                const double sum = block_sum(nacc, red);
                if (threadIdx.x == 0) partial[(int64_t)c * kEPart + kNorm] = sum;
            }
        }
    }
}

// TC -= sum_a coef[a] V[a] (a < keff) for kGrow slots; with NORM, partial[c][kNorm] = |TC|^2 after
// SECOND: the second Gram-Schmidt pass, only for slots whose first pass asked for it
template <bool NORM, bool SECOND>
__global__ void __launch_bounds__(kEThreads) e_axpy_kernel(const Header *hdr, const SlotDev *slots,
                                                          const int *chunk_slot, const int64_t *chunk_off,
                                                          double *partial)
{
    __shared__ F2 cs[kEMaxSub];
    __shared__ double red[kEThreads / 32];
    const int nchunk = hdr->nchunk;
    for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
        const SlotDev &d = slots[chunk_slot[c]];
        if (!(d.kind & kGrow)) continue;
        if (SECOND && d.red[kRedNeed2] == 0.0) continue;
        const int ke = keff(d);
        __syncthreads();
        for (int a = threadIdx.x; a < ke; a += kEThreads) cs[a] = f2_split(d.coef[a]);
        __syncthreads();
        const int64_t e0 = chunk_off[c], e1 = min(e0 + kChunk, d.N);
        double nacc = 0.0;
        for (int64_t i = e0 + threadIdx.x; i < e1; i += kEThreads) {
            F2 sp(0.f);  // sum_a coef[a] V[a] in pairs, subtracted in FP64
            for (int a0 = 0; a0 < ke; a0 += kLoadE) {
                double x[kLoadE];
#pragma unroll
                for (int q = 0; q < kLoadE; ++q) x[q] = a0 + q < ke ? d.V[(int64_t)(a0 + q) * d.N + i] : 0.0;
#pragma unroll
                for (int q = 0; q < kLoadE; ++q)
                    if (a0 + q < ke) f2_mac(sp, cs[a0 + q], f2_split(x[q]));
            }
            const double t = d.TC[i] - f2_value(sp);
            d.TC[i] = t;
            if (NORM) nacc += t * t;
        }
        if (NORM) {
            const double sum = block_sum(nacc, red);
            if (threadIdx.x == 0) partial[(int64_t)c * kEPart + kNorm] = sum;
        }
    }
}

// Per-slot reduction of the chunk partial sums in a fixed order (lane l sums chunks l, l+32, ...
// of the slot, then a butterfly over the lanes); one warp per output.  What is reduced and where
// it goes depends on the phase:
enum : int { kFinRitz, kFinGS1, kFinAfter1, kFinGS2, kFinAfter, kFinExtend, kFinCheck1, kFinCheck2 };

__global__ void e_final_kernel(const Header *hdr, SlotDev *slots, const double *partial, int phase)
{
    const int s = blockIdx.x;
    if (s >= hdr->nslot) return;
    const SlotDev d = slots[s];
    const int mask = (phase == kFinRitz) ? kRitz : ((phase == kFinCheck1 || phase == kFinCheck2) ? kCheck : kGrow);
    if (!(d.kind & mask)) return;
    if ((phase == kFinGS2 || phase == kFinAfter) && d.red[kRedNeed2] == 0.0) return;
    const int ke = keff(d);
    int cnt = 0;  // dot outputs 0..cnt-1
    bool norm = false;
    switch (phase) {
    case kFinRitz: cnt = 1; break;
    case kFinGS1: cnt = ke; norm = true; break;
    case kFinAfter1: norm = true; break;
    case kFinGS2: cnt = ke; break;
    case kFinAfter: norm = true; break;
    case kFinExtend: cnt = ke + 1; break;
    case kFinCheck1: cnt = 1; norm = true; break;
    case kFinCheck2: cnt = 1; break;
    }
    __shared__ double out[kEPart];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nout = cnt + (norm ? 1 : 0);
    for (int o = warp; o < nout; o += nw) {
        const int j = o < cnt ? o : kNorm;
        double v = 0.0;
        for (int64_t c = d.chunk0 + lane; c < d.chunk1; c += 32) v += partial[c * kEPart + j];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) out[j] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    switch (phase) {
    case kFinRitz: d.red[kRedResid] = out[0]; break;
    case kFinGS1:
        for (int a = 0; a < ke; ++a) d.coef[a] = out[a];
        d.red[kRedBefore] = out[kNorm];
        break;
    case kFinGS2:
        for (int a = 0; a < ke; ++a) d.coef[a] = out[a];
        break;
    case kFinAfter1:
    case kFinAfter: {
        const double before = d.red[kRedBefore], after = out[kNorm];
        // a second pass when the first removed more than half of |t|^2 (the DGKS criterion)
        if (phase == kFinAfter1) d.red[kRedNeed2] = (ke > 0 && !(after > 0.5 * before)) ? 1.0 : 0.0;
        d.red[kRedAfter] = after;
        // keep the correction unless Gram-Schmidt removed all but 1e-10 of its norm
        const bool keep = after > 1e-20 * before && isfinite(after) && after > 0.0;
        d.red[kRedScale] = keep ? 1.0 / sqrt(after) : 0.0;
        break;
    }
    case kFinExtend:
        for (int a = 0; a <= ke; ++a) {
            d.T[a * kEMaxSub + ke] = out[a];
            d.T[ke * kEMaxSub + a] = out[a];
        }
        break;
    case kFinCheck1:
        d.red[kRedUH] = out[0];
        d.red[kRedUU] = out[kNorm];
        d.red[kRedTheta64] = out[0] / out[kNorm];
        break;
    case kFinCheck2: d.red[kRedR64] = out[0]; break;
    }
}

// thick restart, in place: V[j] = sum_a Y[a][j] V[a], W likewise, j < nk, a < k (each thread reads
// all k inputs of its element before writing any output)
__global__ void __launch_bounds__(kEThreads) e_compress_kernel(const Header *hdr, const SlotDev *slots,
                                                              const int *chunk_slot, const int64_t *chunk_off)
{
    __shared__ F2 ys[kEMaxSub * kEMaxSub];
    const int nchunk = hdr->nchunk;
    for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
        const SlotDev &d = slots[chunk_slot[c]];
        if (!(d.kind & kRestart)) continue;
        const int k = d.k, nk = d.nk;
        __syncthreads();
        for (int t = threadIdx.x; t < k * nk; t += kEThreads) ys[t] = f2_split(d.Y[(t / nk) * kEMaxSub + (t % nk)]);
        __syncthreads();
        const int64_t e0 = chunk_off[c], e1 = min(e0 + kChunk, d.N);
        for (int64_t i = e0 + threadIdx.x; i < e1; i += kEThreads) {
#pragma unroll 1
            for (int m = 0; m < 2; ++m) {
                double *X = m == 0 ? d.V : d.W;
                F2 x[kEMaxSub];
#pragma unroll
                for (int a = 0; a < kEMaxSub; ++a) x[a] = a < k ? f2_split(X[(int64_t)a * d.N + i]) : F2(0.f);
                for (int j = 0; j < nk; ++j) {
                    F2 v(0.f);
#pragma unroll
                    for (int a = 0; a < kEMaxSub; ++a)
                        if (a < k) f2_mac(v, ys[a * nk + j], x[a]);
                    X[(int64_t)j * d.N + i] = f2_value(v);
                }
            }
        }
    }
}

// per-slot bookkeeping before Gram-Schmidt: after a restart T = diag(theta[0..nk))
__global__ void e_restart_T_kernel(const Header *hdr, const SlotDev *slots)
{
    const int s = blockIdx.x;
    if (s >= hdr->nslot) return;
    const SlotDev &d = slots[s];
    if (!(d.kind & kRestart)) return;
    for (int t = threadIdx.x; t < kEMaxSub * kEMaxSub; t += blockDim.x) {
        const int a = t / kEMaxSub, b = t % kEMaxSub;
        d.T[t] = (a == b && a < d.nk) ? d.theta[a] : 0.0;
    }
}

// V[keff] = TC / |TC| and its FP32 copy (zero when the correction was dropped)
__global__ void __launch_bounds__(kEThreads) e_scale_kernel(const Header *hdr, const SlotDev *slots,
                                                           const int *chunk_slot, const int64_t *chunk_off)
{
    const int nchunk = hdr->nchunk;
    for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
        const SlotDev &d = slots[chunk_slot[c]];
        if (!(d.kind & kGrow)) continue;
        const double f = d.red[kRedScale];
        double *v = d.V + (int64_t)keff(d) * d.N;
        const int64_t e0 = chunk_off[c], e1 = min(e0 + kChunk, d.N);
        for (int64_t i = e0 + threadIdx.x; i < e1; i += kEThreads) {
            const double x = d.TC[i] * f;
            v[i] = x;
            d.c32[i] = __double2float_rn(x);
        }
    }
}

// partial[c][0] = |H64 u - theta64 u|^2 over the chunk (check slots; H64 u is in TC)
__global__ void __launch_bounds__(kEThreads) e_check_resid_kernel(const Header *hdr, const SlotDev *slots,
                                                                 const int *chunk_slot, const int64_t *chunk_off,
                                                                 double *partial)
{
    __shared__ double red[kEThreads / 32];
    const int nchunk = hdr->nchunk;
    for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
        const SlotDev &d = slots[chunk_slot[c]];
        if (!(d.kind & kCheck)) continue;
        const double th = d.red[kRedTheta64];
        const int64_t e0 = chunk_off[c], e1 = min(e0 + kChunk, d.N);
        double acc = 0.0;
        for (int64_t i = e0 + threadIdx.x; i < e1; i += kEThreads) {
            const double r = d.TC[i] - th * d.U[i];
            acc += r * r;
        }
        const double sum = block_sum(acc, red);
        if (threadIdx.x == 0) partial[(int64_t)c * kEPart + 0] = sum;
    }
}

__global__ void e_status_kernel(const Header *hdr, const SlotDev *slots, Status *st)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < hdr->nslot; s += gridDim.x * blockDim.x) {
        const SlotDev &d = slots[s];
        Status o{};
        if (d.N == 0) {
            st[s] = o;
            continue;
        }
        o.theta0 = d.theta[0];
        o.resid2 = d.red[kRedResid];
        o.scale = d.red[kRedScale];
        o.theta64 = d.red[kRedTheta64];
        o.r64sq = d.red[kRedR64];
        o.uu = d.red[kRedUU];
        st[s] = o;
    }
}

// index of the lowest entry (ties: lowest index), two stages
__global__ void e_argmin_partial(const double *x, int64_t n, double *pv, int64_t *pi)
{
    __shared__ double sv[kEThreads];
    __shared__ int64_t si[kEThreads];
    double bv = INFINITY;
    int64_t bi = -1;
    for (int64_t i = blockIdx.x * (int64_t)kEThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kEThreads)
        if (bi < 0 || x[i] < bv) {
            bv = x[i];
            bi = i;
        }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int w = kEThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double ov = sv[threadIdx.x + w];
            const int64_t oi = si[threadIdx.x + w];
            if (oi >= 0 && (si[threadIdx.x] < 0 || ov < sv[threadIdx.x] ||
                            (ov == sv[threadIdx.x] && oi < si[threadIdx.x]))) {
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

// index of the largest |entry| (ties: lowest index)
__global__ void e_argmaxabs_partial(const double *x, int64_t n, double *pv, int64_t *pi)
{
    __shared__ double sv[kEThreads];
    __shared__ int64_t si[kEThreads];
    double bv = -1.0;
    int64_t bi = -1;
    for (int64_t i = blockIdx.x * (int64_t)kEThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kEThreads)
        if (fabs(x[i]) > bv) {
            bv = fabs(x[i]);
            bi = i;
        }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int w = kEThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double ov = sv[threadIdx.x + w];
            const int64_t oi = si[threadIdx.x + w];
            if (oi >= 0 && (si[threadIdx.x] < 0 || ov > sv[threadIdx.x] ||
                            (ov == sv[threadIdx.x] && oi < si[threadIdx.x]))) {
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

__global__ void e_unit_kernel(double *x, int64_t n, int64_t idx)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = i == idx ? 1.0 : 0.0;
}

__global__ void e_negate_kernel(double *x, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = -x[i];
}

double now_seconds(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace sbd

using namespace sbd;

struct Job {
    int64_t id = 0;
    int norb = 0, na = 0, nb = 0;
    std::vector<double> h, eri;
    std::vector<uint64_t> A, B;
    double ecore = 0.0, tol = 1e-6, tol_energy = 0.0;
    bool keep_vector = false;
    bool finished = false;
    sbd_job_result res{};
    std::vector<double> vec;
};

struct Slot {
    Job *job = nullptr;
    sbd_handle handle = nullptr;
    int64_t N = 0;
    double *V = nullptr, *W = nullptr, *U = nullptr, *HU = nullptr, *TC = nullptr, *small = nullptr;
    float *c32 = nullptr;
    size_t bytes = 0;
    int k = 0;              // basis vectors
    int kind = 0;           // for the graph being built
    int nk = 0;
    double theta_prev = NAN, thr = 0.0, r_mixed = INFINITY;
    std::vector<double> hist;  // mixed residuals since the last FP64 check
    int64_t chunk0 = 0, chunk1 = 0;
    double pass = 0.0;      // fair schedule: device work taken so far, in determinants per iteration
    bool run = false;       // takes part in the current iteration
};

struct sbd_engine_s {
    sbd_engine_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;  // created here because the caller passed the legacy stream (not capturable)
    int device = 0, num_sms = 0, nkeep = 4;
    std::chrono::steady_clock::time_point t0;
    std::deque<Job *> pending;
    std::map<int64_t, std::unique_ptr<Job>> jobs;
    std::vector<Slot> slots;
    int64_t next_id = 0;
    size_t bytes_in_use = 0, bytes_peak = 0;
    double vtime = 0.0;  // fair schedule: smallest pass of the running jobs at the last iteration
    int64_t max_chunks = 0;
    // device staging block: header, slot descriptors, chunk table (+ pinned host mirror)
    size_t off_hdr = 0, off_slots = 0, off_cslot = 0, off_coff = 0, stage_bytes = 0;
    unsigned char *dstage = nullptr, *hstage = nullptr;
    double *partial = nullptr;
    Status *dstatus = nullptr, *hstatus = nullptr;
    double *small_scratch = nullptr;  // argmin / argmaxabs partials
    int64_t *small_idx = nullptr;
    SigmaBatch *sb32 = nullptr, *sb64 = nullptr;
    int rows_per_item = 0;
    double tune_ms[4] = {0, 0, 0, 0};
    cudaGraphExec_t gA = nullptr, gB = nullptr;
    int64_t launches_A = 0, launches_B = 0;
    int64_t steps = 0, graph_launches = 0, kernel_launches = 0;
    int64_t requeued = 0;  // admissions undone because the job's tables exceeded the budget left
    int grid_vec = 0;
    std::vector<SigmaSlot> s32, s64;

    Header *d_hdr() { return reinterpret_cast<Header *>(dstage + off_hdr); }
    SlotDev *d_slots() { return reinterpret_cast<SlotDev *>(dstage + off_slots); }
    int *d_cslot() { return reinterpret_cast<int *>(dstage + off_cslot); }
    int64_t *d_coff() { return reinterpret_cast<int64_t *>(dstage + off_coff); }
    Header *h_hdr() { return reinterpret_cast<Header *>(hstage + off_hdr); }
    SlotDev *h_slots() { return reinterpret_cast<SlotDev *>(hstage + off_slots); }
    int *h_cslot() { return reinterpret_cast<int *>(hstage + off_cslot); }
    int64_t *h_coff() { return reinterpret_cast<int64_t *>(hstage + off_coff); }

    void *alloc(size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        void *p = nullptr;
        if (opt.alloc) {
            p = opt.alloc(opt.alloc_ctx, bytes, (void *)stream);
            if (!p) fail(SBD_ERR_OUT_OF_MEMORY, "device allocator returned NULL");
        } else {
            cudaError_t e = cudaMallocAsync(&p, bytes, stream);
            if (e != cudaSuccess || !p) {
                (void)cudaGetLastError();
                fail(SBD_ERR_OUT_OF_MEMORY, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
            }
        }
        return p;
    }
    void release(void *p)
    {
        if (!p) return;
        if (opt.free) opt.free(opt.alloc_ctx, p, (void *)stream);
        else (void)cudaFreeAsync(p, stream);
    }

    int max_sub() const { return opt.max_subspace; }
    size_t basis_bytes(int64_t N) const
    {
        return (size_t)N * 8 * (2 * (size_t)opt.max_subspace + 3) + (size_t)N * 4 + 256 * 6 +
               sizeof(double) * (3 * kEMaxSub * kEMaxSub);
    }

    void init();
    void destroy();
    bool admit_one();
    void free_slot(Slot &s);
    void finish(Slot &s, int status, bool with_vector);
    void write_stage();
    void build_sigma_lists();
    void capture();
    void autotune();
    int step();
    void replay(cudaGraphExec_t g, int64_t launches);
};

void sbd_engine_s::init()
{
    SBD_CUDA(cudaGetDevice(&device));
    if (!stream) {
        SBD_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
        own_stream = true;
    }
    SBD_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
    grid_vec = 4 * num_sms;
    nkeep = std::max(2, opt.max_subspace / 3);
    t0 = std::chrono::steady_clock::now();
    slots.resize(opt.max_slots);
    // chunk capacity: the budget's worth of determinants (or 2^31 without a budget) plus one
    // partial chunk per slot
    int64_t max_dets = (int64_t)1 << 31;
    if (opt.hbm_budget_bytes) max_dets = (int64_t)(opt.hbm_budget_bytes / (8 * (2 * (size_t)opt.max_subspace + 3)));
    max_chunks = max_dets / kChunk + opt.max_slots + 1;
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t at = o;
        o = (o + b + 255) & ~(size_t)255;
        return at;
    };
    off_hdr = take(sizeof(Header));
    off_slots = take(sizeof(SlotDev) * opt.max_slots);
    off_cslot = take(sizeof(int) * max_chunks);
    off_coff = take(sizeof(int64_t) * max_chunks);
    stage_bytes = o;
    SBD_CUDA(cudaMalloc(&dstage, stage_bytes));
    SBD_CUDA(cudaMallocHost(&hstage, stage_bytes));
    memset(hstage, 0, stage_bytes);
    SBD_CUDA(cudaMalloc(&partial, sizeof(double) * kEPart * (size_t)max_chunks));
    SBD_CUDA(cudaMalloc(&dstatus, sizeof(Status) * opt.max_slots));
    SBD_CUDA(cudaMallocHost(&hstatus, sizeof(Status) * opt.max_slots));
    SBD_CUDA(cudaMalloc(&small_scratch, sizeof(double) * grid_vec));
    SBD_CUDA(cudaMalloc(&small_idx, sizeof(int64_t) * grid_vec));
    SBD_CUDA(cudaFuncSetAttribute(e_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(2 * sizeof(double) * kEMaxSub * kEMaxSub)));
    const int ms = std::max(opt.max_strings, 1);
    // FP64-accurate sigma for the checks (FP32 pairs): the largest rows per item that fits
    for (int R : {2, 1})
        if (sigma_batch_smem(SBD_F32X2, R, ms, opt.max_norb) <= sigma_batch_smem_limit(device)) {
            sb64 = sigma_batch_create(opt.max_slots, SBD_F32X2, R, ms, opt.max_norb, device);
            break;
        }
    if (!sb64) fail(SBD_ERR_UNSUPPORTED, "engine: max_strings/max_norb too large for the FP64 sigma staging");
    if (opt.rows_per_item) {
        sb32 = sigma_batch_create(opt.max_slots, SBD_MIXED, opt.rows_per_item, ms, opt.max_norb, device);
        rows_per_item = opt.rows_per_item;
    }
}

void sbd_engine_s::destroy()
{
    if (stream) (void)cudaStreamSynchronize(stream);
    for (Slot &s : slots)
        if (s.job) free_slot(s);
    if (gA) (void)cudaGraphExecDestroy(gA);
    if (gB) (void)cudaGraphExecDestroy(gB);
    sigma_batch_destroy(sb32);
    sigma_batch_destroy(sb64);
    if (stream) (void)cudaStreamSynchronize(stream);
    if (dstage) (void)cudaFree(dstage);
    if (hstage) (void)cudaFreeHost(hstage);
    if (partial) (void)cudaFree(partial);
    if (dstatus) (void)cudaFree(dstatus);
    if (hstatus) (void)cudaFreeHost(hstatus);
    if (small_scratch) (void)cudaFree(small_scratch);
    if (small_idx) (void)cudaFree(small_idx);
    if (own_stream && stream) (void)cudaStreamDestroy(stream);
}

void sbd_engine_s::free_slot(Slot &s)
{
    release(s.V);
    release(s.W);
    release(s.U);
    release(s.HU);
    release(s.TC);
    release(s.c32);
    release(s.small);
    if (s.handle) sbd_destroy(s.handle);
    bytes_in_use -= std::min(bytes_in_use, s.bytes);
    s = Slot{};
}

// Admits the head of the queue if a slot is free and its memory fits the budget.
bool sbd_engine_s::admit_one()
{
    if (pending.empty()) return false;
    int free_idx = -1;
    for (int i = 0; i < (int)slots.size(); ++i)
        if (!slots[i].job) {
            free_idx = i;
            break;
        }
    if (free_idx < 0) return false;
    Job *j = pending.front();
    const int64_t nA = (int64_t)j->A.size(), nB = (int64_t)j->B.size();
    const int64_t N = nA * nB;
    // device bytes: basis and vectors, Hamiltonian diagonal + transposed work vector, and a
    // reserve per string for the excitation tables (an estimate: the handle's own allocations are
    // held to the budget left after the basis when the job is created, below)
    const size_t est = basis_bytes(N) + (size_t)N * 16 + (size_t)(nA + nB) * opt.table_bytes_per_string;
    if (opt.hbm_budget_bytes && bytes_in_use + est > opt.hbm_budget_bytes) {
        if (bytes_in_use == 0) {
            // cannot fit even alone: fail the job instead of blocking the queue
            pending.pop_front();
            j->res.status = SBD_ERR_OVER_BUDGET;
            j->res.t_admit = j->res.t_done = now_seconds(t0);
            j->finished = true;
            return true;
        }
        return false;
    }
    int64_t used_chunks = 0;
    for (const Slot &s : slots)
        if (s.job) used_chunks += (s.N + kChunk - 1) / kChunk;
    if (used_chunks + (N + kChunk - 1) / kChunk > max_chunks) {
        if (used_chunks == 0) {
            pending.pop_front();
            j->res.status = SBD_ERR_OVER_BUDGET;
            j->res.t_admit = j->res.t_done = now_seconds(t0);
            j->finished = true;
            set_thread_error("engine job larger than the engine's vector capacity");
            return true;
        }
        return false;
    }
    pending.pop_front();
    double pass0 = vtime;  // a new job starts at the smallest pass of the running ones
    for (const Slot &r : slots)
        if (r.job) pass0 = std::min(pass0, r.pass);
    Slot &s = slots[free_idx];
    s = Slot{};
    s.job = j;
    s.N = N;
    s.pass = pass0;
    j->res.t_admit = now_seconds(t0);
    j->res.ndets = N;
    try {
        sbd_options o;
        sbd_default_options(&o);
        o.alloc = opt.alloc;
        o.free = opt.free;
        o.alloc_ctx = opt.alloc_ctx;
        o.ecore = j->ecore;
        // the tables, diagonal and work vectors of the handle (and whatever sbd_create holds while it
        // runs) must fit what the budget leaves after the jobs in use and this job's basis
        if (opt.hbm_budget_bytes) o.hbm_budget_bytes = opt.hbm_budget_bytes - bytes_in_use - basis_bytes(N);
        int rc = sbd_create(&s.handle, j->norb, j->na, j->nb, j->h.data(), j->eri.data(), j->A.data(), nA,
                            j->B.data(), nB, &o, (void *)stream);
        if (rc == SBD_ERR_OVER_BUDGET && bytes_in_use > 0) {
            // the estimate was too low: wait at the head of the queue until running jobs free memory
            s = Slot{};
            j->res.t_admit = 0.0;
            j->res.ndets = 0;
            pending.push_front(j);
            requeued++;
            return false;
        }
        if (rc != SBD_OK) fail(rc, std::string("engine job: ") + sbd_last_error(nullptr));
        const Ctx &c = ctx_of(s.handle);
        if (std::max(c.nA, c.nB) > opt.max_strings || c.norb > opt.max_norb)
            fail(SBD_ERR_UNSUPPORTED, "engine job exceeds max_strings or max_norb");
        const size_t nb8 = (size_t)N * 8;
        s.V = (double *)alloc(nb8 * opt.max_subspace);
        s.W = (double *)alloc(nb8 * opt.max_subspace);
        s.U = (double *)alloc(nb8);
        s.HU = (double *)alloc(nb8);
        s.TC = (double *)alloc(nb8);
        s.c32 = (float *)alloc((size_t)N * 4);
        s.small = (double *)alloc(sizeof(double) * (3 * kEMaxSub * kEMaxSub));
        s.bytes = basis_bytes(N) + c.bytes_held;
        SBD_CUDA(cudaMemsetAsync(s.small, 0, sizeof(double) * (3 * kEMaxSub * kEMaxSub), stream));
        SBD_CUDA(cudaMemsetAsync(s.c32, 0, (size_t)N * 4, stream));
        // initial vector: unit vector on the lowest diagonal entry (ties: lowest index)
        const int g = (int)std::min<int64_t>(grid_vec, std::max<int64_t>(1, (N + kEThreads - 1) / kEThreads));
        e_argmin_partial<<<g, kEThreads, 0, stream>>>(c.hd, N, small_scratch, small_idx);
        SBD_LAUNCH("e_argmin_partial");
        std::vector<double> pv(g);
        std::vector<int64_t> pi(g);
        SBD_CUDA(cudaMemcpyAsync(pv.data(), small_scratch, sizeof(double) * g, cudaMemcpyDeviceToHost, stream));
        SBD_CUDA(cudaMemcpyAsync(pi.data(), small_idx, sizeof(int64_t) * g, cudaMemcpyDeviceToHost, stream));
        SBD_CUDA(cudaStreamSynchronize(stream));
        int64_t bi = -1;
        double bv = INFINITY;
        for (int b = 0; b < g; ++b)
            if (pi[b] >= 0 && (bi < 0 || pv[b] < bv || (pv[b] == bv && pi[b] < bi))) {
                bv = pv[b];
                bi = pi[b];
            }
        e_unit_kernel<<<g, kEThreads, 0, stream>>>(s.TC, N, bi);
        SBD_LAUNCH("e_unit_kernel");
        s.k = 0;
        s.thr = j->tol;
        bytes_in_use += s.bytes;
        bytes_peak = std::max(bytes_peak, bytes_in_use);
    } catch (const Error &e) {
        j->res.status = e.code;
        j->res.t_done = now_seconds(t0);
        j->finished = true;
        s.bytes = 0;
        free_slot(s);
        set_thread_error(e.msg);
    }
    return true;
}

void sbd_engine_s::finish(Slot &s, int status, bool with_vector)
{
    Job *j = s.job;
    j->res.status = status;
    if (with_vector && j->keep_vector) {
        // sign convention: the largest-magnitude component is positive
        const int g = (int)std::min<int64_t>(grid_vec, std::max<int64_t>(1, (s.N + kEThreads - 1) / kEThreads));
        e_argmaxabs_partial<<<g, kEThreads, 0, stream>>>(s.U, s.N, small_scratch, small_idx);
        SBD_LAUNCH("e_argmaxabs_partial");
        std::vector<double> pv(g);
        std::vector<int64_t> pi(g);
        SBD_CUDA(cudaMemcpyAsync(pv.data(), small_scratch, sizeof(double) * g, cudaMemcpyDeviceToHost, stream));
        SBD_CUDA(cudaMemcpyAsync(pi.data(), small_idx, sizeof(int64_t) * g, cudaMemcpyDeviceToHost, stream));
        SBD_CUDA(cudaStreamSynchronize(stream));
        int64_t bi = -1;
        double bv = -1.0;
        for (int b = 0; b < g; ++b)
            if (pi[b] >= 0 && (pv[b] > bv || (pv[b] == bv && pi[b] < bi))) {
                bv = pv[b];
                bi = pi[b];
            }
        double val = 0.0;
        if (bi >= 0) SBD_CUDA(cudaMemcpyAsync(&val, s.U + bi, sizeof(double), cudaMemcpyDeviceToHost, stream));
        SBD_CUDA(cudaStreamSynchronize(stream));
        if (val < 0.0) {
            e_negate_kernel<<<g, kEThreads, 0, stream>>>(s.U, s.N);
            SBD_LAUNCH("e_negate_kernel");
        }
        j->vec.resize((size_t)s.N);
        SBD_CUDA(cudaMemcpyAsync(j->vec.data(), s.U, (size_t)s.N * 8, cudaMemcpyDeviceToHost, stream));
        SBD_CUDA(cudaStreamSynchronize(stream));
    }
    j->res.t_done = now_seconds(t0);
    j->finished = true;
    free_slot(s);
}

// descriptors and chunk table of the current slots into the pinned staging block
void sbd_engine_s::write_stage()
{
    Header *h = h_hdr();
    SlotDev *sd = h_slots();
    int *cs = h_cslot();
    int64_t *co = h_coff();
    int nchunk = 0;
    h->nslot = (int)slots.size();
    for (int i = 0; i < (int)slots.size(); ++i) {
        Slot &s = slots[i];
        SlotDev d{};
        if (s.job) {
            const Ctx &c = ctx_of(s.handle);
            d.N = s.N;
            d.V = s.V;
            d.W = s.W;
            d.U = s.U;
            d.HU = s.HU;
            d.TC = s.TC;
            d.c32 = s.c32;
            d.hd = c.hd;
            d.T = s.small;
            d.Y = s.small + kEMaxSub * kEMaxSub;
            d.theta = s.small + 2 * kEMaxSub * kEMaxSub;
            d.coef = d.theta + kEMaxSub;
            d.red = d.coef + kEMaxSub;
            d.delta = opt.delta;
            d.k = s.k;
            d.kind = s.kind;
            d.nk = s.nk;
            d.chunk0 = nchunk;
            for (int64_t off = 0; off < s.N; off += kChunk) {
                cs[nchunk] = i;
                co[nchunk] = off;
                ++nchunk;
            }
            d.chunk1 = nchunk;
            s.chunk0 = d.chunk0;
            s.chunk1 = d.chunk1;
        }
        sd[i] = d;
    }
    h->nchunk = nchunk;
}

// the batched sigma slot lists: mixed for kGrow slots (new basis vector), FP64 for kCheck slots (Ritz vector)
void sbd_engine_s::build_sigma_lists()
{
    s32.clear();
    s64.clear();
    for (Slot &s : slots) {
        if (!s.job) continue;
        Ctx &c = ctx_of(s.handle);
        const int ke = (s.kind & kRestart) ? s.nk : s.k;
        if (s.kind & kGrow) s32.push_back(SigmaSlot{&c, s.c32, s.W + (int64_t)ke * s.N, s.V + (int64_t)ke * s.N, c.work_t});
        if (s.kind & kCheck) s64.push_back(SigmaSlot{&c, s.U, s.TC, nullptr, c.work_t});
    }
    sigma_batch_set(sb32, s32.data(), (int)s32.size());
    sigma_batch_set(sb64, s64.data(), (int)s64.size());
}

void sbd_engine_s::capture()
{
    Header *hd = d_hdr();
    SlotDev *sd = d_slots();
    const int *cs = d_cslot();
    const int64_t *co = d_coff();
    const int nsl = (int)slots.size();
    const int gv = grid_vec;
    auto begin = [&]() {
        SBD_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        return sbd_launch_count();
    };
    auto end = [&](cudaGraphExec_t &exec) {
        cudaGraph_t g = nullptr;
        SBD_CUDA(cudaStreamEndCapture(stream, &g));
        SBD_CUDA(cudaGraphInstantiate(&exec, g, 0));
        (void)cudaGraphDestroy(g);
    };
    // graph A: Rayleigh-Ritz and the corrections
    int64_t l0 = begin();
    SBD_CUDA(cudaMemcpyAsync(dstage, hstage, stage_bytes, cudaMemcpyHostToDevice, stream));
    e_jacobi_kernel<<<nsl, 256, 2 * sizeof(double) * kEMaxSub * kEMaxSub, stream>>>(hd, sd);
    SBD_LAUNCH("e_jacobi_kernel");
    e_ritz_kernel<<<gv, kEThreads, 0, stream>>>(hd, sd, cs, co, partial);
    SBD_LAUNCH("e_ritz_kernel");
    e_final_kernel<<<nsl, 256, 0, stream>>>(hd, sd, partial, kFinRitz);
    SBD_LAUNCH("e_final_kernel");
    e_status_kernel<<<(nsl + 127) / 128, 128, 0, stream>>>(hd, sd, dstatus);
    SBD_LAUNCH("e_status_kernel");
    SBD_CUDA(cudaMemcpyAsync(hstatus, dstatus, sizeof(Status) * nsl, cudaMemcpyDeviceToHost, stream));
    launches_A = sbd_launch_count() - l0;
    end(gA);
    // graph B: restart, Gram-Schmidt, new basis vector and its sigma, T extension, FP64 checks
    l0 = begin();
    SBD_CUDA(cudaMemcpyAsync(dstage, hstage, stage_bytes, cudaMemcpyHostToDevice, stream));
    e_compress_kernel<<<gv, kEThreads, 0, stream>>>(hd, sd, cs, co);
    SBD_LAUNCH("e_compress_kernel");
    e_restart_T_kernel<<<nsl, 256, 0, stream>>>(hd, sd);
    SBD_LAUNCH("e_restart_T_kernel");
    e_dots_kernel<0, true><<<gv, kEThreads, 0, stream>>>(hd, sd, cs, co, partial);
    SBD_LAUNCH("e_dots_kernel");
    e_final_kernel<<<nsl, 256, 0, stream>>>(hd, sd, partial, kFinGS1);
    SBD_LAUNCH("e_final_kernel");
    e_axpy_kernel<true, false><<<gv, kEThreads, 0, stream>>>(hd, sd, cs, co, partial);
    SBD_LAUNCH("e_axpy_kernel");
    e_final_kernel<<<nsl, 256, 0, stream>>>(hd, sd, partial, kFinAfter1);
    SBD_LAUNCH("e_final_kernel");
    e_dots_kernel<0, false><<<gv, kEThreads, 0, stream>>>(hd, sd, cs, co, partial);
    SBD_LAUNCH("e_dots_kernel");
    e_final_kernel<<<nsl, 256, 0, stream>>>(hd, sd, partial, kFinGS2);
    SBD_LAUNCH("e_final_kernel");
    e_axpy_kernel<true, true><<<gv, kEThreads, 0, stream>>>(hd, sd, cs, co, partial);
    SBD_LAUNCH("e_axpy_kernel");
    e_final_kernel<<<nsl, 256, 0, stream>>>(hd, sd, partial, kFinAfter);
    SBD_LAUNCH("e_final_kernel");
    e_scale_kernel<<<gv, kEThreads, 0, stream>>>(hd, sd, cs, co);
    SBD_LAUNCH("e_scale_kernel");
    sigma_batch_launch(sb32, stream);
    e_dots_kernel<1, false><<<gv, kEThreads, 0, stream>>>(hd, sd, cs, co, partial);
    SBD_LAUNCH("e_dots_kernel");
    e_final_kernel<<<nsl, 256, 0, stream>>>(hd, sd, partial, kFinExtend);
    SBD_LAUNCH("e_final_kernel");
    sigma_batch_launch(sb64, stream);
    e_dots_kernel<2, true><<<gv, kEThreads, 0, stream>>>(hd, sd, cs, co, partial);
    SBD_LAUNCH("e_dots_kernel");
    e_final_kernel<<<nsl, 256, 0, stream>>>(hd, sd, partial, kFinCheck1);
    SBD_LAUNCH("e_final_kernel");
    e_check_resid_kernel<<<gv, kEThreads, 0, stream>>>(hd, sd, cs, co, partial);
    SBD_LAUNCH("e_check_resid_kernel");
    e_final_kernel<<<nsl, 256, 0, stream>>>(hd, sd, partial, kFinCheck2);
    SBD_LAUNCH("e_final_kernel");
    e_status_kernel<<<(nsl + 127) / 128, 128, 0, stream>>>(hd, sd, dstatus);
    SBD_LAUNCH("e_status_kernel");
    SBD_CUDA(cudaMemcpyAsync(hstatus, dstatus, sizeof(Status) * nsl, cudaMemcpyDeviceToHost, stream));
    launches_B = sbd_launch_count() - l0;
    end(gB);
}

void sbd_engine_s::replay(cudaGraphExec_t g, int64_t launches)
{
    SBD_CUDA(cudaGraphLaunch(g, stream));
    SBD_CUDA(cudaStreamSynchronize(stream));
    graph_launches++;
    kernel_launches += launches;
}

// Autotuner for the mixed batched sigma: times one launch sequence for each rows-per-item
// candidate that fits shared memory, on the slots admitted so far, and keeps the fastest.
void sbd_engine_s::autotune()
{
    const int ms = std::max(opt.max_strings, 1);
    std::vector<SigmaSlot> list;
    for (Slot &s : slots)
        if (s.job) {
            Ctx &c = ctx_of(s.handle);
            list.push_back(SigmaSlot{&c, s.c32, s.W, s.V, c.work_t});
        }
    cudaEvent_t a, b;
    SBD_CUDA(cudaEventCreate(&a));
    SBD_CUDA(cudaEventCreate(&b));
    const int cand[4] = {8, 4, 2, 1};
    float best = INFINITY;
    int best_r = 0;
    for (int ci = 0; ci < 4; ++ci) {
        const int R = cand[ci];
        if (!sigma_batch_fits(SBD_MIXED, R, ms, opt.max_norb, device)) continue;
        SigmaBatch *sb = sigma_batch_create(opt.max_slots, SBD_MIXED, R, ms, opt.max_norb, device);
        float t = INFINITY;
        for (int rep = 0; rep < 3; ++rep) {
            sigma_batch_set(sb, list.data(), (int)list.size());
            SBD_CUDA(cudaEventRecord(a, stream));
            sigma_batch_launch(sb, stream);
            SBD_CUDA(cudaEventRecord(b, stream));
            SBD_CUDA(cudaEventSynchronize(b));
            float ms_t = 0.f;
            SBD_CUDA(cudaEventElapsedTime(&ms_t, a, b));
            if (rep > 0) t = std::min(t, ms_t);  // the first run warms up
        }
        tune_ms[ci] = t;
        if (t < best) {
            best = t;
            best_r = R;
        }
        sigma_batch_destroy(sb);
    }
    (void)cudaEventDestroy(a);
    (void)cudaEventDestroy(b);
    if (!best_r) fail(SBD_ERR_UNSUPPORTED, "engine: no sigma configuration fits shared memory");
    rows_per_item = best_r;
    sb32 = sigma_batch_create(opt.max_slots, SBD_MIXED, best_r, ms, opt.max_norb, device);
}

int sbd_engine_s::step()
{
    // admission, in submission order
    while (admit_one()) {
    }
    bool any = false;
    for (Slot &s : slots) any |= s.job != nullptr;
    if (!any) return (int)pending.size();
    if (!sb32) autotune();
    if (!gA) capture();
    steps++;

    // the jobs of this iteration: all, or (fair schedule) those within one smallest-job quantum of
    // the smallest pass (stride scheduling by N; the slot with the smallest pass always runs)
    {
        double pmin = INFINITY;
        int64_t nmin = INT64_MAX;
        for (const Slot &s : slots)
            if (s.job) {
                pmin = std::min(pmin, s.pass);
                nmin = std::min(nmin, s.N);
            }
        vtime = pmin;
        for (Slot &s : slots) {
            s.run = s.job && (opt.schedule == SBD_SCHED_LOCKSTEP || s.pass < pmin + (double)std::max<int64_t>(nmin, 1));
            if (s.run) s.pass += (double)s.N;
        }
    }

    // graph A: Rayleigh-Ritz for every running slot with a basis
    bool anyA = false;
    for (Slot &s : slots) {
        s.kind = 0;
        if (s.run && s.k >= 1) {
            s.kind = kRitz;
            anyA = true;
        }
    }
    if (anyA) {
        write_stage();
        replay(gA, launches_A);
    }
    // decisions
    for (int i = 0; i < (int)slots.size(); ++i) {
        Slot &s = slots[i];
        if (!s.run) continue;
        Job *j = s.job;
        if (s.k == 0) {
            s.kind = kGrow;  // seed: the initial unit vector enters the basis
            s.nk = 0;
            continue;
        }
        const Status &st = hstatus[i];
        const double th = st.theta0, r = sqrt(std::max(0.0, st.resid2));
        j->res.iterations++;
        j->res.energy_mixed = th + j->ecore;
        s.r_mixed = r;
        const bool de_ok = !(j->tol_energy > 0.0) || (std::isfinite(s.theta_prev) && fabs(th - s.theta_prev) <= j->tol_energy);
        s.theta_prev = th;
        if (!std::isfinite(th) || !std::isfinite(r)) {
            finish(s, SBD_ERR_BREAKDOWN, false);
            continue;
        }
        s.hist.push_back(r);
        // the mixed residual has stopped halving at a level where FP32 rounding can matter
        const size_t nh = s.hist.size();
        const bool stalled = nh > 8 && r > 0.5 * s.hist[nh - 9] && r < 1e-4 * fabs(th);
        if ((r <= s.thr && de_ok) || stalled || j->res.iterations >= opt.max_iter) {
            s.kind = kCheck;
        } else {
            s.kind = kGrow;
            if (s.k + 1 > opt.max_subspace) {
                s.kind |= kRestart;
                s.nk = std::min(nkeep, s.k);
            }
        }
    }
    // graph B
    bool anyB = false;
    for (Slot &s : slots) anyB |= s.run && s.kind;
    if (anyB) {
        write_stage();
        build_sigma_lists();
        replay(gB, launches_B);
    }
    for (int i = 0; i < (int)slots.size(); ++i) {
        Slot &s = slots[i];
        if (!s.run || !s.kind) continue;
        Job *j = s.job;
        const Status &st = hstatus[i];
        if (s.kind & kGrow) {
            const int ke = (s.kind & kRestart) ? s.nk : s.k;
            if (s.kind & kRestart) j->res.restarts++;
            if (st.scale > 0.0) {
                s.k = ke + 1;
                j->res.sigma_mixed++;
            } else {
                s.k = ke;
                if (s.k == 0) {
                    finish(s, SBD_ERR_BREAKDOWN, false);
                    continue;
                }
                // no new direction: check what we have
                s.thr = INFINITY;
            }
        }
        if (s.kind & kCheck) {
            j->res.sigma_fp64++;
            const double uu = st.uu > 0.0 ? st.uu : 1.0;
            const double r64 = sqrt(std::max(0.0, st.r64sq) / uu);
            j->res.energy = st.theta64 + j->ecore;
            j->res.residual = r64;
            if (r64 <= j->tol) {
                finish(s, SBD_OK, true);
            } else if (j->res.iterations >= opt.max_iter) {
                finish(s, SBD_NOT_CONVERGED, true);
            } else {
                // FP32 noise or a premature stop: iterate on to half the mixed residual seen here
                s.thr = std::min(j->tol, 0.5 * s.r_mixed);
                s.hist.clear();
            }
        }
    }
    int remaining = (int)pending.size();
    for (Slot &s : slots) remaining += s.job != nullptr;
    return remaining;
}

namespace {


template <typename F>
int eguard(F &&f)
{
    try {
        return f();
    } catch (const Error &e) {
        set_thread_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_thread_error("host allocation failed");
        return SBD_ERR_OUT_OF_MEMORY;
    } catch (...) {
        set_thread_error("unexpected internal error");
        return SBD_ERR_CUDA;
    }
}

}  // namespace

extern "C" {

void sbd_engine_default_options(sbd_engine_options *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->max_slots = 64;
    o->max_subspace = 12;
    o->max_iter = 200;
    o->max_norb = 64;
    o->max_strings = 20000;
    o->rows_per_item = 0;
    o->delta = 1e-4;
    o->table_bytes_per_string = 16384;
    o->schedule = SBD_SCHED_FAIR;
}

int sbd_engine_create(sbd_engine *out, const sbd_engine_options *opt, void *stream)
{
    if (!out) return SBD_ERR_INVALID_ARG;
    *out = nullptr;
    sbd_engine_options o;
    sbd_engine_default_options(&o);
    if (opt) o = *opt;
    if (o.max_slots < 1 || o.max_slots > 1024 || o.max_subspace < 3 || o.max_subspace > kEMaxSub ||
        o.max_iter < 1 || o.max_norb < 1 || o.max_norb > 64 || o.max_strings < 1 ||
        o.max_strings > (int)kMaxStringsPerSpin || !(o.rows_per_item == 0 || o.rows_per_item == 1 ||
                                                     o.rows_per_item == 2 || o.rows_per_item == 4 ||
                                                     o.rows_per_item == 8) ||
        !(o.delta > 0.0) || !(o.schedule == SBD_SCHED_FAIR || o.schedule == SBD_SCHED_LOCKSTEP)) {
        set_thread_error("invalid engine options");
        return SBD_ERR_INVALID_ARG;
    }
    if ((o.alloc == nullptr) != (o.free == nullptr)) {
        set_thread_error("engine allocator: give both alloc and free, or neither");
        return SBD_ERR_INVALID_ARG;
    }
    auto *e = new (std::nothrow) sbd_engine_s();
    if (!e) return SBD_ERR_OUT_OF_MEMORY;
    e->opt = o;
    e->stream = (cudaStream_t)stream;
    const int rc = eguard([&] {
        e->init();
        return SBD_OK;
    });
    if (rc != SBD_OK) {
        e->destroy();
        delete e;
        return rc;
    }
    *out = e;
    return SBD_OK;
}

int sbd_engine_destroy(sbd_engine e)
{
    if (!e) return SBD_ERR_INVALID_ARG;
    const int rc = eguard([&] {
        e->destroy();
        return SBD_OK;
    });
    delete e;
    return rc;
}

int sbd_engine_submit(sbd_engine e, int norb, int nalpha, int nbeta, const double *h, const double *eri,
                      const uint64_t *A, int64_t nA, const uint64_t *B, int64_t nB, double ecore, double tol,
                      double tol_energy, int keep_vector, int64_t *job)
{
    if (!e || !job || !h || !eri || !A || !B || nA < 1 || nB < 1 || !(tol > 0.0) || tol_energy < 0.0) {
        set_thread_error("sbd_engine_submit: invalid argument");
        return SBD_ERR_INVALID_ARG;
    }
    if (norb < 1 || norb > 64) {
        set_thread_error("norb must be in 1..64");
        return SBD_ERR_NORB;
    }
    if (norb > e->opt.max_norb || nA > e->opt.max_strings || nB > e->opt.max_strings) {
        set_thread_error("job exceeds the engine's max_norb or max_strings");
        return SBD_ERR_UNSUPPORTED;
    }
    return eguard([&] {
        auto j = std::make_unique<Job>();
        j->id = e->next_id++;
        j->norb = norb;
        j->na = nalpha;
        j->nb = nbeta;
        const size_t n2 = (size_t)norb * norb;
        j->h.resize(n2);
        j->eri.resize(n2 * n2);
        j->A.resize((size_t)nA);
        j->B.resize((size_t)nB);
        SBD_CUDA(cudaMemcpy(j->h.data(), h, n2 * 8, cudaMemcpyDefault));
        SBD_CUDA(cudaMemcpy(j->eri.data(), eri, n2 * n2 * 8, cudaMemcpyDefault));
        SBD_CUDA(cudaMemcpy(j->A.data(), A, (size_t)nA * 8, cudaMemcpyDefault));
        SBD_CUDA(cudaMemcpy(j->B.data(), B, (size_t)nB * 8, cudaMemcpyDefault));
        j->ecore = ecore;
        j->tol = tol;
        j->tol_energy = tol_energy;
        j->keep_vector = keep_vector != 0;
        j->res.status = SBD_PENDING;
        j->res.t_submit = now_seconds(e->t0);
        j->res.ndets = nA * nB;
        *job = j->id;
        e->pending.push_back(j.get());
        e->jobs[j->id] = std::move(j);
        return SBD_OK;
    });
}

int sbd_engine_step(sbd_engine e, int *remaining)
{
    if (!e) return SBD_ERR_INVALID_ARG;
    return eguard([&] {
        const int r = e->step();
        if (remaining) *remaining = r;
        return SBD_OK;
    });
}

int sbd_engine_run(sbd_engine e)
{
    if (!e) return SBD_ERR_INVALID_ARG;
    return eguard([&] {
        while (e->step() > 0) {
        }
        return SBD_OK;
    });
}

int sbd_engine_result(sbd_engine e, int64_t job, sbd_job_result *out)
{
    if (!e || !out) return SBD_ERR_INVALID_ARG;
    auto it = e->jobs.find(job);
    if (it == e->jobs.end()) {
        set_thread_error("unknown job id");
        return SBD_ERR_INVALID_ARG;
    }
    *out = it->second->res;
    return it->second->finished ? SBD_OK : SBD_PENDING;
}

int sbd_engine_vector(sbd_engine e, int64_t job, double *out, int64_t n)
{
    if (!e || !out) return SBD_ERR_INVALID_ARG;
    auto it = e->jobs.find(job);
    if (it == e->jobs.end() || !it->second->finished || it->second->vec.empty() ||
        n != (int64_t)it->second->vec.size()) {
        set_thread_error("job unknown, unfinished, without a kept vector, or n != nA*nB");
        return SBD_ERR_INVALID_ARG;
    }
    return eguard([&] {
        SBD_CUDA(cudaMemcpy(out, it->second->vec.data(), (size_t)n * 8, cudaMemcpyDefault));
        return SBD_OK;
    });
}

int sbd_engine_release(sbd_engine e, int64_t job)
{
    if (!e) return SBD_ERR_INVALID_ARG;
    auto it = e->jobs.find(job);
    if (it == e->jobs.end() || !it->second->finished) {
        set_thread_error("job unknown or unfinished");
        return SBD_ERR_INVALID_ARG;
    }
    e->jobs.erase(it);
    return SBD_OK;
}

int sbd_engine_get_stats(sbd_engine e, sbd_engine_stats *out)
{
    if (!e || !out) return SBD_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->steps = e->steps;
    out->graph_launches = e->graph_launches;
    out->kernel_launches = e->kernel_launches;
    out->rows_per_item = e->rows_per_item;
    for (int i = 0; i < 4; ++i) out->tune_ms[i] = e->tune_ms[i];
    out->bytes_in_use = e->bytes_in_use;
    out->bytes_peak = e->bytes_peak;
    out->requeued = e->requeued;
    for (const Slot &s : e->slots) out->active += s.job != nullptr;
    out->pending = (int)e->pending.size();
    for (const auto &kv : e->jobs) out->done += kv.second->finished;
    return SBD_OK;
}

double sbd_engine_clock(sbd_engine e) { return e ? now_seconds(e->t0) : 0.0; }

}  // extern "C"
