// Matrix-free sigma product s = H c on the selected space A x B (paper
// Sec. II-A/B, Eq. 4; the three task types of Sec. III-B).
//
// With E_pq split by spin, H = H_alpha (x) 1 + 1 (x) H_beta + V_ab where
//   H_alpha(I,J) = <I| sum h_pq E_pq + 1/2 sum (pq|rs)(E_pq E_rs - d_qr E_ps) |J>
// evaluated by the same-spin Slater-Condon rules between alpha strings, and
//   V_ab = sum_pqrs (pq|rs) E^alpha_pq E^beta_rs.
// Because every alpha operator pair commutes with the beta creators, the
// phases factorise: <Ia Ib|E^a_pq E^b_rs|Ja Jb> = <Ia|E_pq|Ja><Ib|E_rs|Jb>.
// With J_x[uv] = sum_{k in x} (uv|kk) this gives, for output (ia, ib):
//   s = Hd(ia,ib) c(ia,ib)                                          diagonal
//     + sum_{jb in doubles(ib)} Hb(ib,jb) c(ia,jb)
//     + sum_{jb in singles(ib), code rs, phase t} [Hb(ib,jb) + t J_ia[rs]] c(ia,jb)
//     + sum_{ja in doubles(ia)} Ha(ia,ja) c(ja,ib)
//     + sum_{ja in singles(ia), code pq, phase u} [Ha(ia,ja) + u J_ib[pq]] c(ja,ib)
//     + sum_{ja in singles(ia)} sum_{jb in singles(ib)} u t (pq|rs) c(ja,jb)
// The first three lines are a gather inside row ia of C ("beta pass"), the
// next two the same gather inside column ib, run on the transpose C^T
// ("alpha pass", same kernel), and the last line is the alpha-beta pass.
//
// Every output element is owned by one thread group in each pass and each
// pass adds into it in program order, so results are deterministic.  Rows of
// C are staged in shared memory, R rows interleaved per column so one vector
// load fetches the same column of all R rows; the inner gathers then hit
// shared memory only.  The lists are the padded sigma copies: each lane of an
// 8-lane group fetches 4 entries with 16-byte loads, and the next column's
// list bounds are prefetched.  The phase of a single is folded into the
// shared-memory coefficient tables, which are indexed by 2*code + (phase<0).
// Precision T = double (FP64), float (mixed: FP32 amplitudes, integrals,
// products and per-list sums, each list sum and the diagonal term accumulated
// into the FP64 output), or F2 (FP64-accurate arithmetic on the FP32 pipe:
// every amplitude, integral and matrix element is an unevaluated sum hi + lo
// of two floats, products are exact hi*hi (a fused multiply-add recovers the
// rounding error, Dekker's product) plus the two cross terms, and sums use
// Knuth's two-sum; on GB300 the FP32 pipe is ~64x the FP64 pipe).
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "pair.cuh"

namespace sbd {

namespace {

constexpr int kGroup = 8;  // lanes cooperating on one output column
constexpr int kGroupsPerWarp = 32 / kGroup;

template <typename T>
constexpr bool kIsF2 = std::is_same<T, F2>::value;

// element type of the vectors a pass reads (the pair precision reads FP64 vectors)
template <typename T>
struct In {
    using type = T;
};
template <>
struct In<F2> {
    using type = double;
};

template <typename T>
__device__ __forceinline__ T conv(double x)
{
    if constexpr (kIsF2<T>) return f2_split(x);
    else return (T)x;
}
template <typename T>
__device__ __forceinline__ T conv(float x)
{
    return (T)x;
}

template <typename T>
struct Threads;
template <>
struct Threads<F2> {
    static constexpr int value = 1024;  // latency-bound at 512 (209 vs 292 ms per sigma at 1.0e8 dets)
};
template <>
struct Threads<float> {
    static constexpr int value = 1024;
};
template <>
struct Threads<double> {
    static constexpr int value = 512;
};

template <typename T, int R>
struct VecIO;
template <>
struct VecIO<float, 4> {
    __device__ static void ld(const float *p, float (&v)[4])
    {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    }
    __device__ static void st(float *p, const float (&v)[4])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct VecIO<float, 2> {
    __device__ static void ld(const float *p, float (&v)[2])
    {
        const float2 x = *reinterpret_cast<const float2 *>(p);
        v[0] = x.x;
        v[1] = x.y;
    }
    __device__ static void st(float *p, const float (&v)[2])
    {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    }
};
template <>
struct VecIO<double, 2> {
    __device__ static void ld(const double *p, double (&v)[2])
    {
        const double2 x = *reinterpret_cast<const double2 *>(p);
        v[0] = x.x;
        v[1] = x.y;
    }
    __device__ static void st(double *p, const double (&v)[2])
    {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
};
template <>
struct VecIO<F2, 2> {
    __device__ static void ld(const F2 *p, F2 (&v)[2])
    {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = F2(x.x, x.y);
        v[1] = F2(x.z, x.w);
    }
    __device__ static void st(F2 *p, const F2 (&v)[2])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
    }
};
template <>
struct VecIO<F2, 1> {
    __device__ static void ld(const F2 *p, F2 (&v)[1])
    {
        const float2 x = *reinterpret_cast<const float2 *>(p);
        v[0] = F2(x.x, x.y);
    }
    __device__ static void st(F2 *p, const F2 (&v)[1]) { *reinterpret_cast<float2 *>(p) = make_float2(v[0].hi, v[0].lo); }
};
template <typename T>
struct VecIO<T, 1> {
    __device__ static void ld(const T *p, T (&v)[1]) { v[0] = *p; }
    __device__ static void st(T *p, const T (&v)[1]) { *p = v[0]; }
};

template <int R, typename T>
__device__ __forceinline__ T pick(const T (&v)[R], int i)
{
    T out = v[0];
#pragma unroll
    for (int r = 1; r < R; ++r)
        if (i == r) out = v[r];
    return out;
}

__host__ __device__ constexpr size_t round16(size_t b) { return (b + 15) & ~(size_t)15; }

__device__ __forceinline__ int pk_j(uint32_t pk) { return (int)(pk & kPackJMask); }
__device__ __forceinline__ int pk_key(uint32_t pk) { return (int)(pk >> kPackKeyShift); }  // 2*code + neg
__device__ __forceinline__ int pk_code(uint32_t pk) { return (int)(pk >> (kPackKeyShift + 1)); }
__device__ __forceinline__ bool pk_neg(uint32_t pk) { return ((pk >> kPackKeyShift) & 1u) != 0u; }

// Excitation lists of the column spin (padded sigma copies), in the layout each precision
// reads.  Every list starts at a multiple of kListPad entries.  The 8 lanes of a group read a
// list in chunks of up to 32 slots: in a chunk, lane l takes slots 4l..4l+3 (two 2-entry loads),
// and entry u of the lane is the slot the u-th 128-bit shared-memory phase of the pass gathers
// for that lane.  (Taking the two halves of a chunk as two contiguous runs instead halves the
// sectors each load touches but loses the L1 hits of the second load, and was slower at 1.0e8
// determinants.)
__device__ __forceinline__ void list_slots(int64_t s0, int cb, int lc, int lig, int64_t &e0, int64_t &e1)
{
    (void)lc;
    e0 = s0 + cb + 4 * lig;
    e1 = e0 + 2;
}

template <typename T>
struct Lists;
template <>
struct Lists<float> {
    const uint2 *s;  // (packed single, value bits)
    const uint2 *d;  // (target, value bits)
    __device__ void singles4(int64_t e0, int64_t e1, uint32_t (&pk)[4], float (&v)[4]) const
    {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(s + e0));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(s + e1));
        pk[0] = a.x, v[0] = __uint_as_float(a.y), pk[1] = a.z, v[1] = __uint_as_float(a.w);
        pk[2] = b.x, v[2] = __uint_as_float(b.y), pk[3] = b.z, v[3] = __uint_as_float(b.w);
    }
    __device__ void doubles4(int64_t e0, int64_t e1, int (&j)[4], float (&v)[4]) const
    {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(d + e0));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(d + e1));
        j[0] = (int)a.x, v[0] = __uint_as_float(a.y), j[1] = (int)a.z, v[1] = __uint_as_float(a.w);
        j[2] = (int)b.x, v[2] = __uint_as_float(b.y), j[3] = (int)b.z, v[3] = __uint_as_float(b.w);
    }
};
template <>
struct Lists<double> {
    const uint32_t *spk;
    const double *sv;
    const int32_t *dj;
    const double *dv;
    __device__ void singles4(int64_t e0, int64_t e1, uint32_t (&pk)[4], double (&v)[4]) const
    {
        const uint2 a = __ldg(reinterpret_cast<const uint2 *>(spk + e0));
        const uint2 a1 = __ldg(reinterpret_cast<const uint2 *>(spk + e1));
        const double2 b = __ldg(reinterpret_cast<const double2 *>(sv + e0));
        const double2 c = __ldg(reinterpret_cast<const double2 *>(sv + e1));
        pk[0] = a.x, pk[1] = a.y, pk[2] = a1.x, pk[3] = a1.y;
        v[0] = b.x, v[1] = b.y, v[2] = c.x, v[3] = c.y;
    }
    __device__ void doubles4(int64_t e0, int64_t e1, int (&j)[4], double (&v)[4]) const
    {
        const int2 a = __ldg(reinterpret_cast<const int2 *>(dj + e0));
        const int2 a1 = __ldg(reinterpret_cast<const int2 *>(dj + e1));
        const double2 b = __ldg(reinterpret_cast<const double2 *>(dv + e0));
        const double2 c = __ldg(reinterpret_cast<const double2 *>(dv + e1));
        j[0] = a.x, j[1] = a.y, j[2] = a1.x, j[3] = a1.y;
        v[0] = b.x, v[1] = b.y, v[2] = c.x, v[3] = c.y;
    }
};

template <>
struct Lists<F2> {
    const uint32_t *spk;
    const float2 *sv;
    const int32_t *dj;
    const float2 *dv;
    __device__ void singles4(int64_t e0, int64_t e1, uint32_t (&pk)[4], F2 (&v)[4]) const
    {
        const uint2 a = __ldg(reinterpret_cast<const uint2 *>(spk + e0));
        const uint2 a1 = __ldg(reinterpret_cast<const uint2 *>(spk + e1));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(sv + e0));
        const float4 c = __ldg(reinterpret_cast<const float4 *>(sv + e1));
        pk[0] = a.x, pk[1] = a.y, pk[2] = a1.x, pk[3] = a1.y;
        v[0] = F2(b.x, b.y), v[1] = F2(b.z, b.w), v[2] = F2(c.x, c.y), v[3] = F2(c.z, c.w);
    }
    __device__ void doubles4(int64_t e0, int64_t e1, int (&j)[4], F2 (&v)[4]) const
    {
        const int2 a = __ldg(reinterpret_cast<const int2 *>(dj + e0));
        const int2 a1 = __ldg(reinterpret_cast<const int2 *>(dj + e1));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(dv + e0));
        const float4 c = __ldg(reinterpret_cast<const float4 *>(dv + e1));
        j[0] = a.x, j[1] = a.y, j[2] = a1.x, j[3] = a1.y;
        v[0] = F2(b.x, b.y), v[1] = F2(b.z, b.w), v[2] = F2(c.x, c.y), v[3] = F2(c.z, c.w);
    }
};

template <typename T>
struct RowArgs {
    const typename In<T>::type *X;  // [nrow][ncol]
    int64_t nrow, ncol;
    int64_t ncol_out;  // output columns (list sources); ncol except for row-block sigma
    double *Y;  // output element (row r, column c) at r*y_rs + c*y_cs
    int64_t y_rs, y_cs;
    int accumulate;
    const double *hd;    // optional diagonal, indexed like Y
    const double *xd64;  // optional FP64 amplitudes [nrow][ncol] for the diagonal term
    float *rowmax;       // optional (FP32 only): rowmax[r] = max_c |X[r][c]| of every row of the pass
    const uint64_t *row_strings;
    int norb;
    const double *eri;  // FP64 integrals, for the J vectors of the staged rows
    const int64_t *s_ptr, *d_ptr;
    Lists<T> lists;
    // mixed passes over column halves (row_halves): the column spin's lists split at `half`
    const int64_t *hls_ptr, *hld_ptr;  // singles, doubles: [2n + 1]
    const uint2 *hls;                  // (packed single, FP32 value bits)
    const float *hldv;                 // doubles: FP32 values
    const uint16_t *hldt;              // doubles: targets relative to their column half
    int64_t half;
};

// Gather pass over rows of X: each CTA stages R consecutive rows, then every
// output column c sums its excitation list (column spin) inside those rows.
// row_group() does one group of rows starting at r0; the single-instance
// kernel strides over the groups, the batched kernel takes (instance, group)
// items from a work counter.
template <typename T, int R, bool STAGED>
__device__ __forceinline__ void row_group(const RowArgs<T> &a, int64_t r0, unsigned char *smem)
{
    constexpr int kThreads = Threads<T>::value;
    const int n2 = a.norb * a.norb;
    const size_t xs_bytes = STAGED ? round16((size_t)a.ncol * R * sizeof(T)) : 0;
    T *Xs = reinterpret_cast<T *>(smem);
    T *Js = reinterpret_cast<T *>(smem + xs_bytes);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gi = lane / kGroup, lig = lane % kGroup;
    const int64_t ngroups = (kThreads / 32) * kGroupsPerWarp;
    {
        const int nr = (int)min((int64_t)R, a.nrow - r0);
        __syncthreads();
        // row maxima (FP32 pass only): largest |x| as the bit pattern of a non-negative float, so a
        // NaN amplitude leaves a NaN maximum
        unsigned rmax[R];
#pragma unroll
        for (int r = 0; r < R; ++r) rmax[r] = 0u;
        constexpr bool kMax = std::is_same<T, float>::value;
        if (STAGED) {
            for (int64_t c = tid; c < a.ncol; c += kThreads) {
                T v[R];
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = r < nr ? conv<T>(a.X[(r0 + r) * a.ncol + c]) : T(0);
                VecIO<T, R>::st(Xs + c * R, v);
                if constexpr (kMax) {
#pragma unroll
                    for (int r = 0; r < R; ++r) rmax[r] = max(rmax[r], __float_as_uint(fabsf(v[r])));
                }
            }
        } else if constexpr (kMax) {
            if (a.rowmax)
                for (int64_t c = tid; c < a.ncol; c += kThreads) rmax[0] = max(rmax[0], __float_as_uint(fabsf(a.X[r0 * a.ncol + c])));
        }
        __shared__ unsigned red_max[kMax ? R : 1][kMax ? kThreads / 32 : 1];
        if constexpr (kMax) {
            if (a.rowmax) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const unsigned w = __reduce_max_sync(0xffffffffu, rmax[r]);
                    if (lane == 0) red_max[r][warp] = w;
                }
            }
        }
        // sign-folded J table: row key = 2*code + neg holds (neg ? -1 : 1) * J_r[code]; code 0 rows
        // stay zero (no single has code 0; padding entries point there)
        for (int key = tid; key < 2 * n2; key += kThreads) {
            const int code = key >> 1;
            T v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                double s = 0.0;
                if (r < nr && code != 0)
                    for (uint64_t m = a.row_strings[r0 + r]; m; m &= m - 1ull) {
                        const int k = __ffsll((long long)m) - 1;
                        s += __ldg(a.eri + (size_t)code * n2 + (size_t)k * (a.norb + 1));
                    }
                v[r] = conv<T>((key & 1) ? -s : s);
            }
            VecIO<T, R>::st(Js + (size_t)key * R, v);
        }
        __syncthreads();
        if constexpr (kMax) {
            if (a.rowmax && tid < nr) {
                unsigned m = 0u;
                for (int w = 0; w < kThreads / 32; ++w) m = max(m, red_max[tid][w]);
                a.rowmax[r0 + tid] = __uint_as_float(m);
            }
        }

        int64_t cb = (int64_t)warp * kGroupsPerWarp;
        int64_t nxt_s0 = 0, nxt_s1 = 0, nxt_d0 = 0, nxt_d1 = 0;
        if (cb + gi < a.ncol_out) {
            nxt_s0 = a.s_ptr[cb + gi];
            nxt_s1 = a.s_ptr[cb + gi + 1];
            nxt_d0 = a.d_ptr[cb + gi];
            nxt_d1 = a.d_ptr[cb + gi + 1];
        }
        for (; cb < a.ncol_out; cb += ngroups) {
            const int64_t c = cb + gi;
            const bool valid = c < a.ncol_out;
            const int64_t s0 = nxt_s0, s1 = nxt_s1, d0 = nxt_d0, d1 = nxt_d1;
            if (c + ngroups < a.ncol_out) {  // prefetch the next column's list bounds
                nxt_s0 = a.s_ptr[c + ngroups];
                nxt_s1 = a.s_ptr[c + ngroups + 1];
                nxt_d0 = a.d_ptr[c + ngroups];
                nxt_d1 = a.d_ptr[c + ngroups + 1];
            }
            T acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = T(0);
            if (valid) {
                const int ls = (int)(s1 - s0), ld = (int)(d1 - d0);
                for (int cb = 0; cb < ls; cb += kGroup * kListPad) {
                    const int lc = min(kGroup * kListPad, ls - cb);
                    if (kListPad * lig >= lc) break;
                    int64_t e0, e1;
                    list_slots(s0, cb, lc, lig, e0, e1);
                    uint32_t pk[4];
                    T v[4];
                    a.lists.singles4(e0, e1, pk, v);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        T xj[R], jv[R];
                        if (STAGED) VecIO<T, R>::ld(Xs + (size_t)pk_j(pk[u]) * R, xj);
                        else xj[0] = conv<T>(a.X[r0 * a.ncol + pk_j(pk[u])]);
                        VecIO<T, R>::ld(Js + (size_t)pk_key(pk[u]) * R, jv);
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            if constexpr (kIsF2<T>) {
                                f2_mac(acc[r], v[u], xj[r]);
                                f2_mac(acc[r], jv[r], xj[r]);
                            } else {
                                acc[r] += (v[u] + jv[r]) * xj[r];
                            }
                        }
                    }
                }
                for (int cb = 0; cb < ld; cb += kGroup * kListPad) {
                    const int lc = min(kGroup * kListPad, ld - cb);
                    if (kListPad * lig >= lc) break;
                    int64_t e0, e1;
                    list_slots(d0, cb, lc, lig, e0, e1);
                    int jj[4];
                    T v[4];
                    a.lists.doubles4(e0, e1, jj, v);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        T xj[R];
                        if (STAGED) VecIO<T, R>::ld(Xs + (size_t)jj[u] * R, xj);
                        else xj[0] = conv<T>(a.X[r0 * a.ncol + jj[u]]);
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            if constexpr (kIsF2<T>) f2_mac(acc[r], v[u], xj[r]);
                            else acc[r] += v[u] * xj[r];
                        }
                    }
                }
            }
#pragma unroll
            for (int off = kGroup / 2; off > 0; off >>= 1)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if constexpr (kIsF2<T>) {
                        const F2 o(__shfl_xor_sync(0xffffffffu, acc[r].hi, off, kGroup),
                                   __shfl_xor_sync(0xffffffffu, acc[r].lo, off, kGroup));
                        acc[r] = f2_add(acc[r], o);
                    } else {
                        acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off, kGroup);
                    }
                }
            if (valid && lig < nr) {
                double out;
                if constexpr (kIsF2<T>) out = f2_value(pick<R>(acc, lig));
                else out = (double)pick<R>(acc, lig);
                const int64_t idx = (r0 + lig) * a.y_rs + c * a.y_cs;
                if (a.hd) {
                    double xc;
                    if constexpr (kIsF2<T>) xc = a.X[(r0 + lig) * a.ncol + c];  // the FP64 input itself
                    else xc = a.xd64 ? a.xd64[(r0 + lig) * a.ncol + c]
                                     : (double)(STAGED ? Xs[(size_t)c * R + lig] : a.X[(r0 + lig) * a.ncol + c]);
                    out += a.hd[idx] * xc;
                }
                a.Y[idx] = a.accumulate ? a.Y[idx] + out : out;
            }
        }
    }
}

template <typename T, int R, bool STAGED>
__global__ void __launch_bounds__(Threads<T>::value) row_pass_kernel(const RowArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < a.nrow; r0 += (int64_t)gridDim.x * R) row_group<T, R, STAGED>(a, r0, smem);
}

// Mixed-precision gather pass over 8 rows, one column half at a time.  With 4 rows the whole row
// range fits shared memory; staging 8 rows of one half ([0, half) or [half, ncol)) in the same space
// lets every excitation-list entry, loaded once from L2, feed 8 multiply-adds instead of 4.  Each
// output column sums its entries with targets in the staged half (the split lists of the column
// spin), writes that half's sum (with the diagonal term), and adds the other half's sum after the
// second staging.  The 8 rows are kept as two 4-row interleaved arrays, so a 16-byte gather per
// array has the bank pattern of the 4-row pass; the coefficient table of the singles likewise.
constexpr int kHalfRows = 8;

__host__ __device__ inline size_t halves_smem(int64_t half, int norb)
{
    return (size_t)32 * half + (size_t)64 * norb * norb;
}

__device__ __forceinline__ void row_halves(const RowArgs<float> &a, int64_t r0, unsigned char *smem)
{
    constexpr int kThreads = Threads<float>::value;
    const int n2 = a.norb * a.norb;
    const int64_t hw = a.half;  // rows of the staged arrays: the lower half is the wider one
    float *Xa = reinterpret_cast<float *>(smem);                   // [hw][4]  rows 0-3
    float *Xb = Xa + 4 * hw;                                        // [hw][4]  rows 4-7
    float *Ja = Xb + 4 * hw;                                        // [2 n2][4]
    float *Jb = Ja + 8 * n2;                                        // [2 n2][4]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gi = lane / kGroup, lig = lane % kGroup;
    const int64_t ngroups = (kThreads / 32) * kGroupsPerWarp;
    const int nr = (int)min((int64_t)kHalfRows, a.nrow - r0);
    unsigned rmax[kHalfRows];
#pragma unroll
    for (int r = 0; r < kHalfRows; ++r) rmax[r] = 0u;
    __shared__ unsigned red_h[kHalfRows];
    __syncthreads();  // the previous row group is finished with shared memory
    if (tid < kHalfRows) red_h[tid] = 0u;
    // sign-folded J table of the 8 rows (row key = 2*code + neg; code 0 rows zero)
    for (int key = tid; key < 2 * n2; key += kThreads) {
        const int code = key >> 1;
        float v[kHalfRows];
#pragma unroll
        for (int r = 0; r < kHalfRows; ++r) {
            double sj = 0.0;
            if (r < nr && code != 0)
                for (uint64_t m = a.row_strings[r0 + r]; m; m &= m - 1ull) {
                    const int k = __ffsll((long long)m) - 1;
                    sj += __ldg(a.eri + (size_t)code * n2 + (size_t)k * (a.norb + 1));
                }
            v[r] = (float)((key & 1) ? -sj : sj);
        }
        *reinterpret_cast<float4 *>(Ja + (size_t)key * 4) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(Jb + (size_t)key * 4) = make_float4(v[4], v[5], v[6], v[7]);
    }
    for (int h = 0; h < 2; ++h) {
        const int64_t c0 = h ? a.half : 0, c1 = h ? a.ncol : a.half;
        if (h) __syncthreads();  // every column is finished with the first half
        for (int64_t c = c0 + tid; c < c1; c += kThreads) {
            float v[kHalfRows];
#pragma unroll
            for (int r = 0; r < kHalfRows; ++r) v[r] = r < nr ? a.X[(r0 + r) * a.ncol + c] : 0.f;
            *reinterpret_cast<float4 *>(Xa + (c - c0) * 4) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4 *>(Xb + (c - c0) * 4) = make_float4(v[4], v[5], v[6], v[7]);
#pragma unroll
            for (int r = 0; r < kHalfRows; ++r) rmax[r] = max(rmax[r], __float_as_uint(fabsf(v[r])));
        }
        __syncthreads();
        for (int64_t cb = (int64_t)warp * kGroupsPerWarp; cb < a.ncol_out; cb += ngroups) {
            const int64_t c = cb + gi;
            const bool valid = c < a.ncol_out;
            float acc[kHalfRows];
#pragma unroll
            for (int r = 0; r < kHalfRows; ++r) acc[r] = 0.f;
            if (valid) {
                const int64_t s0 = a.hls_ptr[2 * c + h], s1 = a.hls_ptr[2 * c + h + 1];
                const int64_t d0 = a.hld_ptr[2 * c + h], d1 = a.hld_ptr[2 * c + h + 1];
                const int ls = (int)(s1 - s0), ld = (int)(d1 - d0);
                for (int cb2 = 0; cb2 < ls; cb2 += kGroup * kListPad) {
                    const int lc = min(kGroup * kListPad, ls - cb2);
                    if (kListPad * lig >= lc) break;
                    int64_t e0, e1;
                    list_slots(s0, cb2, lc, lig, e0, e1);
                    const uint4 p0 = __ldg(reinterpret_cast<const uint4 *>(a.hls + e0));
                    const uint4 p1 = __ldg(reinterpret_cast<const uint4 *>(a.hls + e1));
                    const uint32_t pk[4] = {p0.x, p0.z, p1.x, p1.z};
                    const float vv[4] = {__uint_as_float(p0.y), __uint_as_float(p0.w), __uint_as_float(p1.y),
                                         __uint_as_float(p1.w)};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int64_t jl = (pk[u] ? (int64_t)pk_j(pk[u]) - c0 : 0);
                        const float4 xa = *reinterpret_cast<const float4 *>(Xa + jl * 4);
                        const float4 xb = *reinterpret_cast<const float4 *>(Xb + jl * 4);
                        const float4 ja = *reinterpret_cast<const float4 *>(Ja + (size_t)pk_key(pk[u]) * 4);
                        const float4 jb = *reinterpret_cast<const float4 *>(Jb + (size_t)pk_key(pk[u]) * 4);
                        acc[0] += (vv[u] + ja.x) * xa.x;
                        acc[1] += (vv[u] + ja.y) * xa.y;
                        acc[2] += (vv[u] + ja.z) * xa.z;
                        acc[3] += (vv[u] + ja.w) * xa.w;
                        acc[4] += (vv[u] + jb.x) * xb.x;
                        acc[5] += (vv[u] + jb.y) * xb.y;
                        acc[6] += (vv[u] + jb.z) * xb.z;
                        acc[7] += (vv[u] + jb.w) * xb.w;
                    }
                }
                for (int cb2 = 0; cb2 < ld; cb2 += kGroup * kListPad) {
                    const int lc = min(kGroup * kListPad, ld - cb2);
                    if (kListPad * lig >= lc) break;
                    int64_t e0, e1;
                    list_slots(d0, cb2, lc, lig, e0, e1);
                    // entries e0 .. e0 + 3: four values (16 bytes) and four 16-bit targets (8 bytes)
                    const float4 v4 = __ldg(reinterpret_cast<const float4 *>(a.hldv + e0));
                    const uint2 t4 = __ldg(reinterpret_cast<const uint2 *>(a.hldt + e0));
                    const uint32_t jj[4] = {t4.x & 0xFFFFu, t4.x >> 16, t4.y & 0xFFFFu, t4.y >> 16};
                    const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        // targets are relative to the staged half; padding entries: target 0, value 0
                        const int64_t jl = (int64_t)jj[u];
                        const float4 xa = *reinterpret_cast<const float4 *>(Xa + jl * 4);
                        const float4 xb = *reinterpret_cast<const float4 *>(Xb + jl * 4);
                        acc[0] += vv[u] * xa.x;
                        acc[1] += vv[u] * xa.y;
                        acc[2] += vv[u] * xa.z;
                        acc[3] += vv[u] * xa.w;
                        acc[4] += vv[u] * xb.x;
                        acc[5] += vv[u] * xb.y;
                        acc[6] += vv[u] * xb.z;
                        acc[7] += vv[u] * xb.w;
                    }
                }
            }
#pragma unroll
            for (int off = kGroup / 2; off > 0; off >>= 1)
#pragma unroll
                for (int r = 0; r < kHalfRows; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off, kGroup);
            if (valid && lig < nr) {
                double out = (double)pick<kHalfRows>(acc, lig);
                const int64_t idx = (r0 + lig) * a.y_rs + c * a.y_cs;
                if (h == 0) {
                    if (a.hd) {
                        const double xc = a.xd64 ? a.xd64[(r0 + lig) * a.ncol + c] : (double)a.X[(r0 + lig) * a.ncol + c];
                        out += a.hd[idx] * xc;
                    }
                    a.Y[idx] = a.accumulate ? a.Y[idx] + out : out;
                } else {
                    a.Y[idx] += out;
                }
            }
        }
    }
    if (a.rowmax) {  // uniform
#pragma unroll
        for (int r = 0; r < kHalfRows; ++r) {
            const unsigned w = __reduce_max_sync(0xffffffffu, rmax[r]);
            if (lane == 0) atomicMax(red_h + r, w);
        }
        __syncthreads();
        if (tid < nr) a.rowmax[r0 + tid] = __uint_as_float(red_h[tid]);
    }
}

__global__ void __launch_bounds__(Threads<float>::value) row_halves_kernel(const RowArgs<float> a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    for (int64_t r0 = (int64_t)blockIdx.x * kHalfRows; r0 < a.nrow; r0 += (int64_t)gridDim.x * kHalfRows)
        row_halves(a, r0, smem);
}

template <typename T>
struct AbArgs {
    const typename In<T>::type *C;  // [nA][nB]
    double *S;                       // [nA][nB], accumulated
    int64_t nA, nB;
    int norb;
    const typename In<T>::type *eri;  // (pq|rs) as a [norb^2][norb^2] matrix
    const int64_t *as_ptr;
    const uint32_t *as_pk;
    const int64_t *bs_ptr;
    const uint32_t *bs_pk;
};

// Alpha-beta pass: CTA per output row ia.  The alpha single excitations of
// ia are taken R at a time: their rows C[ja,:] are staged interleaved and
// W[rs][k] = u_k (p_k q_k|rs) is tabulated; each output column ib then
// runs over its beta singles (jb, rs, t): acc += t * sum_k W[rs][k] C[ja_k, jb],
// and adds acc to s(ia, ib) with a fire-and-forget reduction (the same thread
// owns (ia, ib) for every group of this row, so the adds land in program order).
template <typename T, int R, bool STAGED>
__device__ __forceinline__ void ab_row(const AbArgs<T> &a, int64_t ia, unsigned char *smem)
{
    constexpr int kThreads = Threads<T>::value;
    const int n2 = a.norb * a.norb;
    const size_t cs_bytes = STAGED ? round16((size_t)a.nB * R * sizeof(T)) : 0;
    T *Cs = reinterpret_cast<T *>(smem);
    T *Ws = reinterpret_cast<T *>(smem + cs_bytes);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gi = lane / kGroup, lig = lane % kGroup;
    const int64_t ngroups = (kThreads / 32) * kGroupsPerWarp;
    {
        const int64_t e0 = a.as_ptr[ia];
        const int K = (int)(a.as_ptr[ia + 1] - e0);
        for (int k0 = 0; k0 < K; k0 += R) {
            const int kr = min(R, K - k0);
            int64_t ja[R];
            int pq[R];
            T u[R];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const bool ok = k < kr;
                const uint32_t pk = ok ? a.as_pk[e0 + k0 + k] : 0u;
                ja[k] = pk_j(pk);
                pq[k] = pk_code(pk);
                u[k] = ok ? (pk_neg(pk) ? T(-1) : T(1)) : T(0);
            }
            __syncthreads();
            if (STAGED) {
                for (int64_t c = tid; c < a.nB; c += kThreads) {
                    T v[R];
#pragma unroll
                    for (int k = 0; k < R; ++k) v[k] = k < kr ? conv<T>(a.C[ja[k] * a.nB + c]) : T(0);
                    VecIO<T, R>::st(Cs + c * R, v);
                }
            }
            // sign-folded W: row key = 2*rs + t holds (t ? -1 : 1) * u_k (p_k q_k|rs); rs = 0 rows zero
            for (int key = tid; key < 2 * n2; key += kThreads) {
                const int code = key >> 1;
                T v[R];
                if constexpr (kIsF2<T>) {
                    const double sg = (key & 1) ? -1.0 : 1.0;
#pragma unroll
                    for (int k = 0; k < R; ++k)
                        v[k] = code ? f2_split(sg * (double)u[k].hi * __ldg(a.eri + (size_t)pq[k] * n2 + code)) : T(0);
                } else {
                    const T sg = (key & 1) ? T(-1) : T(1);
#pragma unroll
                    for (int k = 0; k < R; ++k) v[k] = code ? sg * u[k] * __ldg(a.eri + (size_t)pq[k] * n2 + code) : T(0);
                }
                VecIO<T, R>::st(Ws + (size_t)key * R, v);
            }
            __syncthreads();

            int64_t cb = (int64_t)warp * kGroupsPerWarp;
            int64_t nxt0 = 0, nxt1 = 0;
            if (cb + gi < a.nB) {
                nxt0 = a.bs_ptr[cb + gi];
                nxt1 = a.bs_ptr[cb + gi + 1];
            }
            for (; cb < a.nB; cb += ngroups) {
                const int64_t ib = cb + gi;
                const bool valid = ib < a.nB;
                const int64_t b0 = nxt0, b1 = nxt1;
                if (ib + ngroups < a.nB) {
                    nxt0 = a.bs_ptr[ib + ngroups];
                    nxt1 = a.bs_ptr[ib + ngroups + 1];
                }
                T acc = T(0);
                if (valid) {
                    const int lb = (int)(b1 - b0);
                    for (int cb = 0; cb < lb; cb += kGroup * kListPad) {
                        const int lc = min(kGroup * kListPad, lb - cb);
                        if (kListPad * lig >= lc) break;
                        int64_t e0, e1;
                        list_slots(b0, cb, lc, lig, e0, e1);
                        const uint2 pa = __ldg(reinterpret_cast<const uint2 *>(a.bs_pk + e0));
                        const uint2 pb = __ldg(reinterpret_cast<const uint2 *>(a.bs_pk + e1));
                        const uint32_t pk[4] = {pa.x, pa.y, pb.x, pb.y};
                        T part[4];
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            T cv[R], wv[R];
                            if (STAGED) VecIO<T, R>::ld(Cs + (size_t)pk_j(pk[t]) * R, cv);
                            else cv[0] = conv<T>(a.C[ja[0] * a.nB + pk_j(pk[t])]);
                            VecIO<T, R>::ld(Ws + (size_t)pk_key(pk[t]) * R, wv);
                            if constexpr (kIsF2<T>) {
#pragma unroll
                                for (int k = 0; k < R; ++k) f2_mac(acc, wv[k], cv[k]);
                            } else if constexpr (sizeof(T) == 4) {
                                // FP32: one short chain per entry keeps the four entries independent
                                part[t] = wv[0] * cv[0];
#pragma unroll
                                for (int k = 1; k < R; ++k) part[t] = fma(wv[k], cv[k], part[t]);
                            } else {
                                // FP64 is bound by the FP64 pipe: a single chain needs the fewest operations
#pragma unroll
                                for (int k = 0; k < R; ++k) acc = fma(wv[k], cv[k], acc);
                            }
                        }
                        if constexpr (sizeof(T) == 4) acc += (part[0] + part[1]) + (part[2] + part[3]);
                    }
                }
                double total;
                if constexpr (kIsF2<T>) {
#pragma unroll
                    for (int off = kGroup / 2; off > 0; off >>= 1) {
                        const F2 o(__shfl_xor_sync(0xffffffffu, acc.hi, off, kGroup),
                                   __shfl_xor_sync(0xffffffffu, acc.lo, off, kGroup));
                        acc = f2_add(acc, o);
                    }
                    total = f2_value(acc);
                } else {
#pragma unroll
                    for (int off = kGroup / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off, kGroup);
                    total = (double)acc;
                }
                if (valid && lig == 0) atomicAdd(a.S + ia * a.nB + ib, total);
            }
        }
    }
}

template <typename T, int R, bool STAGED>
__global__ void __launch_bounds__(Threads<T>::value) ab_pass_kernel(const AbArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    for (int64_t ia = blockIdx.x; ia < a.nA; ia += gridDim.x) ab_row<T, R, STAGED>(a, ia, smem);
}

// ---------------------------------------------------------------------------
// Column-stationary alpha-beta pass of the mixed sigma.
//
// For output row ia with alpha singles (ja_k, pq_k, u_k), k < K, and the beta singles of each
// string (ib <- jb with orbital pair {r, s}, phase t; by Hermiticity the singles list of jb names
// every ib that has jb among its singles, with the same phase):
//   s(ia, ib) += sum_{jb} sum_{ib in singles(jb)} t * sum_k W[{r,s}][k] C(ja_k, jb),
//   W[{r,s}][k] = u_k (p_k q_k|rs)                       ((pq|rs) = (pq|sr) for real orbitals)
// The alpha singles are taken in chunks of KC <= 32.  A lane owns one column jb: it holds the KC
// amplitudes C(ja_k, jb) in registers and walks the singles of jb; for each it gathers one
// 4*KC-byte row of W from shared memory (the only shared-memory operand of the multiply-adds,
// 4 bytes per FMA) and adds the FP32 dot product to the row accumulator of ib.
//
// Bank conflicts: a W row is 128 bytes (eight 16-byte chunks).  With KC = 32 lane l reads chunk
// (step + l) mod 8 at each step, so the 8 lanes of a 128-bit phase hit 8 distinct bank groups
// whatever rows they read; with KC = 16 (8) each row holds 2 (4) copies and lanes read their own
// copy, rotated within it.  The lane's registers hold the amplitudes in the same rotated order.
// For large norb the rows are 64 bytes (RS = 4 chunks, KC <= 16): with KC = 16 a row holds one
// copy, the rotation spreads lanes l and l + 4 of a phase over the same four chunks, and two of
// them conflict when their rows lie in the same half of the 128-byte bank window.
//
// Determinism: each FP32 dot product is rounded once onto a fixed-point grid with one scale 2^e per
// output row and added as an integer, and integer addition is exact and order independent, so the
// result does not depend on the order of the shared-memory atomics.  An element of the row receives
// at most m = maxdeg_beta * (chunks of the row) contributions v.  Each v is split as
// v = hi * 2^L + lo with 0 <= lo < 2^L, L = 32 - bitlength(m), and lo and hi are added with 32-bit
// integer atomics into two words per element (random 32-bit shared-memory atomics run several times
// faster than 64-bit ones): the lo word cannot overflow (m * 2^L < 2^32), and e is chosen so that
// the largest possible row sum of |v|,
//   maxdeg_beta * max|(pq|rs)| * sum_k max_jb |C(ja_k, jb)|  (times 2^e),
// stays below 2^(30+L), which keeps the sum of the hi words inside a signed 32-bit word.  The grid
// step is then about 2^-(30+L) >= 2^-52 of that bound, far below FP32 rounding of the products.
// The element is hi_sum * 2^L + lo_sum exactly; the row is added to s(ia, :) in FP64 by the CTA
// that owns the row.

constexpr int kSrcThreads = 896;

struct AbSrcArgs {
    const float *C;  // [nA][nB] FP32 amplitudes
    double *S;       // [nA][nB], accumulated
    int64_t nA, nB;
    int norb, npair;
    const float *eri;         // FP32 (pq|rs) as [norb^2][norb^2]
    const int64_t *as_ptr;    // alpha singles, canonical CSR
    const uint32_t *as_pk;
    const uint32_t *src_item; // beta singles, source-major items (string | entries << 18)
    const uint32_t *src_ent;
    int64_t src_nitem;
    const float *rowmax;      // [nA] max |C(ja, :)|
    float bound;              // maxdeg_beta * max |(pq|rs)|
    int maxdeg;               // maxdeg_beta: most singles of a beta string
    int rs;                   // W row stride in float4: 8 (chunks of up to 32 alpha singles) or 4 (up to 16)
};

// shared memory of one CTA: W [npair][rs] float4, accumulator [nB] u64, pair -> rs code.  rs = 4
// (64-byte W rows, chunks of at most 16 alpha singles) is the layout for large norb, where the
// 128-byte rows and the row accumulator do not fit together (norb 58: 1,653 pairs, 211 KB of rows)
__host__ __device__ constexpr size_t src_w_bytes(int npair, int rs) { return (size_t)npair * rs * 16; }
__host__ __device__ inline size_t src_smem(int npair, int64_t nB, int rs)
{
    return src_w_bytes(npair, rs) + (size_t)nB * 8 + round16((size_t)npair * 2);
}
// the W row stride that fits `limit` bytes (8 preferred), 0 if neither does
__host__ __device__ inline int src_rs(int npair, int64_t nB, size_t limit)
{
    return src_smem(npair, nB, 8) <= limit ? 8 : (src_smem(npair, nB, 4) <= limit ? 4 : 0);
}

// adds t * f to element ib of the row accumulator (words lo[ib], hi[ib]; see above)
__device__ __forceinline__ void src_add(unsigned *acc_lo, unsigned *acc_hi, uint32_t e, float f, float scale,
                                        int lbits)
{
    long long v = __float2ll_rn(f * scale);
    if ((e >> kSrcNegBit) & 1u) v = -v;
    const int ib = (int)(e & kPackJMask);
    atomicAdd(acc_lo + ib, (unsigned)v & ((1u << lbits) - 1u));
    atomicAdd(acc_hi + ib, (unsigned)(int)(v >> lbits));
}

template <int KC, int RS>
__device__ __forceinline__ void src_chunk(const AbSrcArgs &a, const float4 *__restrict__ Wt, unsigned *acc_lo,
                                          unsigned *acc_hi, const int *ja_s, int kc, float scale, int lbits,
                                          int *ctr)
{
    static_assert(KC / 4 <= RS, "a W row holds at least one copy of the chunk");
    constexpr int CPW = KC / 4;  // 16-byte chunks per copy of a W row
    const int lane = threadIdx.x & 31;
    const int rot = lane & (CPW - 1);
    const int base = ((lane / CPW) & (RS / CPW - 1)) * CPW;  // first chunk of this lane's copy
    const int nsl = (int)((a.src_nitem + 31) >> 5);
    while (true) {
        int sl = 0;
        if (lane == 0) sl = atomicAdd(ctr, 1);
        sl = __shfl_sync(0xffffffffu, sl, 0);
        if (sl >= nsl) break;
        // one item per lane: a string jb (column of C) and at most kSrcItem of its singles
        const int64_t t = (int64_t)sl * 32 + lane;
        const uint32_t info = t < a.src_nitem ? __ldg(a.src_item + t) : 0u;
        const int64_t jb = info & kPackJMask;
        const int cnt = (int)(info >> kSrcPairShift);
        const uint32_t *ent = a.src_ent + (int64_t)sl * 32 * kSrcItem + lane;
        uint32_t e[kSrcItem];
#pragma unroll
        for (int i = 0; i < kSrcItem; ++i) e[i] = i < cnt ? __ldg(ent + 32 * i) : 0u;
        // amplitudes of the chunk's alpha singles at column jb (consecutive lanes: consecutive or equal
        // columns), then rotated by `rot` chunks so that register chunk s holds amplitude chunk
        // (s + rot) mod CPW
        float cv[KC];
#pragma unroll
        for (int k4 = 0; k4 < KC; k4 += 4) {
            const int4 j4 = *reinterpret_cast<const int4 *>(ja_s + k4);  // one broadcast load per 4 rows
            const int jr[4] = {j4.x, j4.y, j4.z, j4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                cv[k4 + i] = (cnt > 0 && k4 + i < kc) ? __ldg(a.C + (int64_t)jr[i] * a.nB + jb) : 0.f;
        }
#pragma unroll
        for (int b = 1; b < CPW; b <<= 1) {
            if (rot & b) {
                float tmp[KC];
#pragma unroll
                for (int s = 0; s < CPW; ++s)
#pragma unroll
                    for (int i = 0; i < 4; ++i) tmp[4 * s + i] = cv[4 * ((s + b) % CPW) + i];
#pragma unroll
                for (int k = 0; k < KC; ++k) cv[k] = tmp[k];
            }
        }
#pragma unroll
        for (int i = 0; i < kSrcItem; i += 2) {  // two singles per round for independent chains
            if (i < cnt) {
                const bool two = i + 1 < cnt;
                const float4 *w0 = Wt + ((e[i] >> kSrcPairShift) & 0x7ffu) * RS + base;
                const float4 *w1 = Wt + ((e[i + 1] >> kSrcPairShift) & 0x7ffu) * RS + base;
                float f0 = 0.f, f1 = 0.f;
#pragma unroll
                for (int s = 0; s < CPW; ++s) {
                    const int q = (s + rot) & (CPW - 1);
                    const float4 x0 = w0[q];
                    const float4 x1 = two ? w1[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                    f0 = fmaf(x0.x, cv[4 * s], f0);
                    f1 = fmaf(x1.x, cv[4 * s], f1);
                    f0 = fmaf(x0.y, cv[4 * s + 1], f0);
                    f1 = fmaf(x1.y, cv[4 * s + 1], f1);
                    f0 = fmaf(x0.z, cv[4 * s + 2], f0);
                    f1 = fmaf(x1.z, cv[4 * s + 2], f1);
                    f0 = fmaf(x0.w, cv[4 * s + 3], f0);
                    f1 = fmaf(x1.w, cv[4 * s + 3], f1);
                }
                src_add(acc_lo, acc_hi, e[i], f0, scale, lbits);
                if (two) src_add(acc_lo, acc_hi, e[i + 1], f1, scale, lbits);
            }
        }
    }
}

// W[x][position p] for the chunk's alpha singles, position p holding amplitude chunk p mod CPW
template <int KC, int RS>
__device__ __forceinline__ void src_build_w(const AbSrcArgs &a, float4 *Wt, const int16_t *rs_of,
                                            const int *pq_s, const float *u_s, int kc)
{
    constexpr int CPW = KC / 4;
    const int n2 = a.norb * a.norb;
    for (int idx = threadIdx.x; idx < a.npair * RS; idx += blockDim.x) {
        const int p = idx / a.npair, x = idx - p * a.npair;
        const int c = p & (CPW - 1);
        const int rs = rs_of[x];
        float v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = 4 * c + i;
            v[i] = k < kc ? u_s[k] * __ldg(a.eri + (size_t)pq_s[k] * n2 + rs) : 0.f;
        }
        Wt[(size_t)x * RS + p] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

template <int RS>
__device__ __forceinline__ void src_row(const AbSrcArgs &a, int64_t ia, unsigned char *smem)
{
    constexpr int KMAX = RS * 4;  // alpha singles per chunk
    float4 *Wt = reinterpret_cast<float4 *>(smem);
    unsigned *acc_lo = reinterpret_cast<unsigned *>(smem + src_w_bytes(a.npair, RS));
    unsigned *acc_hi = acc_lo + a.nB;
    const int16_t *rs_of = reinterpret_cast<const int16_t *>(smem + src_w_bytes(a.npair, RS) + (size_t)a.nB * 8);
    __shared__ __align__(16) int ja_s[32];
    __shared__ int pq_s[32];
    __shared__ float u_s[32];
    __shared__ int ctr;
    __shared__ float s_scale;
    __shared__ double s_inv;
    __shared__ int s_lbits;
    __shared__ int s_state;  // 0 skip the row, 1 accumulate, 2 non-finite amplitudes
    const int tid = threadIdx.x;
    const int64_t e0 = a.as_ptr[ia];
    const int K = (int)(a.as_ptr[ia + 1] - e0);
    __syncthreads();  // the previous row is finished with shared memory
    for (int64_t ib = tid; ib < a.nB; ib += blockDim.x) acc_lo[ib] = acc_hi[ib] = 0u;
    {
        int16_t *rs_w = reinterpret_cast<int16_t *>(smem + src_w_bytes(a.npair, RS) + (size_t)a.nB * 8);
        for (int r = 1; r < a.norb; ++r)
            for (int s = tid; s < r; s += blockDim.x) rs_w[r * (r - 1) / 2 + s] = (int16_t)(r * a.norb + s);
    }
    if (tid < 32) {
        float m = 0.f;
        for (int k = tid; k < K; k += 32) m += __ldg(a.rowmax + (a.as_pk[e0 + k] & kPackJMask));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m += __shfl_xor_sync(0xffffffffu, m, off);
        if (tid == 0) {
            const double bnd = (double)m * (double)a.bound;
            if (!(bnd <= 1e300)) {
                s_state = 2;
            } else if (bnd == 0.0) {
                s_state = 0;
            } else {
                // contributions per element: at most maxdeg per chunk of the row
                const long long m = (long long)max(a.maxdeg, 1) * ((K + KMAX - 1) / KMAX);
                const int lbits = max(1, 32 - (64 - __clzll(m)));
                int e = 30 + lbits - ilogb(bnd) - 1;  // bnd < 2^(ilogb+1), so bnd * 2^e < 2^(30+lbits)
                e = max(-120, min(120, e));
                s_scale = ldexpf(1.f, e);
                s_inv = ldexp(1.0, -e);
                s_lbits = lbits;
                s_state = 1;
            }
        }
    }
    __syncthreads();
    const int state = s_state;
    if (state == 0) return;
    if (state == 2) {
        for (int64_t ib = tid; ib < a.nB; ib += blockDim.x) a.S[ia * a.nB + ib] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const float scale = s_scale;
    const int lbits = s_lbits;
    for (int k0 = 0; k0 < K; k0 += KMAX) {
        const int kc = min(KMAX, K - k0);
        __syncthreads();  // the previous chunk is finished with W and the chunk arrays
        if (tid < kc) {
            const uint32_t pk = a.as_pk[e0 + k0 + tid];
            ja_s[tid] = (int)(pk & kPackJMask);
            pq_s[tid] = (int)(pk >> (kPackKeyShift + 1));
            u_s[tid] = ((pk >> kPackKeyShift) & 1u) ? -1.f : 1.f;
        }
        if (tid == 0) ctr = 0;
        __syncthreads();
        if (kc <= 8) {
            src_build_w<8, RS>(a, Wt, rs_of, pq_s, u_s, kc);
            __syncthreads();
            src_chunk<8, RS>(a, Wt, acc_lo, acc_hi, ja_s, kc, scale, lbits, &ctr);
        } else if (RS == 4 || kc <= 16) {
            src_build_w<16, RS>(a, Wt, rs_of, pq_s, u_s, kc);
            __syncthreads();
            src_chunk<16, RS>(a, Wt, acc_lo, acc_hi, ja_s, kc, scale, lbits, &ctr);
        } else {
            src_build_w<(RS == 8 ? 32 : 16), RS>(a, Wt, rs_of, pq_s, u_s, kc);
            __syncthreads();
            src_chunk<(RS == 8 ? 32 : 16), RS>(a, Wt, acc_lo, acc_hi, ja_s, kc, scale, lbits, &ctr);
        }
    }
    __syncthreads();
    const double inv = s_inv;
    for (int64_t ib = tid; ib < a.nB; ib += blockDim.x) {
        const long long v = (long long)(int)acc_hi[ib] * (1ll << lbits) + (long long)acc_lo[ib];
        a.S[ia * a.nB + ib] += (double)v * inv;
    }
}

// one instance per W row stride (the host launches the one a.rs names)
template <int RS>
__global__ void __launch_bounds__(kSrcThreads, 1) ab_src_kernel(const AbSrcArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    for (int64_t ia = blockIdx.x; ia < a.nA; ia += gridDim.x) src_row<RS>(a, ia, smem);
}

// out[c][r] = in[r][c]; with rowmax (FP32 only, zeroed beforehand): rowmax[r] = max_c |in[r][c]|,
// accumulated as the bit patterns of non-negative floats (a NaN row stays NaN)
template <typename T>
__global__ void transpose_kernel(const T *__restrict__ in, T *__restrict__ out, int64_t rows, int64_t cols,
                                 float *rowmax = nullptr)
{
    __shared__ T tile[32][33];
    const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int64_t r = by + j, c = bx + threadIdx.x;
        T v = T(0);
        if (r < rows && c < cols) {
            v = in[r * cols + c];
            tile[j][threadIdx.x] = v;
        }
        if constexpr (sizeof(T) == 4) {
            if (rowmax) {  // uniform per launch
                const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf((float)v)));
                if (threadIdx.x == 0 && r < rows) atomicMax(reinterpret_cast<unsigned *>(rowmax) + r, m);
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int64_t c = bx + j, r = by + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][j];
    }
}

struct PassCfg {
    int R = 1;
    bool staged = false;
    size_t smem = 0;
};

PassCfg choose(int64_t ncol, int n2, size_t elem, int rmax, size_t limit)
{
    PassCfg p;
    for (int R = rmax; R >= 1; R /= 2) {
        size_t b = round16((size_t)ncol * R * elem) + (size_t)2 * n2 * R * elem;
        if (b <= limit) {
            p.R = R;
            p.staged = true;
            p.smem = b;
            return p;
        }
    }
    p.R = 1;
    p.staged = false;
    p.smem = (size_t)2 * n2 * elem;
    return p;
}

size_t smem_limit(const Ctx &c) { return (size_t)c.smem_optin - 1024; }

// max |x| over n floats, as the bit pattern of a non-negative float (out zeroed beforehand)
__global__ void absmax_kernel(const float *__restrict__ x, int64_t n, unsigned *out)
{
    unsigned m = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(x[i])));
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

int npairs(int norb) { return norb * (norb - 1) / 2; }

// the column-stationary alpha-beta pass applies when its W table (128- or 64-byte rows) and row
// accumulator fit
int src_rs_of(const Ctx &c)
{
    return (c.norb >= 2 && c.sp[1].src_ent) ? src_rs(npairs(c.norb), c.nB, smem_limit(c)) : 0;
}
bool src_fits(const Ctx &c) { return src_rs_of(c) > 0; }

AbSrcArgs src_args(const Ctx &c, const float *C, double *S, const float *rowmax)
{
    const SpinTables &ta = c.sp[0], &tb = c.sp[1];
    AbSrcArgs a{};
    a.C = C;
    a.S = S;
    a.nA = c.nA;
    a.nB = c.nB;
    a.norb = c.norb;
    a.npair = npairs(c.norb);
    a.eri = c.eri32;
    a.as_ptr = ta.s_ptr;
    a.as_pk = ta.s_pk;
    a.src_item = tb.src_item;
    a.src_ent = tb.src_ent;
    a.src_nitem = tb.src_nitem;
    a.rowmax = rowmax;
    a.bound = (float)((double)tb.src_maxdeg * (double)c.eri_absmax);
    a.maxdeg = tb.src_maxdeg;
    a.rs = src_rs_of(c);
    return a;
}

void launch_ab_src(const AbSrcArgs &a, int num_sms, cudaStream_t s)
{
    const int grid = (int)std::min<int64_t>(a.nA, (int64_t)num_sms);
    if (a.rs == 8) ab_src_kernel<8><<<grid, kSrcThreads, src_smem(a.npair, a.nB, 8), s>>>(a);
    else ab_src_kernel<4><<<grid, kSrcThreads, src_smem(a.npair, a.nB, 4), s>>>(a);
    SBD_LAUNCH("ab_src_kernel");
}

template <typename T>
void set_attrs(int optin)
{
    if constexpr (sizeof(T) == 4) {
        SBD_CUDA(cudaFuncSetAttribute(row_pass_kernel<T, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        SBD_CUDA(cudaFuncSetAttribute(ab_pass_kernel<T, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    }
    SBD_CUDA(cudaFuncSetAttribute(row_pass_kernel<T, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    SBD_CUDA(cudaFuncSetAttribute(row_pass_kernel<T, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    SBD_CUDA(cudaFuncSetAttribute(row_pass_kernel<T, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    SBD_CUDA(cudaFuncSetAttribute(ab_pass_kernel<T, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    SBD_CUDA(cudaFuncSetAttribute(ab_pass_kernel<T, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    SBD_CUDA(cudaFuncSetAttribute(ab_pass_kernel<T, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
}

// the mixed 8-row pass over column halves applies when its staged half and tables fit
bool halves_fit(const RowArgs<float> &a, size_t limit)
{
    return a.hls_ptr && a.ncol_out == a.ncol && a.half > 0 && halves_smem(a.half, a.norb) <= limit;
}

void launch_halves(const RowArgs<float> &a, cudaStream_t s)
{
    const int64_t groups = (a.nrow + kHalfRows - 1) / kHalfRows;
    const int grid = (int)(groups < 65535 ? groups : 65535);
    row_halves_kernel<<<grid, Threads<float>::value, halves_smem(a.half, a.norb), s>>>(a);
    SBD_LAUNCH("row_halves_kernel");
}

template <typename T>
void launch_row(const RowArgs<T> &a, const PassCfg &p, cudaStream_t s)
{
    constexpr int kThreads = Threads<T>::value;
    const int64_t groups = (a.nrow + p.R - 1) / p.R;
    const int grid = (int)(groups < 65535 ? groups : 65535);
    if (!p.staged) row_pass_kernel<T, 1, false><<<grid, kThreads, p.smem, s>>>(a);
    else if (p.R == 4) row_pass_kernel<T, (sizeof(T) == 4 ? 4 : 2), true><<<grid, kThreads, p.smem, s>>>(a);
    else if (p.R == 2) row_pass_kernel<T, 2, true><<<grid, kThreads, p.smem, s>>>(a);
    else row_pass_kernel<T, 1, true><<<grid, kThreads, p.smem, s>>>(a);
    SBD_LAUNCH("row_pass_kernel");
}

template <typename T>
void launch_ab(const AbArgs<T> &a, const PassCfg &p, cudaStream_t s)
{
    constexpr int kThreads = Threads<T>::value;
    const int grid = (int)(a.nA < 65535 ? a.nA : 65535);
    if (!p.staged) ab_pass_kernel<T, 1, false><<<grid, kThreads, p.smem, s>>>(a);
    else if (p.R == 4) ab_pass_kernel<T, (sizeof(T) == 4 ? 4 : 2), true><<<grid, kThreads, p.smem, s>>>(a);
    else if (p.R == 2) ab_pass_kernel<T, 2, true><<<grid, kThreads, p.smem, s>>>(a);
    else ab_pass_kernel<T, 1, true><<<grid, kThreads, p.smem, s>>>(a);
    SBD_LAUNCH("ab_pass_kernel");
}

template <typename T>
void transpose(const T *in, T *out, int64_t rows, int64_t cols, cudaStream_t s, float *rowmax = nullptr)
{
    const int64_t gy = (rows + 31) / 32;
    if (gy > 65535) fail(SBD_ERR_UNSUPPORTED, "alpha string set too large for the transpose");
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)gy);
    if (rowmax) SBD_CUDA(cudaMemsetAsync(rowmax, 0, (size_t)rows * sizeof(float), s));
    transpose_kernel<T><<<grid, dim3(32, 8), 0, s>>>(in, out, rows, cols, rowmax);
    SBD_LAUNCH("transpose_kernel");
}

template <typename T>
Lists<T> lists_of(const SpinTables &t);
template <>
Lists<float> lists_of<float>(const SpinTables &t)
{
    return Lists<float>{t.s_pkv32, t.d_jv32};
}
template <>
Lists<double> lists_of<double>(const SpinTables &t)
{
    return Lists<double>{t.s_pk_sig, t.s_v64_sig, t.d_j_sig, t.d_v64_sig};
}
template <>
Lists<F2> lists_of<F2>(const SpinTables &t)
{
    return Lists<F2>{t.s_pk_sig, t.s_vx2, t.d_j_sig, t.d_vx2};
}

// timing slot of the first sigma kernel of a precision (transpose, beta, alpha, alpha-beta follow)
template <typename T>
constexpr int kSlotBase = kIsF2<T> ? 8 : (sizeof(T) == 4 ? 4 : 0);
template <typename T>
constexpr int kRowsMax = sizeof(T) == 4 ? 4 : 2;

// Runs launch(); when timing is on, brackets it with events on stream s and
// queues the pair for sbd_kernel_times (slot: kernel kind, +4 for FP32).
template <typename F>
void timed(Ctx &c, int slot, cudaStream_t s, F &&launch)
{
    if (!c.opt.timing) {
        launch();
        return;
    }
    cudaEvent_t a = take_event(c), b = take_event(c);
    SBD_CUDA(cudaEventRecord(a, s));
    launch();
    SBD_CUDA(cudaEventRecord(b, s));
    c.pending.push_back({slot, a, b});
}

// Arguments of the three gather passes of one instance: beta pass on C, alpha pass on its
// transpose Ct, alpha-beta pass on C (the single-instance and the batched launches share them).
template <typename T>
void make_args(const Ctx &c, const typename In<T>::type *C, double *S, const double *c64,
               const typename In<T>::type *Ct, RowArgs<T> &rb, RowArgs<T> &ra, AbArgs<T> &ab)
{
    const SpinTables &ta = c.sp[0], &tb = c.sp[1];
    rb = RowArgs<T>{};
    rb.X = C;
    rb.nrow = c.nA;
    rb.ncol = c.nB;
    rb.ncol_out = c.nB;
    rb.Y = S;
    rb.y_rs = c.nB;
    rb.y_cs = 1;
    rb.accumulate = 0;
    rb.hd = c.hd;
    rb.xd64 = c64;
    rb.row_strings = ta.strings;
    rb.norb = c.norb;
    rb.eri = c.eri64;
    rb.s_ptr = tb.sig_s_ptr;
    rb.d_ptr = tb.sig_d_ptr;
    rb.lists = lists_of<T>(tb);
    rb.hls_ptr = tb.hs_ptr;
    rb.hld_ptr = tb.hd_ptr;
    rb.hls = tb.hs;
    rb.hldv = tb.hdv;
    rb.hldt = tb.hdt;
    rb.half = tb.half;

    ra = rb;
    ra.X = Ct;
    ra.nrow = c.nB;
    ra.ncol = c.nA;
    ra.ncol_out = c.nA;
    ra.y_rs = 1;
    ra.y_cs = c.nB;
    ra.accumulate = 1;
    ra.hd = nullptr;
    ra.xd64 = nullptr;
    ra.row_strings = tb.strings;
    ra.s_ptr = ta.sig_s_ptr;
    ra.d_ptr = ta.sig_d_ptr;
    ra.lists = lists_of<T>(ta);
    ra.hls_ptr = ta.hs_ptr;
    ra.hld_ptr = ta.hd_ptr;
    ra.hls = ta.hs;
    ra.hldv = ta.hdv;
    ra.hldt = ta.hdt;
    ra.half = ta.half;

    ab = AbArgs<T>{};
    ab.C = C;
    ab.S = S;
    ab.nA = c.nA;
    ab.nB = c.nB;
    ab.norb = c.norb;
    using E = typename In<T>::type;
    ab.eri = sizeof(E) == 4 ? (const E *)(const void *)c.eri32 : (const E *)(const void *)c.eri64;
    ab.as_ptr = ta.s_ptr;      // canonical alpha lists: exact counts for the row groups
    ab.as_pk = ta.s_pk;
    ab.bs_ptr = tb.sig_s_ptr;  // padded beta lists for 16-byte loads
    ab.bs_pk = tb.s_pk_sig;
}

template <typename T>
void apply(Ctx &c, const typename In<T>::type *C, double *S, const double *c64, cudaStream_t s)
{
    using E = typename In<T>::type;
    const int n2 = c.norb * c.norb;
    const int rmax = kRowsMax<T>;
    const size_t lim = smem_limit(c);
    const int base = kSlotBase<T>;
    E *Ct = static_cast<E *>(c.work_t);
    // the mixed alpha-beta pass takes the row maxima of C from the beta pass
    const bool src = std::is_same<T, float>::value && src_fits(c);
    timed(c, base + 0, s, [&] { transpose<E>(C, Ct, c.nA, c.nB, s); });
    RowArgs<T> rb, ra;
    AbArgs<T> ab;
    make_args<T>(c, C, S, c64, Ct, rb, ra, ab);
    if (src) rb.rowmax = c.rowmax;
    if constexpr (std::is_same<T, float>::value) {
        // 8 rows over column halves where they fit, else 4 rows over the whole row
        timed(c, base + 1, s, [&] {
            if (halves_fit(rb, lim)) launch_halves(rb, s);
            else launch_row<T>(rb, choose(c.nB, n2, sizeof(T), rmax, lim), s);
        });
        timed(c, base + 2, s, [&] {
            if (halves_fit(ra, lim)) launch_halves(ra, s);
            else launch_row<T>(ra, choose(c.nA, n2, sizeof(T), rmax, lim), s);
        });
    } else {
        timed(c, base + 1, s, [&] { launch_row<T>(rb, choose(c.nB, n2, sizeof(T), rmax, lim), s); });
        timed(c, base + 2, s, [&] { launch_row<T>(ra, choose(c.nA, n2, sizeof(T), rmax, lim), s); });
    }
    if constexpr (std::is_same<T, float>::value) {
        if (src) {
            timed(c, base + 3, s, [&] { launch_ab_src(src_args(c, C, S, c.rowmax), c.num_sms, s); });
            return;
        }
    }
    timed(c, base + 3, s, [&] { launch_ab<T>(ab, choose(c.nB, n2, sizeof(T), rmax, lim), s); });
}

// ---------------------------------------------------------------------------
// Batched sigma.  One descriptor block holds, for every slot, the arguments of its passes and
// the prefix sums of its work items (transpose tiles, beta row groups, alpha row groups, alpha-beta
// rows).  Persistent CTAs take items from a counter and run the same per-item device functions as
// the single-instance kernels, so every output element is computed by the same arithmetic.

template <typename T>
struct TDesc {
    const T *in;
    T *out;
    int64_t rows, cols;
};

struct Layout {
    size_t n, off_t, off_b, off_a, off_ab, td, rb, ra, ab, src, total;
};

template <typename T>
Layout layout_for(int m)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 255) & ~(size_t)255;
        return at;
    };
    L.n = take(sizeof(int));
    L.off_t = take(sizeof(int64_t) * (m + 1));
    L.off_b = take(sizeof(int64_t) * (m + 1));
    L.off_a = take(sizeof(int64_t) * (m + 1));
    L.off_ab = take(sizeof(int64_t) * (m + 1));
    L.td = take(sizeof(TDesc<typename In<T>::type>) * m);
    L.rb = take(sizeof(RowArgs<T>) * m);
    L.ra = take(sizeof(RowArgs<T>) * m);
    L.ab = take(sizeof(AbArgs<T>) * m);
    L.src = take(sizeof(AbSrcArgs) * m);
    L.total = o;
    return L;
}

// slot s with off[s] <= item < off[s + 1] (empty slots are skipped)
__device__ __forceinline__ int find_slot(const int64_t *off, int n, int64_t item)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename T>
__global__ void transpose_batch_kernel(const int *pn, const int64_t *off, const TDesc<T> *td)
{
    __shared__ T tile[32][33];
    const int n = *pn;
    const int64_t total = off[n];
    for (int64_t it = blockIdx.x; it < total; it += gridDim.x) {
        const int sl = find_slot(off, n, it);
        const TDesc<T> d = td[sl];
        const int64_t lt = it - off[sl], tx = (d.cols + 31) / 32;
        const int64_t by = (lt / tx) * 32, bx = (lt % tx) * 32;
        __syncthreads();
        for (int j = threadIdx.y; j < 32; j += 8) {
            const int64_t r = by + j, c = bx + threadIdx.x;
            if (r < d.rows && c < d.cols) tile[j][threadIdx.x] = d.in[r * d.cols + c];
        }
        __syncthreads();
        for (int j = threadIdx.y; j < 32; j += 8) {
            const int64_t c = bx + j, r = by + threadIdx.x;
            if (r < d.rows && c < d.cols) d.out[c * d.rows + r] = tile[threadIdx.x][j];
        }
    }
}

// Work-item loop of the persistent pass kernels: thread 0 takes the next item from the counter,
// the CTA copies the slot's arguments to shared memory when the slot changes, then runs body().
template <typename Args, typename F>
__device__ __forceinline__ void item_loop(const int *pn, const int64_t *off, const Args *args,
                                          unsigned long long *counter, Args &sa, F &&body)
{
    __shared__ int64_t s_item;
    __shared__ int s_slot;
    const int n = *pn;
    const int64_t total = off[n];
    int cur = -1;
    while (true) {
        __syncthreads();  // the previous item is finished with shared memory
        if (threadIdx.x == 0) {
            const int64_t it = (int64_t)atomicAdd(counter, 1ull);
            s_item = it;
            s_slot = it < total ? find_slot(off, n, it) : -1;
        }
        __syncthreads();
        const int64_t it = s_item;
        const int sl = s_slot;
        if (it >= total) break;
        if (sl != cur) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(args + sl);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&sa);
            for (int i = threadIdx.x; i < (int)(sizeof(Args) / 4); i += blockDim.x) dst[i] = src[i];
            cur = sl;
            __syncthreads();
        }
        body(it - off[sl]);
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(Threads<T>::value) row_batch_kernel(const int *pn, const int64_t *off,
                                                                      const RowArgs<T> *args,
                                                                      unsigned long long *counter)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ RowArgs<T> sa;
    item_loop(pn, off, args, counter, sa, [&](int64_t li) { row_group<T, R, true>(sa, li * R, smem); });
}

template <typename T, int R>
__global__ void __launch_bounds__(Threads<T>::value) ab_batch_kernel(const int *pn, const int64_t *off,
                                                                     const AbArgs<T> *args,
                                                                     unsigned long long *counter)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ AbArgs<T> sa;
    item_loop(pn, off, args, counter, sa, [&](int64_t li) { ab_row<T, R, true>(sa, li, smem); });
}

template <int RS>
__global__ void __launch_bounds__(kSrcThreads, 1) ab_src_batch_kernel(const int *pn, const int64_t *off,
                                                                      const AbSrcArgs *args,
                                                                      unsigned long long *counter)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ AbSrcArgs sa;
    item_loop(pn, off, args, counter, sa, [&](int64_t li) { src_row<RS>(sa, li, smem); });
}

__global__ void __launch_bounds__(Threads<float>::value) row_halves_batch_kernel(const int *pn, const int64_t *off,
                                                                               const RowArgs<float> *args,
                                                                               unsigned long long *counter)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ RowArgs<float> sa;
    item_loop(pn, off, args, counter, sa, [&](int64_t li) { row_halves(sa, li * kHalfRows, smem); });
}

size_t batch_smem(size_t elem, int R, int max_strings, int max_norb)
{
    if (R == kHalfRows) return halves_smem((max_strings + 1) / 2, max_norb);
    return round16((size_t)max_strings * R * elem) + (size_t)2 * max_norb * max_norb * R * elem;
}

}  // namespace

struct SigmaBatch {
    sbd_precision prec = SBD_MIXED;
    int max_slots = 0, R = 1, device = 0, grid_pass = 0, grid_t = 0, grid_src = 0;
    size_t smem = 0;
    bool src = false;     // mixed: the column-stationary alpha-beta pass (when its table and accumulator fit)
    int src_rs = 0;       // its W row stride for the largest slot (8 or 4 float4)
    size_t src_smem = 0;
    Layout L{};
    unsigned char *dev = nullptr, *host = nullptr;
    unsigned long long *counters = nullptr;  // [3]: beta, alpha, alpha-beta
};

namespace {

template <typename T>
void batch_set(SigmaBatch *b, const SigmaSlot *slots, int n)
{
    const Layout &L = b->L;
    unsigned char *h = b->host;
    *reinterpret_cast<int *>(h + L.n) = n;
    int64_t *ot = reinterpret_cast<int64_t *>(h + L.off_t), *ob = reinterpret_cast<int64_t *>(h + L.off_b);
    int64_t *oa = reinterpret_cast<int64_t *>(h + L.off_a), *oab = reinterpret_cast<int64_t *>(h + L.off_ab);
    using E = typename In<T>::type;
    TDesc<E> *td = reinterpret_cast<TDesc<E> *>(h + L.td);
    RowArgs<T> *rb = reinterpret_cast<RowArgs<T> *>(h + L.rb), *ra = reinterpret_cast<RowArgs<T> *>(h + L.ra);
    AbArgs<T> *ab = reinterpret_cast<AbArgs<T> *>(h + L.ab);
    ot[0] = ob[0] = oa[0] = oab[0] = 0;
    for (int i = 0; i < n; ++i) {
        const SigmaSlot &sl = slots[i];
        const Ctx &c = *sl.c;
        const E *x = static_cast<const E *>(sl.x);
        E *xt = static_cast<E *>(sl.xt);
        make_args<T>(c, x, sl.y, sl.x64, xt, rb[i], ra[i], ab[i]);
        if constexpr (std::is_same<T, float>::value) {
            if (b->src) {
                rb[i].rowmax = c.rowmax;
                AbSrcArgs sa = src_args(c, x, sl.y, c.rowmax);
                sa.rs = b->src_rs;  // every slot in the layout the batch's shared memory was sized for
                reinterpret_cast<AbSrcArgs *>(h + L.src)[i] = sa;
            }
        }
        td[i] = TDesc<E>{x, xt, c.nA, c.nB};
        ot[i + 1] = ot[i] + ((c.nA + 31) / 32) * ((c.nB + 31) / 32);
        ob[i + 1] = ob[i] + (c.nA + b->R - 1) / b->R;
        oa[i + 1] = oa[i] + (c.nB + b->R - 1) / b->R;
        oab[i + 1] = oab[i] + c.nA;
    }
}

template <typename T, int R>
void batch_launch_r(SigmaBatch *b, cudaStream_t s)
{
    constexpr int kThreads = Threads<T>::value;
    const Layout &L = b->L;
    unsigned char *d = b->dev;
    const int *pn = reinterpret_cast<const int *>(d + L.n);
    using E = typename In<T>::type;
    transpose_batch_kernel<E><<<b->grid_t, dim3(32, 8), 0, s>>>(pn, reinterpret_cast<const int64_t *>(d + L.off_t),
                                                                reinterpret_cast<const TDesc<E> *>(d + L.td));
    SBD_LAUNCH("transpose_batch_kernel");
    if constexpr (R == kHalfRows) {
        row_halves_batch_kernel<<<b->grid_pass, kThreads, b->smem, s>>>(
            pn, reinterpret_cast<const int64_t *>(d + L.off_b), reinterpret_cast<const RowArgs<float> *>(d + L.rb),
            b->counters);
        SBD_LAUNCH("row_halves_batch_kernel");
        row_halves_batch_kernel<<<b->grid_pass, kThreads, b->smem, s>>>(
            pn, reinterpret_cast<const int64_t *>(d + L.off_a), reinterpret_cast<const RowArgs<float> *>(d + L.ra),
            b->counters + 1);
        SBD_LAUNCH("row_halves_batch_kernel");
    } else {
        row_batch_kernel<T, R><<<b->grid_pass, kThreads, b->smem, s>>>(
            pn, reinterpret_cast<const int64_t *>(d + L.off_b), reinterpret_cast<const RowArgs<T> *>(d + L.rb),
            b->counters);
        SBD_LAUNCH("row_batch_kernel");
        row_batch_kernel<T, R><<<b->grid_pass, kThreads, b->smem, s>>>(
            pn, reinterpret_cast<const int64_t *>(d + L.off_a), reinterpret_cast<const RowArgs<T> *>(d + L.ra),
            b->counters + 1);
        SBD_LAUNCH("row_batch_kernel");
    }
    if (std::is_same<T, float>::value && b->src) {
        const int64_t *off_ab = reinterpret_cast<const int64_t *>(d + L.off_ab);
        const AbSrcArgs *src_args_d = reinterpret_cast<const AbSrcArgs *>(d + L.src);
        if (b->src_rs == 8)
            ab_src_batch_kernel<8><<<b->grid_src, kSrcThreads, b->src_smem, s>>>(pn, off_ab, src_args_d, b->counters + 2);
        else
            ab_src_batch_kernel<4><<<b->grid_src, kSrcThreads, b->src_smem, s>>>(pn, off_ab, src_args_d, b->counters + 2);
        SBD_LAUNCH("ab_src_batch_kernel");
        return;
    }
    if constexpr (R != kHalfRows) {  // 8 rows per item only come with the column-stationary pass
        ab_batch_kernel<T, R><<<b->grid_pass, kThreads, b->smem, s>>>(
            pn, reinterpret_cast<const int64_t *>(d + L.off_ab), reinterpret_cast<const AbArgs<T> *>(d + L.ab),
            b->counters + 2);
        SBD_LAUNCH("ab_batch_kernel");
    }
}

template <typename T, int R>
void batch_attrs(SigmaBatch *b)
{
    constexpr int kThreads = Threads<T>::value;
    int occ_row = 0, occ_ab = 1 << 20;
    if constexpr (R == kHalfRows) {
        SBD_CUDA(cudaFuncSetAttribute(row_halves_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)b->smem));
        SBD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_row, row_halves_batch_kernel, kThreads, b->smem));
    } else {
        SBD_CUDA(cudaFuncSetAttribute(row_batch_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
        SBD_CUDA(cudaFuncSetAttribute(ab_batch_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
        SBD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_row, row_batch_kernel<T, R>, kThreads, b->smem));
        SBD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_ab, ab_batch_kernel<T, R>, kThreads, b->smem));
    }
    const int occ = std::max(1, std::min(occ_row, occ_ab));
    int sms = 0;
    SBD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    b->grid_pass = sms * occ;
    b->grid_t = sms * 8;
    if (b->src) {
        int occ_src = 0;
        if (b->src_rs == 8) {
            SBD_CUDA(cudaFuncSetAttribute(ab_src_batch_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)b->src_smem));
            SBD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_src, ab_src_batch_kernel<8>, kSrcThreads,
                                                                   b->src_smem));
        } else {
            SBD_CUDA(cudaFuncSetAttribute(ab_src_batch_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)b->src_smem));
            SBD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_src, ab_src_batch_kernel<4>, kSrcThreads,
                                                                   b->src_smem));
        }
        b->grid_src = sms * std::max(1, occ_src);
    }
}

}  // namespace

void sigma_prepare(Ctx &c)
{
    // dynamic shared memory up to smem_limit(): the kernels' static shared memory (at most 1 KB) and
    // the dynamic part must stay within the opt-in maximum together
    const int lim = (int)smem_limit(c);
    set_attrs<double>(lim);
    set_attrs<float>(lim);
    set_attrs<F2>(lim);
    SBD_CUDA(cudaFuncSetAttribute(ab_src_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    SBD_CUDA(cudaFuncSetAttribute(ab_src_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    SBD_CUDA(cudaFuncSetAttribute(row_halves_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    // max |(pq|rs)| of the FP32 integrals, for the fixed-point scale of the alpha-beta pass
    const int64_t n4 = (int64_t)c.norb * c.norb * c.norb * c.norb;
    unsigned *m = reinterpret_cast<unsigned *>(c.dstat);  // status words are free after create
    SBD_CUDA(cudaMemsetAsync(m, 0, sizeof(unsigned), c.stream));
    absmax_kernel<<<(int)std::min<int64_t>((n4 + 255) / 256, 1024), 256, 0, c.stream>>>(c.eri32, n4, m);
    SBD_LAUNCH("absmax_kernel");
    unsigned bits = 0;
    SBD_CUDA(cudaMemcpyAsync(&bits, m, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
    SBD_CUDA(cudaStreamSynchronize(c.stream));
    memcpy(&c.eri_absmax, &bits, sizeof(float));
    c.rowmax = dalloc_n<float>(c, (size_t)c.nA);
}

size_t sigma_batch_smem(sbd_precision prec, int R, int max_strings, int max_norb)
{
    return batch_smem(prec == SBD_MIXED ? 4 : 8, R, max_strings, max_norb);
}

bool sigma_batch_fits(sbd_precision prec, int R, int max_strings, int max_norb, int device)
{
    const size_t lim = sigma_batch_smem_limit(device);
    if (R == kHalfRows)
        return prec == SBD_MIXED && max_norb >= 2 && sigma_batch_smem(prec, R, max_strings, max_norb) <= lim &&
               src_rs(npairs(max_norb), max_strings, lim) > 0;
    if (R == 4 && prec != SBD_MIXED) return false;
    return sigma_batch_smem(prec, R, max_strings, max_norb) <= lim;
}

size_t sigma_batch_smem_limit(int device)
{
    int optin = 0;
    SBD_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    return (size_t)optin - 1024;  // headroom for the kernels' static shared memory
}

SigmaBatch *sigma_batch_create(int max_slots, sbd_precision prec, int R, int max_strings, int max_norb, int device)
{
    if (max_slots < 1) fail(SBD_ERR_INVALID_ARG, "batched sigma needs at least one slot");
    if (!(R == 1 || R == 2 || ((R == 4 || R == kHalfRows) && prec == SBD_MIXED)) || prec < SBD_FP64 ||
        prec > SBD_F32X2)
        fail(SBD_ERR_INVALID_ARG, "rows per work item must be 1, 2 or (mixed only) 4 or 8");
    const size_t smem = sigma_batch_smem(prec, R, max_strings, max_norb);
    if (smem > sigma_batch_smem_limit(device))
        fail(SBD_ERR_UNSUPPORTED, "batched sigma: staged rows do not fit in shared memory");
    auto *b = new SigmaBatch();
    b->prec = prec;
    b->max_slots = max_slots;
    b->R = R;
    b->device = device;
    b->smem = smem;
    b->src_rs = max_norb >= 2 ? src_rs(npairs(max_norb), max_strings, sigma_batch_smem_limit(device)) : 0;
    b->src_smem = b->src_rs ? src_smem(npairs(max_norb), max_strings, b->src_rs) : 0;
    b->src = prec == SBD_MIXED && b->src_rs > 0;
    if (R == kHalfRows && !b->src) {
        delete b;
        fail(SBD_ERR_UNSUPPORTED, "batched sigma: 8 rows per item need the column-stationary alpha-beta pass, "
                                  "whose table and accumulator do not fit shared memory here");
    }
    b->L = prec == SBD_FP64 ? layout_for<double>(max_slots)
                            : (prec == SBD_F32X2 ? layout_for<F2>(max_slots) : layout_for<float>(max_slots));
    try {
        SBD_CUDA(cudaMalloc(&b->dev, b->L.total));
        SBD_CUDA(cudaMallocHost(&b->host, b->L.total));
        SBD_CUDA(cudaMalloc(&b->counters, 3 * sizeof(unsigned long long)));
        memset(b->host, 0, b->L.total);
        if (prec == SBD_FP64) {
            if (R == 2) batch_attrs<double, 2>(b);
            else batch_attrs<double, 1>(b);
        } else if (prec == SBD_F32X2) {
            if (R == 2) batch_attrs<F2, 2>(b);
            else batch_attrs<F2, 1>(b);
        } else {
            if (R == kHalfRows) batch_attrs<float, kHalfRows>(b);
            else if (R == 4) batch_attrs<float, 4>(b);
            else if (R == 2) batch_attrs<float, 2>(b);
            else batch_attrs<float, 1>(b);
        }
    } catch (...) {
        sigma_batch_destroy(b);
        throw;
    }
    return b;
}

void sigma_batch_set(SigmaBatch *b, const SigmaSlot *slots, int n)
{
    if (n < 0 || n > b->max_slots) fail(SBD_ERR_INVALID_ARG, "batched sigma: too many slots");
    for (int i = 0; i < n; ++i) {
        const Ctx &c = *slots[i].c;
        if (sigma_batch_smem(b->prec, b->R, (int)std::max(c.nA, c.nB), c.norb) > b->smem)
            fail(SBD_ERR_UNSUPPORTED, "batched sigma: an instance exceeds the string or orbital limit of the batch");
    }
    if (b->prec == SBD_FP64) batch_set<double>(b, slots, n);
    else if (b->prec == SBD_F32X2) batch_set<F2>(b, slots, n);
    else batch_set<float>(b, slots, n);
}

void sigma_batch_launch(SigmaBatch *b, cudaStream_t s)
{
    SBD_CUDA(cudaMemcpyAsync(b->dev, b->host, b->L.total, cudaMemcpyHostToDevice, s));
    SBD_CUDA(cudaMemsetAsync(b->counters, 0, 3 * sizeof(unsigned long long), s));
    if (b->prec == SBD_FP64) {
        if (b->R == 2) batch_launch_r<double, 2>(b, s);
        else batch_launch_r<double, 1>(b, s);
    } else if (b->prec == SBD_F32X2) {
        if (b->R == 2) batch_launch_r<F2, 2>(b, s);
        else batch_launch_r<F2, 1>(b, s);
    } else {
        if (b->R == kHalfRows) batch_launch_r<float, kHalfRows>(b, s);
        else if (b->R == 4) batch_launch_r<float, 4>(b, s);
        else if (b->R == 2) batch_launch_r<float, 2>(b, s);
        else batch_launch_r<float, 1>(b, s);
    }
}

int64_t sigma_batch_launches(const SigmaBatch *) { return 4; }

void sigma_batch_destroy(SigmaBatch *b)
{
    if (!b) return;
    if (b->dev) (void)cudaFree(b->dev);
    if (b->host) (void)cudaFreeHost(b->host);
    if (b->counters) (void)cudaFree(b->counters);
    delete b;
}

namespace {

// The three passes of one source block for the output rows of a plan (see BlockPlan).
template <typename T>
void apply_block(BlockPlan &p, const typename In<T>::type *Cb, double *S, cudaStream_t s, const double *x64)
{
    using E = typename In<T>::type;
    Ctx &c = *p.c;
    const int n2 = c.norb * c.norb;
    const int rmax = kRowsMax<T>;
    const size_t lim = smem_limit(c);
    const int64_t nj = p.j1 - p.j0, nr = p.r1 - p.r0;
    const SpinTables &ta = c.sp[0], &tb = c.sp[1];
    E *Ct = static_cast<E *>(p.work_t);
    // mixed: the column-stationary alpha-beta pass takes the source rows' maxima from the transpose
    const bool src = std::is_same<T, float>::value && src_fits(c);
    transpose<E>(Cb, Ct, nj, c.nB, s, src ? p.rowmax : nullptr);
    // beta pass: the output rows inside the block
    const int64_t lo = std::max(p.r0, p.j0), hi = std::min(p.r1, p.j1);
    RowArgs<T> rb, ra;
    AbArgs<T> ab;
    make_args<T>(c, Cb, S, nullptr, Ct, rb, ra, ab);
    if (lo < hi) {
        RowArgs<T> b = rb;
        b.X = Cb + (lo - p.j0) * c.nB;
        b.nrow = hi - lo;
        b.Y = S + (lo - p.r0) * c.nB;
        b.accumulate = 1;
        b.hd = c.hd + lo * c.nB;
        b.xd64 = x64 ? x64 + (lo - p.r0) * c.nB : nullptr;
        b.row_strings = ta.strings + lo;
        launch_row<T>(b, choose(c.nB, n2, sizeof(T), rmax, lim), s);
    }
    // alpha pass: rows of the transposed block, output columns r0..r1, lists restricted to the block
    ra.X = Ct;
    ra.nrow = c.nB;
    ra.ncol = nj;
    ra.ncol_out = nr;
    ra.Y = S;
    ra.y_rs = 1;
    ra.y_cs = c.nB;
    ra.accumulate = 1;
    ra.s_ptr = p.sig_s_ptr;
    ra.d_ptr = p.sig_d_ptr;
    if constexpr (kIsF2<T>) ra.lists = Lists<F2>{p.s_pk_sig, p.s_vx2, p.d_j_sig, p.d_vx2};
    else if constexpr (sizeof(T) == 4) ra.lists = Lists<float>{p.s_pkv32, p.d_jv32};
    else ra.lists = Lists<double>{p.s_pk_sig, p.s_v64_sig, p.d_j_sig, p.d_v64_sig};
    launch_row<T>(ra, choose(nj, n2, sizeof(T), rmax, lim), s);
    // alpha-beta pass: output rows r0..r1, their alpha singles inside the block
    if constexpr (std::is_same<T, float>::value) {
        if (src) {
            AbSrcArgs a = src_args(c, Cb, S, p.rowmax);
            a.nA = nr;
            a.as_ptr = p.s_ptr;
            a.as_pk = p.s_pk;
            launch_ab_src(a, c.num_sms, s);
            return;
        }
    }
    ab.C = Cb;
    ab.S = S;
    ab.nA = nr;
    ab.as_ptr = p.s_ptr;
    ab.as_pk = p.s_pk;
    (void)tb;
    launch_ab<T>(ab, choose(c.nB, n2, sizeof(T), rmax, lim), s);
}

}  // namespace

void sigma_block_apply(BlockPlan &p, const void *cblock, double *sigma_rows, sbd_precision prec, cudaStream_t s,
                       const double *x64_rows)
{
    if (prec == SBD_FP64) apply_block<double>(p, static_cast<const double *>(cblock), sigma_rows, s, nullptr);
    else if (prec == SBD_F32X2) apply_block<F2>(p, static_cast<const double *>(cblock), sigma_rows, s, nullptr);
    else apply_block<float>(p, static_cast<const float *>(cblock), sigma_rows, s, x64_rows);
}

void sigma_apply(Ctx &c, const void *cvec, double *svec, sbd_precision prec, cudaStream_t s, const double *c64)
{
    if (prec == SBD_FP64) apply<double>(c, static_cast<const double *>(cvec), svec, nullptr, s);
    else if (prec == SBD_F32X2) apply<F2>(c, static_cast<const double *>(cvec), svec, nullptr, s);
    else apply<float>(c, static_cast<const float *>(cvec), svec, c64, s);
}

}  // namespace sbd
