// String ingestion: validation, LSD radix sort, duplicate detection and the
// warp-cooperative lookup of strings in a sorted set.
//
// The selected determinant space is the product of an alpha-string set A and
// a beta-string set B (paper Sec. II-F, "half-bitstring"); every other part
// of the library addresses strings by their position in the ascending
// unsigned order of their set, so these kernels fix that order.
#include "common.cuh"

namespace sbd {

namespace {

constexpr int kSortThreads = 1024;
constexpr int kSortWarps = kSortThreads / 32;

__global__ void validate_kernel(const uint64_t *s, int64_t n, int norb, int nel, DevStatus *st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t x = s[i];
        bool bad = __popcll(x) != nel || (norb < 64 && (x >> norb) != 0);
        if (bad) atomicMin(&st->first_bad, (unsigned long long)i);
    }
}

__global__ void duplicate_kernel(const uint64_t *s, int64_t n, DevStatus *st)
{
    for (int64_t i = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (s[i] == s[i - 1]) atomicMin(&st->first_dup, (unsigned long long)i);
}

__global__ void compare_kernel(const uint64_t *a, const uint64_t *b, int64_t n, DevStatus *st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (a[i] != b[i]) st->differ = 1;
}

__global__ void finite_kernel(const double *x, int64_t n, DevStatus *st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) st->nonfinite = 1;
}

// Stable LSD radix sort over 8-bit digits inside one CTA.  Each pass:
// global histogram, exclusive scan into bucket bases, then a tile-by-tile
// stable scatter in which the rank of an element among equal digits of its
// tile is its rank inside its warp (__match_any_sync) plus the counts of the
// warps before it.
__global__ void __launch_bounds__(kSortThreads) radix_sort_kernel(uint64_t *keys, uint64_t *tmp, int n,
                                                                 int passes)
{
    __shared__ int hist[256];
    __shared__ int base[256];
    __shared__ int warp_cnt[kSortWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    uint64_t *src = keys, *dst = tmp;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        if (tid < 256) hist[tid] = 0;
        __syncthreads();
        for (int i = tid; i < n; i += kSortThreads) atomicAdd(&hist[(src[i] >> shift) & 255], 1);
        __syncthreads();
        if (tid == 0) {
            int run = 0;
            for (int d = 0; d < 256; ++d) {
                base[d] = run;
                run += hist[d];
            }
        }
        __syncthreads();
        for (int t0 = 0; t0 < n; t0 += kSortThreads) {
            const int i = t0 + tid;
            const bool valid = i < n;
            const uint64_t key = valid ? src[i] : 0ull;
            const int d = valid ? (int)((key >> shift) & 255) : 256;
            for (int k = tid; k < kSortWarps * 256; k += kSortThreads) (&warp_cnt[0][0])[k] = 0;
            __syncthreads();
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const int rank = __popc(peers & lt_mask);
            if (valid && rank == 0) warp_cnt[warp][d] = __popc(peers);
            __syncthreads();
            int tile_total = 0;
            if (tid < 256) {
                for (int w = 0; w < kSortWarps; ++w) {
                    int cnt = warp_cnt[w][tid];
                    warp_cnt[w][tid] = tile_total;
                    tile_total += cnt;
                }
            }
            __syncthreads();
            if (valid) dst[base[d] + warp_cnt[warp][d] + rank] = key;
            __syncthreads();
            if (tid < 256) base[tid] += tile_total;
            __syncthreads();
        }
        uint64_t *t = src;
        src = dst;
        dst = t;
    }
    if (src != keys) {
        for (int i = tid; i < n; i += kSortThreads) keys[i] = src[i];
    }
}

__global__ void lookup_kernel(const uint64_t *sorted, int64_t n, const uint64_t *keys, int64_t nq,
                              int64_t *idx)
{
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    for (int64_t q = w0; q < nq; q += warps) {
        const uint64_t key = keys[q];
        const int64_t r = warp_find(sorted, n, key);
        if ((threadIdx.x & 31) == 0) idx[q] = r;
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535) g = 65535;
    return (int)g;
}

}  // namespace

void validate_strings(Ctx &c, const uint64_t *s, int64_t n, int norb, int nel)
{
    validate_kernel<<<grid_for(n, 256), 256, 0, c.stream>>>(s, n, norb, nel, c.dstat);
    SBD_LAUNCH("validate_kernel");
}

void radix_sort_strings(Ctx &c, uint64_t *keys, int64_t n, int nbits)
{
    if (n <= 1) return;
    if (n > (int64_t)0x7fffffff) fail(SBD_ERR_UNSUPPORTED, "string set larger than 2^31-1");
    uint64_t *tmp = dalloc_n<uint64_t>(c, (size_t)n);
    int passes = (nbits + 7) / 8;
    radix_sort_kernel<<<1, kSortThreads, 0, c.stream>>>(keys, tmp, (int)n, passes);
    SBD_LAUNCH("radix_sort_kernel");
    dfree(c, tmp);
}

void check_duplicates(Ctx &c, const uint64_t *sorted, int64_t n)
{
    if (n < 2) return;
    duplicate_kernel<<<grid_for(n, 256), 256, 0, c.stream>>>(sorted, n, c.dstat);
    SBD_LAUNCH("duplicate_kernel");
}

void compare_sets(Ctx &c, const uint64_t *a, const uint64_t *b, int64_t n)
{
    compare_kernel<<<grid_for(n, 256), 256, 0, c.stream>>>(a, b, n, c.dstat);
    SBD_LAUNCH("compare_kernel");
}

void check_finite(Ctx &c, const double *x, int64_t n)
{
    finite_kernel<<<grid_for(n, 256), 256, 0, c.stream>>>(x, n, c.dstat);
    SBD_LAUNCH("finite_kernel");
}

void lookup_strings(const uint64_t *sorted, int64_t n, const uint64_t *keys, int64_t nq, int64_t *idx,
                    cudaStream_t s)
{
    if (nq <= 0) return;
    int64_t blocks = (nq + 7) / 8;  // 8 warps per block, one query per warp per step
    if (blocks > 4096) blocks = 4096;
    lookup_kernel<<<(int)blocks, 256, 0, s>>>(sorted, n, keys, nq, idx);
    SBD_LAUNCH("lookup_kernel");
}

// Copies n strings to `out`, validates them, sorts `out` ascending and checks
// for duplicates, using caller-provided work space: tmp (n uint64) and the
// status words st.  Enqueued on s; nothing is allocated.
void sort_validate_into(const uint64_t *in, int64_t n, int norb, int nel, uint64_t *out, uint64_t *tmp,
                        DevStatus *st, cudaStream_t s)
{
    SBD_CUDA(cudaMemsetAsync(st, 0xff, 2 * sizeof(unsigned long long), s));
    SBD_CUDA(cudaMemsetAsync(&st->nonfinite, 0, 2 * sizeof(int), s));
    if (n <= 0) return;
    SBD_CUDA(cudaMemcpyAsync(out, in, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    validate_kernel<<<grid_for(n, 256), 256, 0, s>>>(out, n, norb, nel, st);
    SBD_LAUNCH("validate_kernel");
    if (n > 1) {
        radix_sort_kernel<<<1, kSortThreads, 0, s>>>(out, tmp, (int)n, (norb + 7) / 8);
        SBD_LAUNCH("radix_sort_kernel");
        duplicate_kernel<<<grid_for(n, 256), 256, 0, s>>>(out, n, st);
        SBD_LAUNCH("duplicate_kernel");
    }
}

}  // namespace sbd
