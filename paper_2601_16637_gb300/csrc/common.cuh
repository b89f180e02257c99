// Internal declarations of the SBD CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sbd.h"

namespace sbd {

// ---------------------------------------------------------------------------
// errors: thrown inside the library, converted to status codes at the ABI

struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg);
void set_thread_error(const std::string &msg);  // sbd_last_error(NULL) on this thread
void check_cuda(cudaError_t e, const char *what, const char *file, int line);
void count_launch();
#define SBD_CUDA(call) ::sbd::check_cuda((call), #call, __FILE__, __LINE__)
#define SBD_LAUNCH(what) (::sbd::count_launch(), ::sbd::check_cuda(cudaGetLastError(), what, __FILE__, __LINE__))

// Packed single-excitation entry: target j in bits 0-17, phase -1 in bit 18, code p*norb+q in
// bits 19-30, so pk >> 18 = 2*code + (phase < 0) indexes sign-folded coefficient tables.  A
// single always has p != q, so code 0 never occurs: pk = 0 is the padding entry, and the
// coefficient-table rows of code 0 are kept zero.  Strings per spin must stay below 2^18.
constexpr int kPackJBits = 18;
constexpr uint32_t kPackJMask = (1u << kPackJBits) - 1u;
constexpr int kPackKeyShift = 18;  // pk >> 18 = 2*code + neg
constexpr int64_t kMaxStringsPerSpin = (int64_t)1 << kPackJBits;
constexpr int kSrcPairShift = 18;  // source-major singles: orbital-pair index at bits 18-28
constexpr int kSrcNegBit = 29;     // and the phase at bit 29
constexpr int kSrcItem = 8;        // source-major singles per work item
constexpr int kBankGroups = 8;     // 16-byte bank groups of shared memory (32 banks x 4 bytes)
constexpr int kListPad = 4;        // sigma lists are padded to multiples of 4 entries (16-byte loads)

// ---------------------------------------------------------------------------
// device status words written by validation kernels

struct DevStatus {
    unsigned long long first_bad;  // smallest index of a malformed string (~0 if none)
    unsigned long long first_dup;  // smallest index i with sorted[i] == sorted[i-1]
    int nonfinite;                 // nonzero if h or eri hold NaN/Inf
    int differ;                    // nonzero if two sorted sets differ
};

// ---------------------------------------------------------------------------
// per-spin tables, all device memory

struct SpinTables {
    int nel = 0;                 // electrons of this spin
    int64_t n = 0;               // |S|
    uint64_t *strings = nullptr; // sorted ascending
    // canonical CSR excitation tables (kind 1 singles, kind 2 doubles)
    int64_t *s_ptr = nullptr, *d_ptr = nullptr;  // [n+1]
    int64_t ns = 0, nd = 0;                      // total entries
    int32_t *s_j = nullptr, *d_j = nullptr;      // target index
    uint8_t *s_orb = nullptr, *d_orb = nullptr;  // p1,p2,q1,q2 per entry
    int8_t *s_sign = nullptr, *d_sign = nullptr; // fermionic phase
    // packed single: target j (bits 0-17) | code p*norb+q (bits 18-29) | phase -1 (bit 30)
    uint32_t *s_pk = nullptr;
    double *s_v64 = nullptr, *d_v64 = nullptr;   // same-spin matrix elements
    // Sigma copies of the lists: the same entries per source, each list padded with zero entries
    // to a multiple of kListPad and reordered so that the 8 entries one 128-bit shared-memory
    // phase gathers have distinct targets modulo 8 where possible (kBankGroups).
    int64_t *sig_s_ptr = nullptr, *sig_d_ptr = nullptr;  // [n+1], padded CSR offsets
    int64_t sig_ns = 0, sig_nd = 0;
    uint32_t *s_pk_sig = nullptr;
    double *s_v64_sig = nullptr;
    int32_t *d_j_sig = nullptr;
    double *d_v64_sig = nullptr;
    uint2 *s_pkv32 = nullptr;  // (s_pk_sig, FP32 value bits), for the mixed sigma
    uint2 *d_jv32 = nullptr;   // (d_j_sig, FP32 value bits), for the mixed sigma
    float2 *s_vx2 = nullptr;   // s_v64_sig as FP32 pairs (hi, lo), for the FP32-pair sigma
    float2 *d_vx2 = nullptr;   // d_v64_sig as FP32 pairs
    // Mixed-sigma lists split at the middle of the string set (half = (n + 1) / 2): virtual list
    // 2i holds the entries of source i with target < half, list 2i + 1 those with target >= half,
    // each padded to kListPad and in sigma order, for row passes that stage one column half at a
    // time (8 rows instead of 4 in the same shared memory).
    int64_t half = 0;
    int64_t *hs_ptr = nullptr, *hd_ptr = nullptr;  // [2n + 1]
    uint2 *hs = nullptr;  // (packed single, FP32 value bits)
    // doubles as two arrays with the same entry index: FP32 values, and targets relative to the
    // list's column half (0 for the lower half, `half` for the upper), which fit 16 bits: the split
    // lists are built only for half <= 65536 (six bytes per entry instead of eight)
    float *hdv = nullptr;
    uint16_t *hdt = nullptr;
    // Source-major singles for the column-stationary alpha-beta pass.  The canonical singles list
    // of each string is cut into items of at most kSrcItem entries (strings in ascending order,
    // each string's items consecutive, then inside each slice of 32 items the full ones first and
    // the partial ones by decreasing length), so that the lanes of a warp, one item each, walk
    // lists of nearly equal length; item t = string | entries << 18 (src_item[t]); entry i of item t is
    // src_ent[(t / 32) * 32 * kSrcItem + 32 * i + t % 32] (coalesced for the 32 items of a warp):
    // target (bits 0-17) | index of the unordered orbital pair {p, q} (bits 18-28) | phase -1 (bit 29).
    uint32_t *src_item = nullptr;
    uint32_t *src_ent = nullptr;
    int64_t src_nitem = 0;
    int src_maxdeg = 0;          // largest singles count of a string
    double *ediag = nullptr;     // [n] same-spin diagonal energies
    bool alias = false;          // storage owned by the other spin (A == B)
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    sbd_options opt{};
    int norb = 0, na = 0, nb = 0;
    int64_t nA = 0, nB = 0, N = 0;
    double *h64 = nullptr, *eri64 = nullptr;
    float *eri32 = nullptr;
    SpinTables sp[2];
    double *hd = nullptr;   // [N] Hamiltonian diagonal
    void *work_t = nullptr; // [N] doubles: transposed copy of one vector
    float *rowmax = nullptr; // [nA] max |c(ia, :)| of the last mixed-precision vector (written by its beta pass)
    float eri_absmax = 0.f;  // max |(pq|rs)| of the FP32 integrals
    size_t bytes_held = 0;
    std::vector<std::pair<void *, size_t>> allocs;
    std::string last_error;
    DevStatus *dstat = nullptr;  // device
    int smem_optin = 0;          // max dynamic shared memory per block
    int num_sms = 0;
    // kernel timing (sbd_options.timing)
    struct Pending {
        int slot;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    double kernel_ms[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    int64_t kernel_n[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
};

// the context inside a C-ABI handle (api.cu)
Ctx &ctx_of(sbd_handle h);

// kernel timing helpers (api.cu)
cudaEvent_t take_event(Ctx &c);
void harvest_timing(Ctx &c);

// device memory through the handle's allocator, with budget accounting
void *dalloc(Ctx &c, size_t bytes);
void dfree(Ctx &c, void *p);
template <typename T>
T *dalloc_n(Ctx &c, size_t n)
{
    return static_cast<T *>(dalloc(c, n * sizeof(T) > 0 ? n * sizeof(T) : 16));
}

// ---------------------------------------------------------------------------
// Diagonal preconditioner of Davidson (paper Eq. 7): t = r / (sign(d) max(|d|, delta)),
// d = Hd - theta.  The factor multiplying r is formed as an FP32 reciprocal: a preconditioner only
// shapes the correction direction (which is then orthogonalised and normalised in FP64), and the
// FP64 division would cost the FP64 pipe as much as a fifth of the Ritz pass.
__device__ __forceinline__ double precond_factor(double d, double delta)
{
    const double den = (d >= 0.0 ? 1.0 : -1.0) * fmax(fabs(d), delta);
    return (double)__frcp_rn((float)den);
}

// ---------------------------------------------------------------------------
// warp-cooperative search, shared by the lookup entry point and the table builder

// Position of `key` in sorted[0, n), or -1.  All 32 lanes call it with the
// same key; each step samples 32 evenly spaced elements of the remaining
// range and narrows it to one gap between samples (a 32-ary search).
__device__ __forceinline__ int64_t warp_find(const uint64_t *__restrict__ sorted, int64_t n, uint64_t key)
{
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = n;  // first element >= key lies in [lo, hi]
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t pos = lo + lane * step;
        const bool below = pos < hi && __ldg(sorted + pos) < key;
        const int c = __popc(__ballot_sync(0xffffffffu, below));
        const int64_t nlo = c == 0 ? lo : lo + (int64_t)(c - 1) * step + 1;
        const int64_t nhi = min(hi, lo + (int64_t)c * step + 1);
        lo = nlo;
        hi = nhi;
    }
    const int64_t pos = lo + lane;
    const bool hit = pos < hi && pos < n && __ldg(sorted + pos) == key;
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    return m ? lo + (__ffs(m) - 1) : -1;
}

// ---------------------------------------------------------------------------
// launchers (each enqueues on c.stream unless a stream is given)

// strings.cu
void validate_strings(Ctx &c, const uint64_t *s, int64_t n, int norb, int nel);
void radix_sort_strings(Ctx &c, uint64_t *keys, int64_t n, int nbits);
void check_duplicates(Ctx &c, const uint64_t *sorted, int64_t n);
void compare_sets(Ctx &c, const uint64_t *a, const uint64_t *b, int64_t n);
void check_finite(Ctx &c, const double *x, int64_t n);
void lookup_strings(const uint64_t *sorted, int64_t n, const uint64_t *keys, int64_t nq, int64_t *idx,
                    cudaStream_t s);
void sort_validate_into(const uint64_t *in, int64_t n, int norb, int nel, uint64_t *out, uint64_t *tmp,
                        DevStatus *st, cudaStream_t s);

// tables.cu
void build_tables(Ctx &c, int spin);
void build_diagonal(Ctx &c);
void to_float(const double *in, float *out, int64_t n, cudaStream_t s);

// sigma.cu
void sigma_prepare(Ctx &c);

// ---------------------------------------------------------------------------
// row-block sigma for alpha-row sharding (shard.cu, sigma.cu)

// The alpha lists of output rows [r0, r1) restricted to sources in [j0, j1), targets renumbered
// from j0, in the layouts of SpinTables (canonical singles; padded sigma singles and doubles).
struct BlockPlan {
    Ctx *c = nullptr;
    int64_t r0 = 0, r1 = 0, j0 = 0, j1 = 0;
    int64_t *s_ptr = nullptr;
    uint32_t *s_pk = nullptr;
    int64_t *sig_s_ptr = nullptr, *sig_d_ptr = nullptr;
    uint32_t *s_pk_sig = nullptr;
    double *s_v64_sig = nullptr;
    uint2 *s_pkv32 = nullptr;
    float2 *s_vx2 = nullptr;
    int32_t *d_j_sig = nullptr;
    double *d_v64_sig = nullptr;
    uint2 *d_jv32 = nullptr;
    float2 *d_vx2 = nullptr;
    void *work_t = nullptr;  // [nB][j1 - j0] doubles: the transposed source block
    float *rowmax = nullptr; // [j1 - j0] max |c| of each source row (mixed alpha-beta pass)
    std::vector<void *> allocs;
};
BlockPlan *block_plan_create(Ctx &c, int64_t r0, int64_t r1, int64_t j0, int64_t j1);
void block_plan_destroy(BlockPlan *p);
// sigma_rows[(ia - r0)*nB + ib] += sum over (ja, jb), ja in [j0, j1), of H[(ia,ib),(ja,jb)] cblock[(ja - j0)*nB + jb]
// x64_rows (optional, mixed precision): FP64 amplitudes of the output rows, for the diagonal term
void sigma_block_apply(BlockPlan &p, const void *cblock, double *sigma_rows, sbd_precision prec, cudaStream_t s,
                       const double *x64_rows = nullptr);

// ---------------------------------------------------------------------------
// batched sigma: many instances in one set of persistent launches (sigma.cu)

// One instance of a batched sigma (host side).
struct SigmaSlot {
    const Ctx *c;
    const void *x;       // amplitudes [nA][nB]: float (mixed) or double (FP64)
    double *y;           // sigma [nA][nB], overwritten
    const double *x64;   // mixed only: FP64 amplitudes for the diagonal term, or null
    void *xt;            // [nA*nB] elements of the precision: transposed copy of x
};
struct SigmaBatch;
// Device descriptors for up to max_slots instances whose string sets have at most max_strings
// entries per spin and norb <= max_norb; R = rows staged per work item (1, 2, or for the mixed
// precision 4, or 8 over column halves).
SigmaBatch *sigma_batch_create(int max_slots, sbd_precision prec, int R, int max_strings, int max_norb, int device);
// Shared memory one work item needs with R staged rows; compare with sigma_batch_smem_limit().
size_t sigma_batch_smem(sbd_precision prec, int R, int max_strings, int max_norb);
size_t sigma_batch_smem_limit(int device);
// whether R rows per item (8: mixed only, over column halves, with the column-stationary alpha-beta
// pass) fits shared memory for max_strings and max_norb
bool sigma_batch_fits(sbd_precision prec, int R, int max_strings, int max_norb, int device);
// Fills the host staging copy of the descriptors (no device work).
void sigma_batch_set(SigmaBatch *b, const SigmaSlot *slots, int n);
// Copies the staged descriptors to the device and runs transpose, beta, alpha and alpha-beta
// passes over every slot: fixed grids and device-resident counts, so the sequence can be
// captured in a CUDA graph once and replayed after each sigma_batch_set.
void sigma_batch_launch(SigmaBatch *b, cudaStream_t s);
void sigma_batch_destroy(SigmaBatch *b);
int64_t sigma_batch_launches(const SigmaBatch *b);  // kernel launches per sigma_batch_launch
// c64 (mixed only, may be NULL): the FP64 amplitudes, used for the diagonal term
void sigma_apply(Ctx &c, const void *cvec, double *svec, sbd_precision prec, cudaStream_t s,
                 const double *c64 = nullptr);

// davidson.cu
// A rank of an alpha-row-sharded solve: its rows [bounds[rank], bounds[rank+1]) of every vector,
// one block plan per source block, two ring buffers and the caller's communication callbacks.
struct ShardCtx {
    int rank = 0, world = 1;
    std::vector<int64_t> bounds;    // world + 1 alpha-row boundaries
    std::vector<BlockPlan *> plans; // plans[b]: this rank's rows, source block b
    void *ring[2] = {nullptr, nullptr};
    sbd_comm comm{};
    int64_t row0() const { return bounds[rank]; }
    int64_t rows() const { return bounds[rank + 1] - bounds[rank]; }
};

int davidson(Ctx &c, int nroots, double tol, sbd_precision prec, double *energies, double *vecs,
             double *resid, sbd_report *rep, ShardCtx *shard = nullptr);
// sigma of this rank's rows: the source blocks pass around the ring of ranks (shard.cu)
void ring_sigma(ShardCtx &sh, Ctx &c, const void *x_rows, double *y_rows, sbd_precision prec, cudaStream_t s,
                const double *x64_rows = nullptr);

}  // namespace sbd
