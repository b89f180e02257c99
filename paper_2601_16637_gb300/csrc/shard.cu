// Row-block sigma for alpha-row sharding (paper Sec. III: the alpha rows of C and sigma are
// distributed over processes and the C blocks travel around a ring, so each process adds, block
// after block, the contribution of every block to its own rows).
//
// A plan fixes the output alpha rows [r0, r1) and the source alpha rows [j0, j1).  It holds the
// alpha excitation lists of the output rows restricted to targets in [j0, j1), with the targets
// renumbered from j0, in every layout the gather passes read (canonical singles for the
// alpha-beta pass; the padded, bank-ordered sigma copies of singles and doubles in the FP64, FP32
// and FP32-pair formats for the alpha pass).  The restriction keeps each list's order, so the
// entries a pass visits for a block are exactly those the full sigma visits with targets in the
// block.  sigma_block_apply (sigma.cu) then runs the three passes on the block with the unchanged
// kernels: beta pass on the output rows that lie inside the block, alpha pass on the transposed
// block, alpha-beta pass on the block's rows.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace sbd {

namespace {

constexpr int kThreadsB = 128;

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(65535, (n + kThreadsB - 1) / kThreadsB)); }

// per output row: entries of the canonical singles list with target in [j0, j1)
__global__ void count_canon_kernel(const int64_t *__restrict__ ptr, const int32_t *__restrict__ tgt, int64_t r0,
                                   int64_t nr, int64_t j0, int64_t j1, int64_t *cnt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = 0;
        for (int64_t e = ptr[r0 + i]; e < ptr[r0 + i + 1]; ++e) k += tgt[e] >= j0 && tgt[e] < j1;
        cnt[i] = k;
    }
}

__global__ void fill_canon_kernel(const int64_t *__restrict__ ptr, const int32_t *__restrict__ tgt,
                                  const uint32_t *__restrict__ pk, int64_t r0, int64_t nr, int64_t j0, int64_t j1,
                                  const int64_t *__restrict__ optr, uint32_t *opk)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = optr[i];
        for (int64_t e = ptr[r0 + i]; e < ptr[r0 + i + 1]; ++e)
            if (tgt[e] >= j0 && tgt[e] < j1) opk[o++] = (pk[e] & ~kPackJMask) | (uint32_t)(tgt[e] - j0);
    }
}

// Padded sigma lists.  A singles entry is real when its packed word is nonzero (code 0 never
// occurs); a doubles entry is real unless both its target and its value are zero (such an entry
// adds nothing either way).  Counts are rounded up to multiples of kListPad.
__global__ void count_sig_kernel(const int64_t *__restrict__ ptr, const uint32_t *__restrict__ spk,
                                 const int32_t *__restrict__ dj, const double *__restrict__ dv, int64_t r0,
                                 int64_t nr, int64_t j0, int64_t j1, int64_t *cnt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = 0;
        for (int64_t e = ptr[r0 + i]; e < ptr[r0 + i + 1]; ++e) {
            int64_t t;
            bool real;
            if (spk) {
                real = spk[e] != 0u;
                t = (int64_t)(spk[e] & kPackJMask);
            } else {
                real = !(dj[e] == 0 && dv[e] == 0.0);
                t = dj[e];
            }
            k += real && t >= j0 && t < j1;
        }
        cnt[i] = (k + kListPad - 1) / kListPad * kListPad;
    }
}

// perm[o] = source entry of output slot o (-1 for padding)
__global__ void fill_sig_kernel(const int64_t *__restrict__ ptr, const uint32_t *__restrict__ spk,
                                const int32_t *__restrict__ dj, const double *__restrict__ dv, int64_t r0, int64_t nr,
                                int64_t j0, int64_t j1, const int64_t *__restrict__ optr, int64_t *perm)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t o = optr[i];
        for (int64_t e = ptr[r0 + i]; e < ptr[r0 + i + 1]; ++e) {
            int64_t t;
            bool real;
            if (spk) {
                real = spk[e] != 0u;
                t = (int64_t)(spk[e] & kPackJMask);
            } else {
                real = !(dj[e] == 0 && dv[e] == 0.0);
                t = dj[e];
            }
            if (real && t >= j0 && t < j1) perm[o++] = e;
        }
        for (; o < optr[i + 1]; ++o) perm[o] = -1;
    }
}

// gathers the restricted entries and renumbers their targets from j0
__global__ void gather_singles_kernel(const int64_t *__restrict__ perm, int64_t n, int64_t j0,
                                      const uint32_t *__restrict__ spk, const double *__restrict__ sv,
                                      const uint2 *__restrict__ spkv, const float2 *__restrict__ svx,
                                      uint32_t *opk, double *ov, uint2 *opkv, float2 *ovx)
{
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = perm[o];
        if (e < 0) {
            opk[o] = 0u;
            ov[o] = 0.0;
            opkv[o] = make_uint2(0u, 0u);
            ovx[o] = make_float2(0.f, 0.f);
        } else {
            const uint32_t p = (spk[e] & ~kPackJMask) | (uint32_t)((int64_t)(spk[e] & kPackJMask) - j0);
            opk[o] = p;
            ov[o] = sv[e];
            opkv[o] = make_uint2(p, spkv[e].y);
            ovx[o] = svx[e];
        }
    }
}

__global__ void gather_doubles_kernel(const int64_t *__restrict__ perm, int64_t n, int64_t j0,
                                      const int32_t *__restrict__ dj, const double *__restrict__ dv,
                                      const uint2 *__restrict__ djv, const float2 *__restrict__ dvx, int32_t *oj,
                                      double *ov, uint2 *ojv, float2 *ovx)
{
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = perm[o];
        if (e < 0) {
            oj[o] = 0;
            ov[o] = 0.0;
            ojv[o] = make_uint2(0u, 0u);
            ovx[o] = make_float2(0.f, 0.f);
        } else {
            const int32_t t = (int32_t)(dj[e] - j0);
            oj[o] = t;
            ov[o] = dv[e];
            ojv[o] = make_uint2((uint32_t)t, djv[e].y);
            ovx[o] = dvx[e];
        }
    }
}

// exclusive prefix sum of n counts into out[0..n] (single CTA, sequential blocks of the block size)
__global__ void scan_counts_kernel(const int64_t *cnt, int64_t n, int64_t *out)
{
    __shared__ int64_t part[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < n; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        part[threadIdx.x] = i < n ? cnt[i] : 0;
        __syncthreads();
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            const int64_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += v;
            __syncthreads();
        }
        if (i < n) out[i + 1] = carry + part[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = 0;
}

}  // namespace

BlockPlan *block_plan_create(Ctx &c, int64_t r0, int64_t r1, int64_t j0, int64_t j1)
{
    if (r0 < 0 || r1 <= r0 || r1 > c.nA || j0 < 0 || j1 <= j0 || j1 > c.nA)
        fail(SBD_ERR_INVALID_ARG, "block plan: row ranges must be non-empty and inside [0, nA)");
    auto *p = new BlockPlan();
    p->c = &c;
    p->r0 = r0;
    p->r1 = r1;
    p->j0 = j0;
    p->j1 = j1;
    const SpinTables &ta = c.sp[0];
    const int64_t nr = r1 - r0;
    cudaStream_t s = c.stream;
    auto grab = [&](size_t bytes) {
        void *q = dalloc(c, bytes);
        p->allocs.push_back(q);
        return q;
    };
    try {
        int64_t *cnt = (int64_t *)grab(sizeof(int64_t) * nr);
        // canonical singles (alpha-beta pass)
        p->s_ptr = (int64_t *)grab(sizeof(int64_t) * (nr + 1));
        count_canon_kernel<<<grid_for(nr), kThreadsB, 0, s>>>(ta.s_ptr, ta.s_j, r0, nr, j0, j1, cnt);
        SBD_LAUNCH("count_canon_kernel");
        scan_counts_kernel<<<1, 1024, 0, s>>>(cnt, nr, p->s_ptr);
        SBD_LAUNCH("scan_counts_kernel");
        int64_t ns = 0;
        SBD_CUDA(cudaMemcpyAsync(&ns, p->s_ptr + nr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SBD_CUDA(cudaStreamSynchronize(s));
        p->s_pk = (uint32_t *)grab(sizeof(uint32_t) * std::max<int64_t>(ns, 1));
        fill_canon_kernel<<<grid_for(nr), kThreadsB, 0, s>>>(ta.s_ptr, ta.s_j, ta.s_pk, r0, nr, j0, j1, p->s_ptr,
                                                             p->s_pk);
        SBD_LAUNCH("fill_canon_kernel");
        // padded sigma lists (alpha pass)
        for (int kind = 0; kind < 2; ++kind) {
            const int64_t *sptr = kind == 0 ? ta.sig_s_ptr : ta.sig_d_ptr;
            int64_t *optr = (int64_t *)grab(sizeof(int64_t) * (nr + 1));
            const uint32_t *spk = kind == 0 ? ta.s_pk_sig : nullptr;
            count_sig_kernel<<<grid_for(nr), kThreadsB, 0, s>>>(sptr, spk, ta.d_j_sig, ta.d_v64_sig, r0, nr, j0, j1,
                                                               cnt);
            SBD_LAUNCH("count_sig_kernel");
            scan_counts_kernel<<<1, 1024, 0, s>>>(cnt, nr, optr);
            SBD_LAUNCH("scan_counts_kernel");
            int64_t m = 0;
            SBD_CUDA(cudaMemcpyAsync(&m, optr + nr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            SBD_CUDA(cudaStreamSynchronize(s));
            const int64_t mm = std::max<int64_t>(m, 1);
            int64_t *perm = (int64_t *)dalloc(c, sizeof(int64_t) * mm);
            fill_sig_kernel<<<grid_for(nr), kThreadsB, 0, s>>>(sptr, spk, ta.d_j_sig, ta.d_v64_sig, r0, nr, j0, j1,
                                                              optr, perm);
            SBD_LAUNCH("fill_sig_kernel");
            const int gm = grid_for(m);
            if (kind == 0) {
                p->sig_s_ptr = optr;
                p->s_pk_sig = (uint32_t *)grab(sizeof(uint32_t) * mm);
                p->s_v64_sig = (double *)grab(sizeof(double) * mm);
                p->s_pkv32 = (uint2 *)grab(sizeof(uint2) * mm);
                p->s_vx2 = (float2 *)grab(sizeof(float2) * mm);
                if (m)
                    gather_singles_kernel<<<gm, kThreadsB, 0, s>>>(perm, m, j0, ta.s_pk_sig, ta.s_v64_sig, ta.s_pkv32,
                                                                   ta.s_vx2, p->s_pk_sig, p->s_v64_sig, p->s_pkv32,
                                                                   p->s_vx2);
            } else {
                p->sig_d_ptr = optr;
                p->d_j_sig = (int32_t *)grab(sizeof(int32_t) * mm);
                p->d_v64_sig = (double *)grab(sizeof(double) * mm);
                p->d_jv32 = (uint2 *)grab(sizeof(uint2) * mm);
                p->d_vx2 = (float2 *)grab(sizeof(float2) * mm);
                if (m)
                    gather_doubles_kernel<<<gm, kThreadsB, 0, s>>>(perm, m, j0, ta.d_j_sig, ta.d_v64_sig, ta.d_jv32,
                                                                   ta.d_vx2, p->d_j_sig, p->d_v64_sig, p->d_jv32,
                                                                   p->d_vx2);
            }
            SBD_LAUNCH("gather_sig_kernel");
            dfree(c, perm);
        }
        // transposed source block, doubles
        p->work_t = grab(sizeof(double) * (size_t)(j1 - j0) * (size_t)c.nB);
        p->rowmax = (float *)grab(sizeof(float) * (size_t)(j1 - j0));
        SBD_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        block_plan_destroy(p);
        throw;
    }
    return p;
}

void ring_sigma(ShardCtx &sh, Ctx &c, const void *x_rows, double *y_rows, sbd_precision prec, cudaStream_t s,
                const double *x64_rows)
{
    const size_t elem = prec == SBD_MIXED ? sizeof(float) : sizeof(double);
    const int W = sh.world, r = sh.rank;
    SBD_CUDA(cudaMemsetAsync(y_rows, 0, sizeof(double) * (size_t)sh.rows() * (size_t)c.nB, s));
    // the rank's own block is complete before the first transfer reads it
    SBD_CUDA(cudaStreamSynchronize(s));
    const void *cur = x_rows;
    for (int step = 0; step < W; ++step) {
        const int b = ((r - step) % W + W) % W;
        sigma_block_apply(*sh.plans[b], cur, y_rows, prec, s, b == r ? x64_rows : nullptr);
        void *nxt = nullptr;
        if (step + 1 < W) {
            // double buffering (Sec. III-E): the transfer runs while the products above are in flight.
            // Both only read cur; nxt was last read by the previous step's products, which have completed.
            const int nb = ((r - step - 1) % W + W) % W;
            nxt = sh.ring[step % 2];
            const size_t sb = (size_t)(sh.bounds[b + 1] - sh.bounds[b]) * (size_t)c.nB * elem;
            const size_t rb = (size_t)(sh.bounds[nb + 1] - sh.bounds[nb]) * (size_t)c.nB * elem;
            if (sh.comm.ring_exchange(sh.comm.ctx, cur, sb, nxt, rb, (void *)s) != 0)
                fail(SBD_ERR_CUDA, "ring_exchange callback failed");
        }
        SBD_CUDA(cudaStreamSynchronize(s));  // this block's products are done before its buffer is reused
        if (nxt) cur = nxt;
    }
}

void block_plan_destroy(BlockPlan *p)
{
    if (!p) return;
    for (void *q : p->allocs) dfree(*p->c, q);
    delete p;
}

}  // namespace sbd
