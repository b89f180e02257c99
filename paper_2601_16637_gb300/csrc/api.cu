// The C ABI declared in include/sbd.h: handle life cycle, argument checks,
// allocation with budget accounting, and conversion of internal errors to
// status codes (no C++ exception leaves this file).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "common.cuh"

namespace sbd {

[[noreturn]] void fail(int code, const std::string &msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char *what, const char *file, int line)
{
    if (e == cudaSuccess) return;
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    fail(e == cudaErrorMemoryAllocation ? SBD_ERR_OUT_OF_MEMORY : SBD_ERR_CUDA, buf);
}

static std::atomic<int64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

cudaEvent_t take_event(Ctx &c)
{
    if (!c.event_pool.empty()) {
        cudaEvent_t e = c.event_pool.back();
        c.event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    SBD_CUDA(cudaEventCreate(&e));
    return e;
}

void harvest_timing(Ctx &c)
{
    for (const Ctx::Pending &p : c.pending) {
        SBD_CUDA(cudaEventSynchronize(p.b));
        float ms = 0.f;
        SBD_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
        c.kernel_ms[p.slot] += ms;
        c.kernel_n[p.slot] += 1;
        c.event_pool.push_back(p.a);
        c.event_pool.push_back(p.b);
    }
    c.pending.clear();
}

static void destroy_events(Ctx &c)
{
    for (const Ctx::Pending &p : c.pending) {
        (void)cudaEventDestroy(p.a);
        (void)cudaEventDestroy(p.b);
    }
    c.pending.clear();
    for (cudaEvent_t e : c.event_pool) (void)cudaEventDestroy(e);
    c.event_pool.clear();
}

void *dalloc(Ctx &c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (c.opt.hbm_budget_bytes && c.bytes_held + bytes > c.opt.hbm_budget_bytes) {
        char buf[160];
        snprintf(buf, sizeof(buf), "allocation of %zu bytes would exceed the budget (%zu held, %zu allowed)", bytes,
                 c.bytes_held, c.opt.hbm_budget_bytes);
        fail(SBD_ERR_OVER_BUDGET, buf);
    }
    void *p = nullptr;
    if (c.opt.alloc) {
        p = c.opt.alloc(c.opt.alloc_ctx, bytes, (void *)c.stream);
        if (!p) fail(SBD_ERR_OUT_OF_MEMORY, "device allocator returned NULL");
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, c.stream);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            fail(SBD_ERR_OUT_OF_MEMORY, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        }
    }
    c.allocs.emplace_back(p, bytes);
    c.bytes_held += bytes;
    return p;
}

void dfree(Ctx &c, void *p)
{
    if (!p) return;
    auto it = std::find_if(c.allocs.begin(), c.allocs.end(), [p](const std::pair<void *, size_t> &a) { return a.first == p; });
    if (it == c.allocs.end()) return;
    c.bytes_held -= it->second;
    c.allocs.erase(it);
    if (c.opt.free) c.opt.free(c.opt.alloc_ctx, p, (void *)c.stream);
    else (void)cudaFreeAsync(p, c.stream);
}

static void free_all(Ctx &c)
{
    while (!c.allocs.empty()) dfree(c, c.allocs.back().first);
}

}  // namespace sbd

using namespace sbd;

struct sbd_ctx {
    Ctx c;
};

Ctx &sbd::ctx_of(sbd_handle h) { return h->c; }

static thread_local std::string g_last_error;

void sbd::set_thread_error(const std::string &msg) { g_last_error = msg; }

template <typename F>
static int guarded(sbd_handle h, F &&f)
{
    try {
        return f();
    } catch (const Error &e) {
        if (h) h->c.last_error = e.msg;
        else g_last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        if (h) h->c.last_error = "host allocation failed";
        else g_last_error = "host allocation failed";
        return SBD_ERR_OUT_OF_MEMORY;
    } catch (...) {
        if (h) h->c.last_error = "unexpected internal error";
        else g_last_error = "unexpected internal error";
        return SBD_ERR_CUDA;
    }
}

extern "C" {

void sbd_default_options(sbd_options *opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->refine_precision = SBD_F32X2;
    opt->delta = 1e-4;
    opt->max_subspace = 0;
    opt->max_iter = 200;
}

const char *sbd_status_string(int status)
{
    switch (status) {
    case SBD_OK: return "ok";
    case SBD_NOT_CONVERGED: return "not converged";
    case SBD_PENDING: return "pending";
    case SBD_ERR_INVALID_ARG: return "invalid argument";
    case SBD_ERR_BAD_STRING: return "bad string";
    case SBD_ERR_DUPLICATE_STRING: return "duplicate string";
    case SBD_ERR_NORB: return "norb out of range";
    case SBD_ERR_OUT_OF_MEMORY: return "out of memory";
    case SBD_ERR_OVER_BUDGET: return "over budget";
    case SBD_ERR_CUDA: return "CUDA error";
    case SBD_ERR_NONFINITE: return "non-finite input";
    case SBD_ERR_BREAKDOWN: return "breakdown";
    case SBD_ERR_UNSUPPORTED: return "unsupported size";
    default: return "unknown status";
    }
}

int sbd_sigma_batched(int n, const sbd_handle *handles, const void *const *c_dev, double *const *sigma_dev,
                      sbd_precision prec, int rows_per_item, void *stream)
{
    if (n < 0 || (n > 0 && (!handles || !c_dev || !sigma_dev)) || prec < SBD_FP64 || prec > SBD_F32X2) {
        g_last_error = "sbd_sigma_batched: invalid argument";
        return SBD_ERR_INVALID_ARG;
    }
    if (n == 0) return SBD_OK;
    return guarded(nullptr, [&]() -> int {
        cudaStream_t s = (cudaStream_t)stream;
        int max_strings = 1, max_norb = 1, device = 0;
        std::vector<SigmaSlot> slots((size_t)n);
        for (int i = 0; i < n; ++i) {
            if (!handles[i] || !c_dev[i] || !sigma_dev[i]) fail(SBD_ERR_INVALID_ARG, "sbd_sigma_batched: NULL entry");
            for (int j = 0; j < i; ++j)
                if (handles[j] == handles[i]) fail(SBD_ERR_INVALID_ARG, "sbd_sigma_batched: a handle appears twice");
            Ctx &c = handles[i]->c;
            if (i == 0) device = c.device;
            else if (c.device != device) fail(SBD_ERR_INVALID_ARG, "sbd_sigma_batched: handles on different devices");
            max_strings = (int)std::max<int64_t>(max_strings, std::max(c.nA, c.nB));
            max_norb = std::max(max_norb, c.norb);
            slots[i] = SigmaSlot{&c, c_dev[i], sigma_dev[i], nullptr, c.work_t};
        }
        int R = rows_per_item;
        if (R == 0) {
            for (int cand : {8, 4, 2, 1}) {
                if (sigma_batch_fits(prec, cand, max_strings, max_norb, device)) {
                    R = cand;
                    break;
                }
            }
            if (R == 0) fail(SBD_ERR_UNSUPPORTED, "sbd_sigma_batched: string sets too large for the staged passes");
        }
        SigmaBatch *b = sigma_batch_create(n, prec, R, max_strings, max_norb, device);
        try {
            sigma_batch_set(b, slots.data(), n);
            sigma_batch_launch(b, s);
            SBD_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            sigma_batch_destroy(b);
            throw;
        }
        sigma_batch_destroy(b);
        return SBD_OK;
    });
}

}  // extern "C"

struct sbd_block_plan_s {
    sbd_handle h;
    BlockPlan *p;
};

extern "C" {

int sbd_block_plan_create(sbd_handle h, int64_t r0, int64_t r1, int64_t j0, int64_t j1, sbd_block_plan *out)
{
    if (!h || !out) return SBD_ERR_INVALID_ARG;
    *out = nullptr;
    return guarded(h, [&]() -> int {
        BlockPlan *p = block_plan_create(h->c, r0, r1, j0, j1);
        auto *bp = new (std::nothrow) sbd_block_plan_s{h, p};
        if (!bp) {
            block_plan_destroy(p);
            fail(SBD_ERR_OUT_OF_MEMORY, "host allocation failed");
        }
        *out = bp;
        return SBD_OK;
    });
}

int sbd_sigma_block(sbd_block_plan bp, const void *c_block_dev, double *sigma_rows_dev, sbd_precision prec,
                    void *stream)
{
    if (!bp || !c_block_dev || !sigma_rows_dev || prec < SBD_FP64 || prec > SBD_F32X2) return SBD_ERR_INVALID_ARG;
    return guarded(nullptr, [&]() -> int {  // errors: sbd_last_error(NULL) on this thread
        sigma_block_apply(*bp->p, c_block_dev, sigma_rows_dev, prec, (cudaStream_t)stream);
        return SBD_OK;
    });
}

int sbd_block_plan_destroy(sbd_block_plan bp)
{
    if (!bp) return SBD_ERR_INVALID_ARG;
    const int rc = guarded(nullptr, [&]() -> int {
        block_plan_destroy(bp->p);
        return SBD_OK;
    });
    delete bp;
    return rc;
}

const char *sbd_last_error(sbd_handle h) { return h ? h->c.last_error.c_str() : g_last_error.c_str(); }

int sbd_create(sbd_handle *out, int norb, int nalpha, int nbeta, const double *h, const double *eri,
               const uint64_t *A, int64_t nA, const uint64_t *B, int64_t nB, const sbd_options *opt, void *stream)
{
    if (!out) {
        g_last_error = "out is NULL";
        return SBD_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (norb < 1 || norb > 64) {
        g_last_error = "norb must be in 1..64";
        return SBD_ERR_NORB;
    }
    if (nalpha < 0 || nbeta < 0 || nalpha > norb || nbeta > norb || !h || !eri || !A || !B || nA < 1 || nB < 1 ||
        nA > 0x7fffffffLL || nB > 0x7fffffffLL) {
        g_last_error = "invalid argument to sbd_create";
        return SBD_ERR_INVALID_ARG;
    }
    sbd_ctx *hd = new (std::nothrow) sbd_ctx;
    if (!hd) {
        g_last_error = "host allocation failed";
        return SBD_ERR_OUT_OF_MEMORY;
    }
    Ctx &c = hd->c;
    if (opt) c.opt = *opt;
    else sbd_default_options(&c.opt);
    c.stream = (cudaStream_t)stream;
    c.norb = norb;
    c.na = nalpha;
    c.nb = nbeta;
    c.nA = nA;
    c.nB = nB;
    c.N = nA * nB;
    int rc = guarded(nullptr, [&]() -> int {
        SBD_CUDA(cudaGetDevice(&c.device));
        SBD_CUDA(cudaDeviceGetAttribute(&c.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device));
        SBD_CUDA(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device));
        const size_t n2 = (size_t)norb * norb;
        c.dstat = dalloc_n<DevStatus>(c, 1);
        SBD_CUDA(cudaMemsetAsync(c.dstat, 0xff, 2 * sizeof(unsigned long long), c.stream));
        SBD_CUDA(cudaMemsetAsync(&c.dstat->nonfinite, 0, 2 * sizeof(int), c.stream));
        c.h64 = dalloc_n<double>(c, n2);
        c.eri64 = dalloc_n<double>(c, n2 * n2);
        c.eri32 = dalloc_n<float>(c, n2 * n2);
        SBD_CUDA(cudaMemcpyAsync(c.h64, h, n2 * sizeof(double), cudaMemcpyDefault, c.stream));
        SBD_CUDA(cudaMemcpyAsync(c.eri64, eri, n2 * n2 * sizeof(double), cudaMemcpyDefault, c.stream));
        check_finite(c, c.h64, (int64_t)n2);
        check_finite(c, c.eri64, (int64_t)(n2 * n2));
        to_float(c.eri64, c.eri32, (int64_t)(n2 * n2), c.stream);
        // strings: copy, validate, sort, look for duplicates
        const uint64_t *src[2] = {A, B};
        const int64_t cnt[2] = {nA, nB};
        const int nel[2] = {nalpha, nbeta};
        DevStatus st{};
        for (int s = 0; s < 2; ++s) {
            SpinTables &t = c.sp[s];
            t.nel = nel[s];
            t.n = cnt[s];
            t.strings = dalloc_n<uint64_t>(c, (size_t)t.n);
            SBD_CUDA(cudaMemcpyAsync(t.strings, src[s], (size_t)t.n * sizeof(uint64_t), cudaMemcpyDefault, c.stream));
            validate_strings(c, t.strings, t.n, norb, t.nel);
            SBD_CUDA(cudaMemcpyAsync(&st, c.dstat, sizeof(st), cudaMemcpyDeviceToHost, c.stream));
            SBD_CUDA(cudaStreamSynchronize(c.stream));
            if (st.nonfinite) fail(SBD_ERR_NONFINITE, "h or eri contains NaN or Inf");
            if (st.first_bad != ~0ull) {
                char buf[160];
                snprintf(buf, sizeof(buf), "%s string at input position %llu has the wrong electron count or a bit >= norb",
                         s == 0 ? "alpha" : "beta", st.first_bad);
                fail(SBD_ERR_BAD_STRING, buf);
            }
            radix_sort_strings(c, t.strings, t.n, norb);
            check_duplicates(c, t.strings, t.n);
            SBD_CUDA(cudaMemcpyAsync(&st, c.dstat, sizeof(st), cudaMemcpyDeviceToHost, c.stream));
            SBD_CUDA(cudaStreamSynchronize(c.stream));
            if (st.first_dup != ~0ull) {
                fail(SBD_ERR_DUPLICATE_STRING, std::string(s == 0 ? "alpha" : "beta") + " strings contain a duplicate");
            }
        }
        // identical sets share their tables
        bool same = false;
        if (nA == nB && nalpha == nbeta) {
            compare_sets(c, c.sp[0].strings, c.sp[1].strings, nA);
            SBD_CUDA(cudaMemcpyAsync(&st, c.dstat, sizeof(st), cudaMemcpyDeviceToHost, c.stream));
            SBD_CUDA(cudaStreamSynchronize(c.stream));
            same = st.differ == 0;
        }
        build_tables(c, 0);
        if (same) {
            uint64_t *own = c.sp[1].strings;
            c.sp[1] = c.sp[0];
            c.sp[1].strings = own;
            c.sp[1].alias = true;
        } else {
            build_tables(c, 1);
        }
        build_diagonal(c);
        c.work_t = dalloc(c, (size_t)c.N * sizeof(double));
        sigma_prepare(c);
        SBD_CUDA(cudaStreamSynchronize(c.stream));
        return SBD_OK;
    });
    if (rc != SBD_OK) {
        // release whatever was allocated; errors here are secondary
        try {
            free_all(c);
            (void)cudaStreamSynchronize(c.stream);
        } catch (...) {
        }
        delete hd;
        return rc;
    }
    *out = hd;
    return SBD_OK;
}

int sbd_destroy(sbd_handle h)
{
    if (!h) return SBD_ERR_INVALID_ARG;
    int rc = guarded(nullptr, [&]() -> int {
        free_all(h->c);
        SBD_CUDA(cudaStreamSynchronize(h->c.stream));
        destroy_events(h->c);
        return SBD_OK;
    });
    delete h;
    return rc;
}

int sbd_dims(sbd_handle h, int64_t *nA, int64_t *nB)
{
    if (!h) return SBD_ERR_INVALID_ARG;
    if (nA) *nA = h->c.nA;
    if (nB) *nB = h->c.nB;
    return SBD_OK;
}

int sbd_memory(sbd_handle h, size_t *bytes)
{
    if (!h || !bytes) return SBD_ERR_INVALID_ARG;
    *bytes = h->c.bytes_held;
    return SBD_OK;
}

int sbd_sorted_strings(sbd_handle h, int spin, uint64_t *out_host)
{
    if (!h || !out_host || spin < 0 || spin > 1) return SBD_ERR_INVALID_ARG;
    return guarded(h, [&]() -> int {
        const SpinTables &t = h->c.sp[spin];
        SBD_CUDA(cudaMemcpyAsync(out_host, t.strings, (size_t)t.n * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                 h->c.stream));
        SBD_CUDA(cudaStreamSynchronize(h->c.stream));
        return SBD_OK;
    });
}

int sbd_table_size(sbd_handle h, int spin, int kind, int64_t *nentries)
{
    if (!h || !nentries || spin < 0 || spin > 1 || kind < 1 || kind > 2) return SBD_ERR_INVALID_ARG;
    *nentries = kind == 1 ? h->c.sp[spin].ns : h->c.sp[spin].nd;
    return SBD_OK;
}

int sbd_tables(sbd_handle h, int spin, int kind, int64_t *ptr_host, int32_t *target_host, uint8_t *orbs_host,
               int8_t *sign_host)
{
    if (!h || spin < 0 || spin > 1 || kind < 1 || kind > 2) return SBD_ERR_INVALID_ARG;
    return guarded(h, [&]() -> int {
        const SpinTables &t = h->c.sp[spin];
        const int64_t m = kind == 1 ? t.ns : t.nd;
        cudaStream_t s = h->c.stream;
        if (ptr_host)
            SBD_CUDA(cudaMemcpyAsync(ptr_host, kind == 1 ? t.s_ptr : t.d_ptr, (size_t)(t.n + 1) * sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, s));
        if (target_host && m)
            SBD_CUDA(cudaMemcpyAsync(target_host, kind == 1 ? t.s_j : t.d_j, (size_t)m * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s));
        if (orbs_host && m)
            SBD_CUDA(cudaMemcpyAsync(orbs_host, kind == 1 ? t.s_orb : t.d_orb, (size_t)m * 4, cudaMemcpyDeviceToHost, s));
        if (sign_host && m)
            SBD_CUDA(cudaMemcpyAsync(sign_host, kind == 1 ? t.s_sign : t.d_sign, (size_t)m, cudaMemcpyDeviceToHost, s));
        SBD_CUDA(cudaStreamSynchronize(s));
        return SBD_OK;
    });
}

int sbd_string_elements(sbd_handle h, int spin, int kind, double *out_host)
{
    if (!h || !out_host || spin < 0 || spin > 1 || kind < 0 || kind > 2) return SBD_ERR_INVALID_ARG;
    return guarded(h, [&]() -> int {
        const SpinTables &t = h->c.sp[spin];
        const double *src = kind == 0 ? t.ediag : (kind == 1 ? t.s_v64 : t.d_v64);
        const int64_t m = kind == 0 ? t.n : (kind == 1 ? t.ns : t.nd);
        if (m) SBD_CUDA(cudaMemcpyAsync(out_host, src, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, h->c.stream));
        SBD_CUDA(cudaStreamSynchronize(h->c.stream));
        return SBD_OK;
    });
}

int sbd_diagonal(sbd_handle h, double *hd_dev, void *stream)
{
    if (!h || !hd_dev) return SBD_ERR_INVALID_ARG;
    return guarded(h, [&]() -> int {
        SBD_CUDA(cudaMemcpyAsync(hd_dev, h->c.hd, (size_t)h->c.N * sizeof(double), cudaMemcpyDeviceToDevice,
                                 (cudaStream_t)stream));
        return SBD_OK;
    });
}

int sbd_lookup(sbd_handle h, int spin, const uint64_t *keys_dev, int64_t n, int64_t *idx_dev, void *stream)
{
    if (!h || spin < 0 || spin > 1 || n < 0 || (n > 0 && (!keys_dev || !idx_dev))) return SBD_ERR_INVALID_ARG;
    return guarded(h, [&]() -> int {
        const SpinTables &t = h->c.sp[spin];
        lookup_strings(t.strings, t.n, keys_dev, n, idx_dev, (cudaStream_t)stream);
        return SBD_OK;
    });
}

int sbd_sigma(sbd_handle h, const void *c_dev, double *sigma_dev, int nvec, sbd_precision prec, void *stream)
{
    if (!h || !c_dev || !sigma_dev || nvec < 1 || prec < SBD_FP64 || prec > SBD_F32X2) return SBD_ERR_INVALID_ARG;
    return guarded(h, [&]() -> int {
        Ctx &c = h->c;
        const size_t elem = prec == SBD_MIXED ? sizeof(float) : sizeof(double);
        for (int v = 0; v < nvec; ++v)
            sigma_apply(c, static_cast<const char *>(c_dev) + (size_t)v * c.N * elem, sigma_dev + (size_t)v * c.N, prec,
                        (cudaStream_t)stream);
        return SBD_OK;
    });
}

int sbd_davidson(sbd_handle h, int nroots, double tol, sbd_precision prec, double *energies_host, double *vecs,
                 double *residuals_host, sbd_report *report)
{
    if (!h || !energies_host || prec < SBD_FP64 || prec > SBD_F32X2) return SBD_ERR_INVALID_ARG;
    return guarded(h, [&]() -> int {
        return davidson(h->c, nroots, tol, prec, energies_host, vecs, residuals_host, report);
    });
}

int sbd_davidson_sharded(sbd_handle h, const int64_t *bounds, const sbd_comm *comm, int nroots, double tol,
                         sbd_precision prec, double *energies_host, double *vecs_rows, double *residuals_host,
                         sbd_report *report)
{
    if (!h || !bounds || !comm || !energies_host || prec < SBD_FP64 || prec > SBD_F32X2) return SBD_ERR_INVALID_ARG;
    return guarded(h, [&]() -> int {
        Ctx &c = h->c;
        ShardCtx sh;
        sh.rank = comm->rank;
        sh.world = comm->world;
        sh.comm = *comm;
        if (sh.world < 1 || sh.rank < 0 || sh.rank >= sh.world || sh.world > c.nA)
            fail(SBD_ERR_INVALID_ARG, "sharded solve: rank/world out of range");
        if (sh.world > 1 && (!comm->allreduce_sum || !comm->ring_exchange))
            fail(SBD_ERR_INVALID_ARG, "sharded solve: communication callbacks missing");
        sh.bounds.assign(bounds, bounds + sh.world + 1);
        if (sh.bounds[0] != 0 || sh.bounds[sh.world] != c.nA)
            fail(SBD_ERR_INVALID_ARG, "sharded solve: bounds must run from 0 to nA");
        int64_t maxrows = 0;
        for (int b = 0; b < sh.world; ++b) {
            if (sh.bounds[b + 1] <= sh.bounds[b]) fail(SBD_ERR_INVALID_ARG, "sharded solve: empty or decreasing block");
            maxrows = std::max(maxrows, sh.bounds[b + 1] - sh.bounds[b]);
        }
        auto cleanup = [&]() {
            for (BlockPlan *p : sh.plans) block_plan_destroy(p);
            sh.plans.clear();
            for (void *&q : sh.ring)
                if (q) {
                    dfree(c, q);
                    q = nullptr;
                }
        };
        try {
            for (int b = 0; b < sh.world; ++b)
                sh.plans.push_back(block_plan_create(c, sh.row0(), sh.row0() + sh.rows(), sh.bounds[b], sh.bounds[b + 1]));
            if (sh.world > 1)
                for (void *&q : sh.ring) q = dalloc(c, sizeof(double) * (size_t)maxrows * (size_t)c.nB);
            const int rc = davidson(c, nroots, tol, prec, energies_host, vecs_rows, residuals_host, report, &sh);
            cleanup();
            return rc;
        } catch (...) {
            cleanup();
            throw;
        }
    });
}

int sbd_kernel_times(sbd_handle h, double *ms_host, int64_t *launches_host, int reset)
{
    if (!h) return SBD_ERR_INVALID_ARG;
    return guarded(h, [&]() -> int {
        harvest_timing(h->c);
        for (int i = 0; i < 12; ++i) {
            if (ms_host) ms_host[i] = h->c.kernel_ms[i];
            if (launches_host) launches_host[i] = h->c.kernel_n[i];
            if (reset) {
                h->c.kernel_ms[i] = 0.0;
                h->c.kernel_n[i] = 0;
            }
        }
        return SBD_OK;
    });
}

int64_t sbd_launch_count(void) { return g_launches.load(); }

}  // extern "C"
