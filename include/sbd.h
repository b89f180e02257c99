/*
 * sbd.h -- C ABI of the GB300 selected-basis diagonalization (SBD) library.
 *
 * The library computes, on one CUDA device, the lowest eigenpairs of the
 * Hamiltonian restricted to a selected determinant space (paper Sec. II,
 * Eqs. 1-2).  Determinants are the product A x B of a selected alpha-string
 * set A and a selected beta-string set B ("half-bitstring" form, Sec. II-F):
 * each string is a uint64 occupation bitstring over norb <= 64 spatial
 * orbitals.  Amplitude vectors are stored row-major as C[|A|][|B|]
 * (index ia*|B| + ib) with both string sets in ascending unsigned order.
 *
 * The Hamiltonian is Eq. 3 with one-electron integrals h_pq and
 * two-electron integrals (pq|rs) in chemists' notation, i.e.
 *   H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps),
 * E_pq = sum_spin a+_p a_q; matrix elements follow the Slater-Condon rules
 * (Eq. 4).  Fermionic phases use the Jordan-Wigner order "all alpha modes
 * ascending, then all beta modes ascending".
 *
 * Conventions for every entry point:
 *  - Return value: 0 = SBD_OK, > 0 = warning, < 0 = error (enum below).
 *    No C++ exception crosses the ABI.  sbd_last_error() describes the most
 *    recent failure on the handle (or, for a NULL handle, on this thread).
 *  - "device pointer": memory the CUDA runtime can address on the handle's
 *    device.  "host or device pointer": any pointer cudaMemcpy can read with
 *    cudaMemcpyDefault (pageable or pinned host memory, or device memory).
 *  - Streams are cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Work is enqueued on that stream; functions that return host
 *    results synchronise it.
 *  - A handle is not thread-safe: one host thread at a time per handle.
 *  - Device memory owned by a handle comes from the allocator in
 *    sbd_options (default: the CUDA stream-ordered allocator) and is freed by
 *    sbd_destroy.  Caller-owned buffers stay caller-owned.
 */
#ifndef SBD_H
#define SBD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbd_ctx *sbd_handle;

typedef enum {
    SBD_FP64 = 0,  /* FP64 amplitudes, integrals, products and sums */
    SBD_MIXED = 1, /* FP32 amplitudes and integrals, FP32 products and inner
                      sums, FP64 accumulation per output element */
    SBD_F32X2 = 2, /* FP64 vectors, FP64-accurate arithmetic on the FP32 pipe:
                      every operand an unevaluated sum of two floats (about
                      48 significant bits), exact FP32 products with their
                      rounding errors recovered by fused multiply-adds, two-sum
                      additions; the same tolerance as SBD_FP64 (1e-12
                      relative), several times faster on GPUs whose FP64 rate
                      is a small fraction of their FP32 rate */
} sbd_precision;

enum {
    SBD_OK = 0,
    SBD_NOT_CONVERGED = 1,        /* warning: best estimates were still written */
    SBD_ERR_INVALID_ARG = -1,     /* NULL pointer, size or count out of range */
    SBD_ERR_BAD_STRING = -2,      /* popcount != electron count, or a bit >= norb */
    SBD_ERR_DUPLICATE_STRING = -3,/* a string occurs twice in A or in B */
    SBD_ERR_NORB = -4,            /* norb outside 1..64 */
    SBD_ERR_OUT_OF_MEMORY = -5,   /* the allocator returned NULL */
    SBD_ERR_OVER_BUDGET = -6,     /* would exceed sbd_options.hbm_budget_bytes */
    SBD_ERR_CUDA = -7,            /* a CUDA runtime call failed */
    SBD_ERR_NONFINITE = -8,       /* NaN or Inf in h or eri */
    SBD_ERR_BREAKDOWN = -9,       /* Davidson could not extend its subspace */
    SBD_ERR_UNSUPPORTED = -10,    /* a size this build does not handle */
    SBD_PENDING = 2,              /* engine job not finished yet (sbd_engine_result) */
};

/* Device allocator hooks.  alloc returns a device pointer (16-byte aligned
 * or better) usable on `stream`, or NULL; free releases it, stream-ordered. */
typedef void *(*sbd_alloc_fn)(void *ctx, size_t bytes, void *stream);
typedef void (*sbd_free_fn)(void *ctx, void *ptr, void *stream);

typedef struct {
    double delta;            /* preconditioner floor delta of Eq. 7 (default 1e-4) */
    int max_subspace;        /* Davidson subspace cap; 0 = max(24, 8*nroots), lowered to fit the budget */
    int max_iter;            /* Davidson iteration cap; 0 = 200 */
    size_t hbm_budget_bytes; /* cap on device bytes the handle may hold; 0 = unlimited */
    double ecore;            /* constant added to reported energies */
    int table_algo;          /* excitation tables: 0 auto, 1 all-pairs XOR-popcount, 2 enumerate + lookup */
    int verbose;             /* > 0: per-iteration log on stderr */
    sbd_alloc_fn alloc;      /* NULL: cudaMallocAsync / cudaFreeAsync */
    sbd_free_fn free;
    void *alloc_ctx;
    int timing;              /* nonzero: time every sigma kernel with CUDA events (sbd_kernel_times) */
    double tol_energy;       /* > 0: a root also needs |theta_k - theta_(k-1)| <= tol_energy between
                                consecutive iterations to count as converged (default 0: off) */
    int refine_precision;    /* FP64-accurate arithmetic of SBD_MIXED solves: SBD_F32X2 (default; the
                                defect-correction sigma and the basis-vector arithmetic in FP32
                                pairs) or SBD_FP64 (both on the FP64 pipe) */
    int restart_keep;        /* Ritz vectors a thick restart keeps; 0 = max(nroots, min(max_subspace -
                                nroots, max(2 nroots, max_subspace/3))) */
} sbd_options;

typedef struct {
    int iterations;       /* Davidson iterations (all phases) */
    int sigma_fp64;       /* vectors multiplied by an FP64-accurate sigma (SBD_FP64 or SBD_F32X2) */
    int sigma_mixed;      /* vectors multiplied by the mixed sigma */
    int restarts;         /* subspace restarts */
    int refinements;      /* FP64 defect-correction steps (mixed mode) */
    int reorthogonalisations; /* second Gram-Schmidt passes (taken when the first removed > 1/sqrt(2)) */
    int status;           /* same as the return value */
    double max_residual;  /* largest final residual norm (FP64-evaluated) */
    double seconds_total; /* wall time inside sbd_davidson */
    double seconds_sigma; /* of which sigma launches (host-timed with events) */
    double gap_estimate;  /* first Ritz value above the roots minus the highest root's Ritz value at
                             the last Rayleigh-Ritz step (0 if the basis held no further vector);
                             residual_j^2 / (gap_estimate + E_last - E_j) estimates the error of
                             energy j (Kato-Temple form, with a Ritz value for the next eigenvalue) */
} sbd_report;

/* Fills *opt with the defaults listed above. */
void sbd_default_options(sbd_options *opt);

/* Human-readable name of a status code (static storage). */
const char *sbd_status_string(int status);

/*
 * sbd_create -- build one instance (paper Sec. II-B/F, III-B).
 *   norb        number of spatial orbitals, 1..64
 *   nalpha/nbeta electrons per spin, 0..norb
 *   h           host or device pointer, norb*norb doubles, row-major h[p*norb+q], symmetric
 *   eri         host or device pointer, norb^4 doubles, (pq|rs) at ((p*norb+q)*norb+r)*norb+s,
 *               8-fold symmetric (real orbitals)
 *   A, B        host or device pointers, nA and nB uint64 strings in any order
 *   opt         NULL for defaults
 *   stream      cudaStream_t used for the build and as the handle's default stream
 * The strings are validated (popcount, bits below norb, no duplicates), sorted
 * ascending, and the excitation tables, string matrix elements and the
 * Hamiltonian diagonal are built on the device.  The inputs are copied; the
 * caller keeps ownership.  On error *out is NULL and nothing is leaked.
 */
int sbd_create(sbd_handle *out, int norb, int nalpha, int nbeta, const double *h, const double *eri,
               const uint64_t *A, int64_t nA, const uint64_t *B, int64_t nB, const sbd_options *opt,
               void *stream);

/* Releases every device buffer of the handle (stream-ordered on its stream). */
int sbd_destroy(sbd_handle handle);

/* |A| and |B|; either output may be NULL. */
int sbd_dims(sbd_handle handle, int64_t *nA, int64_t *nB);

/* Device bytes currently held by the handle. */
int sbd_memory(sbd_handle handle, size_t *bytes);

/* Copies the sorted strings of one spin (0 alpha, 1 beta) to host memory
 * (nA or nB uint64).  Synchronises the handle's stream. */
int sbd_sorted_strings(sbd_handle handle, int spin, uint64_t *out_host);

/*
 * Excitation tables (paper Sec. III-B, the per-string singles/doubles lists).
 * kind 1 = single, 2 = double excitations within one spin's sorted set.
 * Canonical CSR: entries of source i at [ptr[i], ptr[i+1]), targets j
 * ascending, no self entry.  orbs[4e..4e+3] = p1, p2, q1, q2 where p's are
 * occupied in string i only and q's in string j only, each pair ascending
 * (singles: p2 = q2 = 255).  sign = <S_i| a+_p1 a+_p2 a_q2 a_q1 |S_j> (singles:
 * <S_i| a+_p a_q |S_j>).  sbd_table_size gives the entry count; sbd_tables
 * copies to host buffers of ptr[n+1] (int64), target[m] (int32),
 * orbs[4m] (uint8), sign[m] (int8); any of them may be NULL.
 */
int sbd_table_size(sbd_handle handle, int spin, int kind, int64_t *nentries);
int sbd_tables(sbd_handle handle, int spin, int kind, int64_t *ptr_host, int32_t *target_host,
               uint8_t *orbs_host, int8_t *sign_host);

/*
 * Same-spin string matrix elements <S_i|H_spin|S_j> (the Slater-Condon rules
 * of Eq. 4 for one spin species alone), FP64, copied to host:
 * kind 0: the diagonal, n values; kind 1/2: aligned with the entries of
 * sbd_tables(spin, kind).
 */
int sbd_string_elements(sbd_handle handle, int spin, int kind, double *out_host);

/* Hamiltonian diagonal H_ii (Sec. II-E, Eq. 5), nA*nB doubles, into a
 * caller-owned device buffer, enqueued on `stream`. */
int sbd_diagonal(sbd_handle handle, double *hd_dev, void *stream);

/*
 * Index lookup of strings in one spin's sorted set: idx[k] = position of
 * keys[k], or -1 when absent (warp-cooperative search).  keys_dev and
 * idx_dev are device pointers of n elements; enqueued on `stream`.
 */
int sbd_lookup(sbd_handle handle, int spin, const uint64_t *keys_dev, int64_t n, int64_t *idx_dev,
               void *stream);

/*
 * sbd_sigma -- sigma = H c for nvec vectors (paper Sec. II-B Eq. 4; the
 * matrix-free product of Sec. II-A), enqueued on `stream`.
 *   c_dev     device pointer, [nvec][nA][nB], double for SBD_FP64 and SBD_F32X2,
 *             float for SBD_MIXED, in sorted-string order
 *   sigma_dev device pointer, [nvec][nA][nB] doubles (written, not accumulated)
 * The handle keeps one transposed copy of a vector as work space (allocated
 * on the first call).  c and sigma must not overlap.
 */
int sbd_sigma(sbd_handle handle, const void *c_dev, double *sigma_dev, int nvec, sbd_precision prec,
              void *stream);

/*
 * sbd_davidson -- lowest nroots eigenpairs by block Davidson (paper Sec. II-C
 * with the damped diagonal preconditioner of Sec. II-E, stopping per
 * Sec. II-G), on the handle's stream.
 *   tol         residual-norm tolerance ||H u - theta u||_2 per root (u normalised)
 *   prec        SBD_FP64; SBD_F32X2 (every sigma FP64-accurate on the FP32 pipe);
 *               or SBD_MIXED: mixed-precision sigma for the bulk of the iterations
 *               with FP64-accurate defect correction (sbd_options.refine_precision;
 *               the converged residual is always FP64-accurate).  Vectors, the projected
 *               eigenproblem, residuals and energies stay FP64; with SBD_F32X2 (the whole
 *               solve, or refine_precision of a mixed one) the Ritz-vector combinations,
 *               the Gram-Schmidt dot products and updates and the projected-matrix dot
 *               products sum in FP32 pairs (48-bit products, one FP64 rounding per stored
 *               value or per block sum); the Rayleigh quotients that decide convergence
 *               after a defect correction are FP64 dot products
 *   energies_host  nroots doubles (ascending), ecore included
 *   vecs        NULL, or host or device pointer for [nroots][nA*nB] doubles
 *   residuals_host NULL or nroots doubles
 *   report      NULL or filled on return
 * Returns SBD_OK, SBD_NOT_CONVERGED (estimates still written) or an error.
 */
int sbd_davidson(sbd_handle handle, int nroots, double tol, sbd_precision prec, double *energies_host,
                 double *vecs, double *residuals_host, sbd_report *report);

/*
 * Per-kernel device time of the sigma kernels launched on this handle since
 * the last reset (only when sbd_options.timing was set), measured with CUDA
 * events recorded on the stream each kernel was launched on.  Slots:
 *   0 transpose of C, 1 beta gather pass (rows of C), 2 alpha gather pass
 *   (rows of C^T), 3 alpha-beta pass; FP64 kernels in 0..3, mixed in 4..7,
 *   SBD_F32X2 in 8..11.
 * ms_host and launches_host: 12 entries each (either may be NULL).  Waits for
 * the recorded events; reset != 0 clears the counters afterwards.
 */
int sbd_kernel_times(sbd_handle handle, double *ms_host, int64_t *launches_host, int reset);

/* Number of kernels this library has launched in the process so far. */
int64_t sbd_launch_count(void);

/*
 * sbd_sort_strings_noalloc -- validate and sort one string set without
 * allocating any device memory.  The paper has no counterpart; this entry
 * point exists for callers that cannot let a library allocate on their
 * behalf (device memory carved up in advance by the caller's own allocator,
 * a plug-in that must not grow its host process's footprint, a loop that may
 * not touch an allocator).  It runs the same validation, stable radix sort and
 * duplicate check as sbd_create, with its work space in a fixed array inside
 * the library (SBD_NOALLOC_MAX_STRINGS strings; about 0.5 MB that every GPU
 * which loads the library holds until the process exits).
 *   keys_dev     device pointer, n uint64 strings (any order; not modified)
 *   n            0..SBD_NOALLOC_MAX_STRINGS; larger n returns SBD_ERR_INVALID_ARG
 *   norb, nel    orbitals (1..64) and electrons per string
 *   sorted_dev   device pointer, n uint64: the strings in ascending order
 *   bad_index_host NULL or one int64: -1, or for SBD_ERR_BAD_STRING the input
 *                position of a malformed string, for SBD_ERR_DUPLICATE_STRING the
 *                sorted position of a repeated string
 * Every call is enqueued on `stream` and synchronises `stream` before it
 * returns (the status words are read back).  The first call on each device
 * looks up the work space's device address (cudaGetSymbolAddress, with that
 * device current) and caches it; make that first call before any stream
 * capture.  The cached address assumes that the device's CUDA context lives
 * as long as the library stays loaded (no cudaDeviceReset in between).  All
 * calls share the work space: calls that overlap on the GPU race and must be
 * serialised by the caller.  Errors are reported by sbd_last_error(NULL) on
 * this thread.
 */
#define SBD_NOALLOC_MAX_STRINGS 65536
int sbd_sort_strings_noalloc(const uint64_t *keys_dev, int64_t n, int norb, int nel, uint64_t *sorted_dev,
                             int64_t *bad_index_host, void *stream);

/*
 * sbd_sigma_batched -- sigma = H c of n instances in one batched launch
 * sequence: a transpose and the beta, alpha and alpha-beta passes each run as
 * one persistent launch whose CTAs take (instance, row-group) work items from
 * a device counter (the batched engine's sigma; paper Sec. II-A/B Eq. 4).
 *   handles      n handles on the same device (distinct)
 *   c_dev[i]     device pointer, handle i's [nA][nB] vector (float for
 *                SBD_MIXED, double for SBD_FP64), sorted-string order
 *   sigma_dev[i] device pointer, [nA][nB] doubles, written
 *   rows_per_item rows of C staged per work item: 1, 2, or for SBD_MIXED 4 or 8
 *                (8: one column half at a time); 0 picks the largest that fits
 *                shared memory for every instance
 * Each output element is computed by the same arithmetic as sbd_sigma with
 * the same rows per item (sbd_sigma takes 8 rows over column halves for
 * SBD_MIXED where they fit, else the largest that fits).  Enqueued on `stream`
 * (the handles' work buffers are used), then synchronised.
 */
int sbd_sigma_batched(int n, const sbd_handle *handles, const void *const *c_dev, double *const *sigma_dev,
                      sbd_precision prec, int rows_per_item, void *stream);

/*
 * Alpha-row sharding (paper Sec. III: the alpha rows of C and sigma are distributed over
 * processes and the C blocks are passed around a ring).  A block plan fixes output alpha rows
 * [r0, r1) and source alpha rows [j0, j1) of the handle's instance; sbd_sigma_block adds the
 * contribution of the source block to the output rows:
 *   sigma_rows[(ia-r0)*nB + ib] += sum_{ja in [j0,j1), jb} H[(ia,ib),(ja,jb)] c_block[(ja-j0)*nB + jb]
 * Summed over the blocks of a partition of [0, nA), this is rows [r0, r1) of sbd_sigma (up to the
 * rounding order of the partial sums).  c_block: device pointer, (j1-j0)*nB elements (float for
 * SBD_MIXED, double otherwise); sigma_rows: device pointer, (r1-r0)*nB doubles, accumulated (zero
 * it before the first block).  A plan holds device memory through the handle's allocator and
 * budget and must be destroyed before the handle; calls on one plan must not overlap.  Errors of
 * sbd_block_plan_create are reported on the handle, those of the other two on the calling thread
 * (sbd_last_error(NULL)).
 */
typedef struct sbd_block_plan_s *sbd_block_plan;
int sbd_block_plan_create(sbd_handle handle, int64_t r0, int64_t r1, int64_t j0, int64_t j1, sbd_block_plan *out);
int sbd_sigma_block(sbd_block_plan plan, const void *c_block_dev, double *sigma_rows_dev, sbd_precision prec,
                    void *stream);
int sbd_block_plan_destroy(sbd_block_plan plan);

/*
 * Alpha-row-sharded Davidson (paper Sec. III: the distributed eigensolver).  Every rank calls
 * sbd_davidson_sharded on its own handle of the same instance, with the same bounds (world + 1
 * alpha-row boundaries, bounds[0] = 0, bounds[world] = nA, increasing) and its own rank; it holds
 * rows [bounds[rank], bounds[rank+1]) of every Davidson vector.  Sigma products run the ring of
 * sbd_sigma_block over the blocks; dot products, norms and the searches for the initial and the
 * sign-fixing components are summed over the ranks with allreduce_sum, so every rank takes the same
 * decisions and returns the same energies.  vecs_rows (NULL or host or device memory) receives this
 * rank's rows of the eigenvectors, [nroots][(bounds[rank+1]-bounds[rank])*nB].
 * Callbacks (called from the thread that called sbd_davidson_sharded, in the same order on every
 * rank; nonzero return = failure, reported as SBD_ERR_CUDA):
 *   allreduce_sum(ctx, buf, n): replace the n host doubles in buf by their sum over the ranks;
 *   ring_exchange(ctx, send, send_bytes, recv, recv_bytes, stream): send the device buffer `send` to
 *     rank (rank+1) mod world and receive into the device buffer `recv` from rank (rank-1) mod world;
 *     `send` holds its data when the call is made, and `recv` must hold the data when the callback
 *     returns.  The products of the block in `send` may still be running on `stream` during the call
 *     (the transfer overlaps them, double buffering): the callback must not write `send`; `recv` is
 *     not in use by the library until the callback returns.
 */
typedef struct {
    int rank, world;
    void *ctx;
    int (*allreduce_sum)(void *ctx, double *buf, int n);
    int (*ring_exchange)(void *ctx, const void *send, size_t send_bytes, void *recv, size_t recv_bytes,
                         void *stream);
} sbd_comm;

int sbd_davidson_sharded(sbd_handle handle, const int64_t *bounds, const sbd_comm *comm, int nroots, double tol,
                         sbd_precision prec, double *energies_host, double *vecs_rows, double *residuals_host,
                         sbd_report *report);

/*
 * Batched and served solves.  No counterpart in the paper: an engine runs the
 * Davidson iterations (Sec. II-C, the Eq. 7 preconditioner) of many
 * independent instances ("jobs") together on one device.  Per engine
 * iteration, one set of persistent kernel launches covers every admitted job
 * (the sigma work items and vector chunks of all jobs share each launch), and
 * the iteration's launch sequence is captured once as two CUDA graphs that
 * are replayed.  Jobs are admitted in submission order while a slot is free
 * and their device memory fits the budget, iterate until converged, and leave,
 * so jobs submitted while others run join them (continuous batching).  A job's
 * arithmetic does not depend on the other jobs: its results are bitwise the
 * same alone and in any mix.
 *
 * Per job: 1 root; sigma in mixed precision (SBD_MIXED) for the iterations;
 * convergence when the mixed residual is <= tol and (tol_energy > 0) the
 * change of the Ritz value since the previous iteration is <= tol_energy; the
 * result is then checked with one FP64 sigma of the Ritz vector, whose FP64
 * residual must also be <= tol (else the job iterates on with a halved mixed
 * threshold).  Reported energy = FP64 Rayleigh quotient + ecore.  The basis
 * vector arithmetic (Ritz combinations, Gram-Schmidt, projected matrix, restart)
 * sums in FP32 pairs (48-bit products); the check is FP64.
 * Orthogonalisation: classical Gram-Schmidt with a second pass when the first removed more than
 * half of the squared norm (the DGKS criterion, decided per job on the device); thick restart
 * to nkeep = max(2, max_subspace/3) Ritz vectors.
 */
typedef struct sbd_engine_s *sbd_engine;

typedef struct {
    int max_slots;           /* jobs on the device at once (default 64, at most 1024) */
    int max_subspace;        /* Davidson basis vectors per job (default 12, 3..32) */
    int max_iter;            /* iterations per job (default 200) */
    int max_norb;            /* largest norb of a job (default 64) */
    int max_strings;         /* largest |A| or |B| of a job (default 20000) */
    int rows_per_item;       /* mixed sigma rows per work item: 1, 2, 4, 8 (over column halves); 0 = autotune at
                                the first step */
    double delta;            /* preconditioner floor (default 1e-4) */
    size_t hbm_budget_bytes; /* admission budget for the jobs' device memory; 0 = unlimited */
    sbd_alloc_fn alloc;      /* NULL: cudaMallocAsync / cudaFreeAsync */
    sbd_free_fn free;
    void *alloc_ctx;
    /* Admission estimate of a job's excitation tables, in bytes per string (default 16384).  The
     * estimate only decides when a job is tried: its handle is then created under the budget left
     * after the running jobs and its own basis, and a job whose tables do not fit returns to the
     * head of the queue until running jobs free memory (or fails with SBD_ERR_OVER_BUDGET when no
     * other job holds memory). */
    size_t table_bytes_per_string;
    /* Which jobs take part in an iteration.  SBD_SCHED_FAIR (default): jobs share the device by
     * cost, stride scheduling on N = nA*nB: every job has a pass value that grows by N each
     * iteration it takes part in, and an iteration runs the jobs whose pass is below the smallest
     * pass plus the smallest N of the running jobs, so a job N times larger than the smallest
     * iterates about once per N/N_min iterations while smaller ones run (equal device time per
     * job; a job admitted later starts at the smallest pass).  SBD_SCHED_LOCKSTEP: every job
     * takes part in every iteration.  The schedule changes when a job finishes, never what it
     * computes. */
    int schedule;
} sbd_engine_options;

enum { SBD_SCHED_FAIR = 0, SBD_SCHED_LOCKSTEP = 1 };

typedef struct {
    int status;          /* SBD_OK, SBD_NOT_CONVERGED, or an error (< 0) */
    int iterations;      /* engine iterations the job took part in */
    int sigma_mixed;     /* mixed sigma products */
    int sigma_fp64;      /* FP64 sigma products (checks) */
    int restarts;
    double energy;       /* FP64 Rayleigh quotient of the returned vector, + ecore */
    double residual;     /* its FP64 residual norm */
    double energy_mixed; /* last mixed Ritz value, + ecore */
    double t_submit;     /* engine clock (seconds since sbd_engine_create) */
    double t_admit;
    double t_done;
    int64_t ndets;       /* nA * nB */
} sbd_job_result;

typedef struct {
    int64_t steps;            /* sbd_engine_step calls that did work */
    int64_t graph_launches;   /* CUDA graph replays */
    int64_t kernel_launches;  /* kernels run by this engine (graph nodes included) */
    int rows_per_item;        /* mixed sigma rows per work item in use */
    double tune_ms[4];        /* autotuner: batched mixed sigma time with 8, 4, 2, 1 rows (0 = not tried) */
    size_t bytes_in_use;      /* device bytes held for admitted jobs */
    size_t bytes_peak;
    int active, pending, done;
    int64_t requeued;         /* admissions undone because a job's tables exceeded the budget left */
} sbd_engine_stats;

void sbd_engine_default_options(sbd_engine_options *opt);
/* One engine per device and stream; the stream is used for all its work. */
int sbd_engine_create(sbd_engine *out, const sbd_engine_options *opt, void *stream);
/* Frees every job's device memory; unfinished jobs are dropped. */
int sbd_engine_destroy(sbd_engine engine);
/*
 * Queues a job (inputs as in sbd_create; host or device pointers, copied
 * before return).  keep_vector != 0 keeps the eigenvector for
 * sbd_engine_vector.  *job receives the job id.  Invalid inputs are reported
 * here; errors found while the job runs are reported in its result.
 */
int sbd_engine_submit(sbd_engine engine, int norb, int nalpha, int nbeta, const double *h, const double *eri,
                      const uint64_t *A, int64_t nA, const uint64_t *B, int64_t nB, double ecore, double tol,
                      double tol_energy, int keep_vector, int64_t *job);
/* One engine iteration: admit, iterate every admitted job once, retire the
 * finished ones.  *remaining (may be NULL) = jobs pending or active after it. */
int sbd_engine_step(sbd_engine engine, int *remaining);
/* Steps until no job is pending or active. */
int sbd_engine_run(sbd_engine engine);
/* SBD_PENDING while the job runs; otherwise fills *out and returns SBD_OK. */
int sbd_engine_result(sbd_engine engine, int64_t job, sbd_job_result *out);
/* Copies a finished job's eigenvector (nA*nB doubles, sorted-string order;
 * largest-magnitude component positive) to a host or device pointer. */
int sbd_engine_vector(sbd_engine engine, int64_t job, double *out, int64_t n);
/* Forgets a finished job (its result and vector). */
int sbd_engine_release(sbd_engine engine, int64_t job);
int sbd_engine_get_stats(sbd_engine engine, sbd_engine_stats *out);
/* Seconds since sbd_engine_create on the engine's clock. */
double sbd_engine_clock(sbd_engine engine);

/* Message for the last failure on `handle` (NULL: on this thread); valid
 * until the next call on the same handle / thread. */
const char *sbd_last_error(sbd_handle handle);

#ifdef __cplusplus
}
#endif
#endif /* SBD_H */
