// Excitation tables, same-spin string matrix elements and the Hamiltonian
// diagonal.
//
// For one spin's sorted string set S, the singles and doubles tables list,
// for every source string S_i, the strings S_j of the set that differ from
// it by moving one (single) or two (double) electrons -- the per-string
// excitation lists the sigma product iterates over (paper Sec. III-B,
// Listing 3) -- in canonical CSR form (targets ascending).  Two builders
// produce identical tables:
//   all-pairs  : XOR-popcount of S_i against every S_j (popcount 2 -> single,
//                4 -> double), a warp per source, ballots place the hits;
//   enumerate  : every single/double move of S_i is generated and looked up
//                with the warp-cooperative search; hits are marked in a
//                per-warp bitmap that is then read back in ascending order.
// Fermionic phases are popcount masks over the ket string (Jordan-Wigner
// order within one spin):
//   single q -> p : (-1)^popcount(S_j & bits strictly between p and q)
//                 = <S_i| a+_p a_q |S_j>;
//   double q1<q2 -> p1<p2 : phase(S_j, q2->p2) * phase(S_j', q1->p1), S_j' =
//                 S_j with q2 -> p2, which equals <S_i|a+_p1 a+_p2 a_q2 a_q1|S_j>.
// Matrix elements (Slater-Condon rules, Sec. II-B Eq. 4, for one spin):
//   diagonal  sum_{i in S} h_ii + 1/2 sum_{i,j in S} [(ii|jj) - (ij|ji)]
//   single    phase * [h_pq + sum_{k in S_j} ((pq|kk) - (pk|kq))]
//   double    phase * [(p1 q1|p2 q2) - (p1 q2|p2 q1)]
#include <algorithm>

#include "common.cuh"

namespace sbd {

namespace {

__device__ __forceinline__ double eri_at(const double *__restrict__ eri, int norb, int p, int q, int r, int s)
{
    return __ldg(eri + ((((size_t)p * norb + q) * norb + r) * norb + s));
}

// bits strictly between positions a and b
__device__ __forceinline__ uint64_t between_mask(int a, int b)
{
    const int lo = min(a, b), hi = max(a, b);
    const uint64_t below_hi = (1ull << hi) - 1ull;  // hi <= 63
    const uint64_t upto_lo = (lo >= 63) ? ~0ull : ((1ull << (lo + 1)) - 1ull);
    return below_hi & ~upto_lo;
}

__device__ __forceinline__ int move_phase(uint64_t ket, int from, int to)
{
    return (__popcll(ket & between_mask(from, to)) & 1) ? -1 : 1;
}

struct Entry {
    int32_t j;
    uint8_t orb[4];
    int8_t sign;
    double val;
};

__device__ Entry make_single(uint64_t si, uint64_t sj, int32_t j, int norb, const double *__restrict__ h,
                             const double *__restrict__ eri)
{
    Entry e;
    const uint64_t x = si ^ sj;
    const int p = __ffsll((long long)(x & si)) - 1;
    const int q = __ffsll((long long)(x & sj)) - 1;
    const int sg = move_phase(sj, q, p);
    double v = __ldg(h + (size_t)p * norb + q);
    for (uint64_t m = sj; m; m &= m - 1ull) {
        const int k = __ffsll((long long)m) - 1;
        v += eri_at(eri, norb, p, q, k, k) - eri_at(eri, norb, p, k, k, q);
    }
    e.j = j;
    e.orb[0] = (uint8_t)p;
    e.orb[1] = 255;
    e.orb[2] = (uint8_t)q;
    e.orb[3] = 255;
    e.sign = (int8_t)sg;
    e.val = sg * v;
    return e;
}

__device__ Entry make_double(uint64_t si, uint64_t sj, int32_t j, int norb, const double *__restrict__ eri)
{
    Entry e;
    const uint64_t x = si ^ sj, pb = x & si, qb = x & sj;
    const int p1 = __ffsll((long long)pb) - 1, p2 = 63 - __clzll((long long)pb);
    const int q1 = __ffsll((long long)qb) - 1, q2 = 63 - __clzll((long long)qb);
    const int s2 = move_phase(sj, q2, p2);
    const uint64_t sj2 = sj ^ (1ull << q2) ^ (1ull << p2);
    const int s1 = move_phase(sj2, q1, p1);
    const int sg = s1 * s2;
    const double v = eri_at(eri, norb, p1, q1, p2, q2) - eri_at(eri, norb, p1, q2, p2, q1);
    e.j = j;
    e.orb[0] = (uint8_t)p1;
    e.orb[1] = (uint8_t)p2;
    e.orb[2] = (uint8_t)q1;
    e.orb[3] = (uint8_t)q2;
    e.sign = (int8_t)sg;
    e.val = sg * v;
    return e;
}

struct TableOut {
    const int64_t *s_ptr, *d_ptr;
    int32_t *s_j, *d_j;
    uint8_t *s_orb, *d_orb;
    int8_t *s_sign, *d_sign;
    uint32_t *s_pk;
    double *s_v, *d_v;
};

__device__ __forceinline__ void store_single(const TableOut &o, int64_t pos, const Entry &e, int norb)
{
    o.s_j[pos] = e.j;
    o.s_orb[4 * pos + 0] = e.orb[0];
    o.s_orb[4 * pos + 1] = e.orb[1];
    o.s_orb[4 * pos + 2] = e.orb[2];
    o.s_orb[4 * pos + 3] = e.orb[3];
    o.s_sign[pos] = e.sign;
    o.s_v[pos] = e.val;
    const uint32_t key = 2u * (uint32_t)(e.orb[0] * norb + e.orb[2]) + (e.sign < 0 ? 1u : 0u);
    o.s_pk[pos] = (uint32_t)e.j | (key << kPackKeyShift);
}

__device__ __forceinline__ void store_double(const TableOut &o, int64_t pos, const Entry &e)
{
    o.d_j[pos] = e.j;
    o.d_orb[4 * pos + 0] = e.orb[0];
    o.d_orb[4 * pos + 1] = e.orb[1];
    o.d_orb[4 * pos + 2] = e.orb[2];
    o.d_orb[4 * pos + 3] = e.orb[3];
    o.d_sign[pos] = e.sign;
    o.d_v[pos] = e.val;
}

// ---- all-pairs builder -----------------------------------------------------

__global__ void pairs_count_kernel(const uint64_t *__restrict__ S, int64_t n, int64_t *cnt_s, int64_t *cnt_d)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; i < n; i += nw) {
        const uint64_t si = S[i];
        int64_t cs = 0, cd = 0;
        for (int64_t j0 = 0; j0 < n; j0 += 32) {
            const int64_t j = j0 + lane;
            const int pc = j < n ? __popcll(si ^ __ldg(S + j)) : 0;
            cs += __popc(__ballot_sync(0xffffffffu, pc == 2));
            cd += __popc(__ballot_sync(0xffffffffu, pc == 4));
        }
        if (lane == 0) {
            cnt_s[i] = cs;
            cnt_d[i] = cd;
        }
    }
}

__global__ void pairs_fill_kernel(const uint64_t *__restrict__ S, int64_t n, int norb,
                                  const double *__restrict__ h, const double *__restrict__ eri, TableOut o)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; i < n; i += nw) {
        const uint64_t si = S[i];
        int64_t ps = o.s_ptr[i], pd = o.d_ptr[i];
        for (int64_t j0 = 0; j0 < n; j0 += 32) {
            const int64_t j = j0 + lane;
            const uint64_t sj = j < n ? __ldg(S + j) : si;
            const int pc = __popcll(si ^ sj);
            const unsigned bs = __ballot_sync(0xffffffffu, pc == 2);
            const unsigned bd = __ballot_sync(0xffffffffu, pc == 4);
            if (pc == 2) store_single(o, ps + __popc(bs & lt), make_single(si, sj, (int32_t)j, norb, h, eri), norb);
            if (pc == 4) store_double(o, pd + __popc(bd & lt), make_double(si, sj, (int32_t)j, norb, eri));
            ps += __popc(bs);
            pd += __popc(bd);
        }
    }
}

// ---- enumerate + lookup builder ---------------------------------------------

constexpr int kEnumWarps = 4;

// pair index k in [0, m(m-1)/2) -> (x, y), x < y, in lexicographic order
__device__ __forceinline__ void unrank_pair(int k, int m, int &x, int &y)
{
    x = 0;
    while (k >= m - 1 - x) {
        k -= m - 1 - x;
        ++x;
    }
    y = x + 1 + k;
}

__device__ void mark_hits(const uint64_t *__restrict__ S, int64_t n, uint64_t t, bool valid, unsigned *bitmap)
{
    const int lane = threadIdx.x & 31;
    unsigned todo = __ballot_sync(0xffffffffu, valid);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1u;
        const uint64_t key = __shfl_sync(0xffffffffu, t, src);
        const int64_t idx = warp_find(S, n, key);
        if (lane == 0 && idx >= 0) atomicOr(bitmap + (idx >> 5), 1u << (idx & 31));
    }
}

// mode 0: counts, mode 1: fill
__global__ void enum_kernel(const uint64_t *__restrict__ S, int64_t n, int norb, int nel, int mode,
                            int64_t *cnt_s, int64_t *cnt_d, const double *__restrict__ h,
                            const double *__restrict__ eri, TableOut o)
{
    extern __shared__ unsigned smem_u[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t words = (n + 31) / 32;
    unsigned *bitmap = smem_u + (size_t)wib * words;
    __shared__ uint8_t occ_s[kEnumWarps][64], vir_s[kEnumWarps][64];
    uint8_t *occ = occ_s[wib], *vir = vir_s[wib];
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nw = (int64_t)gridDim.x * kEnumWarps;
    const int no = nel, nv = norb - nel;
    for (int64_t i = blockIdx.x * (int64_t)kEnumWarps + wib; i < n; i += nw) {
        const uint64_t si = S[i];
        int oseen = 0, vseen = 0;
        for (int half = 0; half < 2; ++half) {
            const int m = lane + 32 * half;
            const bool inr = m < norb;
            const bool isocc = inr && ((si >> m) & 1ull);
            const unsigned mo = __ballot_sync(0xffffffffu, isocc);
            const unsigned mv = __ballot_sync(0xffffffffu, inr && !isocc);
            if (isocc) occ[oseen + __popc(mo & lt)] = (uint8_t)m;
            if (inr && !isocc) vir[vseen + __popc(mv & lt)] = (uint8_t)m;
            oseen += __popc(mo);
            vseen += __popc(mv);
        }
        for (int64_t w = lane; w < words; w += 32) bitmap[w] = 0u;
        __syncwarp();
        const int nsc = no * nv;
        for (int c0 = 0; c0 < nsc; c0 += 32) {
            const int cidx = c0 + lane;
            const bool valid = cidx < nsc;
            uint64_t t = 0;
            if (valid) t = si ^ (1ull << occ[cidx / nv]) ^ (1ull << vir[cidx % nv]);
            mark_hits(S, n, t, valid, bitmap);
        }
        const int npo = no * (no - 1) / 2, npv = nv * (nv - 1) / 2;
        const int64_t ndc = (int64_t)npo * npv;
        for (int64_t c0 = 0; c0 < ndc; c0 += 32) {
            const int64_t cidx = c0 + lane;
            const bool valid = cidx < ndc;
            uint64_t t = 0;
            if (valid) {
                int a1, a2, b1, b2;
                unrank_pair((int)(cidx / npv), no, a1, a2);
                unrank_pair((int)(cidx % npv), nv, b1, b2);
                t = si ^ (1ull << occ[a1]) ^ (1ull << occ[a2]) ^ (1ull << vir[b1]) ^ (1ull << vir[b2]);
            }
            mark_hits(S, n, t, valid, bitmap);
        }
        __syncwarp();
        int64_t ps = mode ? o.s_ptr[i] : 0, pd = mode ? o.d_ptr[i] : 0;
        for (int64_t w0 = 0; w0 < words; w0 += 32) {
            const int64_t w = w0 + lane;
            const unsigned bits = w < words ? bitmap[w] : 0u;
            int cs = 0, cd = 0;
            for (unsigned b = bits; b; b &= b - 1u) {
                const int64_t j = w * 32 + (__ffs(b) - 1);
                const int pc = __popcll(si ^ __ldg(S + j));
                cs += pc == 2;
                cd += pc == 4;
            }
            // exclusive warp prefix of (cs, cd)
            int xs = cs, xd = cd;
            for (int off = 1; off < 32; off <<= 1) {
                const int ys = __shfl_up_sync(0xffffffffu, xs, off);
                const int yd = __shfl_up_sync(0xffffffffu, xd, off);
                if (lane >= off) {
                    xs += ys;
                    xd += yd;
                }
            }
            const int ts = __shfl_sync(0xffffffffu, xs, 31), td = __shfl_sync(0xffffffffu, xd, 31);
            if (mode) {
                int64_t qs = ps + xs - cs, qd = pd + xd - cd;
                for (unsigned b = bits; b; b &= b - 1u) {
                    const int64_t j = w * 32 + (__ffs(b) - 1);
                    const uint64_t sj = __ldg(S + j);
                    const int pc = __popcll(si ^ sj);
                    if (pc == 2) store_single(o, qs++, make_single(si, sj, (int32_t)j, norb, h, eri), norb);
                    else if (pc == 4) store_double(o, qd++, make_double(si, sj, (int32_t)j, norb, eri));
                }
            }
            ps += ts;
            pd += td;
        }
        if (!mode && lane == 0) {
            cnt_s[i] = ps;
            cnt_d[i] = pd;
        }
        __syncwarp();
    }
    (void)lt;
}

// ---- scan, diagonal energies, conversions, Hamiltonian diagonal ---------------

// ptr[0] = 0, ptr[i+1] = ptr[i] + cnt[i]; one CTA, each thread a contiguous chunk
__global__ void __launch_bounds__(1024) scan_kernel(const int64_t *cnt, int64_t n, int64_t *ptr)
{
    __shared__ int64_t part[1024];
    const int tid = threadIdx.x;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t b = tid * chunk, e = min(n, b + chunk);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += cnt[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int64_t run = 0;
        for (int t = 0; t < 1024; ++t) {
            const int64_t v = part[t];
            part[t] = run;
            run += v;
        }
    }
    __syncthreads();
    int64_t run = part[tid];
    if (tid == 0) ptr[0] = 0;
    for (int64_t i = b; i < e; ++i) {
        run += cnt[i];
        ptr[i + 1] = run;
    }
}

__global__ void ediag_kernel(const uint64_t *S, int64_t n, int norb, const double *__restrict__ h,
                             const double *__restrict__ eri, double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t s = S[i];
        double one = 0.0, two = 0.0;
        for (uint64_t a = s; a; a &= a - 1ull) {
            const int p = __ffsll((long long)a) - 1;
            one += __ldg(h + (size_t)p * norb + p);
            for (uint64_t b = s; b; b &= b - 1ull) {
                const int q = __ffsll((long long)b) - 1;
                two += eri_at(eri, norb, p, p, q, q) - eri_at(eri, norb, p, q, q, p);
            }
        }
        out[i] = one + 0.5 * two;
    }
}

// Sigma order of each source's list.  The list is padded with empty slots to a multiple of
// kListPad and laid out for 16-byte loads: lane l of an 8-lane group fetches slots 4l..4l+3 of
// each 32-slot chunk, and one 128-bit shared-memory phase gathers slot 4l+u of every lane.
// Entries are first ranked as rounds "rank 0 of every target residue mod 8, rank 1 of every
// residue, ...", so that consecutive entries in that order have distinct residues where the
// residue counts allow; each phase then receives a run of consecutive positions.
// round-order position q of a list of Lp slots -> slot: in a chunk of Lc slots (32, or what is left of
// a short list) m = Lc/4 lanes each fetch 4 slots, and phase u gathers slot 4*l + u of every lane l;
// position m*u + l goes to slot 4*l + u, so each phase reads m consecutive round-order positions
__device__ __forceinline__ int slot_of(int q, int Lp)
{
    const int chunk = q / 32, within = q % 32;
    const int m = min(32, Lp - chunk * 32) / 4;
    return chunk * 32 + 4 * (within % m) + within / m;
}

// Singles lists, where the gathers read two tables: staged amplitudes by target j and coefficient
// rows by key = 2*code + neg (16-byte rows, bank group = index mod 8).  Each phase of m positions is
// filled one entry at a time with the untaken entry that scores highest: residues new to the phase
// first (both sides, then one), and among those the residues most frequent among the untaken
// entries, since the busiest residue classes bound the number of conflict-free phases.  Lists longer
// than kJointMax keep the target-only order.
constexpr int kJointMax = 1024;
__device__ bool joint_order(int64_t b, int64_t e, int64_t sb, int Lp, const int32_t *__restrict__ j_src,
                            const uint32_t *__restrict__ pk, int64_t *perm)
{
    const int L = (int)(e - b);
    if (L > kJointMax) return false;
    uint32_t taken[kJointMax / 32];
    for (int w = 0; w < (L + 31) / 32; ++w) taken[w] = 0u;
    int cj[kBankGroups] = {0, 0, 0, 0, 0, 0, 0, 0}, ck[kBankGroups] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int x = 0; x < L; ++x) {
        ++cj[j_src[b + x] & (kBankGroups - 1)];
        ++ck[(pk[b + x] >> kPackKeyShift) & (kBankGroups - 1)];
    }
    int q = 0;
    while (q < L) {
        const int chunk = q / 32;
        const int m = min(32, Lp - chunk * 32) / 4;
        const int phase_end = min(L, q + m - (q - chunk * 32) % m);  // end of the phase q lies in
        unsigned int usedJ = 0u, usedK = 0u;
        for (; q < phase_end; ++q) {
            int best = -1, best_score = -1, brj = 0, brk = 0;
            for (int x = 0; x < L; ++x) {
                if (taken[x >> 5] >> (x & 31) & 1u) continue;
                const int rj = j_src[b + x] & (kBankGroups - 1);
                const int rk = (pk[b + x] >> kPackKeyShift) & (kBankGroups - 1);
                const int fresh = (int)!((usedJ >> rj) & 1u) + (int)!((usedK >> rk) & 1u);
                const int score = fresh * 4096 + cj[rj] + ck[rk];
                if (score > best_score) {
                    best_score = score;
                    best = x;
                    brj = rj;
                    brk = rk;
                }
            }
            taken[best >> 5] |= 1u << (best & 31);
            usedJ |= 1u << brj;
            usedK |= 1u << brk;
            --cj[brj];
            --ck[brk];
            perm[sb + slot_of(q, Lp)] = b + best;
        }
    }
    return true;
}

// perm[sig_ptr[i] + slot] = index of the canonical entry, or -1 for padding.  One thread per source.
// pk (singles only): packed entries, for the joint target/key order.
__global__ void sigma_order_kernel(const int64_t *__restrict__ ptr, const int64_t *__restrict__ sig_ptr, int64_t n,
                                   const int32_t *__restrict__ j_src, const uint32_t *__restrict__ pk, int64_t *perm)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = ptr[i], e = ptr[i + 1], sb = sig_ptr[i], se = sig_ptr[i + 1];
        const int Lp = (int)(se - sb);
        for (int q = 0; q < Lp; ++q) perm[sb + q] = -1;  // slots no entry lands on stay padding
        if (pk && joint_order(b, e, sb, Lp, j_src, pk, perm)) continue;
        int count[kBankGroups] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t x = b; x < e; ++x) ++count[j_src[x] & (kBankGroups - 1)];
        int seen[kBankGroups] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t x = b; x < e; ++x) {
            const int r = j_src[x] & (kBankGroups - 1);
            const int t = seen[r]++;
            int q = 0;  // position in round order
#pragma unroll
            for (int w = 0; w < kBankGroups; ++w) q += min(count[w], t) + ((w < r && count[w] > t) ? 1 : 0);
            perm[sb + slot_of(q, Lp)] = x;
        }
    }
}

template <typename V>
__global__ void gather_kernel(const V *__restrict__ src, const int64_t *__restrict__ perm, V *dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = perm[i];
        dst[i] = p >= 0 ? src[p] : V(0);
    }
}

// padded counts: cnt[i] = ceil((ptr[i+1]-ptr[i]) / kListPad) * kListPad
__global__ void padded_count_kernel(const int64_t *__restrict__ ptr, int64_t n, int64_t *cnt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L = ptr[i + 1] - ptr[i];
        cnt[i] = (L + kListPad - 1) / kListPad * kListPad;
    }
}

// Source-major singles (column-stationary alpha-beta pass): cnt[i] = items of string i (its singles
// in pieces of kSrcItem); *maxdeg = largest singles count.
__global__ void src_count_kernel(const int64_t *__restrict__ ptr, int64_t n, int64_t *cnt, int *maxdeg)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(ptr[i + 1] - ptr[i]);
        cnt[i] = (d + kSrcItem - 1) / kSrcItem;
        atomicMax(maxdeg, d);
    }
}

// items of string i from item ioff[i] on; each entry keeps the target and phase of the canonical
// single and replaces its orbital code p*norb+q by the index r(r-1)/2 + s of the pair r = max, s = min
__global__ void src_fill_kernel(const int64_t *__restrict__ ptr, const uint32_t *__restrict__ pk, int64_t n,
                                int norb, const int64_t *__restrict__ ioff, uint32_t *item, uint32_t *ent)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = ptr[i], e = ptr[i + 1];
        for (int64_t x = b; x < e; ++x) {
            const int64_t t = ioff[i] + (x - b) / kSrcItem;
            const int slot = (int)((x - b) % kSrcItem);
            if (slot == 0) item[t] = (uint32_t)i | ((uint32_t)min((int64_t)kSrcItem, e - x) << kSrcPairShift);
            const uint32_t v = pk[x];
            const int code = (int)(v >> (kPackKeyShift + 1));
            const int p = code / norb, q = code - p * norb;
            const int r = max(p, q), s = min(p, q);
            const uint32_t pair = (uint32_t)(r * (r - 1) / 2 + s);
            const uint32_t neg = (v >> kPackKeyShift) & 1u;
            ent[(t / 32) * 32 * kSrcItem + 32 * slot + (t % 32)] =
                (v & kPackJMask) | (pair << kSrcPairShift) | (neg << kSrcNegBit);
        }
    }
}

// Order of the items inside each slice of 32: full items first, then the partial ones by decreasing
// length (stable), so that in every round of the alpha-beta pass the lanes that still have a single
// form a prefix of the warp and whole quarter-warps go idle together.  One warp per slice.
__global__ void src_slice_order_kernel(const uint32_t *__restrict__ item_in, const uint32_t *__restrict__ ent_in,
                                       int64_t nsl, uint32_t *item_out, uint32_t *ent_out)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; s < nsl;
         s += (int64_t)gridDim.x * blockDim.x / 32) {
        const uint32_t it = item_in[s * 32 + lane];
        const int key = (int)(it >> kSrcPairShift);  // entries of the item, 0 for an empty slot
        int rank = 0;
        for (int c = kSrcItem; c >= 0; --c) {
            const unsigned m = __ballot_sync(0xffffffffu, key == c);
            if (c > key) rank += __popc(m);
            else if (c == key) rank += __popc(m & lt);
        }
        item_out[s * 32 + rank] = it;
        const int64_t base = s * 32 * kSrcItem;
        for (int i = 0; i < kSrcItem; ++i) ent_out[base + 32 * i + rank] = ent_in[base + 32 * i + lane];
    }
}

// Split of each source list at target `half`: ptr2[2i] = start of list i, ptr2[2i+1] = its first
// entry with target >= half (targets ascend in the canonical lists), ptr2[2n] = end of the last list
__global__ void half_split_kernel(const int64_t *__restrict__ ptr, const int32_t *__restrict__ tgt, int64_t n,
                                  int64_t half, int64_t *ptr2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = ptr[i], hi = ptr[i + 1];
        ptr2[2 * i] = lo;
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if (tgt[mid] < half) lo = mid + 1;
            else hi = mid;
        }
        ptr2[2 * i + 1] = lo;
        if (i == n - 1) ptr2[2 * n] = ptr[n];
    }
}

// Doubles of the half-split lists: val[o] = FP32 of v[perm[o]], tgt[o] = its target relative to
// the column half it lies in (target - half for targets >= half); zeros for padding
__global__ void gather_half_doubles_kernel(const int64_t *__restrict__ perm, int64_t m,
                                           const int32_t *__restrict__ j, const double *__restrict__ v,
                                           int64_t half, float *val, uint16_t *tgt)
{
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < m; o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = perm[o];
        const int64_t jj = e >= 0 ? (int64_t)j[e] : 0;
        val[o] = e >= 0 ? __double2float_rn(v[e]) : 0.f;
        tgt[o] = (uint16_t)(jj >= half ? jj - half : jj);
    }
}

// out[o] = (key[perm[o]], FP32 of val[perm[o]]), zeros for padding
__global__ void gather_pair_kernel(const int64_t *__restrict__ perm, int64_t m, const uint32_t *__restrict__ key,
                                   const double *__restrict__ val, uint2 *out)
{
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < m; o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = perm[o];
        out[o] = e >= 0 ? make_uint2(key[e], __float_as_uint(__double2float_rn(val[e]))) : make_uint2(0u, 0u);
    }
}

// Order of the entries inside the items of each slice: in round i every lane of the warp adds the
// dot product of its item's i-th entry into the row accumulator at the entry's target (32-bit shared
// atomics, bank = target mod 32).  Round by round, each lane takes, of its entries not yet placed,
// one whose bank no earlier lane of that round has taken (the first such), else its first remaining
// entry, so the 32 atomics of a round hit distinct banks where the slice's targets allow.  Any order
// gives the same sums; one thread per slice.
__global__ void src_entry_order_kernel(const uint32_t *__restrict__ item, uint32_t *ent, int64_t nsl)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nsl; s += (int64_t)gridDim.x * blockDim.x) {
        uint32_t *e = ent + s * 32 * kSrcItem;
        uint32_t loc[32][kSrcItem];
        int cnt[32];
        unsigned left[32];
        for (int l = 0; l < 32; ++l) {
            cnt[l] = (int)(item[s * 32 + l] >> kSrcPairShift);
            left[l] = (1u << cnt[l]) - 1u;
            for (int i = 0; i < kSrcItem; ++i) loc[l][i] = e[32 * i + l];
        }
        for (int i = 0; i < kSrcItem; ++i) {
            unsigned used = 0u;
            for (int l = 0; l < 32; ++l) {
                if (i >= cnt[l]) continue;
                int pick = -1;
                for (int x = 0; x < cnt[l]; ++x) {
                    if (!((left[l] >> x) & 1u)) continue;
                    if (pick < 0) pick = x;
                    if (!((used >> (loc[l][x] & 31u)) & 1u)) {
                        pick = x;
                        break;
                    }
                }
                left[l] &= ~(1u << pick);
                used |= 1u << (loc[l][pick] & 31u);
                e[32 * i + l] = loc[l][pick];
            }
        }
    }
}

// (key, FP32 value) pairs for single 8-byte loads in the mixed sigma
__global__ void pair_kernel(const uint32_t *__restrict__ key, const double *__restrict__ val, uint2 *out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_uint2(key[i], __float_as_uint(__double2float_rn(val[i])));
}

// x = hi + lo with hi the FP32 rounding of x and lo the FP32 rounding of the remainder
__global__ void split_kernel(const double *__restrict__ in, float2 *out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = in[i];
        const float hi = __double2float_rn(x);
        out[i] = make_float2(hi, __double2float_rn(x - (double)hi));
    }
}

__global__ void to_float_kernel(const double *in, float *out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __double2float_rn(in[i]);
}

// Hd[ia, ib] = E_alpha(ia) + E_beta(ib) + sum_{p in ia, r in ib} (pp|rr)   (Sec. II-E)
__global__ void hdiag_kernel(const uint64_t *__restrict__ A, const uint64_t *__restrict__ B,
                             const double *__restrict__ eA, const double *__restrict__ eB,
                             const double *__restrict__ eri, int norb, int64_t nA, int64_t nB, double *hd)
{
    __shared__ double jd[64];
    for (int64_t ia = blockIdx.x; ia < nA; ia += gridDim.x) {
        const uint64_t a = A[ia];
        if (threadIdx.x < norb) {
            const int r = threadIdx.x;
            double s = 0.0;
            for (uint64_t m = a; m; m &= m - 1ull) {
                const int p = __ffsll((long long)m) - 1;
                s += eri_at(eri, norb, p, p, r, r);
            }
            jd[r] = s;
        }
        __syncthreads();
        const double ea = eA[ia];
        for (int64_t ib = threadIdx.x; ib < nB; ib += blockDim.x) {
            double v = ea + eB[ib];
            for (uint64_t m = B[ib]; m; m &= m - 1ull) v += jd[__ffsll((long long)m) - 1];
            hd[ia * nB + ib] = v;
        }
        __syncthreads();
    }
}

int blocks_for(int64_t n, int threads, int cap = 65535)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

void to_float(const double *in, float *out, int64_t n, cudaStream_t s)
{
    if (n <= 0) return;
    to_float_kernel<<<blocks_for(n, 256, 16384), 256, 0, s>>>(in, out, n);
    SBD_LAUNCH("to_float_kernel");
}

void build_tables(Ctx &c, int spin)
{
    SpinTables &t = c.sp[spin];
    const int64_t n = t.n;
    const int norb = c.norb;
    if (n >= kMaxStringsPerSpin) fail(SBD_ERR_UNSUPPORTED, "at most 262143 strings per spin are supported");
    int64_t *cnt = dalloc_n<int64_t>(c, 2 * (size_t)n);
    t.s_ptr = dalloc_n<int64_t>(c, n + 1);
    t.d_ptr = dalloc_n<int64_t>(c, n + 1);

    int algo = c.opt.table_algo;
    if (algo == 0) {
        // all-pairs costs n^2/32 warp steps; enumeration about n * moves * (log32 n + 1)
        double moves = (double)t.nel * (norb - t.nel) +
                       0.25 * t.nel * (t.nel - 1.0) * (norb - t.nel) * (norb - t.nel - 1.0);
        double steps = 1.0;
        for (double r = (double)n; r > 32.0; r /= 32.0) steps += 1.0;
        algo = ((double)n / 32.0 > moves * steps && n <= (1 << 17)) ? 2 : 1;
    }
    if (algo == 2 && n > (1 << 17)) fail(SBD_ERR_UNSUPPORTED, "enumerate+lookup tables need |S| <= 131072");
    const int64_t words = (n + 31) / 32;
    const size_t enum_smem = (size_t)kEnumWarps * words * sizeof(unsigned);
    int warps_per_block = 8, threads = 256;
    int grid = blocks_for(n, warps_per_block, 4 * 65535);
    grid = grid > 65535 ? 65535 : grid;
    TableOut o{};
    if (algo == 1) {
        pairs_count_kernel<<<grid, threads, 0, c.stream>>>(t.strings, n, cnt, cnt + n);
        SBD_LAUNCH("pairs_count_kernel");
    } else {
        SBD_CUDA(cudaFuncSetAttribute(enum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)enum_smem));
        int eg = blocks_for(n, kEnumWarps, 65535);
        enum_kernel<<<eg, 32 * kEnumWarps, enum_smem, c.stream>>>(t.strings, n, norb, t.nel, 0, cnt, cnt + n,
                                                                  c.h64, c.eri64, o);
        SBD_LAUNCH("enum_kernel(count)");
    }
    scan_kernel<<<1, 1024, 0, c.stream>>>(cnt, n, t.s_ptr);
    scan_kernel<<<1, 1024, 0, c.stream>>>(cnt + n, n, t.d_ptr);
    SBD_LAUNCH("scan_kernel");
    SBD_CUDA(cudaMemcpyAsync(&t.ns, t.s_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
    SBD_CUDA(cudaMemcpyAsync(&t.nd, t.d_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
    SBD_CUDA(cudaStreamSynchronize(c.stream));
    if (t.ns > 0x7fffffffLL || t.nd > 0x7fffffffLL) fail(SBD_ERR_UNSUPPORTED, "excitation table too large");

    t.s_j = dalloc_n<int32_t>(c, t.ns);
    t.s_orb = dalloc_n<uint8_t>(c, 4 * t.ns);
    t.s_sign = dalloc_n<int8_t>(c, t.ns);
    t.s_pk = dalloc_n<uint32_t>(c, t.ns);
    t.s_v64 = dalloc_n<double>(c, t.ns);
    t.d_j = dalloc_n<int32_t>(c, t.nd);
    t.d_orb = dalloc_n<uint8_t>(c, 4 * t.nd);
    t.d_sign = dalloc_n<int8_t>(c, t.nd);
    t.d_v64 = dalloc_n<double>(c, t.nd);
    o.s_ptr = t.s_ptr;
    o.d_ptr = t.d_ptr;
    o.s_j = t.s_j;
    o.d_j = t.d_j;
    o.s_orb = t.s_orb;
    o.d_orb = t.d_orb;
    o.s_sign = t.s_sign;
    o.d_sign = t.d_sign;
    o.s_pk = t.s_pk;
    o.s_v = t.s_v64;
    o.d_v = t.d_v64;
    if (algo == 1) {
        pairs_fill_kernel<<<grid, threads, 0, c.stream>>>(t.strings, n, norb, c.h64, c.eri64, o);
        SBD_LAUNCH("pairs_fill_kernel");
    } else {
        int eg = blocks_for(n, kEnumWarps, 65535);
        enum_kernel<<<eg, 32 * kEnumWarps, enum_smem, c.stream>>>(t.strings, n, norb, t.nel, 1, nullptr, nullptr,
                                                                  c.h64, c.eri64, o);
        SBD_LAUNCH("enum_kernel(fill)");
    }
    // sigma copies: padded, bank-aware order
    t.sig_s_ptr = dalloc_n<int64_t>(c, n + 1);
    t.sig_d_ptr = dalloc_n<int64_t>(c, n + 1);
    padded_count_kernel<<<blocks_for(n, 256), 256, 0, c.stream>>>(t.s_ptr, n, cnt);
    padded_count_kernel<<<blocks_for(n, 256), 256, 0, c.stream>>>(t.d_ptr, n, cnt + n);
    SBD_LAUNCH("padded_count_kernel");
    scan_kernel<<<1, 1024, 0, c.stream>>>(cnt, n, t.sig_s_ptr);
    scan_kernel<<<1, 1024, 0, c.stream>>>(cnt + n, n, t.sig_d_ptr);
    SBD_LAUNCH("scan_kernel(sigma lists)");
    SBD_CUDA(cudaMemcpyAsync(&t.sig_ns, t.sig_s_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
    SBD_CUDA(cudaMemcpyAsync(&t.sig_nd, t.sig_d_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
    SBD_CUDA(cudaStreamSynchronize(c.stream));
    t.s_pk_sig = dalloc_n<uint32_t>(c, t.sig_ns);
    t.s_v64_sig = dalloc_n<double>(c, t.sig_ns);
    t.s_pkv32 = dalloc_n<uint2>(c, t.sig_ns);
    t.d_j_sig = dalloc_n<int32_t>(c, t.sig_nd);
    t.d_v64_sig = dalloc_n<double>(c, t.sig_nd);
    t.d_jv32 = dalloc_n<uint2>(c, t.sig_nd);
    t.s_vx2 = dalloc_n<float2>(c, t.sig_ns);
    t.d_vx2 = dalloc_n<float2>(c, t.sig_nd);
    int64_t *perm = dalloc_n<int64_t>(c, (size_t)std::max<int64_t>(std::max(t.sig_ns, t.sig_nd), 1));
    const int ob = blocks_for(n, 128);
    if (t.sig_ns) {
        sigma_order_kernel<<<ob, 128, 0, c.stream>>>(t.s_ptr, t.sig_s_ptr, n, t.s_j, t.s_pk, perm);
        SBD_LAUNCH("sigma_order_kernel(singles)");
        const int gb = blocks_for(t.sig_ns, 256, 16384);
        gather_kernel<uint32_t><<<gb, 256, 0, c.stream>>>(t.s_pk, perm, t.s_pk_sig, t.sig_ns);
        gather_kernel<double><<<gb, 256, 0, c.stream>>>(t.s_v64, perm, t.s_v64_sig, t.sig_ns);
        SBD_LAUNCH("gather_kernel(singles)");
        pair_kernel<<<gb, 256, 0, c.stream>>>(t.s_pk_sig, t.s_v64_sig, t.s_pkv32, t.sig_ns);
        SBD_LAUNCH("pair_kernel(singles)");
        split_kernel<<<gb, 256, 0, c.stream>>>(t.s_v64_sig, t.s_vx2, t.sig_ns);
        SBD_LAUNCH("split_kernel(singles)");
    }
    if (t.sig_nd) {
        sigma_order_kernel<<<ob, 128, 0, c.stream>>>(t.d_ptr, t.sig_d_ptr, n, t.d_j, nullptr, perm);
        SBD_LAUNCH("sigma_order_kernel(doubles)");
        const int gb = blocks_for(t.sig_nd, 256, 16384);
        gather_kernel<int32_t><<<gb, 256, 0, c.stream>>>(t.d_j, perm, t.d_j_sig, t.sig_nd);
        gather_kernel<double><<<gb, 256, 0, c.stream>>>(t.d_v64, perm, t.d_v64_sig, t.sig_nd);
        SBD_LAUNCH("gather_kernel(doubles)");
        pair_kernel<<<gb, 256, 0, c.stream>>>(reinterpret_cast<const uint32_t *>(t.d_j_sig), t.d_v64_sig, t.d_jv32,
                                               t.sig_nd);
        SBD_LAUNCH("pair_kernel(doubles)");
        split_kernel<<<gb, 256, 0, c.stream>>>(t.d_v64_sig, t.d_vx2, t.sig_nd);
        SBD_LAUNCH("split_kernel(doubles)");
    }
    dfree(c, perm);
    // mixed-sigma lists split at the middle of the set (row passes over column halves); their
    // 16-bit doubles targets need half <= 65536 (the staged halves fit shared memory only far below)
    if ((n + 1) / 2 <= 65536) {
        t.half = (n + 1) / 2;
        int64_t *ptr2 = dalloc_n<int64_t>(c, 2 * (size_t)n + 1);
        int64_t *cnt2 = dalloc_n<int64_t>(c, 2 * (size_t)n);
        for (int kind = 0; kind < 2; ++kind) {
            const int64_t *ptr = kind == 0 ? t.s_ptr : t.d_ptr;
            const int32_t *tgt = kind == 0 ? t.s_j : t.d_j;
            int64_t *&hptr = kind == 0 ? t.hs_ptr : t.hd_ptr;
            half_split_kernel<<<blocks_for(n, 256), 256, 0, c.stream>>>(ptr, tgt, n, t.half, ptr2);
            SBD_LAUNCH("half_split_kernel");
            hptr = dalloc_n<int64_t>(c, 2 * (size_t)n + 1);
            padded_count_kernel<<<blocks_for(2 * n, 256), 256, 0, c.stream>>>(ptr2, 2 * n, cnt2);
            SBD_LAUNCH("padded_count_kernel(halves)");
            scan_kernel<<<1, 1024, 0, c.stream>>>(cnt2, 2 * n, hptr);
            SBD_LAUNCH("scan_kernel(halves)");
            int64_t m = 0;
            SBD_CUDA(cudaMemcpyAsync(&m, hptr + 2 * n, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
            SBD_CUDA(cudaStreamSynchronize(c.stream));
            const size_t mm = (size_t)std::max<int64_t>(m, 1);
            if (kind == 0) {
                t.hs = dalloc_n<uint2>(c, mm);
            } else {
                t.hdv = dalloc_n<float>(c, mm);
                t.hdt = dalloc_n<uint16_t>(c, mm);
            }
            if (m) {
                int64_t *hperm = dalloc_n<int64_t>(c, (size_t)m);
                sigma_order_kernel<<<blocks_for(2 * n, 128), 128, 0, c.stream>>>(ptr2, hptr, 2 * n, tgt,
                                                                                  kind == 0 ? t.s_pk : nullptr, hperm);
                SBD_LAUNCH("sigma_order_kernel(halves)");
                if (kind == 0) {
                    gather_pair_kernel<<<blocks_for(m, 256, 16384), 256, 0, c.stream>>>(hperm, m, t.s_pk, t.s_v64,
                                                                                         t.hs);
                    SBD_LAUNCH("gather_pair_kernel(halves)");
                } else {
                    gather_half_doubles_kernel<<<blocks_for(m, 256, 16384), 256, 0, c.stream>>>(
                        hperm, m, t.d_j, t.d_v64, t.half, t.hdv, t.hdt);
                    SBD_LAUNCH("gather_half_doubles_kernel");
                }
                dfree(c, hperm);
            }
        }
        dfree(c, cnt2);
        dfree(c, ptr2);
    }
    // source-major singles: items of at most kSrcItem singles, 32 items per slice
    {
        int64_t *ioff = dalloc_n<int64_t>(c, n + 1);
        int *dmax = reinterpret_cast<int *>(cnt + n);  // the doubles counts are no longer needed
        SBD_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), c.stream));
        src_count_kernel<<<blocks_for(n, 256), 256, 0, c.stream>>>(t.s_ptr, n, cnt, dmax);
        SBD_LAUNCH("src_count_kernel");
        scan_kernel<<<1, 1024, 0, c.stream>>>(cnt, n, ioff);
        SBD_LAUNCH("scan_kernel(source-major singles)");
        SBD_CUDA(cudaMemcpyAsync(&t.src_nitem, ioff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
        SBD_CUDA(cudaMemcpyAsync(&t.src_maxdeg, dmax, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
        SBD_CUDA(cudaStreamSynchronize(c.stream));
        const int64_t nsl = std::max<int64_t>((t.src_nitem + 31) / 32, 1);
        t.src_item = dalloc_n<uint32_t>(c, (size_t)nsl * 32);
        t.src_ent = dalloc_n<uint32_t>(c, (size_t)nsl * 32 * kSrcItem);
        SBD_CUDA(cudaMemsetAsync(t.src_item, 0, (size_t)nsl * 32 * sizeof(uint32_t), c.stream));
        SBD_CUDA(cudaMemsetAsync(t.src_ent, 0, (size_t)nsl * 32 * kSrcItem * sizeof(uint32_t), c.stream));
        src_fill_kernel<<<blocks_for(n, 128), 128, 0, c.stream>>>(t.s_ptr, t.s_pk, n, norb, ioff, t.src_item,
                                                                  t.src_ent);
        SBD_LAUNCH("src_fill_kernel");
        dfree(c, ioff);
        uint32_t *item2 = dalloc_n<uint32_t>(c, (size_t)nsl * 32);
        uint32_t *ent2 = dalloc_n<uint32_t>(c, (size_t)nsl * 32 * kSrcItem);
        src_slice_order_kernel<<<blocks_for(nsl * 32, 256), 256, 0, c.stream>>>(t.src_item, t.src_ent, nsl, item2,
                                                                                ent2);
        SBD_LAUNCH("src_slice_order_kernel");
        dfree(c, t.src_item);
        dfree(c, t.src_ent);
        t.src_item = item2;
        t.src_ent = ent2;
        src_entry_order_kernel<<<blocks_for(nsl, 64), 64, 0, c.stream>>>(t.src_item, t.src_ent, nsl);
        SBD_LAUNCH("src_entry_order_kernel");
    }
    t.ediag = dalloc_n<double>(c, n);
    ediag_kernel<<<blocks_for(n, 128), 128, 0, c.stream>>>(t.strings, n, norb, c.h64, c.eri64, t.ediag);
    SBD_LAUNCH("ediag_kernel");
    dfree(c, cnt);
}

void build_diagonal(Ctx &c)
{
    c.hd = dalloc_n<double>(c, (size_t)c.N);
    int grid = (int)(c.nA < 65535 ? c.nA : 65535);
    hdiag_kernel<<<grid, 256, 0, c.stream>>>(c.sp[0].strings, c.sp[1].strings, c.sp[0].ediag, c.sp[1].ediag,
                                             c.eri64, c.norb, c.nA, c.nB, c.hd);
    SBD_LAUNCH("hdiag_kernel");
}

}  // namespace sbd
