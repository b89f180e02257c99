/*
 * sbd_oracle.c -- plain, slow CPU FP64 oracle for selected-basis diagonalization.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg load this file; the CUDA library never links, includes or
 * calls it, and it shares no code, header or table with the CUDA library.
 *
 * What it computes (paper Sec. II, Eqs. 1-4):
 *   H_ij = <Phi_i|H|Phi_j> on the selected determinant space Phi = A x B, the
 *   Hamiltonian being the second-quantised H of Eq. 3 with one-electron
 *   integrals h_pq and two-electron integrals (pq|rs).  Eq. 3 is read in
 *   chemists' notation, the creation operator of each electron pairing with
 *   the first index of its bracket:
 *     H = sum_{pq,s} h_pq a+_{p s} a_{q s}
 *       + 1/2 sum_{pqrs} sum_{s,t} (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s}
 *   (s, t: spin labels).  This is the convention under which the integrals
 *   (pq|rs) = sum_L B^L_pq B^L_rs of the synthetic workloads are defined.
 *
 * Formulation (deliberately different from the CUDA path, which factorises
 * by spin strings):
 *   - a determinant is a full spin-orbital bitstring over 2*norb modes, alpha
 *     modes 0..norb-1 first, then beta modes norb..2norb-1 (Jordan-Wigner
 *     order); |D> = a+_{m1} a+_{m2} ... |0> with m1 < m2 < ...;
 *   - phases come from applying annihilation/creation operators one at a
 *     time, each contributing (-1)^(number of occupied modes below it);
 *   - matrix elements are the textbook spin-orbital Slater-Condon rules with
 *     antisymmetrised integrals <PQ||RS> = <PQ|RS> - <PQ|SR>,
 *     <PQ|RS> = (pr|qs) delta(spin P, spin R) delta(spin Q, spin S)
 *     (Eq. 4 neighbourhood: at most two spin-orbital differences);
 *   - sigma_i = sum_j H_ij x_j over every determinant of the space that
 *     differs from D_i by at most two spin-orbitals (Eq. 4);
 *   - Davidson follows the steps of Sec. II-C in order, with the damped
 *     diagonal preconditioner of Eqs. 6-7 and a cyclic Jacobi eigensolver.
 *
 * Determinant order: ascending unsigned value of the alpha string (major)
 * then of the beta string (minor), i.e. index = ia*|B| + ib over the sorted
 * sets.
 *
 * ORACLE_MUTATION (compile-time, default 0) plants one known mistake; it is
 * used only by the test that checks that the pins catch such mistakes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_MUTATION
#define ORACLE_MUTATION 0
#endif
#define PLANTED(k) (ORACLE_MUTATION == (k))

typedef struct {
    uint64_t w[2]; /* w[0]: alpha occupations, w[1]: beta occupations */
} det_t;

typedef struct {
    int norb, na, nb;
    double *h;   /* norb*norb, row-major */
    double *eri; /* norb^4, (pq|rs) at ((p*norb+q)*norb+r)*norb+s */
    uint64_t *A; /* sorted alpha strings */
    uint64_t *B; /* sorted beta strings */
    int64_t nA, nB;
} oracle_t;

/* ------------------------------------------------------------------------ */
/* modes and fermionic operators                                            */

static int popc(uint64_t x) { return __builtin_popcountll(x); }

static uint64_t low_mask(int k) { return k >= 64 ? ~0ull : ((1ull << k) - 1ull); }

static int mode_occupied(const det_t *d, int norb, int m)
{
    return m < norb ? (int)((d->w[0] >> m) & 1ull) : (int)((d->w[1] >> (m - norb)) & 1ull);
}

/* number of occupied modes with index below m (Jordan-Wigner string) */
static int modes_below(const det_t *d, int norb, int m)
{
    if (m < norb) return popc(d->w[0] & low_mask(m));
    return popc(d->w[0]) + popc(d->w[1] & low_mask(m - norb));
}

static void mode_flip(det_t *d, int norb, int m)
{
    if (m < norb) d->w[0] ^= 1ull << m;
    else d->w[1] ^= 1ull << (m - norb);
}

/* a_m |d>: returns the sign (0 when m is empty) and updates d */
static int annihilate(det_t *d, int norb, int m)
{
    if (!mode_occupied(d, norb, m)) return 0;
    int s = (modes_below(d, norb, m) & 1) ? -1 : 1;
    mode_flip(d, norb, m);
    return s;
}

/* a+_m |d>: returns the sign (0 when m is occupied) and updates d */
static int create(det_t *d, int norb, int m)
{
    if (mode_occupied(d, norb, m)) return 0;
    int s = (modes_below(d, norb, m) & 1) ? -1 : 1;
    mode_flip(d, norb, m);
    return s;
}

/* ------------------------------------------------------------------------ */
/* spin-orbital integrals                                                   */

static double eri_chem(const oracle_t *o, int p, int q, int r, int s)
{
    int n = o->norb;
    return o->eri[(((size_t)p * n + q) * n + r) * n + s];
}

static double h_so(const oracle_t *o, int P, int R)
{
    int n = o->norb;
    if ((P >= n) != (R >= n)) return 0.0;
    return o->h[(size_t)(P % n) * n + (R % n)];
}

/* physicists' <PQ|RS> = (pr|qs), spin-diagonal in (P,R) and in (Q,S) */
static double g_phys(const oracle_t *o, int P, int Q, int R, int S)
{
    int n = o->norb;
    if ((P >= n) != (R >= n) || (Q >= n) != (S >= n)) return 0.0;
    if (PLANTED(3)) return eri_chem(o, P % n, Q % n, R % n, S % n);
    return eri_chem(o, P % n, R % n, Q % n, S % n);
}

static double g_anti(const oracle_t *o, int P, int Q, int R, int S)
{
    if (PLANTED(1)) return g_phys(o, P, Q, R, S);
    return g_phys(o, P, Q, R, S) - g_phys(o, P, Q, S, R);
}

/* ascending list of modes set in (w0, w1) */
static int list_modes(int norb, uint64_t w0, uint64_t w1, int *out)
{
    int k = 0;
    for (int m = 0; m < norb; ++m)
        if ((w0 >> m) & 1ull) out[k++] = m;
    for (int m = 0; m < norb; ++m)
        if ((w1 >> m) & 1ull) out[k++] = m + norb;
    return k;
}

/* <Di|H|Dj> by the spin-orbital Slater-Condon rules */
static double slater_condon(const oracle_t *o, det_t di, det_t dj)
{
    int norb = o->norb;
    uint64_t xa = di.w[0] ^ dj.w[0], xb = di.w[1] ^ dj.w[1];
    int ndiff = popc(xa) + popc(xb);
    int occ[128], nocc;

    if (ndiff == 0) {
        double e = 0.0;
        nocc = list_modes(norb, di.w[0], di.w[1], occ);
        for (int i = 0; i < nocc; ++i) e += h_so(o, occ[i], occ[i]);
        double two = 0.0;
        for (int i = 0; i < nocc; ++i)
            for (int j = 0; j < nocc; ++j) two += g_anti(o, occ[i], occ[j], occ[i], occ[j]);
        return e + (PLANTED(5) ? two : 0.5 * two);
    }
    if (ndiff == 2) {
        int P, R, tmp[2];
        list_modes(norb, xa & di.w[0], xb & di.w[1], tmp);
        P = tmp[0];
        list_modes(norb, xa & dj.w[0], xb & dj.w[1], tmp);
        R = tmp[0];
        det_t t = dj;
        int s = annihilate(&t, norb, R);
        s *= create(&t, norb, P);
        double v = PLANTED(4) ? 0.0 : h_so(o, P, R);
        nocc = list_modes(norb, dj.w[0], dj.w[1], occ);
        for (int i = 0; i < nocc; ++i)
            if (occ[i] != R) v += g_anti(o, P, occ[i], R, occ[i]);
        return s * v;
    }
    if (ndiff == 4) {
        int pp[2], rr[2];
        list_modes(norb, xa & di.w[0], xb & di.w[1], pp); /* P < Q in Di only */
        list_modes(norb, xa & dj.w[0], xb & dj.w[1], rr); /* R < S in Dj only */
        int P = pp[0], Q = pp[1], R = rr[0], S = rr[1];
        det_t t = dj;
        /* <Di| a+_P a+_Q a_S a_R |Dj> : rightmost operator acts first */
        int s = annihilate(&t, norb, R);
        s *= annihilate(&t, norb, S);
        s *= create(&t, norb, Q);
        s *= create(&t, norb, P);
        if (PLANTED(2)) s = -s;
        return s * g_anti(o, P, Q, R, S);
    }
    return 0.0;
}

/* ------------------------------------------------------------------------ */
/* the selected space                                                       */

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static int64_t find_string(const uint64_t *S, int64_t n, uint64_t key)
{
    const uint64_t *hit = (const uint64_t *)bsearch(&key, S, (size_t)n, sizeof(uint64_t), cmp_u64);
    return hit ? (int64_t)(hit - S) : -1;
}

static int valid_string(uint64_t s, int norb, int n)
{
    if (norb < 64 && (s >> norb) != 0) return 0;
    return popc(s) == n;
}

/* Returns 0, or -1 (bad argument), -2 (bad string), -3 (duplicate). */
int oracle_create(int norb, int na, int nb, const double *h, const double *eri, const uint64_t *A,
                  int64_t nA, const uint64_t *B, int64_t nB, void **out)
{
    *out = NULL;
    if (norb < 1 || norb > 64 || na < 0 || nb < 0 || na > norb || nb > norb || nA < 1 || nB < 1)
        return -1;
    oracle_t *o = (oracle_t *)calloc(1, sizeof(oracle_t));
    size_t n2 = (size_t)norb * norb;
    o->norb = norb;
    o->na = na;
    o->nb = nb;
    o->h = (double *)malloc(n2 * sizeof(double));
    o->eri = (double *)malloc(n2 * n2 * sizeof(double));
    o->A = (uint64_t *)malloc((size_t)nA * sizeof(uint64_t));
    o->B = (uint64_t *)malloc((size_t)nB * sizeof(uint64_t));
    memcpy(o->h, h, n2 * sizeof(double));
    memcpy(o->eri, eri, n2 * n2 * sizeof(double));
    memcpy(o->A, A, (size_t)nA * sizeof(uint64_t));
    memcpy(o->B, B, (size_t)nB * sizeof(uint64_t));
    o->nA = nA;
    o->nB = nB;
    qsort(o->A, (size_t)nA, sizeof(uint64_t), cmp_u64);
    qsort(o->B, (size_t)nB, sizeof(uint64_t), cmp_u64);
    int rc = 0;
    for (int64_t i = 0; i < nA && !rc; ++i)
        if (!valid_string(o->A[i], norb, na)) rc = -2;
    for (int64_t i = 0; i < nB && !rc; ++i)
        if (!valid_string(o->B[i], norb, nb)) rc = -2;
    for (int64_t i = 1; i < nA && !rc; ++i)
        if (o->A[i] == o->A[i - 1]) rc = -3;
    for (int64_t i = 1; i < nB && !rc; ++i)
        if (o->B[i] == o->B[i - 1]) rc = -3;
    *out = o;
    return rc;
}

void oracle_destroy(void *p)
{
    oracle_t *o = (oracle_t *)p;
    if (!o) return;
    free(o->h);
    free(o->eri);
    free(o->A);
    free(o->B);
    free(o);
}

int64_t oracle_ndets(void *p) { return ((oracle_t *)p)->nA * ((oracle_t *)p)->nB; }

void oracle_sorted(void *p, int spin, uint64_t *out)
{
    oracle_t *o = (oracle_t *)p;
    if (spin == 0) memcpy(out, o->A, (size_t)o->nA * sizeof(uint64_t));
    else memcpy(out, o->B, (size_t)o->nB * sizeof(uint64_t));
}

static det_t det_of(const oracle_t *o, int64_t idx)
{
    det_t d;
    d.w[0] = o->A[idx / o->nB];
    d.w[1] = o->B[idx % o->nB];
    return d;
}

double oracle_hij(void *p, int64_t i, int64_t j)
{
    oracle_t *o = (oracle_t *)p;
    return slater_condon(o, det_of(o, i), det_of(o, j));
}

void oracle_diag(void *p, double *out)
{
    oracle_t *o = (oracle_t *)p;
    int64_t N = o->nA * o->nB;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) out[i] = slater_condon(o, det_of(o, i), det_of(o, i));
}

/* every H_ij over all pairs: the plainest definition, for N up to a few thousand */
void oracle_dense(void *p, double *out)
{
    oracle_t *o = (oracle_t *)p;
    int64_t N = o->nA * o->nB;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) out[i * N + j] = slater_condon(o, det_of(o, i), det_of(o, j));
}

/* Strings of one spin reachable from s by moving `level` (0, 1 or 2)
 * electrons and present in the set S.  Appends indices to idx[]. */
static int64_t reachable(const uint64_t *S, int64_t n, int norb, uint64_t s, int level, int64_t *idx)
{
    int occ[64], vir[64], no = 0, nv = 0;
    int64_t k = 0;
    for (int m = 0; m < norb; ++m) {
        if ((s >> m) & 1ull) occ[no++] = m;
        else vir[nv++] = m;
    }
    if (level == 0) {
        int64_t j = find_string(S, n, s);
        if (j >= 0) idx[k++] = j;
    } else if (level == 1) {
        for (int a = 0; a < no; ++a)
            for (int b = 0; b < nv; ++b) {
                int64_t j = find_string(S, n, s ^ (1ull << occ[a]) ^ (1ull << vir[b]));
                if (j >= 0) idx[k++] = j;
            }
    } else {
        for (int a1 = 0; a1 < no; ++a1)
            for (int a2 = a1 + 1; a2 < no; ++a2)
                for (int b1 = 0; b1 < nv; ++b1)
                    for (int b2 = b1 + 1; b2 < nv; ++b2) {
                        uint64_t t = s ^ (1ull << occ[a1]) ^ (1ull << occ[a2]) ^ (1ull << vir[b1]) ^
                                     (1ull << vir[b2]);
                        int64_t j = find_string(S, n, t);
                        if (j >= 0) idx[k++] = j;
                    }
    }
    return k;
}

static int64_t max_reachable(int norb, int n)
{
    int64_t v = norb - n;
    return 1 + (int64_t)n * v + (int64_t)n * (n - 1) / 2 * v * (v - 1) / 2;
}

/* sigma for a list of rows: out[v*nrows + r] = sum_j H_{rows[r], j} x[v*N + j] */
void oracle_sigma_rows(void *p, const double *x, int nvec, const int64_t *rows, int64_t nrows,
                       double *out)
{
    oracle_t *o = (oracle_t *)p;
    int64_t N = o->nA * o->nB;
    int64_t capA = max_reachable(o->norb, o->na), capB = max_reachable(o->norb, o->nb);
#pragma omp parallel
    {
        int64_t *la[3], *lb[3];
        int64_t na_[3], nb_[3];
        for (int l = 0; l < 3; ++l) {
            la[l] = (int64_t *)malloc((size_t)capA * sizeof(int64_t));
            lb[l] = (int64_t *)malloc((size_t)capB * sizeof(int64_t));
        }
        double *acc = (double *)malloc((size_t)nvec * sizeof(double));
#pragma omp for schedule(dynamic, 4)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t i = rows[r];
            det_t di = det_of(o, i);
            for (int l = 0; l < 3; ++l) {
                na_[l] = reachable(o->A, o->nA, o->norb, di.w[0], l, la[l]);
                nb_[l] = reachable(o->B, o->nB, o->norb, di.w[1], l, lb[l]);
            }
            for (int v = 0; v < nvec; ++v) acc[v] = 0.0;
            /* every (alpha level, beta level) with at most two differences in total */
            for (int lA = 0; lA <= 2; ++lA)
                for (int lB = 0; lA + lB <= 2; ++lB)
                    for (int64_t a = 0; a < na_[lA]; ++a)
                        for (int64_t b = 0; b < nb_[lB]; ++b) {
                            int64_t j = la[lA][a] * o->nB + lb[lB][b];
                            double hij = slater_condon(o, di, det_of(o, j));
                            for (int v = 0; v < nvec; ++v) acc[v] += hij * x[(size_t)v * N + j];
                        }
            for (int v = 0; v < nvec; ++v) out[(size_t)v * nrows + r] = acc[v];
        }
        for (int l = 0; l < 3; ++l) {
            free(la[l]);
            free(lb[l]);
        }
        free(acc);
    }
}

/* The explicit Hamiltonian in CSR form (Sec. II-A, "explicit assembly"):
 * row i lists every determinant j of the space within two spin-orbital
 * differences (including i itself) with H_ij, in the enumeration order of
 * oracle_sigma_rows.  oracle_csr_counts fills counts[i]; oracle_csr_fill
 * writes cols/vals at ptr[i] (ptr = exclusive prefix of the counts). */
static void row_neighbours(const oracle_t *o, int64_t i, int64_t **la, int64_t **lb, int64_t *na_, int64_t *nb_)
{
    det_t di = det_of(o, i);
    for (int l = 0; l < 3; ++l) {
        na_[l] = reachable(o->A, o->nA, o->norb, di.w[0], l, la[l]);
        nb_[l] = reachable(o->B, o->nB, o->norb, di.w[1], l, lb[l]);
    }
}

void oracle_csr_counts(void *p, int64_t *counts)
{
    oracle_t *o = (oracle_t *)p;
    int64_t N = o->nA * o->nB;
    int64_t capA = max_reachable(o->norb, o->na), capB = max_reachable(o->norb, o->nb);
#pragma omp parallel
    {
        int64_t *la[3], *lb[3], na_[3], nb_[3];
        for (int l = 0; l < 3; ++l) {
            la[l] = (int64_t *)malloc((size_t)capA * sizeof(int64_t));
            lb[l] = (int64_t *)malloc((size_t)capB * sizeof(int64_t));
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < N; ++i) {
            row_neighbours(o, i, la, lb, na_, nb_);
            int64_t c = 0;
            for (int lA = 0; lA <= 2; ++lA)
                for (int lB = 0; lA + lB <= 2; ++lB) c += na_[lA] * nb_[lB];
            counts[i] = c;
        }
        for (int l = 0; l < 3; ++l) {
            free(la[l]);
            free(lb[l]);
        }
    }
}

void oracle_csr_fill(void *p, const int64_t *ptr, int64_t *cols, double *vals)
{
    oracle_t *o = (oracle_t *)p;
    int64_t N = o->nA * o->nB;
    int64_t capA = max_reachable(o->norb, o->na), capB = max_reachable(o->norb, o->nb);
#pragma omp parallel
    {
        int64_t *la[3], *lb[3], na_[3], nb_[3];
        for (int l = 0; l < 3; ++l) {
            la[l] = (int64_t *)malloc((size_t)capA * sizeof(int64_t));
            lb[l] = (int64_t *)malloc((size_t)capB * sizeof(int64_t));
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < N; ++i) {
            row_neighbours(o, i, la, lb, na_, nb_);
            det_t di = det_of(o, i);
            int64_t e = ptr[i];
            for (int lA = 0; lA <= 2; ++lA)
                for (int lB = 0; lA + lB <= 2; ++lB)
                    for (int64_t a = 0; a < na_[lA]; ++a)
                        for (int64_t b = 0; b < nb_[lB]; ++b) {
                            int64_t j = la[lA][a] * o->nB + lb[lB][b];
                            cols[e] = j;
                            vals[e] = slater_condon(o, di, det_of(o, j));
                            ++e;
                        }
        }
        for (int l = 0; l < 3; ++l) {
            free(la[l]);
            free(lb[l]);
        }
    }
}

void oracle_sigma(void *p, const double *x, int nvec, double *out)
{
    oracle_t *o = (oracle_t *)p;
    int64_t N = o->nA * o->nB;
    int64_t *rows = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    for (int64_t i = 0; i < N; ++i) rows[i] = i;
    oracle_sigma_rows(p, x, nvec, rows, N, out);
    free(rows);
}

/* ------------------------------------------------------------------------ */
/* single-spin excitation tables (the lists of Sec. III-B, Listing 3)      */
/* kind 1: singles, kind 2: doubles.  Canonical order: source i ascending,  */
/* target j ascending; no self entry.  orbs[4e..4e+3] = p1, p2, q1, q2 with */
/* p's occupied in S[i] only and q's occupied in S[j] only (ascending; for  */
/* singles p2 = q2 = 255).  sign = <S_i| a+_p1 a+_p2 a_q2 a_q1 |S_j>  (or   */
/* <S_i| a+_p a_q |S_j> for singles), from sequential operator application. */

int64_t oracle_table_count(const uint64_t *S, int64_t n, int kind)
{
    int64_t total = 0;
#pragma omp parallel for reduction(+ : total) schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            if (popc(S[i] ^ S[j]) == 2 * kind) ++total;
    return total;
}

void oracle_table_fill(const uint64_t *S, int64_t n, int norb, int kind, int64_t *ptr, int32_t *tgt,
                       uint8_t *orbs, int8_t *sign)
{
    ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j)
            if (popc(S[i] ^ S[j]) == 2 * kind) ++c;
        ptr[i + 1] = ptr[i] + c;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        int64_t e = ptr[i];
        for (int64_t j = 0; j < n; ++j) {
            uint64_t x = S[i] ^ S[j];
            if (popc(x) != 2 * kind) continue;
            int pm[2] = {255, 255}, qm[2] = {255, 255}, k;
            k = 0;
            for (int m = 0; m < norb; ++m)
                if ((x & S[i]) >> m & 1ull) pm[k++] = m;
            k = 0;
            for (int m = 0; m < norb; ++m)
                if ((x & S[j]) >> m & 1ull) qm[k++] = m;
            det_t t = {{S[j], 0}};
            int s;
            if (kind == 1) {
                s = annihilate(&t, norb, qm[0]);
                s *= create(&t, norb, pm[0]);
            } else {
                s = annihilate(&t, norb, qm[0]);
                s *= annihilate(&t, norb, qm[1]);
                s *= create(&t, norb, pm[1]);
                s *= create(&t, norb, pm[0]);
            }
            tgt[e] = (int32_t)j;
            orbs[4 * e + 0] = (uint8_t)pm[0];
            orbs[4 * e + 1] = (uint8_t)pm[1];
            orbs[4 * e + 2] = (uint8_t)qm[0];
            orbs[4 * e + 3] = (uint8_t)qm[1];
            sign[e] = (int8_t)s;
            ++e;
        }
    }
}

/* same-spin string Hamiltonian <S_i|H|S_j> for one spin alone (other spin empty) */
double oracle_string_element(int norb, const double *h, const double *eri, uint64_t si, uint64_t sj)
{
    oracle_t o;
    memset(&o, 0, sizeof(o));
    o.norb = norb;
    o.h = (double *)h;
    o.eri = (double *)eri;
    det_t di = {{si, 0}}, dj = {{sj, 0}};
    return slater_condon(&o, di, dj);
}

/* ------------------------------------------------------------------------ */
/* dense symmetric eigensolver: cyclic Jacobi rotations                     */
/* a: k*k symmetric (destroyed); evals ascending; evecs column j = vector j */

int oracle_jacobi(int k, double *a, double *evals, double *evecs)
{
    double *v = (double *)calloc((size_t)k * k, sizeof(double));
    for (int i = 0; i < k; ++i) v[i * k + i] = 1.0;
    double fro = 0.0;
    for (int i = 0; i < k * k; ++i) fro += a[i] * a[i];
    fro = sqrt(fro);
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) off += a[p * k + q] * a[p * k + q];
        if (sqrt(off) <= 1e-17 * (fro > 0 ? fro : 1.0)) break;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                double apq = a[p * k + q];
                if (apq == 0.0) continue;
                double theta = (a[q * k + q] - a[p * k + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < k; ++r) { /* columns p, q */
                    double arp = a[r * k + p], arq = a[r * k + q];
                    a[r * k + p] = c * arp - s * arq;
                    a[r * k + q] = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) { /* rows p, q */
                    double apr = a[p * k + r], aqr = a[q * k + r];
                    a[p * k + r] = c * apr - s * aqr;
                    a[q * k + r] = s * apr + c * aqr;
                }
                for (int r = 0; r < k; ++r) {
                    double vrp = v[r * k + p], vrq = v[r * k + q];
                    v[r * k + p] = c * vrp - s * vrq;
                    v[r * k + q] = s * vrp + c * vrq;
                }
            }
    }
    /* sort ascending (selection sort keeps it plain) */
    int *ord = (int *)malloc((size_t)k * sizeof(int));
    for (int i = 0; i < k; ++i) ord[i] = i;
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j)
            if (a[ord[j] * k + ord[j]] < a[ord[i] * k + ord[i]]) {
                int t = ord[i];
                ord[i] = ord[j];
                ord[j] = t;
            }
    for (int j = 0; j < k; ++j) {
        evals[j] = a[ord[j] * k + ord[j]];
        for (int r = 0; r < k; ++r) evecs[r * k + j] = v[r * k + ord[j]];
    }
    free(ord);
    free(v);
    return sweep;
}

/* ------------------------------------------------------------------------ */
/* Davidson (Sec. II-C), block form for several roots                       */

static double dotN(const double *x, const double *y, int64_t N)
{
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s += x[i] * y[i];
    return s;
}

/* Returns the iteration count, or -1 if not converged within max_iter. */
int oracle_davidson(void *p, int nroots, double tol, int max_iter, int max_sub, double delta,
                    double *energies, double *vecs, double *resnorms)
{
    oracle_t *o = (oracle_t *)p;
    int64_t N = o->nA * o->nB;
    if (max_sub < 2 * nroots) max_sub = 2 * nroots;
    if (max_sub > N) max_sub = (int)N;
    double *Hd = (double *)malloc((size_t)N * sizeof(double));
    double *V = (double *)calloc((size_t)max_sub * N, sizeof(double));
    double *W = (double *)calloc((size_t)max_sub * N, sizeof(double));
    double *U = (double *)malloc((size_t)nroots * N * sizeof(double));
    double *HU = (double *)malloc((size_t)nroots * N * sizeof(double));
    double *T = (double *)malloc((size_t)max_sub * max_sub * sizeof(double));
    double *Tw = (double *)malloc((size_t)max_sub * max_sub * sizeof(double));
    double *ev = (double *)malloc((size_t)max_sub * sizeof(double));
    double *Y = (double *)malloc((size_t)max_sub * max_sub * sizeof(double));
    double *t = (double *)malloc((size_t)N * sizeof(double));
    oracle_diag(p, Hd);

    /* 1. initial vectors: unit vectors on the lowest diagonal entries */
    int k = 0;
    {
        char *used = (char *)calloc((size_t)N, 1);
        for (int r = 0; r < nroots && r < N; ++r) {
            int64_t best = -1;
            for (int64_t i = 0; i < N; ++i)
                if (!used[i] && (best < 0 || Hd[i] < Hd[best])) best = i;
            used[best] = 1;
            V[(size_t)k * N + best] = 1.0;
            ++k;
        }
        free(used);
    }
    oracle_sigma(p, V, k, W);
    int iter, converged = 0;
    for (iter = 1; iter <= max_iter; ++iter) {
        /* 2b. projected matrix T = V^T W (symmetrised) */
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b) T[a * k + b] = dotN(V + (size_t)a * N, W + (size_t)b * N, N);
        for (int a = 0; a < k; ++a)
            for (int b = a + 1; b < k; ++b) {
                double s = 0.5 * (T[a * k + b] + T[b * k + a]);
                T[a * k + b] = T[b * k + a] = s;
            }
        /* 2c. smallest Ritz pairs */
        memcpy(Tw, T, (size_t)k * k * sizeof(double));
        oracle_jacobi(k, Tw, ev, Y);
        /* 2d. Ritz vectors and residuals */
        int nconv = 0;
        for (int r = 0; r < nroots; ++r) {
            double *u = U + (size_t)r * N, *hu = HU + (size_t)r * N;
            memset(u, 0, (size_t)N * sizeof(double));
            memset(hu, 0, (size_t)N * sizeof(double));
            for (int a = 0; a < k; ++a) {
                double y = Y[a * k + r];
                const double *va = V + (size_t)a * N, *wa = W + (size_t)a * N;
                for (int64_t i = 0; i < N; ++i) {
                    u[i] += y * va[i];
                    hu[i] += y * wa[i];
                }
            }
            double rn = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double ri = hu[i] - ev[r] * u[i];
                rn += ri * ri;
            }
            resnorms[r] = sqrt(rn);
            energies[r] = ev[r];
            /* 2e. convergence test */
            if (resnorms[r] <= tol) ++nconv;
        }
        if (nconv == nroots) {
            converged = 1;
            break;
        }
        /* 2h. thick restart when the subspace would overflow: keep the lowest
         * nkeep Ritz vectors V Y[:, :nkeep] and their images W Y[:, :nkeep] */
        int nnew = nroots - nconv;
        if (k + nnew > max_sub) {
            int nkeep = max_sub / 3;
            if (nkeep < 2 * nroots) nkeep = 2 * nroots;
            if (nkeep > max_sub - nroots) nkeep = max_sub - nroots;
            if (nkeep < nroots) nkeep = nroots;
            if (nkeep > k) nkeep = k;
            double *V2 = (double *)calloc((size_t)nkeep * N, sizeof(double));
            double *W2 = (double *)calloc((size_t)nkeep * N, sizeof(double));
            for (int c = 0; c < nkeep; ++c)
                for (int a = 0; a < k; ++a) {
                    double y = Y[a * k + c];
                    for (int64_t i = 0; i < N; ++i) {
                        V2[(size_t)c * N + i] += y * V[(size_t)a * N + i];
                        W2[(size_t)c * N + i] += y * W[(size_t)a * N + i];
                    }
                }
            memcpy(V, V2, (size_t)nkeep * N * sizeof(double));
            memcpy(W, W2, (size_t)nkeep * N * sizeof(double));
            free(V2);
            free(W2);
            k = nkeep;
        }
        /* 2f-2g. precondition each unconverged residual, orthogonalise, append */
        int added = 0;
        for (int r = 0; r < nroots; ++r) {
            if (resnorms[r] <= tol) continue;
            const double *u = U + (size_t)r * N, *hu = HU + (size_t)r * N;
            for (int64_t i = 0; i < N; ++i) {
                double d = Hd[i] - ev[r];
                double den = (d >= 0 ? 1.0 : -1.0) * (fabs(d) > delta ? fabs(d) : delta);
                t[i] = (hu[i] - ev[r] * u[i]) / den;
            }
            double n0 = sqrt(dotN(t, t, N));
            for (int pass = 0; pass < 2; ++pass) /* Gram-Schmidt, then once more */
                for (int a = 0; a < k; ++a) {
                    double c = dotN(V + (size_t)a * N, t, N);
                    for (int64_t i = 0; i < N; ++i) t[i] -= c * V[(size_t)a * N + i];
                }
            double n1 = sqrt(dotN(t, t, N));
            if (!(n1 > 1e-10 * n0) || k >= max_sub) continue;
            for (int64_t i = 0; i < N; ++i) V[(size_t)k * N + i] = t[i] / n1;
            ++k;
            ++added;
        }
        if (added == 0) break;
        oracle_sigma(p, V + (size_t)(k - added) * N, added, W + (size_t)(k - added) * N);
    }
    if (vecs) memcpy(vecs, U, (size_t)nroots * N * sizeof(double));
    free(Hd);
    free(V);
    free(W);
    free(U);
    free(HU);
    free(T);
    free(Tw);
    free(ev);
    free(Y);
    free(t);
    return converged ? iter : -1;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
