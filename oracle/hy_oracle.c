/*
 * hy_oracle.c -- plain, slow, FP64 CPU oracle for the state-vector ADAPT-VQE
 * hot path.  TEST INFRASTRUCTURE ONLY: nothing in the product library may
 * link, load or call this file.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * What it follows (paper: "Sparse State-Vector Emulation" section):
 *   - the real molecular Hamiltonian (variational framework, Eq. "ev"),
 *     written in second quantisation over 2n spin orbitals in blocked order
 *     (spin orbital p = orbital p alpha for p < n, n + p = orbital p beta);
 *   - the state restricted to the particle- and S_z-conserving determinant
 *     space Omega_CIk (Table 1 gives its sizes);
 *   - determinants enumerated as all n-bit alpha (beta) strings with the
 *     right popcount in increasing numeric order, index I = i_a * N_b + i_b;
 *   - sigma = H psi by the Slater-Condon rules, each element computed from
 *     the spin-orbital integrals, one output determinant at a time;
 *   - operator strings (creation / annihilation) applied to occupation
 *     vectors straight from their definition, with the sign
 *     (-1)^(number of occupied modes below the acted-on mode);
 *   - exp(theta * (C - C^dagger)) applied as the exact rotation on each
 *     connected pair (the closed form of a nilpotent-squared generator);
 *   - pool gradients g = 2 <H psi | A psi> with A psi built term by term.
 * Parity pins for all of it live in tests/test_oracle_pins.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n, na, nb;
    int64_t Na, Nb, N;
    uint32_t *astr, *bstr;     /* strings in index order                   */
    int64_t *alook, *blook;    /* 2^n lookup: string -> position, else -1 */
    double *h1;                /* n*n                                       */
    double *h2;                /* n^4, (pq|rs) at ((p*n+q)*n+r)*n+s         */
    double e_core;
} orc_sys;

static int popc64(uint64_t x) { return __builtin_popcountll(x); }

/* ------------------------------------------------------------------ */
/* determinant space                                                    */
/* ------------------------------------------------------------------ */

int64_t orc_binom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

/* All n-bit masks with popcount k, increasing numeric order. */
static int64_t enumerate(int n, int k, uint32_t **out, int64_t **look)
{
    int64_t cnt = 0;
    int64_t *lk = (int64_t *)malloc(sizeof(int64_t) << n);
    for (uint64_t m = 0; m < (1ull << n); ++m) lk[m] = -1;
    for (uint64_t m = 0; m < (1ull << n); ++m)
        if (popc64(m) == k) lk[m] = cnt++;
    uint32_t *s = (uint32_t *)malloc(sizeof(uint32_t) * (cnt ? cnt : 1));
    for (uint64_t m = 0; m < (1ull << n); ++m)
        if (lk[m] >= 0) s[lk[m]] = (uint32_t)m;
    *out = s;
    *look = lk;
    return cnt;
}

orc_sys *orc_create(int n, int na, int nb, const double *h1, const double *h2,
                    double e_core)
{
    if (n < 1 || n > 20 || na < 0 || nb < 0 || na > n || nb > n) return NULL;
    orc_sys *s = (orc_sys *)calloc(1, sizeof(orc_sys));
    s->n = n; s->na = na; s->nb = nb;
    s->Na = enumerate(n, na, &s->astr, &s->alook);
    s->Nb = enumerate(n, nb, &s->bstr, &s->blook);
    s->N = s->Na * s->Nb;
    s->h1 = (double *)malloc(sizeof(double) * n * n);
    memcpy(s->h1, h1, sizeof(double) * n * n);
    size_t n4 = (size_t)n * n * n * n;
    s->h2 = (double *)malloc(sizeof(double) * n4);
    memcpy(s->h2, h2, sizeof(double) * n4);
    s->e_core = e_core;
    return s;
}

void orc_destroy(orc_sys *s)
{
    if (!s) return;
    free(s->astr); free(s->bstr); free(s->alook); free(s->blook);
    free(s->h1); free(s->h2); free(s);
}

int64_t orc_ndet(const orc_sys *s) { return s->N; }
int64_t orc_nalpha_str(const orc_sys *s) { return s->Na; }
int64_t orc_nbeta_str(const orc_sys *s) { return s->Nb; }

/* determinant (2n-bit occupation, alpha block low) of index I */
uint64_t orc_det(const orc_sys *s, int64_t I)
{
    uint64_t a = s->astr[I / s->Nb], b = s->bstr[I % s->Nb];
    return a | (b << s->n);
}

void orc_dets(const orc_sys *s, uint64_t *out)
{
    for (int64_t I = 0; I < s->N; ++I) out[I] = orc_det(s, I);
}

int64_t orc_index(const orc_sys *s, uint64_t det)
{
    uint64_t mask = (1ull << s->n) - 1;
    if (det >> (2 * s->n)) return -1;
    int64_t ia = s->alook[det & mask], ib = s->blook[(det >> s->n) & mask];
    if (ia < 0 || ib < 0) return -1;
    return ia * s->Nb + ib;
}

/* ------------------------------------------------------------------ */
/* second quantisation by definition                                    */
/* ------------------------------------------------------------------ */

/* Apply a product of fermion operators, rightmost first.  ops[t] =
 * 2*mode + dagger.  Returns 1 and sets *out / *sign when the result is
 * nonzero, 0 otherwise. */
int orc_apply_ops(const int *ops, int nops, uint64_t det, uint64_t *out,
                  int *sign)
{
    int sg = 1;
    for (int t = nops - 1; t >= 0; --t) {
        int mode = ops[t] >> 1, dag = ops[t] & 1;
        uint64_t bit = 1ull << mode;
        int occ = (det & bit) != 0;
        if (dag == occ) return 0;          /* create on full / destroy empty */
        if (popc64(det & (bit - 1)) & 1) sg = -sg;
        det ^= bit;
    }
    *out = det;
    *sign = sg;
    return 1;
}

/* spin-orbital integrals in chemists' notation */
static double h1so(const orc_sys *s, int P, int Q)
{
    int n = s->n;
    if ((P < n) != (Q < n)) return 0.0;
    return s->h1[(P % n) * n + (Q % n)];
}

static double h2so(const orc_sys *s, int P, int Q, int R, int S)
{
    int n = s->n;
    if ((P < n) != (Q < n) || (R < n) != (S < n)) return 0.0;
    int p = P % n, q = Q % n, r = R % n, t = S % n;
    return s->h2[(((size_t)p * n + q) * n + r) * n + t];
}

/* H psi applied term by term from
 *   H = E_core + sum_PQ h_PQ a+_P a_Q + 1/2 sum_PQRS [PQ|RS] a+_P a+_R a_S a_Q
 * over all spin orbitals.  Cost (2n)^4 * N: tiny systems only. */
void orc_apply_h_definition(const orc_sys *s, const double *psi, double *sigma)
{
    int M = 2 * s->n;
    for (int64_t I = 0; I < s->N; ++I) sigma[I] = s->e_core * psi[I];
    for (int64_t J = 0; J < s->N; ++J) {
        double x = psi[J];
        if (x == 0.0) continue;
        uint64_t d = orc_det(s, J), o;
        int sg;
        for (int P = 0; P < M; ++P)
            for (int Q = 0; Q < M; ++Q) {
                double c = h1so(s, P, Q);
                if (c == 0.0) continue;
                int ops[2] = {2 * P + 1, 2 * Q};
                if (orc_apply_ops(ops, 2, d, &o, &sg)) {
                    int64_t K = orc_index(s, o);
                    if (K >= 0) sigma[K] += c * sg * x;
                }
            }
        for (int P = 0; P < M; ++P)
            for (int Q = 0; Q < M; ++Q)
                for (int R = 0; R < M; ++R)
                    for (int S = 0; S < M; ++S) {
                        double c = h2so(s, P, Q, R, S);
                        if (c == 0.0) continue;
                        int ops[4] = {2 * P + 1, 2 * R + 1, 2 * S, 2 * Q};
                        if (orc_apply_ops(ops, 4, d, &o, &sg)) {
                            int64_t K = orc_index(s, o);
                            if (K >= 0) sigma[K] += 0.5 * c * sg * x;
                        }
                    }
    }
}

/* ------------------------------------------------------------------ */
/* Slater-Condon rules                                                  */
/* ------------------------------------------------------------------ */

static int lowest_bit(uint64_t x) { return __builtin_ctzll(x); }

/* <bra|H|ket> for two determinants of the same particle numbers. */
double orc_matrix_element(const orc_sys *s, uint64_t bra, uint64_t ket)
{
    uint64_t diff = bra ^ ket;
    int lvl = popc64(diff);
    int M = 2 * s->n;
    if (lvl == 0) {
        double e = s->e_core;
        for (int P = 0; P < M; ++P) {
            if (!((bra >> P) & 1)) continue;
            e += h1so(s, P, P);
            for (int R = 0; R < M; ++R) {
                if (!((bra >> R) & 1)) continue;
                e += 0.5 * (h2so(s, P, P, R, R) - h2so(s, P, R, R, P));
            }
        }
        return e;
    }
    if (lvl == 2) {
        int P = lowest_bit(bra & diff);    /* occupied in bra only */
        int Q = lowest_bit(ket & diff);    /* occupied in ket only */
        int ops[2] = {2 * P + 1, 2 * Q};
        uint64_t o;
        int sg;
        if (!orc_apply_ops(ops, 2, ket, &o, &sg) || o != bra) return 0.0;
        double v = h1so(s, P, Q);
        uint64_t common = bra & ket;
        for (int R = 0; R < M; ++R) {
            if (!((common >> R) & 1)) continue;
            v += h2so(s, P, Q, R, R) - h2so(s, P, R, R, Q);
        }
        return sg * v;
    }
    if (lvl == 4) {
        uint64_t up = bra & diff, dn = ket & diff;
        if (popc64(up) != 2) return 0.0;
        int P = lowest_bit(up), R = lowest_bit(up & (up - 1));
        int Q = lowest_bit(dn), S = lowest_bit(dn & (dn - 1));
        int ops[4] = {2 * P + 1, 2 * R + 1, 2 * S, 2 * Q};
        uint64_t o;
        int sg;
        if (!orc_apply_ops(ops, 4, ket, &o, &sg) || o != bra) return 0.0;
        return sg * (h2so(s, P, Q, R, S) - h2so(s, P, S, R, Q));
    }
    return 0.0;
}

/* sigma(I) for one output determinant: sum over itself, its singles and
 * doubles inside Omega_CIk. */
static double sigma_one(const orc_sys *s, const double *psi, int64_t I)
{
    uint64_t d = orc_det(s, I);
    int M = 2 * s->n;
    double acc = orc_matrix_element(s, d, d) * psi[I];
    int occ[64], vir[64], no = 0, nv = 0;
    for (int P = 0; P < M; ++P) {
        if ((d >> P) & 1) occ[no++] = P; else vir[nv++] = P;
    }
    int n = s->n;
    /* singles: same spin */
    for (int i = 0; i < no; ++i)
        for (int a = 0; a < nv; ++a) {
            if ((occ[i] < n) != (vir[a] < n)) continue;
            uint64_t k = d ^ (1ull << occ[i]) ^ (1ull << vir[a]);
            int64_t K = orc_index(s, k);
            if (K < 0) continue;
            double x = psi[K];
            if (x != 0.0) acc += orc_matrix_element(s, d, k) * x;
        }
    /* doubles: spin multiset preserved */
    for (int i = 0; i < no; ++i)
        for (int j = i + 1; j < no; ++j)
            for (int a = 0; a < nv; ++a)
                for (int b = a + 1; b < nv; ++b) {
                    int so = (occ[i] < n) + (occ[j] < n);
                    int sv = (vir[a] < n) + (vir[b] < n);
                    if (so != sv) continue;
                    uint64_t k = d ^ (1ull << occ[i]) ^ (1ull << occ[j]) ^
                                 (1ull << vir[a]) ^ (1ull << vir[b]);
                    int64_t K = orc_index(s, k);
                    if (K < 0) continue;
                    double x = psi[K];
                    if (x != 0.0) acc += orc_matrix_element(s, d, k) * x;
                }
    return acc;
}

int orc_threads_used(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) return nthreads;
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

void orc_sigma(const orc_sys *s, const double *psi, double *sigma, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t I = 0; I < s->N; ++I) sigma[I] = sigma_one(s, psi, I);
    (void)nthreads;
}

void orc_sigma_rows(const orc_sys *s, const double *psi, const int64_t *rows,
                    int64_t m, double *out, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t t = 0; t < m; ++t) out[t] = sigma_one(s, psi, rows[t]);
    (void)nthreads;
}

/* dense H over Omega_CIk (small systems) */
void orc_dense_h(const orc_sys *s, double *H)
{
    for (int64_t I = 0; I < s->N; ++I) {
        uint64_t d = orc_det(s, I);
        for (int64_t J = 0; J < s->N; ++J)
            H[I * s->N + J] = orc_matrix_element(s, d, orc_det(s, J));
    }
}

/* ------------------------------------------------------------------ */
/* operator pool (spin-adapted singles and doubles relative to HF)      */
/* ------------------------------------------------------------------ */
/* Op descriptor: 11 int32 = [nc, (rank, c0, c1, a1, a0) x 2]; a rank-1
 * constituent is a+_{c0} a_{a0}; rank 2 is a+_{c0} a+_{c1} a_{a1} a_{a0}.
 * Modes are spin orbitals in blocked order.  A = sum_c (C_c - C_c^dagger). */

static int hf_occ(const orc_sys *s, int mode)
{
    int n = s->n;
    return mode < n ? (mode < s->na) : ((mode - n) < s->nb);
}

static int valid1(const orc_sys *s, int c0, int a0)
{
    return hf_occ(s, a0) && !hf_occ(s, c0);
}

static int valid2(const orc_sys *s, int c0, int c1, int a1, int a0)
{
    return hf_occ(s, a0) && hf_occ(s, a1) && !hf_occ(s, c0) && !hf_occ(s, c1);
}

static int64_t push_op(int32_t *desc, int64_t k, int64_t cap, int nc,
                       const int32_t *cons)
{
    if (nc == 0) return k;
    if (desc && k < cap) {
        int32_t *d = desc + 11 * k;
        memset(d, 0, sizeof(int32_t) * 11);
        d[0] = nc;
        memcpy(d + 1, cons, sizeof(int32_t) * 5 * nc);
    }
    return k + 1;
}

int64_t orc_pool_build(const orc_sys *s, int32_t *desc, int64_t cap)
{
    int n = s->n;
    int64_t k = 0;
    int32_t c[10];
    /* singles i -> a, i < a */
    for (int i = 0; i < n; ++i)
        for (int a = i + 1; a < n; ++a) {
            int nc = 0;
            for (int sp = 0; sp < 2; ++sp) {
                int ci = a + sp * n, ai = i + sp * n;
                if (valid1(s, ci, ai)) {
                    int32_t t[5] = {1, ci, 0, 0, ai};
                    memcpy(c + 5 * nc++, t, sizeof t);
                }
            }
            k = push_op(desc, k, cap, nc, c);
        }
    /* same-spin doubles i<j -> a<b */
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            for (int a = 0; a < n; ++a)
                for (int b = a + 1; b < n; ++b) {
                    int nc = 0;
                    for (int sp = 0; sp < 2; ++sp) {
                        int o = sp * n;
                        if (valid2(s, a + o, b + o, j + o, i + o)) {
                            int32_t t[5] = {2, a + o, b + o, j + o, i + o};
                            memcpy(c + 5 * nc++, t, sizeof t);
                        }
                    }
                    k = push_op(desc, k, cap, nc, c);
                }
    /* opposite-spin doubles i<=j, a<=b */
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j)
            for (int a = 0; a < n; ++a)
                for (int b = a; b < n; ++b) {
                    /* coupling 0: C1 = a+_{a,al} a+_{b,be} a_{j,be} a_{i,al}
                     *             C2 = a+_{a,be} a+_{b,al} a_{j,al} a_{i,be} */
                    int32_t C1[5] = {2, a, b + n, j + n, i};
                    int32_t C2[5] = {2, a + n, b, j, i + n};
                    int v1 = valid2(s, C1[1], C1[2], C1[3], C1[4]);
                    int v2 = valid2(s, C2[1], C2[2], C2[3], C2[4]);
                    if (i < j && a < b) {
                        int nc = 0;
                        if (v1) memcpy(c + 5 * nc++, C1, sizeof C1);
                        if (v2) memcpy(c + 5 * nc++, C2, sizeof C2);
                        k = push_op(desc, k, cap, nc, c);
                        /* coupling 1: i <-> j */
                        int32_t D1[5] = {2, a, b + n, i + n, j};
                        int32_t D2[5] = {2, a + n, b, i, j + n};
                        nc = 0;
                        if (valid2(s, D1[1], D1[2], D1[3], D1[4]))
                            memcpy(c + 5 * nc++, D1, sizeof D1);
                        if (valid2(s, D2[1], D2[2], D2[3], D2[4]))
                            memcpy(c + 5 * nc++, D2, sizeof D2);
                        k = push_op(desc, k, cap, nc, c);
                    } else if (i == j && a == b) {
                        k = push_op(desc, k, cap, v1, C1);
                    } else {
                        k = push_op(desc, k, cap, v1, C1);
                        k = push_op(desc, k, cap, v2, C2);
                    }
                }
    return k;
}

static int cons_ops(const int32_t *t, int *ops)
{
    if (t[0] == 1) {
        ops[0] = 2 * t[1] + 1; ops[1] = 2 * t[4];
        return 2;
    }
    ops[0] = 2 * t[1] + 1; ops[1] = 2 * t[2] + 1;
    ops[2] = 2 * t[3];     ops[3] = 2 * t[4];
    return 4;
}

/* psi <- exp(theta A) psi for one pool op. */
void orc_apply_excitation(const orc_sys *s, const int32_t *op, double theta,
                          double *psi)
{
    double c = cos(theta), sn = sin(theta);
    for (int q = 0; q < op[0]; ++q) {
        int ops[4];
        int no = cons_ops(op + 1 + 5 * q, ops);
        for (int64_t J = 0; J < s->N; ++J) {
            uint64_t o;
            int sg;
            if (!orc_apply_ops(ops, no, orc_det(s, J), &o, &sg)) continue;
            int64_t K = orc_index(s, o);
            if (K < 0) continue;
            double x = psi[J], y = psi[K];
            psi[J] = c * x - sg * sn * y;
            psi[K] = c * y + sg * sn * x;
        }
    }
}

/* out = A psi for one pool op (A = sum_c C_c - C_c^dagger). */
void orc_apply_generator(const orc_sys *s, const int32_t *op, const double *psi,
                         double *out)
{
    memset(out, 0, sizeof(double) * s->N);
    for (int q = 0; q < op[0]; ++q) {
        int ops[4];
        int no = cons_ops(op + 1 + 5 * q, ops);
        for (int64_t J = 0; J < s->N; ++J) {
            uint64_t o;
            int sg;
            if (!orc_apply_ops(ops, no, orc_det(s, J), &o, &sg)) continue;
            int64_t K = orc_index(s, o);
            if (K < 0) continue;
            out[K] += sg * psi[J];   /*  C psi        */
            out[J] -= sg * psi[K];   /* -C^dagger psi */
        }
    }
}

/* g = 2 <sigma | A psi> */
double orc_op_gradient(const orc_sys *s, const int32_t *op, const double *psi,
                       const double *sigma)
{
    double *t = (double *)malloc(sizeof(double) * s->N);
    orc_apply_generator(s, op, psi, t);
    double g = 0.0;
    for (int64_t I = 0; I < s->N; ++I) g += sigma[I] * t[I];
    free(t);
    return 2.0 * g;
}

void orc_pool_gradients(const orc_sys *s, const int32_t *desc, int64_t K,
                        const double *psi, const double *sigma, double *g,
                        int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t k = 0; k < K; ++k)
        g[k] = orc_op_gradient(s, desc + 11 * k, psi, sigma);
    (void)nthreads;
}
