/*
 * ntc_oracle.c -- FP64 CPU oracle for AO accelerated stochastic nonnegative
 * tensor completion (arXiv 2109.09534).  TEST INFRASTRUCTURE ONLY: see the
 * header.  Plain C, no blocking, no fusion, no reordering beyond what the
 * paper's equations and algorithms state.
 */
#include "ntc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from the published description (Salmon et al., SC'11,
 * Sec. 4.2 and Table 2): ten rounds of two 32x32->64 multiplies whose high
 * halves are xored with the other two words and the round key; the round key
 * is bumped by the Weyl constants between rounds. */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Sample key of bucket position q: word q mod 4 of Philox4x32-10 with
 * counter {mode, ao_iter, inner, floor(q / 4)} and the 64-bit seed as the key
 * (low word first), so that one block gives the keys of four consecutive
 * positions.  The paper only says "sample, uniformly at random" (Sec. II-B,
 * Alg. 1 line 5); this counter-based key makes the sample reproducible. */
uint32_t orc_sample_key(uint64_t seed, uint32_t mode, uint64_t ao_iter, uint32_t inner, int64_t q) {
    uint32_t ctr[4] = {mode, (uint32_t)ao_iter, inner, (uint32_t)(q / 4)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[q % 4];
}

/* B_{l,p} = floor(c ||M(p,:)||_0), Sec. II-B. */
int64_t orc_sample_count(double c, int64_t n) {
    return (int64_t)floor(c * (double)n);
}

typedef struct {
    uint32_t key;
    int64_t pos;
} orc_keypos;

static int orc_cmp_keypos(const void* a, const void* b) {
    const orc_keypos* x = (const orc_keypos*)a;
    const orc_keypos* y = (const orc_keypos*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return 0;
}

/* The k-subset of row positions q0..q0+n-1 with the smallest (key, q):
 * every k-subset is equally likely because the keys are i.i.d. uniform and
 * ties are broken by a fixed rule (Sec. II-B, "sample uniformly at random
 * B_{l,p} nonzero elements"). */
/* Epoch-permutation variant of the sampling: within an epoch of T AO
 * iterations every row is read in the order of one pseudo-random permutation
 * and the minibatch slots take disjoint consecutive stretches of it (the
 * epoch of Sec. IV touches every entry once).  The permutation of [0, n) is a
 * 8-round balanced Feistel network on the smallest even number of bits (at
 * least 8) that covers n, walked until the value falls below n; its eight round keys are
 * the words of two Philox4x32-10 blocks (counters {0xF2000000 | mode, epoch,
 * row, 0 or 1}, key seed) and its round function is the 32-bit finaliser of
 * MurmurHash3 (Appleby), applied to the right half xor the round key. */
static uint32_t orc_fmix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

int64_t orc_perm_index(uint64_t seed, uint32_t mode, uint32_t epoch, uint32_t row, int64_t n, int64_t i) {
    if (n <= 1) return 0;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t K[8];
    for (uint32_t blk = 0; blk < 2; ++blk) {
        const uint32_t ctr[4] = {0xF2000000u | mode, epoch, row, blk};
        orc_philox4x32_10(ctr, key, K + 4 * blk);
    }
    int bits = 0;
    while ((1ll << bits) < n) ++bits;         /* 2^bits >= n */
    int half = (bits + 1) / 2;                 /* domain 2^(2 half) >= n ... */
    if (half < 4) half = 4;                    /* ... and >= 256: short rows walk further */
    const uint32_t mask = (1u << half) - 1u;
    uint64_t x = (uint64_t)i;
    do {
        uint32_t L = (uint32_t)(x >> half), Rh = (uint32_t)x & mask;
        for (int r = 0; r < 8; ++r) {
            const uint32_t t = L ^ (orc_fmix32(Rh ^ K[r]) & mask);
            L = Rh;
            Rh = t;
        }
        x = ((uint64_t)L << half) | Rh;
    } while (x >= (uint64_t)n);
    return (int64_t)x;
}

int orc_sample_row(uint64_t seed, uint32_t mode, uint64_t ao_iter, uint32_t inner,
                   int64_t q0, int64_t n, int64_t k, int64_t* out) {
    if (n < 0 || k < 0 || k > n) return -1;
    if (k == 0) return 0;
    orc_keypos* kp = (orc_keypos*)malloc(sizeof(orc_keypos) * (size_t)n);
    if (!kp) return -1;
    for (int64_t j = 0; j < n; ++j) {
        kp[j].pos = q0 + j;
        kp[j].key = orc_sample_key(seed, mode, ao_iter, inner, q0 + j);
    }
    qsort(kp, (size_t)n, sizeof(orc_keypos), orc_cmp_keypos);
    for (int64_t j = 0; j < k; ++j) out[j] = kp[j].pos;
    free(kp);
    return 0;
}

/* Stable counting sort by row index of the mode-i unfolding (Sec. II):
 * count, exclusive prefix sum, then place entries in input order. */
int orc_bucket(int order, int64_t nnz, const int32_t* idx, int mode, int64_t dim,
               int64_t* row_ptr, int64_t* perm) {
    for (int64_t p = 0; p <= dim; ++p) row_ptr[p] = 0;
    for (int64_t e = 0; e < nnz; ++e) {
        int64_t r = idx[e * order + mode];
        if (r < 0 || r >= dim) return -1;
        row_ptr[r + 1] += 1;
    }
    for (int64_t p = 0; p < dim; ++p) row_ptr[p + 1] += row_ptr[p];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(dim > 0 ? dim : 1));
    if (!fill) return -1;
    for (int64_t p = 0; p < dim; ++p) fill[p] = row_ptr[p];
    for (int64_t e = 0; e < nnz; ++e) {
        int64_t r = idx[e * order + mode];
        perm[fill[r]++] = e;
    }
    free(fill);
    return 0;
}

/* L_p = max eig(H_{l,p}) (Alg. 1 line 10) by the power method (Sec. II-B,
 * cost item 4): v0 = ones/sqrt(R); w = H v; mu = v'w; v = w/||w||. */
double orc_power_lmax(int R, const double* H, int iters) {
    return orc_power_lmax_v(R, H, iters, NULL);
}

/* The same from the start vector v_io (NULL: ones/sqrt(R)); on return v_io
 * holds the last normalised iterate (the warm start of the next call). */
double orc_power_lmax_v(int R, const double* H, int iters, double* v_io) {
    double* v = (double*)malloc(sizeof(double) * (size_t)R);
    double* w = (double*)malloc(sizeof(double) * (size_t)R);
    double mu = 0.0;
    for (int r = 0; r < R; ++r) v[r] = v_io ? v_io[r] : 1.0 / sqrt((double)R);
    for (int t = 0; t < iters; ++t) {
        for (int i = 0; i < R; ++i) {
            double acc = 0.0;
            for (int j = 0; j < R; ++j) acc += H[i * R + j] * v[j];
            w[i] = acc;
        }
        double vw = 0.0, ww = 0.0;
        for (int i = 0; i < R; ++i) {
            vw += v[i] * w[i];
            ww += w[i] * w[i];
        }
        mu = vw;
        if (ww <= 0.0) {
            mu = 0.0;
            break;
        }
        double nrm = sqrt(ww);
        for (int i = 0; i < R; ++i) v[i] = w[i] / nrm;
    }
    if (v_io)
        for (int r = 0; r < R; ++r) v_io[r] = v[r];
    free(v);
    free(w);
    return mu;
}

/* Largest eigenvalue of a symmetric matrix: cyclic Jacobi rotations
 * (Golub & Van Loan, Matrix Computations, Sec. 8.5) until the off-diagonal
 * mass is negligible. */
double orc_jacobi_lmax(int R, const double* H) {
    double* a = (double*)malloc(sizeof(double) * (size_t)R * (size_t)R);
    memcpy(a, H, sizeof(double) * (size_t)R * (size_t)R);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < R; ++i)
            for (int j = 0; j < R; ++j) {
                tot += a[i * R + j] * a[i * R + j];
                if (i != j) off += a[i * R + j] * a[i * R + j];
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < R - 1; ++p)
            for (int q = p + 1; q < R; ++q) {
                double apq = a[p * R + q];
                if (apq == 0.0) continue;
                double app = a[p * R + p], aqq = a[q * R + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < R; ++k) {
                    double akp = a[k * R + p], akq = a[k * R + q];
                    a[k * R + p] = cs * akp - sn * akq;
                    a[k * R + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < R; ++k) {
                    double apk = a[p * R + k], aqk = a[q * R + k];
                    a[p * R + k] = cs * apk - sn * aqk;
                    a[q * R + k] = sn * apk + cs * aqk;
                }
            }
    }
    double mx = a[0];
    for (int i = 1; i < R; ++i)
        if (a[i * R + i] > mx) mx = a[i * R + i];
    free(a);
    return mx;
}

/* ------------------------------------------------------------------------- */
struct orc_state {
    int order;
    int64_t dims[ORC_MAX_ORDER];
    int rank;
    double lambda;
    int max_inner;
    int power_iters;
    int power_warm;     /* 1: each row's power method starts from its last vector */
    int sampler;        /* 0: independent samples; 1: epoch permutation */
    int lp_exact;
    int debug;
    uint64_t ao_iter;
    int64_t nnz;
    int32_t* idx;
    double* vals;
    double* U[ORC_MAX_ORDER];
    int64_t* row_ptr[ORC_MAX_ORDER];
    int64_t* perm[ORC_MAX_ORDER];
    double* V[ORC_MAX_ORDER];   /* last power-method vector per row (power_warm) */
    /* debug views of the last orc_snmc */
    int dbg_mode;
    double* dbg_H;
    double* dbg_grad;
    double* dbg_L;
    double* dbg_Lx;
    double* dbg_beta;
    int64_t* dbg_kp;
    int64_t rows_skipped;
    int64_t visits;
};

orc_state* orc_create(int order, const int64_t* dims, int rank, double lambda) {
    if (order < 2 || order > ORC_MAX_ORDER || rank < 1 || !(lambda >= 0.0)) return NULL;
    for (int i = 0; i < order; ++i)
        if (dims[i] < 1) return NULL;
    orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
    s->order = order;
    s->rank = rank;
    s->lambda = lambda;
    s->max_inner = 1;
    s->power_iters = 10;
    s->dbg_mode = -1;
    for (int i = 0; i < order; ++i) {
        s->dims[i] = dims[i];
        s->U[i] = (double*)calloc((size_t)dims[i] * (size_t)rank, sizeof(double));
    }
    return s;
}

static void orc_free_debug(orc_state* s) {
    free(s->dbg_H); free(s->dbg_grad); free(s->dbg_L); free(s->dbg_Lx);
    free(s->dbg_beta); free(s->dbg_kp);
    s->dbg_H = s->dbg_grad = s->dbg_L = s->dbg_Lx = s->dbg_beta = NULL;
    s->dbg_kp = NULL;
    s->dbg_mode = -1;
}

void orc_destroy(orc_state* s) {
    if (!s) return;
    for (int i = 0; i < s->order; ++i) {
        free(s->U[i]);
        free(s->row_ptr[i]);
        free(s->perm[i]);
        free(s->V[i]);
    }
    free(s->idx);
    free(s->vals);
    orc_free_debug(s);
    free(s);
}

int orc_set_param(orc_state* s, const char* key, double value) {
    if (!strcmp(key, "max_inner")) {
        if (value < 1) return -1;
        s->max_inner = (int)value;
    } else if (!strcmp(key, "power_iters")) {
        if (value < 1) return -1;
        s->power_iters = (int)value;
    } else if (!strcmp(key, "sampler")) {
        if (value != 0.0 && value != 1.0) return -1;
        s->sampler = (int)value;
    } else if (!strcmp(key, "power_warm")) {
        s->power_warm = value != 0.0;
    } else if (!strcmp(key, "lp_exact")) {
        s->lp_exact = value != 0.0;
    } else if (!strcmp(key, "debug")) {
        s->debug = value != 0.0;
    } else {
        return -1;
    }
    return 0;
}

int orc_set_observed(orc_state* s, int64_t nnz, const int32_t* idx, const double* vals) {
    if (nnz < 0) return -1;
    int N = s->order;
    for (int64_t e = 0; e < nnz; ++e)
        for (int i = 0; i < N; ++i)
            if (idx[e * N + i] < 0 || idx[e * N + i] >= s->dims[i]) return -1;
    free(s->idx);
    free(s->vals);
    s->nnz = nnz;
    s->idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz * N + 1));
    s->vals = (double*)malloc(sizeof(double) * (size_t)(nnz + 1));
    memcpy(s->idx, idx, sizeof(int32_t) * (size_t)(nnz * N));
    memcpy(s->vals, vals, sizeof(double) * (size_t)nnz);
    for (int i = 0; i < N; ++i) {
        free(s->row_ptr[i]);
        free(s->perm[i]);
        free(s->V[i]);       /* new observations: the power method starts cold again */
        s->V[i] = NULL;
        s->row_ptr[i] = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->dims[i] + 1));
        s->perm[i] = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz + 1));
        if (orc_bucket(N, nnz, s->idx, i, s->dims[i], s->row_ptr[i], s->perm[i]) != 0) return -1;
    }
    return 0;
}

int orc_set_factor(orc_state* s, int mode, const double* in) {
    if (mode < 0 || mode >= s->order) return -1;
    size_t n = (size_t)s->dims[mode] * (size_t)s->rank;
    for (size_t j = 0; j < n; ++j)
        if (!(in[j] >= 0.0)) return -1;
    memcpy(s->U[mode], in, sizeof(double) * n);
    return 0;
}

int orc_get_factor(const orc_state* s, int mode, double* out) {
    if (mode < 0 || mode >= s->order) return -1;
    memcpy(out, s->U[mode], sizeof(double) * (size_t)s->dims[mode] * (size_t)s->rank);
    return 0;
}

/* Initial values U_0^(i) (Alg. 2 input; the paper does not say how they are
 * drawn): i.i.d. U[0, 2a] with a = (mean(x)/R)^(1/N), so that the expected
 * model value equals the mean observation. */
int orc_init_factors(orc_state* s, uint64_t init_seed) {
    double mean = 0.0;
    for (int64_t e = 0; e < s->nnz; ++e) mean += s->vals[e];
    mean = s->nnz > 0 ? mean / (double)s->nnz : 0.0;
    double a = mean > 0.0 ? pow(mean / (double)s->rank, 1.0 / (double)s->order) : 0.0;
    uint32_t key[2] = {(uint32_t)init_seed, (uint32_t)(init_seed >> 32)};
    for (int i = 0; i < s->order; ++i)
        for (int64_t p = 0; p < s->dims[i]; ++p)
            for (int r = 0; r < s->rank; ++r) {
                uint32_t ctr[4] = {0xFFFFu, (uint32_t)i, (uint32_t)p, (uint32_t)r};
                uint32_t out[4];
                orc_philox4x32_10(ctr, key, out);
                double u = ((double)out[0] + 0.5) * (1.0 / 4294967296.0);
                s->U[i][p * s->rank + r] = 2.0 * a * u;
            }
    return 0;
}

uint64_t orc_get_ao_iter(const orc_state* s) { return s->ao_iter; }
void orc_set_ao_iter(orc_state* s, uint64_t k) { s->ao_iter = k; }

/* Alg. 1 lines 5-13 for one row p of the mode-`mode` unfolding.  The row's
 * observations are given explicitly in bucket order: idx[n][order], vals[n],
 * the first at bucket position q0.  The row of K_k^(i) for an observation is
 * the Hadamard product of the other factors' rows at its indices (Sec. II,
 * unfolding eq.; Sec. III, K definition); it is never formed as a matrix.
 * y = Y_l(p,:), a = A_l(p,:) on input; a_out = A_{l+1}(p,:), y_out =
 * Y_{l+1}(p,:) on output (unchanged copies when the row is skipped).
 * Optional outputs (may be NULL): H[R*R], grad[R], L (used), L_exact, beta.
 * Returns k = B_{l,p}, or -1 when L_p <= 0 made the row skip. */
int64_t orc_row_update(int order, int mode, int rank, double lambda, int power_iters, int lp_exact,
                       const double* const* U, int64_t n, const int32_t* idx, const double* vals,
                       int64_t q0, double c, uint64_t seed, uint64_t ao_iter, int inner,
                       const double* y, const double* a, double* a_out, double* y_out,
                       double* H_out, double* grad_out, double* L_out, double* Lx_out,
                       double* beta_out) {
    return orc_row_update_v(order, mode, rank, lambda, power_iters, lp_exact, U, n, idx, vals, q0, c, seed,
                            ao_iter, inner, y, a, a_out, y_out, H_out, grad_out, L_out, Lx_out, beta_out, NULL);
}

int64_t orc_row_update_v(int order, int mode, int rank, double lambda, int power_iters, int lp_exact,
                         const double* const* U, int64_t n, const int32_t* idx, const double* vals,
                         int64_t q0, double c, uint64_t seed, uint64_t ao_iter, int inner,
                         const double* y, const double* a, double* a_out, double* y_out,
                         double* H_out, double* grad_out, double* L_out, double* Lx_out,
                         double* beta_out, double* v_io) {
    return orc_row_update_s(order, mode, rank, lambda, power_iters, lp_exact, U, n, idx, vals, q0, c, seed,
                            ao_iter, inner, y, a, a_out, y_out, H_out, grad_out, L_out, Lx_out, beta_out, v_io,
                            0, 0, 1);
}

int64_t orc_row_update_s(int order, int mode, int rank, double lambda, int power_iters, int lp_exact,
                         const double* const* U, int64_t n, const int32_t* idx, const double* vals,
                         int64_t q0, double c, uint64_t seed, uint64_t ao_iter, int inner,
                         const double* y, const double* a, double* a_out, double* y_out,
                         double* H_out, double* grad_out, double* L_out, double* Lx_out,
                         double* beta_out, double* v_io, int perm_sampler, int64_t row, int max_inner) {
    const int N = order, R = rank;
    const double lam = lambda;
    for (int r = 0; r < R; ++r) {
        a_out[r] = a[r];
        y_out[r] = y[r];
    }
    const int64_t k = orc_sample_count(c, n);
    if (k == 0) return 0;                          /* B_{l,p} = 0: skip the row */
    int64_t* sel = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    double* W = (double*)calloc((size_t)R, sizeof(double));
    double* Z = (double*)calloc((size_t)R, sizeof(double));
    double* G = (double*)calloc((size_t)R, sizeof(double));
    double* H = (double*)calloc((size_t)R * R, sizeof(double));
    double* kr = (double*)malloc(sizeof(double) * (size_t)R);

    /* line 5: M_hat_l(p,:) = sample(M(p,:)) */
    if (perm_sampler) {
        /* epoch e = floor(k / T) of T = ceil(1/c) AO iterations; slot s of
         * the epoch takes positions pi((s k_p + j) mod n_p), j < k_p */
        const uint64_t T = (uint64_t)ceil(1.0 / c - 1e-12);
        const uint32_t epoch = (uint32_t)(ao_iter / T);
        const int64_t s = (int64_t)(ao_iter % T) * max_inner + inner;
        for (int64_t j = 0; j < k; ++j)
            sel[j] = q0 + orc_perm_index(seed, (uint32_t)mode, epoch, (uint32_t)row, n, (s * k + j) % n);
    } else {
        orc_sample_row(seed, (uint32_t)mode, ao_iter, (uint32_t)inner, q0, n, k, sel);
    }

    for (int64_t t = 0; t < k; ++t) {
        const int64_t j = sel[t] - q0;
        const int32_t* ix = idx + j * N;
        const double x = vals[j];
        /* row of B = K_k^(i) at this observation's column */
        for (int r = 0; r < R; ++r) kr[r] = 1.0;
        for (int m = 0; m < N; ++m) {
            if (m == mode) continue;
            const double* u = U[m] + (int64_t)ix[m] * R;
            for (int r = 0; r < R; ++r) kr[r] *= u[r];
        }
        /* line 6: W_l(p,:) = -(M_hat(p,:) .* X(p,:)) B */
        for (int r = 0; r < R; ++r) W[r] -= x * kr[r];
        /* line 7: Z_l(p,:) = (M_hat(p,:) .* (Y_l(p,:) B^T)) B */
        double yb = 0.0;
        for (int r = 0; r < R; ++r) yb += y[r] * kr[r];
        for (int r = 0; r < R; ++r) Z[r] += yb * kr[r];
        /* line 9: H_{l,p} = B^T diag(M_hat(p,:)) B + lambda I */
        for (int r = 0; r < R; ++r)
            for (int q = 0; q < R; ++q) H[r * R + q] += kr[r] * kr[q];
    }
    for (int r = 0; r < R; ++r) H[r * R + r] += lam;
    /* line 8: gradient = W + Z + lambda Y_l(p,:) */
    for (int r = 0; r < R; ++r) G[r] = W[r] + Z[r] + lam * y[r];
    /* line 10: L_p = max(eig(H_{l,p})) */
    const double Lpm = orc_power_lmax_v(R, H, power_iters, v_io);
    const double L = lp_exact ? orc_jacobi_lmax(R, H) : Lpm;
    if (H_out) memcpy(H_out, H, sizeof(double) * (size_t)R * R);
    if (grad_out) memcpy(grad_out, G, sizeof(double) * (size_t)R);
    if (L_out) *L_out = L;
    if (Lx_out) *Lx_out = orc_jacobi_lmax(R, H);
    int64_t ret = k;
    if (L > 0.0) {
        /* line 11: A_{l+1}(p,:) = (Y_l(p,:) - grad / L_p)_+ */
        /* line 12: beta = (sqrt(L_p) - sqrt(lambda)) / (sqrt(L_p) + sqrt(lambda)) */
        const double beta = (sqrt(L) - sqrt(lam)) / (sqrt(L) + sqrt(lam));
        for (int r = 0; r < R; ++r) {
            double anew = y[r] - G[r] / L;
            if (!(anew > 0.0)) anew = 0.0;
            /* line 13: Y_{l+1} = A_{l+1} + beta (A_{l+1} - A_l) */
            a_out[r] = anew;
            y_out[r] = anew + beta * (anew - a[r]);
        }
        if (beta_out) *beta_out = beta;
    } else {
        ret = -1;                                  /* L_p <= 0: skip as well */
    }
    free(sel); free(W); free(Z); free(G); free(H); free(kr);
    return ret;
}

/* Algorithm 1, S_NMC(X_(i), M_(i), K_k^(i), U_k^(i), lambda): MAX_INNER
 * passes of the row update over every row (Alg. 3: rows in parallel), with
 * the factors of the other modes as they are now, so that modes already
 * visited in this AO iteration contribute their updated values. */
int orc_snmc(orc_state* s, int mode, double c, uint64_t seed) {
    if (mode < 0 || mode >= s->order || !(c > 0.0) || c > 1.0) return -1;
    if (!s->row_ptr[0]) return -1;
    const int N = s->order, R = s->rank;
    const int64_t P = s->dims[mode];
    double* A = s->U[mode];                      /* A_l, updated in place */
    if (s->power_warm && !s->V[mode]) {          /* first warm use: v0 = ones/sqrt(R) */
        s->V[mode] = (double*)malloc(sizeof(double) * (size_t)P * (size_t)R);
        for (int64_t q = 0; q < P * R; ++q) s->V[mode][q] = 1.0 / sqrt((double)R);
    }
    double* Y = (double*)malloc(sizeof(double) * (size_t)P * (size_t)R);
    memcpy(Y, A, sizeof(double) * (size_t)P * (size_t)R); /* Y_0 = A_0 = A_* */
    const double* const* U = (const double* const*)s->U;

    if (s->debug) {
        orc_free_debug(s);
        s->dbg_mode = mode;
        s->dbg_H = (double*)calloc((size_t)P * R * R, sizeof(double));
        s->dbg_grad = (double*)calloc((size_t)P * R, sizeof(double));
        s->dbg_L = (double*)calloc((size_t)P, sizeof(double));
        s->dbg_Lx = (double*)calloc((size_t)P, sizeof(double));
        s->dbg_beta = (double*)calloc((size_t)P, sizeof(double));
        s->dbg_kp = (int64_t*)calloc((size_t)P, sizeof(int64_t));
    }
    int64_t skipped = 0, visits = 0;

    for (int l = 0; l < s->max_inner; ++l) {       /* while (l < MAX_INNER) */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : skipped, visits)
#endif
        for (int64_t p = 0; p < P; ++p) {          /* for p = 1..P (Alg. 3: in parallel) */
            const int64_t q0 = s->row_ptr[mode][p];
            const int64_t n = s->row_ptr[mode][p + 1] - q0;
            int32_t* ridx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n * N + 1));
            double* rval = (double*)malloc(sizeof(double) * (size_t)(n + 1));
            for (int64_t j = 0; j < n; ++j) {
                const int64_t e = s->perm[mode][q0 + j];
                memcpy(ridx + j * N, s->idx + e * N, sizeof(int32_t) * (size_t)N);
                rval[j] = s->vals[e];
            }
            double* a = A + p * R;
            double* y = Y + p * R;
            double* anew = (double*)malloc(sizeof(double) * (size_t)R);
            double* ynew = (double*)malloc(sizeof(double) * (size_t)R);
            const int dbg = s->debug && l == s->max_inner - 1;
            const int64_t k = orc_row_update_s(N, mode, R, s->lambda, s->power_iters, s->lp_exact, U, n,
                                               ridx, rval, q0, c, seed, s->ao_iter, l, y, a, anew, ynew,
                                               dbg ? s->dbg_H + p * R * R : NULL,
                                               dbg ? s->dbg_grad + p * R : NULL,
                                               dbg ? s->dbg_L + p : NULL, dbg ? s->dbg_Lx + p : NULL,
                                               dbg ? s->dbg_beta + p : NULL,
                                               s->power_warm ? s->V[mode] + p * R : NULL, s->sampler, p,
                                               s->max_inner);
            if (dbg) s->dbg_kp[p] = k > 0 ? k : orc_sample_count(c, n);
            if (k <= 0 && l == 0) skipped += 1;
            if (k != 0) visits += k > 0 ? k : orc_sample_count(c, n);
            memcpy(a, anew, sizeof(double) * (size_t)R);
            memcpy(y, ynew, sizeof(double) * (size_t)R);
            free(ridx); free(rval); free(anew); free(ynew);
        }
    }
    free(Y);
    s->rows_skipped = skipped;
    s->visits = visits;
    return 0;
}

/* Algorithm 2 for one epoch: an epoch touches every observed entry once on
 * average (Sec. IV), i.e. ceil(1/c) AO iterations at minibatch fraction c. */
int orc_epoch(orc_state* s, const int* mode_order, double c, uint64_t seed) {
    if (!(c > 0.0) || c > 1.0) return -1;
    const int N = s->order;
    int ord[ORC_MAX_ORDER];
    int seen[ORC_MAX_ORDER] = {0};
    for (int i = 0; i < N; ++i) {
        ord[i] = mode_order ? mode_order[i] : i;
        if (ord[i] < 0 || ord[i] >= N || seen[ord[i]]) return -1;
        seen[ord[i]] = 1;
    }
    int64_t T = (int64_t)ceil(1.0 / c - 1e-12);
    int64_t skipped = 0, visits = 0;
    for (int64_t t = 0; t < T; ++t) {
        for (int i = 0; i < N; ++i) {
            if (orc_snmc(s, ord[i], c, seed) != 0) return -1;
            skipped += s->rows_skipped;
            visits += s->visits;
        }
        s->ao_iter += 1;
    }
    s->rows_skipped = skipped;
    s->visits = visits;
    return 0;
}

/* CPD model value (eq. 1) at one index: sum_r prod_i U^(i)(i_i, r). */
static double orc_model_at(const orc_state* s, const int32_t* ix) {
    double acc = 0.0;
    for (int r = 0; r < s->rank; ++r) {
        double prod = 1.0;
        for (int i = 0; i < s->order; ++i) prod *= s->U[i][(int64_t)ix[i] * s->rank + r];
        acc += prod;
    }
    return acc;
}

int orc_predict(const orc_state* s, int64_t n, const int32_t* idx, double* out) {
    for (int64_t e = 0; e < n; ++e) {
        for (int i = 0; i < s->order; ++i)
            if (idx[e * s->order + i] < 0 || idx[e * s->order + i] >= s->dims[i]) return -1;
        out[e] = orc_model_at(s, idx + e * s->order);
    }
    return 0;
}

double orc_rmse(const orc_state* s, int64_t n, const int32_t* idx, const double* vals) {
    if (n <= 0) return 0.0;
    double acc = 0.0;
    for (int64_t e = 0; e < n; ++e) {
        double d = vals[e] - orc_model_at(s, idx + e * s->order);
        acc += d * d;
    }
    return sqrt(acc / (double)n);
}

/* Eq. 3: f_Omega(U) + lambda/2 sum_i ||U^(i)||_F^2 over the observed set. */
double orc_cost(const orc_state* s) {
    double fit = 0.0, reg = 0.0;
    for (int64_t e = 0; e < s->nnz; ++e) {
        double d = s->vals[e] - orc_model_at(s, s->idx + e * s->order);
        fit += d * d;
    }
    for (int i = 0; i < s->order; ++i) {
        size_t n = (size_t)s->dims[i] * (size_t)s->rank;
        for (size_t j = 0; j < n; ++j) reg += s->U[i][j] * s->U[i][j];
    }
    return 0.5 * fit + 0.5 * s->lambda * reg;
}

int orc_debug_row(const orc_state* s, int64_t row, double* H, double* grad,
                  double* L, double* L_exact, double* beta, int64_t* kp) {
    if (s->dbg_mode < 0 || row < 0 || row >= s->dims[s->dbg_mode]) return -1;
    const int R = s->rank;
    if (H) memcpy(H, s->dbg_H + row * R * R, sizeof(double) * (size_t)R * R);
    if (grad) memcpy(grad, s->dbg_grad + row * R, sizeof(double) * (size_t)R);
    if (L) *L = s->dbg_L[row];
    if (L_exact) *L_exact = s->dbg_Lx[row];
    if (beta) *beta = s->dbg_beta[row];
    if (kp) *kp = s->dbg_kp[row];
    return 0;
}

int orc_get_bucket(const orc_state* s, int mode, int64_t* row_ptr, int64_t* perm) {
    if (mode < 0 || mode >= s->order || !s->row_ptr[mode]) return -1;
    memcpy(row_ptr, s->row_ptr[mode], sizeof(int64_t) * (size_t)(s->dims[mode] + 1));
    memcpy(perm, s->perm[mode], sizeof(int64_t) * (size_t)s->nnz);
    return 0;
}

int64_t orc_rows_skipped(const orc_state* s) { return s->rows_skipped; }
int64_t orc_visits(const orc_state* s) { return s->visits; }
