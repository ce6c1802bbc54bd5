/*
 * ntc_oracle.h -- FP64 CPU oracle for AO accelerated stochastic nonnegative
 * tensor completion (Siaminou, Papagiannakos, Kolomvakis, Liavas,
 * arXiv 2109.09534).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library
 * against a plain, slow, obviously correct restatement of the paper.  Only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the CUDA library, and
 * it includes nothing from it.
 *
 * Everything here is double precision and single threaded, except that the
 * row loop of Algorithm 1 carries an OpenMP "parallel for" (Algorithm 3) which
 * is active only in the -fopenmp build used as the timed CPU baseline.  Rows
 * are independent inside one inner iteration, so both builds give bit-identical
 * results.
 *
 * Readings of points where the paper is silent (each is repeated beside the
 * code that applies it):
 *   - sample (Alg. 1 line 5, Sec. II-B): a uniform k_p-subset without
 *     replacement, k_p = floor(c * n_p) in IEEE double; the subset is the k_p
 *     bucket positions with the smallest (key, position), key = word
 *     (position mod 4) of Philox4x32-10(counter = {mode, ao_iter, inner,
 *     floor(position / 4)}, key = seed).
 *   - L_p (Alg. 1 line 10): power method from v0 = 1/sqrt(R) * ones, a fixed
 *     number of iterations, Rayleigh quotient of the last iterate.  An exact
 *     Jacobi eigenvalue solve is kept for reporting and for the step-size pins.
 *   - beta (Alg. 1 line 12) uses lambda exactly.
 *   - skipped rows (k_p = 0, or L_p <= 0) keep their A and Y rows.
 *   - epoch (Sec. IV): ceil(1/c) AO iterations of Algorithm 2.
 */
#ifndef NTC_ORACLE_H
#define NTC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_ORDER 8

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11, Sec. 4 and Table 2). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Sample key of bucket position q (Alg. 1 line 5 reading above). */
uint32_t orc_sample_key(uint64_t seed, uint32_t mode, uint64_t ao_iter, uint32_t inner, int64_t q);

/* B_{l,p} = floor(c * ||M(p,:)||_0) (Sec. II-B). */
int64_t orc_sample_count(double c, int64_t n);

/* The k smallest (key, position) positions among bucket positions q0..q0+n-1,
 * written in ascending (key, position) order.  out[] holds absolute bucket
 * positions.  Returns 0, or -1 on bad arguments. */
/* Epoch-permutation variant: image of i under the pseudo-random permutation
 * of [0, n) of row `row` in epoch `epoch` (8-round Feistel network with cycle
 * walking, round keys from two Philox blocks, MurmurHash3's finaliser as round
 * function). */
int64_t orc_perm_index(uint64_t seed, uint32_t mode, uint32_t epoch, uint32_t row, int64_t n, int64_t i);

int orc_sample_row(uint64_t seed, uint32_t mode, uint64_t ao_iter, uint32_t inner,
                   int64_t q0, int64_t n, int64_t k, int64_t* out);

/* Stable counting sort of the nnz entries by their mode-`mode` index
 * (the rows of the mode-`mode` unfolding X_(i), Sec. II).  row_ptr[dim+1],
 * perm[nnz]: bucket position q holds entry perm[q].  Returns 0 or -1 when an
 * index is out of range. */
int orc_bucket(int order, int64_t nnz, const int32_t* idx, int mode, int64_t dim,
               int64_t* row_ptr, int64_t* perm);

/* Power method for the largest eigenvalue of the symmetric R x R matrix H
 * (row-major), fixed iteration count (reading above). */
double orc_power_lmax(int R, const double* H, int iters);
/* The same from start vector v_io (NULL: ones/sqrt(R)); v_io receives the
 * last normalised iterate.  A warm start of the next call on a nearby H (the
 * estimation of L_p is an open topic of Sec. II-B; this reading keeps each
 * row's last vector between S_NMC calls). */
double orc_power_lmax_v(int R, const double* H, int iters, double* v_io);

/* Largest eigenvalue of a symmetric matrix by cyclic Jacobi rotations. */
double orc_jacobi_lmax(int R, const double* H);

/* Alg. 1 lines 5-13 for one row, with the row's observations given in bucket
 * order (idx[n][order], vals[n]; the first at bucket position q0) and all
 * factors U[order] ([dims][rank] row-major).  y/a: Y_l(p,:), A_l(p,:); outputs
 * A_{l+1}(p,:), Y_{l+1}(p,:) and optionally H, gradient, L, exact L, beta.
 * Returns B_{l,p} (0 when skipped), or -1 when L_p <= 0 skipped the row. */
int64_t orc_row_update(int order, int mode, int rank, double lambda, int power_iters, int lp_exact,
                       const double* const* U, int64_t n, const int32_t* idx, const double* vals,
                       int64_t q0, double c, uint64_t seed, uint64_t ao_iter, int inner,
                       const double* y, const double* a, double* a_out, double* y_out,
                       double* H_out, double* grad_out, double* L_out, double* Lx_out,
                       double* beta_out);
/* The same with the power method started from v_io (NULL: cold start), which
 * receives the row's last power-method vector. */
int64_t orc_row_update_v(int order, int mode, int rank, double lambda, int power_iters, int lp_exact,
                         const double* const* U, int64_t n, const int32_t* idx, const double* vals,
                         int64_t q0, double c, uint64_t seed, uint64_t ao_iter, int inner,
                         const double* y, const double* a, double* a_out, double* y_out,
                         double* H_out, double* grad_out, double* L_out, double* Lx_out,
                         double* beta_out, double* v_io);
/* The same with the sampling reading chosen: perm_sampler 0 = independent
 * samples, 1 = epoch permutation (slot (k mod T) * max_inner + inner of the
 * epoch floor(k / T), T = ceil(1/c), of row `row`). */
int64_t orc_row_update_s(int order, int mode, int rank, double lambda, int power_iters, int lp_exact,
                         const double* const* U, int64_t n, const int32_t* idx, const double* vals,
                         int64_t q0, double c, uint64_t seed, uint64_t ao_iter, int inner,
                         const double* y, const double* a, double* a_out, double* y_out,
                         double* H_out, double* grad_out, double* L_out, double* Lx_out,
                         double* beta_out, double* v_io, int perm_sampler, int64_t row, int max_inner);

/* ---- whole-problem state (Algorithms 1-2) ---- */
typedef struct orc_state orc_state;

orc_state* orc_create(int order, const int64_t* dims, int rank, double lambda);
void orc_destroy(orc_state* s);
/* keys: "max_inner", "power_iters", "lp_exact" (0 power method, 1 Jacobi),
 *       "sampler" (0: independent samples per AO iteration, 1: epoch
 *       permutation -- the minibatches of an epoch are disjoint stretches of
 *       one pseudo-random permutation of each row),
 *       "power_warm" (1: each row's power method starts from the vector its
 *       previous update of this mode ended with; ones/sqrt(R) the first time),
 *       "debug" (1: keep per-row H, gradient, L of the last row update). */
int orc_set_param(orc_state* s, const char* key, double value);
/* Copies the COO tensor (idx[nnz][order], zero based) and buckets every mode. */
int orc_set_observed(orc_state* s, int64_t nnz, const int32_t* idx, const double* vals);
int orc_set_factor(orc_state* s, int mode, const double* in);
int orc_get_factor(const orc_state* s, int mode, double* out);
/* Initial factors i.i.d. U[0, 2a], a = (mean(x)/R)^(1/N), from Philox with
 * counter {0xFFFF, mode, row, col} and key init_seed. */
int orc_init_factors(orc_state* s, uint64_t init_seed);
uint64_t orc_get_ao_iter(const orc_state* s);
void orc_set_ao_iter(orc_state* s, uint64_t k);

/* Algorithm 1 (S_NMC) on mode `mode` with minibatch fraction c, at the
 * current AO iteration counter (which it does not advance). */
int orc_snmc(orc_state* s, int mode, double c, uint64_t seed);
/* Algorithm 2: ceil(1/c) AO iterations over mode_order (NULL = 0..N-1);
 * advances the AO iteration counter by that many. */
int orc_epoch(orc_state* s, const int* mode_order, double c, uint64_t seed);

/* CPD model (eq. 1) at n indices; RMSE against vals; cost (eq. 3) on the
 * observed set. */
int orc_predict(const orc_state* s, int64_t n, const int32_t* idx, double* out);
double orc_rmse(const orc_state* s, int64_t n, const int32_t* idx, const double* vals);
double orc_cost(const orc_state* s);

/* Debug views of the most recent orc_snmc (only with "debug" = 1):
 * H[dims][R][R], grad[dims][R], L (power method) and L_exact per row,
 * beta per row, k_p per row. */
int orc_debug_row(const orc_state* s, int64_t row, double* H, double* grad,
                  double* L, double* L_exact, double* beta, int64_t* kp);
/* Bucket of mode `mode`: row_ptr[dim+1] and perm[nnz]. */
int orc_get_bucket(const orc_state* s, int mode, int64_t* row_ptr, int64_t* perm);
/* Counters: rows skipped by the last orc_snmc/orc_epoch call, total visits. */
int64_t orc_rows_skipped(const orc_state* s);
int64_t orc_visits(const orc_state* s);

#ifdef __cplusplus
}
#endif
#endif
