/*
 * muca_oracle.h -- plain CPU oracle for the parallel multicanonical (MUCA)
 * Blume-Capel hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct reference
 * that the CUDA library is checked against.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library, and neither side
 * includes the other.
 *
 * Model (paper, Eq. 1): H = -J sum_<ij> s_i s_j + Delta sum_i s_i^2
 *                         = E_J + Delta * E_Delta,  s_i in {-1,0,+1}, J = 1,
 * simple-cubic L^3 lattice with periodic boundaries (Sec. I, Sec. II).
 * MUCA replaces exp(-beta Delta E_Delta) by a weight W(E_Delta) (Sec. II, Eq. after
 * Eq. 2) and time series are reweighted back to any Delta with Eq. 3.
 *
 * Readings where the paper is silent (update order, proposal, random numbers,
 * weight recursion, histogram cadence) are listed in the implementation file
 * next to the code that takes them.
 *
 * All functions return 0 on success and a negative code on error.
 */
#ifndef MUCA_ORACLE_H
#define MUCA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_TALLY (-5)
#define OR_ERR_WINDOW (-7)
#define OR_ERR_NOMEM (-3)

/* Number of logical threshold entries per (E_Delta, d) pair: dE_J in [-12, 12]. */
#define OR_NK 25

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): out = Philox(ctr, key). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Initial spins of one walker: i.i.d. uniform on {-1,0,+1}.  spins is [L^3]. */
int or_init_spins(int L, uint32_t seed, uint32_t walker_id, int8_t *spins);

/* E_J, E_Delta and M of one configuration, recomputed from scratch (Eq. 1). */
int or_energies(int L, const int8_t *spins, int64_t out[3]);

/* Logical acceptance-threshold table thr[nE][3][25] (index [E-e_min][d+1][dEJ+12])
 * built in FP64 from lnW[nE] at temperature T. */
int or_build_table(int L, double T, int e_min, int e_max, const double *lnW, uint32_t *thr);

/* n_sweeps typewriter Metropolis sweeps of one walker with a fixed table.
 * state: spins[L^3] (in/out); tallies[3] = (E_J, E_Delta, M) (in/out).
 * hist[nE] is incremented once per sweep at the walker's E_Delta (may be NULL).
 * ts, if not NULL, receives [n_sweeps][3] (E_J, E_Delta, M) after each sweep.
 * check != 0 recomputes the energies after every sweep and fails on mismatch. */
int or_sweeps(int L, int e_min, int e_max, const uint32_t *thr, uint32_t seed,
              uint32_t walker_id, uint64_t sweep0, int n_sweeps, int8_t *spins,
              int32_t tallies[3], uint64_t *hist, int32_t *ts, int check);

/* Weight recursion: lnW[E] -= ln H[E] wherever H[E] > 0. */
int or_update_lnW(int nE, const uint64_t *H, double *lnW);

/* Accumulated, error-weighted weight recursion (reading R13 in the .c file):
 * acc[nE - 1] holds the accumulated pair weights (zero before the first
 * iteration) and is updated with lnW. */
int or_update_lnW_acc(int nE, const uint64_t *H, double *lnW, double *acc);

/* A whole parallel MUCA run of one (L, T) group (init, n_iter weight
 * iterations of sweeps_per_iter sweeps with merge + update + table rebuild,
 * then n_meas measurement sweeps under the final weights).
 *   lnW[nE]            in: initial weights, out: final weights
 *   hist_iter          [n_iter][nE] merged histogram of every iteration, or NULL
 *   spins_out          [n_walkers][L^3] final spins, or NULL
 *   tallies_out        [n_walkers][3] final (E_J, E_Delta, M), or NULL
 *   ts                 [n_walkers][n_meas][3] measurement time series, or NULL
 *   n_threads          worker threads over walkers (>= 1)
 * Walker w of the group has global id walker_id0 + w. */
int or_muca_run(int L, double T, int n_walkers, int e_min, int e_max, uint32_t seed,
                uint32_t walker_id0, int n_iter, int sweeps_per_iter, int n_meas,
                double *lnW, uint64_t *hist_iter, int8_t *spins_out,
                int32_t *tallies_out, int32_t *ts, int check, int n_threads);

/* The same run with a choice of weight recursion: 0 the plain one
 * (or_update_lnW), 1 the accumulated one (or_update_lnW_acc, with its pair
 * weights in acc[nE - 1], in/out). */
int or_muca_run_rec(int L, double T, int n_walkers, int e_min, int e_max, uint32_t seed,
                    uint32_t walker_id0, int n_iter, int sweeps_per_iter, int n_meas,
                    double *lnW, uint64_t *hist_iter, int8_t *spins_out,
                    int32_t *tallies_out, int32_t *ts, int check, int n_threads,
                    int recursion, double *acc);

/* The same run in an adaptive E_Delta window (reading R15 in the .c file):
 * the walkers move in [win_lo, win_hi] (inside [e_min, e_max]; every initial
 * E_Delta must lie in it, else OR_ERR_WINDOW), which grows by grow_step bins
 * on each side after every iteration whose merged histogram has
 * min H / mean H >= grow_flat over it (grow_flat = 0: a fixed window).
 * win_iter [n_iter][2] receives the window after each iteration (the window
 * of the next one), or NULL.  lnW, acc and hist_iter cover [e_min, e_max]. */
int or_muca_run_win(int L, double T, int n_walkers, int e_min, int e_max, uint32_t seed,
                    uint32_t walker_id0, int n_iter, int sweeps_per_iter, int n_meas,
                    double *lnW, uint64_t *hist_iter, int8_t *spins_out,
                    int32_t *tallies_out, int32_t *ts, int check, int n_threads,
                    int recursion, double *acc, int win_lo, int win_hi, double grow_flat,
                    int grow_step, int32_t *win_iter);

/* The disordered model (reading R16 in the .c file): couplings J[3 i + mu]
 * of the forward bonds (integers in [-jmax, jmax], 1 <= jmax <= OR_MAX_JMAX).
 * The table has rows of 24 jmax + 1 entries, index
 * [(E_Delta - e_min) * 3 + d + 1][dE_J + 12 jmax].  or_muca_run_bonds is
 * or_muca_run_win with couplings (J = NULL: the clean model). */
#define OR_MAX_JMAX 8
int or_energies_bonds(int L, const int8_t *s, const int8_t *J, int64_t out[3]);
int or_build_table_bonds(int L, double T, int jmax, int e_min, int e_max, const double *lnW,
                         uint32_t *thr);
int or_sweeps_bonds(int L, const int8_t *J, int jmax, int e_min, int e_max, const uint32_t *thr,
                    uint32_t seed, uint32_t walker_id, uint64_t sweep0, int n_sweeps,
                    int8_t *spins, int32_t tallies[3], uint64_t *hist, int32_t *ts, int check);
int or_muca_run_bonds(int L, double T, int n_walkers, int e_min, int e_max, uint32_t seed,
                      uint32_t walker_id0, int n_iter, int sweeps_per_iter, int n_meas,
                      double *lnW, uint64_t *hist_iter, int8_t *spins_out,
                      int32_t *tallies_out, int32_t *ts, int check, int n_threads,
                      int recursion, double *acc, int win_lo, int win_hi, double grow_flat,
                      int grow_step, int32_t *win_iter, const int8_t *J, int jmax);

/* Time-series reweighting (Eq. 3) to each Delta_k of grid[n_grid], FP64 with
 * compensated sums.  Samples: e_j[n], e_d[n], m[n].  lnW[nE] indexed by
 * E_Delta - e_min.  out[n_grid][5] = <E_J>, <E_Delta>, C (Eq. 6),
 * chi = beta V (<m^2> - <|m|>^2), U4 = 1 - <m^4> / (3 <m^2>^2), m = M/V. */
int or_reweight(const int32_t *e_j, const int32_t *e_d, const int32_t *m, int64_t n,
                const double *lnW, int e_min, int nE, double beta, int V,
                const double *grid, int n_grid, int n_threads, double *out);

/* The same in binary128 arithmetic (results rounded to double). */
int or_reweight_q(const int32_t *e_j, const int32_t *e_d, const int32_t *m, int64_t n,
                  const double *lnW, int e_min, int nE, double beta, int V,
                  const double *grid, int n_grid, int n_threads, double *out);

/* Pseudo-transition point (Sec. III): Delta*_L (the maximum of C, Eq. 6)
 * by n_iter bisection steps on the zero of dC/dDelta inside [lo, hi], and
 * C*_L, for the full series (n_rows x row_len samples, row-major) and for the
 * n_jack subsets (0 or >= 2) that each leave out one block of n_rows / n_jack
 * consecutive rows.  out[2 b], out[2 b + 1] = Delta*, C* of data set b
 * (b = 0 full, b = 1 + i leaves out block i).  OR_ERR_ARG when [lo, hi] does
 * not bracket the maximum for some data set. */
int or_find_peak(const int32_t *e_j, const int32_t *e_d, int64_t n_rows, int32_t row_len,
                 const double *lnW, int e_min, int nE, double beta, double lo, double hi,
                 int n_iter, int n_jack, int n_threads, double *out);

/* Equal-height field Delta_eqh and barrier B = ln(P_max/P_min)/(2 beta Delta)
 * of the reweighted E_Delta distribution (peaks: the highest occupied bins
 * below and at or above split), by n_iter bisection steps in [lo, hi], for
 * the full series and the n_jack leave-one-block-out subsets.  out[5 b ..]:
 * Delta_eqh, B, E of the left peak, E of the right peak, E of the minimum. */
int or_equal_height(const int32_t *e_d, int64_t n_rows, int32_t row_len, const double *lnW,
                    int e_min, int nE, double beta, int split, double lo, double hi, int n_iter,
                    int n_jack, int n_threads, double *out);

#ifdef __cplusplus
}
#endif
#endif
