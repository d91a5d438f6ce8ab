/*
 * muca.h -- C ABI of the GB300 library for the parallel multicanonical (MUCA)
 * simulation of the three-dimensional Blume-Capel model.
 *
 * The method (Zierenberg, Fytas, Janke, "Parallel multicanonical study of the
 * three-dimensional Blume-Capel model"):
 *   Eq. 1   H = -J sum_<ij> s_i s_j + Delta sum_i s_i^2 = E_J + Delta E_Delta,
 *           s_i in {-1, 0, +1}, J = 1, L^3 simple-cubic lattice, periodic.
 *   Sec. II the weight exp(-beta Delta E_Delta) is replaced by W(E_Delta), adapted
 *           iteratively towards a flat E_Delta histogram; p walkers share W and
 *           their histograms are merged after every iteration.
 *   Eq. 3   time-series reweighting to any Delta at fixed beta.
 *   Eq. 6   C(Delta) = -beta (<E_J E_Delta> - <E_J><E_Delta>).
 *
 * Conventions of every entry point:
 *   - returns MUCA_OK (0) or a negative MUCA_ERR_* code; no exception or
 *     abort crosses the ABI; muca_last_error() gives a one-line reason;
 *   - a muca_ctx owns all device memory it allocates (freed by muca_destroy);
 *   - pointers passed in are borrowed for the duration of the call only;
 *     "host" pointers are ordinary CPU memory, "device" pointers are CUDA
 *     global-memory addresses on the context's device (e.g. a torch tensor's
 *     data_ptr());
 *   - work is issued on the context's CUDA stream (the one passed to
 *     muca_init); calls that return host data synchronise that stream;
 *   - walker ids are global over the groups of a context, in group order.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key
 * (global walker id, seed) and counter (site >> 2, sweep low, sweep high,
 * stream); stream 0 drives the updates and stream 1 the initial spins.  Each
 * 32-bit word serves one site (site & 3): bit 31 chooses the proposal (the
 * smaller or larger of the two other spin values), bits 0..30 are the uniform
 * draw u.  A proposal is accepted iff u < thr[E_Delta][d][dE_J] with
 * thr = 2^31 when x >= 0, else floor(exp(x) 2^31), x = -beta dE_J +
 * lnW[E_Delta + d] - lnW[E_Delta], d = s'^2 - s^2, and thr = 0 when E_Delta + d
 * leaves the window.  The table is built on the host in FP64.
 */
#ifndef MUCA_H
#define MUCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MUCA_OK 0
#define MUCA_ERR_INVALID_ARG (-1)
#define MUCA_ERR_CUDA (-2)
#define MUCA_ERR_OOM (-3)
#define MUCA_ERR_TIMEOUT (-4)
#define MUCA_ERR_TALLY_MISMATCH (-5)
#define MUCA_ERR_NOT_SUPPORTED (-6)
#define MUCA_ERR_WINDOW (-7)
#define MUCA_ERR_IO (-8)

/* Largest supported linear size (V = L^3 sites per walker). */
#define MUCA_MAX_L 64

/* Number of logical threshold entries per (E_Delta, d): dE_J = -12 .. 12. */
#define MUCA_NK 25
/* Largest |coupling| of the disordered model (muca_set_bonds). */
#define MUCA_MAX_JMAX 8

typedef struct muca_ctx muca_ctx;

/* One (L, T) group of walkers sharing one weight function W(E_Delta)
 * (Sec. II: walkers at the same temperature share W and merge histograms). */
typedef struct {
    int32_t L;         /* linear size, 2 <= L <= MUCA_MAX_L */
    double T;          /* temperature > 0, beta = 1 / T */
    int32_t n_walkers; /* >= 1 */
    int32_t e_min;     /* E_Delta window [e_min, e_max]; 0 <= e_min <= e_max <= L^3 */
    int32_t e_max;     /* a negative e_max means L^3 (the full range, Sec. II) */
} muca_group;

/* Lattice residency of the sweep kernel. */
#define MUCA_RES_AUTO 0   /* chosen by the autotuner (measured) */
#define MUCA_RES_GLOBAL 1 /* spins stay in HBM/L2, site-major walker-minor */
#define MUCA_RES_SMEM 2   /* each block keeps its walkers' lattices in shared memory */
#define MUCA_RES_SPLIT 3  /* spins in HBM/L2; each block has one warp that runs the
                             walkers' Metropolis chains and three warps that prepare
                             and finish the rows around it (L % 4 == 0, 8 <= L <= 48;
                             other sizes fall back to MUCA_RES_GLOBAL) */
#define MUCA_RES_SCAN 4   /* spins in HBM/L2; one lane per packed word of a row
                             (a segment of the next power of 2 >= L / 4 lanes per
                             walker) resolves every row of L sites at once: the
                             acceptances that depend on the left neighbour by a
                             prefix scan of bit masks, re-run from each accepted
                             move that changes E_Delta (L % 4 == 0, 4 <= L <= 64;
                             other sizes fall back to MUCA_RES_GLOBAL) */
#define MUCA_RES_BONDS 5  /* the disordered model's kernel (muca_set_bonds): one thread
                             per walker, couplings per bond; reported by
                             muca_get_config, not selectable in muca_options */

/* debug_flags bits */
#define MUCA_DEBUG_TALLY_CHECK 1 /* recompute E_J, E_Delta, M after every sweep call */

typedef struct {
    uint32_t seed;             /* Philox key word 1 */
    int32_t debug_flags;       /* MUCA_DEBUG_* bits */
    int32_t residency;         /* MUCA_RES_* */
    int32_t walkers_per_block; /* 0 = automatic; else 1 .. 32; a block is one warp, so
                                  walkers_per_block x lanes_per_walker <= 32 (== 32 for
                                  global residency); fixed by L for MUCA_RES_SCAN */
    int32_t lanes_per_walker;  /* 0 = automatic; else 1, 2, 4 or 8 threads serve one
                                  walker (they share its random numbers); fixed by L
                                  (1 .. 16) for MUCA_RES_SCAN */
    int32_t shard_rank;        /* walker sharding over contexts (e.g. one per GPU):
                                  with shard_count = N > 1 the context holds shard
                                  shard_rank (0 .. N-1) of every group, walkers
                                  [floor(W r / N), floor(W (r + 1) / N)) of its W
                                  (n_walkers is the group's total), with the global
                                  walker ids of the unsharded context; 0 / 0 = all */
    int32_t shard_count;
} muca_options;

/* ---------------------------------------------------------------- lifetime */

/* Create a context: allocates the spins (int8, site-major walker-minor), the
 * running tallies (E_J, E_Delta, M as int32), the histograms and the threshold
 * tables of every group on the current CUDA device, draws the initial spins
 * i.i.d. uniform on {-1, 0, +1} (Philox stream 1), computes the tallies, sets
 * lnW = 0 and uploads the first table.  stream: a cudaStream_t (NULL = the
 * legacy default stream).  If an initial E_Delta lies outside a restricted
 * window, the group must receive a state through muca_set_state before the
 * first sweep (muca_sweep_iter and muca_run_graph fail with MUCA_ERR_WINDOW
 * until then).  On error *out is NULL. */
int muca_init(const muca_group *groups, int n_groups, const muca_options *opt,
              void *stream, muca_ctx **out);

/* Release every resource of ctx (NULL is accepted). */
void muca_destroy(muca_ctx *ctx);

/* Reason for the most recent failure on ctx; with ctx == NULL, the most recent
 * failure of any call in this thread (e.g. of muca_init).  Never NULL. */
const char *muca_last_error(const muca_ctx *ctx);

/* Wait for all work issued on the context's stream. */
int muca_sync(muca_ctx *ctx);

/* ----------------------------------------------------------- the hot path */

/* n_sweeps typewriter Metropolis sweeps of every walker of every group (Sec. II
 * acceptance with the current table).  After each sweep the walker's E_Delta
 * is added to its group's histogram (one entry per walker per sweep).  With
 * record != 0 each sweep also appends (E_J, E_Delta, M) of every walker to the
 * time series, which must have room (muca_reserve_timeseries).  Asynchronous
 * unless MUCA_DEBUG_TALLY_CHECK is set. */
int muca_sweep_iter(muca_ctx *ctx, int n_sweeps, int record);

/* The merge and weight update of one MUCA iteration for every group (Sec. II):
 * the merged histogram H is read back, the flatness of H over the group's
 * active window is recorded (muca_get_flatness), lnW is updated in FP64 on
 * the host by the context's weight recursion (muca_set_recursion; by default
 * lnW[E] -= ln H[E] wherever H[E] > 0), an adaptive window grows if H was
 * flat over it (muca_set_window), the threshold table is rebuilt in FP64 and
 * uploaded, and H is cleared.  Synchronises the stream. */
int muca_merge_update(muca_ctx *ctx);

/* The batched form: n_iters x (sweeps_per_iter sweeps of all groups in one
 * launch, then merge + update of every group) captured by each call as one
 * CUDA graph (the FP64 update runs in a host node) and launched once; the
 * graph is destroyed before the call returns (its kernels carry the call's
 * sweep counter).  Results are bit-identical to calling muca_sweep_iter +
 * muca_merge_update n_iters times.  Synchronises the stream. */
int muca_run_graph(muca_ctx *ctx, int n_iters, int sweeps_per_iter);

/* ------------------------------------------------ weight-iteration variants */

/* Weight recursions.  Sec. II adapts W iteratively by the recursion of the
 * multicanonical method it cites (Berg and Neuhaus; Janke) without printing
 * it.  With r(E) = lnW[E+1] - lnW[E] the ratio of neighbouring weights:
 *   MUCA_REC_PLAIN        lnW[E] -= ln H[E] wherever H[E] > 0 (the default).
 *   MUCA_REC_ACCUMULATED  the accumulated, error-weighted form: every
 *       iteration estimates r(E) as r(E) + ln H[E] - ln H[E+1] with inverse
 *       variance p(E) = H[E] H[E+1] / (H[E] + H[E+1]); then acc(E) += p(E) and
 *       r(E) += (p(E) / acc(E)) (ln H[E] - ln H[E+1]), which keeps r(E) the
 *       p-weighted mean of the estimates of every iteration that hit both
 *       bins.  In an iteration with H[E] = 0 or H[E+1] = 0 the pair takes the
 *       plain step instead (the empty bin counted as 1, which is what the
 *       plain recursion does to the ratio) and acc(E) is unchanged.  lnW[0]
 *       is kept and lnW[E+1] = lnW[E] + r(E). */
#define MUCA_REC_PLAIN 0
#define MUCA_REC_ACCUMULATED 1

/* One weight update on the host; no device work, no context (the merge of
 * muca_merge_update and muca_run_graph runs this same function).
 *   kind   MUCA_REC_PLAIN or MUCA_REC_ACCUMULATED
 *   hist   host uint64 [n_e]: the merged histogram of the iteration
 *   lnW    host FP64 [n_e], updated in place
 *   acc    host FP64 [n_e - 1]: the accumulated pair weights, updated in place
 *          (zeros before the first iteration); unused, and may be NULL, for
 *          MUCA_REC_PLAIN or n_e == 1
 * MUCA_ERR_INVALID_ARG for an unknown kind, n_e < 1 or a missing array. */
int muca_weight_update(int32_t kind, int32_t n_e, const uint64_t *hist, double *lnW,
                       double *acc);

/* The acceptance-threshold table of a weight function on the host; no device
 * work, no context (the table that muca_merge_update builds and uploads).
 *   L, T, e_min, e_max   the group (window [e_min, e_max], e_max >= e_min)
 *   lnW                  host FP64 [e_max - e_min + 1]
 *   out                  host uint32 [n_e][3][MUCA_NK], index
 *                        [E_Delta - e_min][d + 1][dE_J + 12] (the layout of
 *                        muca_get_table; every entry follows the formula, also
 *                        for (d, dE_J) pairs that no move produces)
 * MUCA_ERR_INVALID_ARG for a bad size or window or a NULL array. */
int muca_build_table(int32_t L, double T, int32_t e_min, int32_t e_max, const double *lnW,
                     uint32_t *out);

/* Select the weight recursion of every group of ctx (MUCA_REC_*) and clear
 * the accumulated pair weights (muca_set_lnW clears a group's as well). */
int muca_set_recursion(muca_ctx *ctx, int32_t kind);

/* Flatness of the histogram H merged by the last weight update of group g
 * (muca_merge_update, muca_run_graph or muca_iterate) over the bins of the
 * active window it was sampled in (all n_e bins unless muca_set_window
 * restricted it): out host FP64 [3] = (min H / mean H, max H / mean H,
 * number of bins with H > 0), mean H = (sum H) / bins; zeros before the
 * first update or when H was empty. */
int muca_get_flatness(muca_ctx *ctx, int group, double *out);

/* The adaptive E_Delta window of the weight iteration.  The paper samples
 * one range, E_Delta in [0, V], and gives no rule for moving a window; this
 * is the library's reading of one.  The walkers of group g move in the active
 * window [lo, hi] inside [e_min, e_max]: a proposal whose E_Delta + d leaves
 * it is rejected (its thresholds are 0), as one leaving [e_min, e_max] is.
 * After each merge and weight update, if grow_flat > 0 and the merged
 * histogram had min H / mean H >= grow_flat over the window, the window grows
 * by grow_step bins on each side, clamped to [e_min, e_max]; each new bin
 * starts from the weight lnW of the old edge next to it, and the accumulated
 * pair weights (MUCA_REC_ACCUMULATED) of the pairs that contain a new bin
 * start from 0.  grow_flat = 0 keeps the window fixed.  Every walker's
 * current E_Delta must lie in [lo, hi] (else MUCA_ERR_WINDOW and nothing
 * changes), so a window set at the start usually spans the walkers' initial
 * E_Delta; a sharded run sets the same window, over all shards' walkers, on
 * every shard.  The table is rebuilt and uploaded; lnW is not changed.
 * MUCA_ERR_INVALID_ARG for lo > hi, a window outside [e_min, e_max], a
 * negative or non-finite grow_flat, or grow_flat > 0 with grow_step < 1.
 * Synchronises the stream.  get_window: out host int32 [2] = the current
 * (lo, hi). */
int muca_set_window(muca_ctx *ctx, int group, int32_t lo, int32_t hi, double grow_flat,
                    int32_t grow_step);
int muca_get_window(muca_ctx *ctx, int group, int32_t *out);

/* The disordered model.  The paper's outlook applies the method to the
 * Blume-Capel model with bond disorder (its random-bond version) without
 * fixing a distribution; this is the library's reading of it.  Every bond
 * carries a quenched integer coupling: E_J = -sum over the forward bonds
 * (i, mu) of J[3 i + mu] s_i s_{i+mu}, the local field of a site weighs each
 * of its six neighbours by the coupling of the bond between them.  E_Delta,
 * W(E_Delta), the histograms, windows, weight recursions and the reweighting
 * in Delta are the clean model's; every walker of the group shares the one
 * realisation.  Integer couplings keep E_J an integer; a bimodal ratio
 * r = J2 / J1 is reached by scaling (couplings q J at temperature q T and
 * field q Delta are the model at J, T, Delta).
 *   J      host int8 [L^3][3]: the couplings of the x, y, z forward bonds of
 *          site i = x + L (y + L z), each in [-jmax, jmax]; NULL returns the
 *          group to the clean model (J = 1)
 *   jmax   1 .. MUCA_MAX_JMAX: the acceptance table covers
 *          dE_J in [-12 jmax, 12 jmax] (rows of 24 jmax + 1 thresholds)
 * The couplings are copied; the running tallies are recomputed from the
 * current spins, the table is rebuilt from lnW, and the group's sweeps run
 * the disordered model's kernel (MUCA_RES_BONDS) from then on.  muca_get_table
 * and muca_set_table refuse such a group (MUCA_ERR_INVALID_ARG).
 * MUCA_ERR_INVALID_ARG for a coupling or jmax out of range.  Synchronises the
 * stream. */
int muca_set_bonds(muca_ctx *ctx, int group, const int8_t *J, int32_t jmax);

/* The disordered model's acceptance table on the host (no context):
 *   out host uint32 [n_e][3][24 jmax + 1], index
 *       [E_Delta - e_min][d + 1][dE_J + 12 jmax]
 * with the thresholds of muca_build_table.  MUCA_ERR_INVALID_ARG for a bad
 * size, window, jmax or a NULL array. */
int muca_build_table_bonds(int32_t L, double T, int32_t jmax, int32_t e_min, int32_t e_max,
                           const double *lnW, uint32_t *out);

/* Weight iteration until the histograms are flat: up to max_iters iterations
 * of sweeps_per_iter sweeps followed by muca_merge_update; stops after the
 * first iteration at which min H / mean H >= flat_min for every group and
 * every group's histogram was taken over its whole [e_min, e_max] (its active
 * window was already full when the iteration ran).
 * *n_done receives the number of iterations run (host int32; max_iters if the
 * histograms never became flat, which is not an error).  Synchronises the
 * stream. */
int muca_iterate(muca_ctx *ctx, int32_t max_iters, int32_t sweeps_per_iter, double flat_min,
                 int32_t *n_done);

/* Time-series reweighting (Eq. 3) of n = n_rows x row_len samples to every
 * Delta_k of delta_grid, with C from Eq. 6.
 *   e_j, e_d, m   device int32; sample (r, c) is at [r * row_stride + c]
 *                 (so the context's [sample][field][walker] series is
 *                 e_j = base, e_d = base + W, m = base + 2 W, row_len = W,
 *                 row_stride = 3 W; plain arrays have n_rows = 1)
 *   lnW           host FP64 [n_e], indexed by E_Delta - e_min; every sample
 *                 must satisfy e_min <= E_Delta < e_min + n_e
 *   beta, V       inverse temperature and number of sites
 *   delta_grid    host FP64 [n_grid]
 *   precision     64: FP64 arithmetic; 32: FP32 arithmetic (max-shifted
 *                 exponents carried as float pairs, Kahan-compensated sums)
 *   out           host FP64 [n_grid][5]: <E_J>, <E_Delta>, C,
 *                 chi = beta V (<m^2> - <|m|>^2), U4 = 1 - <m^4> / (3 <m^2>^2),
 *                 m = M / V
 *   stream        cudaStream_t for the work (NULL = legacy default stream)
 * Working memory (per-bin sums, and up to 8 bytes per sample for at most 2^26
 * samples at a time) comes from a device memory pool that the library creates
 * on the device at the first call and keeps until the process exits; the pool
 * keeps what it has held, so it holds the largest call's working memory.
 * Synchronises the stream before returning. */
int muca_reweight(const int32_t *e_j, const int32_t *e_d, const int32_t *m, int64_t n_rows,
                  int32_t row_len, int64_t row_stride, const double *lnW, int32_t e_min,
                  int32_t n_e, double beta, int32_t V, const double *delta_grid, int32_t n_grid,
                  int32_t precision, double *out, void *stream);

/* muca_reweight without any device allocation (the paper has no counterpart:
 * this is a deployment variant of the same computation).  For callers that
 * cannot allocate device memory at the point of the call: services that
 * reserve all device memory up front, real-time loops that cannot afford an
 * allocator's synchronisation, bindings without a device allocator.
 * Arguments, layouts, results and errors are those of muca_reweight.  Its
 * working memory is a fixed 4 MiB array in the library's device memory,
 * present on every GPU that loads the library until the process exits; this
 * covers n_e <= 32769 (an L = 32 lattice) with n_grid <= 4096 in either
 * precision, and larger problems fail with MUCA_ERR_INVALID_ARG.  The first
 * call on a device looks the array's address up (cudaGetSymbolAddress with
 * that device current) and keeps it; make that first call before any stream
 * capture, and do not call this entry point on a device after
 * cudaDeviceReset of that device.  All calls share the array and it keeps the
 * last call's contents (the parts that must start at zero are cleared by each
 * call); calls whose GPU work overlaps race on it and must be ordered.
 * Synchronises the stream. */
int muca_reweight_noalloc(const int32_t *e_j, const int32_t *e_d, const int32_t *m,
                          int64_t n_rows, int32_t row_len, int64_t row_stride, const double *lnW,
                          int32_t e_min, int32_t n_e, double beta, int32_t V,
                          const double *delta_grid, int32_t n_grid, int32_t precision,
                          double *out, void *stream);

/* Pseudo-transition point (Sec. III): Delta*_L, the crystal field where C of
 * Eq. 6 is largest, and C*_L = C(Delta*_L), with jackknife errors.  Delta*_L
 * is the zero crossing of dC/dDelta = beta^2 <(E_J - <E_J>)(E_Delta - <E_Delta>)^2>,
 * found by n_iter bisection steps in [delta_lo, delta_hi] with time-series
 * reweighting (Eq. 3): each step keeps the half whose ends still bracket it
 * (mid = lo + (hi - lo) / 2; dC/dDelta(mid) > 0 moves lo, else hi), and the
 * result is the last interval's midpoint.  This is done for the full series
 * and for n_jack subsets (0, or 2 .. 1024) that each leave out one block of
 * rows [i n_rows / n_jack, (i + 1) n_rows / n_jack).
 *   e_j, e_d      device int32, sample (r, c) at [r * row_stride + c]; a row
 *                 is one sweep of all walkers (as muca_reweight)
 *   lnW, e_min, n_e, beta   as muca_reweight
 *   n_iter        bisection steps (0 .. 200; 60 reach FP64 resolution)
 *   out           host FP64 [4 + 2 n_jack]: Delta*_L, its jackknife error,
 *                 C*_L, its jackknife error (errors 0 when n_jack = 0), then
 *                 (Delta*, C*) of each subset; the error of x is
 *                 sqrt((w - 1) / w sum_i (x_i - mean x_i)^2), w = n_jack
 * MUCA_ERR_INVALID_ARG when [delta_lo, delta_hi] does not bracket the maximum
 * for the full series or a subset (dC/dDelta must be > 0 at delta_lo and < 0
 * at delta_hi); MUCA_ERR_WINDOW for a sample outside the window.  Allocates
 * its scratch with cudaMallocAsync on the stream; synchronises the stream. */
int muca_find_peak(const int32_t *e_j, const int32_t *e_d, int64_t n_rows, int32_t row_len,
                   int64_t row_stride, const double *lnW, int32_t e_min, int32_t n_e,
                   double beta, double delta_lo, double delta_hi, int32_t n_iter, int32_t n_jack,
                   double *out, void *stream);

/* Equal-height field and barrier (Sec. II, Eq. of B in Sec. IV): the series'
 * reweighted E_Delta distribution at field Delta is
 * P(E) ~ n(E) exp(-beta Delta E) / W(E), n(E) its samples in bin E.  Its peaks
 * are the highest occupied bins below and at or above split; Delta_eqh is
 * where they are equally high, found by n_iter bisection steps in
 * [delta_lo, delta_hi] (the lower-E peak must be lower at delta_lo and higher
 * at delta_hi; mid = lo + (hi - lo) / 2, lower at mid moves lo, else hi; the
 * result is the last midpoint; ties between bins go to the smaller E), and
 * B = ln(P_max / P_min) / (2 beta Delta_eqh) with P_min the lowest occupied
 * bin between the peaks.  Full series and n_jack leave-one-block-out subsets
 * as muca_find_peak.
 *   e_d, n_rows, row_len, row_stride, lnW, e_min, n_e, beta   as muca_find_peak
 *   out   host FP64 [7 + 2 n_jack]: Delta_eqh, its jackknife error, B, its
 *         jackknife error, E of the lower peak, E of the upper peak, E of the
 *         minimum (full series), then (Delta_eqh, B) of each subset
 * MUCA_ERR_INVALID_ARG when the interval does not bracket Delta_eqh for the
 * full series or a subset; MUCA_ERR_WINDOW for a sample outside the window.
 * Allocates its scratch with cudaMallocAsync on the stream; synchronises the
 * stream. */
int muca_equal_height(const int32_t *e_d, int64_t n_rows, int32_t row_len, int64_t row_stride,
                      const double *lnW, int32_t e_min, int32_t n_e, double beta, int32_t split,
                      double delta_lo, double delta_hi, int32_t n_iter, int32_t n_jack,
                      double *out, void *stream);

/* ------------------------------------------------------------ time series */

/* Reserve room for n_samples recorded sweeps per walker (device memory,
 * [sample][3][n_walkers] int32 per group) and reset the recorded length to 0.
 * Asking again for the current capacity only rewinds (no allocation). */
int muca_reserve_timeseries(muca_ctx *ctx, int64_t n_samples);

/* Recorded length (samples per walker) and the device address of group g's
 * series, laid out [sample][field][walker] with field 0 = E_J, 1 = E_Delta,
 * 2 = M and a walker stride of n_walkers of the group. */
int muca_timeseries_device(muca_ctx *ctx, int group, const int32_t **dev, int64_t *n_samples);

/* Copy group g's series to host int32 [n_samples][3][n_walkers]. */
int muca_get_timeseries(muca_ctx *ctx, int group, int32_t *out);

/* ----------------------------------------------------- inspection / parity */

/* Number of sweeps done so far by group g (the next sweep's Philox index). */
int muca_get_sweep_count(muca_ctx *ctx, int group, uint64_t *out);

/* lnW of group g, host FP64 [n_e]. set replaces it, clears the accumulated
 * pair weights of the weight recursion and rebuilds the table. */
int muca_get_lnW(muca_ctx *ctx, int group, double *out);
int muca_set_lnW(muca_ctx *ctx, int group, const double *in);

/* Threshold table of group g in the logical layout, host uint32
 * [n_e][3][MUCA_NK], index [E_Delta - e_min][d + 1][dE_J + 12].  set uploads a
 * given table (its d = 0 entries must not depend on E_Delta). */
int muca_get_table(muca_ctx *ctx, int group, uint32_t *out);
int muca_set_table(muca_ctx *ctx, int group, const uint32_t *in);

/* Merged histogram of group g since the last merge, host uint64 [n_e]. */
int muca_get_hist(muca_ctx *ctx, int group, uint64_t *out);
int muca_set_hist(muca_ctx *ctx, int group, const uint64_t *in);

/* The same with device buffers (uint64 [n_e] on the context's device), for
 * merging the histograms of walker shards with a device all-reduce (Sec. II:
 * the walkers' histograms are summed after every iteration).  get copies the
 * histogram into dev_out and synchronises the context's stream; set copies
 * dev_in over the histogram on the context's stream (dev_in must be complete
 * when it is called, e.g. the caller's all-reduce stream synchronised). */
int muca_get_hist_device(muca_ctx *ctx, int group, uint64_t *dev_out);
int muca_set_hist_device(muca_ctx *ctx, int group, const uint64_t *dev_in);

/* Walkers of group g held by this context (its shard) and the global Philox
 * id of the first of them; either output may be NULL. */
int muca_get_walkers(muca_ctx *ctx, int group, int32_t *n_local, uint32_t *first_id);

/* Walker state of group g: spins host int8 [n_walkers][L^3] (site i =
 * x + L (y + L z)), tallies host int32 [n_walkers][3] = (E_J, E_Delta, M).
 * Either output may be NULL.  set_state uploads spins and recomputes the
 * tallies on the device; fails with MUCA_ERR_WINDOW if an E_Delta leaves the
 * active window (muca_set_window), MUCA_ERR_INVALID_ARG if a spin is not in
 * {-1, 0, +1}. */
int muca_get_state(muca_ctx *ctx, int group, int8_t *spins, int32_t *tallies);
int muca_set_state(muca_ctx *ctx, int group, const int8_t *spins);

/* Recompute E_J, E_Delta, M of every walker on the device and compare with the
 * running tallies: MUCA_OK or MUCA_ERR_TALLY_MISMATCH. */
int muca_check_tallies(muca_ctx *ctx);

/* Kernel configuration chosen for group g: residency (MUCA_RES_GLOBAL,
 * MUCA_RES_SMEM or MUCA_RES_SPLIT), walkers per block and lanes per walker
 * (0 for MUCA_RES_SPLIT).  Any output may be NULL. */
int muca_get_config(muca_ctx *ctx, int group, int32_t *residency, int32_t *walkers_per_block,
                    int32_t *lanes_per_walker);

/* Checkpoint / restore: spins, tallies, lnW, histograms, the weight
 * recursion with its accumulated pair weights, the active window with its
 * growth rule, the couplings of the disordered model, sweep counters and the
 * seed, to / from a file.  Philox is
 * counter-based, so a restored run continues bit-identically.  restore
 * requires a context with the same groups and the same shard
 * (muca_options.shard_rank / shard_count); it also reads files of the earlier
 * formats without the couplings (the clean model), without the window (the
 * fixed window [e_min, e_max]), without the
 * shard record (every walker of a group) or without the recursion (plain
 * recursion, no accumulated weights). */
int muca_checkpoint(muca_ctx *ctx, const char *path);
int muca_restore(muca_ctx *ctx, const char *path);

#ifdef __cplusplus
}
#endif
#endif /* MUCA_H */
