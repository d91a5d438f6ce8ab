/*
 * muca_oracle.c -- plain CPU oracle for the parallel multicanonical (MUCA)
 * Blume-Capel hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library; it is written to be read against the paper, not to be
 * fast: every random word is regenerated where it is used, every neighbour sum
 * is taken with explicit modular coordinates, and the table and the
 * reweighting follow their definitions term by term.
 *
 * What the paper fixes (Zierenberg, Fytas, Janke, "Parallel multicanonical
 * study of the three-dimensional Blume-Capel model"):
 *   - Eq. 1: H = -J sum_<ij> s_i s_j + Delta sum_i s_i^2 = E_J + Delta E_Delta,
 *     s_i in {-1, 0, +1}, J = 1, k_B = 1, periodic simple-cubic lattice (Sec. I).
 *   - Sec. II: the Boltzmann factor exp(-beta E_J) exp(-beta Delta E_Delta) is
 *     replaced by exp(-beta E_J) W(E_Delta); W is adapted iteratively to a flat
 *     E_Delta histogram; p walkers share W and their histograms are merged.
 *   - Sec. II, Eq. 3: time-series reweighting to (beta, Delta) with the factor
 *     exp(-beta Delta E_Delta) / W(E_Delta).
 *   - Eq. 6: C(Delta) = -beta (<E_J E_Delta> - <E_J><E_Delta>).
 *   - Sec. II: E_Delta is an integer in [0, V].
 *
 * Readings where the paper is silent (each one is also a decision the CUDA
 * library takes independently):
 *   R1 site index i = x + L (y + L z); E_J sums the three forward bonds of every
 *      site (at L = 2 the two bonds between a pair are both counted, matching
 *      the six-neighbour local field).
 *   R2 single-site Metropolis in typewriter order i = 0 .. V-1; the proposal is
 *      one of the two values different from s_i, picked with probability 1/2.
 *   R3 random numbers: Philox4x32-10 with key (walker id, seed) and counter
 *      (site >> 2, sweep low word, sweep high word, stream); stream 0 drives the
 *      updates, stream 1 the initial spins.  Each 32-bit output word serves one
 *      site (site & 3 selects the word): bit 31 picks the proposal (0 = the
 *      smaller, 1 = the larger of the two other values), bits 0..30 are the
 *      uniform draw u in [0, 2^31).
 *   R4 acceptance: the proposal is rejected if E_Delta + d leaves the window
 *      [e_min, e_max]; otherwise it is accepted iff u < thr[E_Delta][d][dE_J]
 *      with thr = 2^31 when x >= 0 and floor(exp(x) 2^31) otherwise, where
 *      x = -beta dE_J + (lnW[E_Delta + d] - lnW[E_Delta]) in FP64.  thr is 0 when
 *      E_Delta + d lies outside the window.
 *   R5 one histogram entry per walker per sweep, after the sweep.
 *   R6 weight recursion lnW <- lnW - ln H where H > 0, starting from lnW = 0
 *      (the paper cites the standard recursion without printing it).
 *   R7 the global sweep index counts every sweep of a walker from 0 (weight
 *      iterations first, then measurement sweeps).
 *   R8 chi = beta V (<m^2> - <|m|>^2) and U4 = 1 - <m^4>/(3 <m^2>^2), m = M/V
 *      (the paper names chi without defining it and does not use U4).
 *   R9, R10 (rounding of the reweighting) are stated where they are used.
 *   R13 the accumulated, error-weighted form of the weight recursion and its
 *       rule for empty bins are stated at or_update_lnW_acc.
 *   R15 the adaptive E_Delta window is stated at or_muca_run_win.
 *   R16 the disordered model (quenched bond couplings) is stated at
 *       or_energies_bonds.
 */
#include "muca_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (SC'11, "Parallel random     */
/* numbers: as easy as 1, 2, 3"): ten rounds of two 32x32->64 multiplies,    */
/* with a Weyl-sequence key schedule between rounds.                          */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t p0 = (uint64_t)mult0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)mult1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* The random word of site i in sweep s on the given stream (reading R3). */
static uint32_t site_word(uint32_t seed, uint32_t walker_id, uint64_t sweep, int64_t site,
                          uint32_t stream)
{
    uint32_t ctr[4], key[2], r[4];
    ctr[0] = (uint32_t)(site >> 2);
    ctr[1] = (uint32_t)(sweep & 0xFFFFFFFFu);
    ctr[2] = (uint32_t)(sweep >> 32);
    ctr[3] = stream;
    key[0] = walker_id;
    key[1] = seed;
    or_philox4x32_10(ctr, key, r);
    return r[site & 3];
}

/* ------------------------------------------------------------------------ */
/* Lattice (Eq. 1, reading R1).                                               */
/* ------------------------------------------------------------------------ */
static int64_t site_of(int L, int x, int y, int z)
{
    return (int64_t)x + (int64_t)L * ((int64_t)y + (int64_t)L * (int64_t)z);
}

static int wrap(int a, int L) { return ((a % L) + L) % L; }

/* Sum of the six nearest neighbours of (x, y, z) as currently stored. */
static int local_field(int L, const int8_t *s, int x, int y, int z)
{
    int h = 0;
    h += s[site_of(L, wrap(x + 1, L), y, z)];
    h += s[site_of(L, wrap(x - 1, L), y, z)];
    h += s[site_of(L, x, wrap(y + 1, L), z)];
    h += s[site_of(L, x, wrap(y - 1, L), z)];
    h += s[site_of(L, x, y, wrap(z + 1, L))];
    h += s[site_of(L, x, y, wrap(z - 1, L))];
    return h;
}

int or_energies(int L, const int8_t *s, int64_t out[3])
{
    if (L < 2 || !s || !out) return OR_ERR_ARG;
    int64_t ej = 0, ed = 0, m = 0;
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int si = s[site_of(L, x, y, z)];
                ej -= si * s[site_of(L, wrap(x + 1, L), y, z)];
                ej -= si * s[site_of(L, x, wrap(y + 1, L), z)];
                ej -= si * s[site_of(L, x, y, wrap(z + 1, L))];
                ed += si * si;
                m += si;
            }
    out[0] = ej;
    out[1] = ed;
    out[2] = m;
    return OR_OK;
}

int or_init_spins(int L, uint32_t seed, uint32_t walker_id, int8_t *spins)
{
    if (L < 2 || !spins) return OR_ERR_ARG;
    int64_t V = (int64_t)L * L * L;
    for (int64_t i = 0; i < V; ++i) {
        uint32_t w = site_word(seed, walker_id, 0, i, 1u);
        /* floor(3 w / 2^32) is uniform on {0, 1, 2} up to 2^-32 bias */
        int v = (int)(((uint64_t)w * 3u) >> 32);
        spins[i] = (int8_t)(v - 1);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Acceptance table (reading R4).                                             */
/* ------------------------------------------------------------------------ */
static uint32_t threshold_of(double x)
{
    if (x >= 0.0) return 0x80000000u;
    double p = exp(x);
    double t = floor(p * 2147483648.0);
    if (t >= 2147483648.0) return 0x80000000u;
    return (uint32_t)t;
}

int or_build_table(int L, double T, int e_min, int e_max, const double *lnW, uint32_t *thr)
{
    if (L < 2 || !(T > 0.0) || !lnW || !thr) return OR_ERR_ARG;
    int64_t V = (int64_t)L * L * L;
    if (e_min < 0 || e_max > V || e_min > e_max) return OR_ERR_ARG;
    double beta = 1.0 / T;
    int nE = e_max - e_min + 1;
    for (int e = 0; e < nE; ++e) {
        for (int d = -1; d <= 1; ++d) {
            for (int dej = -12; dej <= 12; ++dej) {
                uint32_t t;
                int en = e + d;
                if (en < 0 || en >= nE) {
                    t = 0u;
                } else {
                    double x = -(beta * (double)dej) + (lnW[en] - lnW[e]);
                    t = threshold_of(x);
                }
                thr[((int64_t)e * 3 + (d + 1)) * OR_NK + (dej + 12)] = t;
            }
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Typewriter Metropolis sweeps (Sec. II; readings R2-R5, R7).                */
/* ------------------------------------------------------------------------ */
int or_sweeps(int L, int e_min, int e_max, const uint32_t *thr, uint32_t seed,
              uint32_t walker_id, uint64_t sweep0, int n_sweeps, int8_t *spins,
              int32_t tallies[3], uint64_t *hist, int32_t *ts, int check)
{
    if (L < 2 || !thr || !spins || !tallies || n_sweeps < 0) return OR_ERR_ARG;
    int64_t ej = tallies[0], ed = tallies[1], m = tallies[2];
    if (ed < e_min || ed > e_max) return OR_ERR_WINDOW;
    for (int k = 0; k < n_sweeps; ++k) {
        uint64_t sweep = sweep0 + (uint64_t)k;
        for (int z = 0; z < L; ++z)
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) {
                    int64_t i = site_of(L, x, y, z);
                    uint32_t w = site_word(seed, walker_id, sweep, i, 0u);
                    uint32_t b = w >> 31;
                    uint32_t u = w & 0x7FFFFFFFu;
                    int s = spins[i];
                    /* the two values different from s, in ascending order */
                    int other[2], n = 0;
                    for (int v = -1; v <= 1; ++v)
                        if (v != s) other[n++] = v;
                    int sp = other[b];
                    int h = local_field(L, spins, x, y, z);
                    int dej = -(sp - s) * h;
                    int d = sp * sp - s * s;
                    int64_t en = ed + d;
                    if (en < e_min || en > e_max) continue;
                    uint32_t t = thr[((ed - e_min) * 3 + (d + 1)) * OR_NK + (dej + 12)];
                    if (u < t) {
                        spins[i] = (int8_t)sp;
                        ej += dej;
                        ed = en;
                        m += sp - s;
                    }
                }
        if (hist) hist[ed - e_min] += 1;
        if (ts) {
            ts[3 * (int64_t)k + 0] = (int32_t)ej;
            ts[3 * (int64_t)k + 1] = (int32_t)ed;
            ts[3 * (int64_t)k + 2] = (int32_t)m;
        }
        if (check) {
            int64_t e[3];
            or_energies(L, spins, e);
            if (e[0] != ej || e[1] != ed || e[2] != m) return OR_ERR_TALLY;
        }
    }
    tallies[0] = (int32_t)ej;
    tallies[1] = (int32_t)ed;
    tallies[2] = (int32_t)m;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Reading R16, the disordered model.  The paper's outlook applies the method */
/* to the Blume-Capel model with bond disorder (its random-bond version) and  */
/* names no distribution or strength.  Here every bond carries its own        */
/* quenched coupling: E_J = -sum_<ij> J_ij s_i s_j, with J[3 i + mu] the       */
/* coupling of the forward bond from site i in direction mu (x, y, z) and     */
/* every J an integer in [-jmax, jmax] (jmax <= 8).  Integer couplings keep   */
/* E_J an integer; a ratio r = J2 / J1 of a bimodal distribution is reached   */
/* by scaling: couplings q J at temperature q T and field q Delta are the     */
/* model at (J, T, Delta).  E_Delta, the weights W(E_Delta) and the           */
/* reweighting in Delta are those of the clean model; all walkers of a group  */
/* share one realisation.  J = 1 everywhere is the clean model.               */
/* The acceptance table of R4 is indexed by dE_J in [-12 jmax, 12 jmax]:      */
/* thr[(E - e_min) * 3 + d + 1][dE_J + 12 jmax], row length 24 jmax + 1.      */
/* ------------------------------------------------------------------------ */
static int bonds_ok(int L, const int8_t *J, int jmax)
{
    if (!J || jmax < 1 || jmax > OR_MAX_JMAX) return 0;
    int64_t V = (int64_t)L * L * L;
    for (int64_t k = 0; k < 3 * V; ++k)
        if (J[k] < -jmax || J[k] > jmax) return 0;
    return 1;
}

/* Coupling-weighted sum of the six neighbours of (x, y, z): the three forward
 * bonds of the site and the forward bonds of its three backward neighbours. */
static int bond_field(int L, const int8_t *s, const int8_t *J, int x, int y, int z)
{
    int64_t i = site_of(L, x, y, z);
    int64_t xm = site_of(L, wrap(x - 1, L), y, z);
    int64_t ym = site_of(L, x, wrap(y - 1, L), z);
    int64_t zm = site_of(L, x, y, wrap(z - 1, L));
    int h = 0;
    h += J[3 * i + 0] * s[site_of(L, wrap(x + 1, L), y, z)];
    h += J[3 * xm + 0] * s[xm];
    h += J[3 * i + 1] * s[site_of(L, x, wrap(y + 1, L), z)];
    h += J[3 * ym + 1] * s[ym];
    h += J[3 * i + 2] * s[site_of(L, x, y, wrap(z + 1, L))];
    h += J[3 * zm + 2] * s[zm];
    return h;
}

int or_energies_bonds(int L, const int8_t *s, const int8_t *J, int64_t out[3])
{
    if (L < 2 || !s || !J || !out) return OR_ERR_ARG;
    int64_t ej = 0, ed = 0, m = 0;
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int64_t i = site_of(L, x, y, z);
                int si = s[i];
                ej -= J[3 * i + 0] * si * s[site_of(L, wrap(x + 1, L), y, z)];
                ej -= J[3 * i + 1] * si * s[site_of(L, x, wrap(y + 1, L), z)];
                ej -= J[3 * i + 2] * si * s[site_of(L, x, y, wrap(z + 1, L))];
                ed += si * si;
                m += si;
            }
    out[0] = ej;
    out[1] = ed;
    out[2] = m;
    return OR_OK;
}

int or_build_table_bonds(int L, double T, int jmax, int e_min, int e_max, const double *lnW,
                         uint32_t *thr)
{
    if (L < 2 || !(T > 0.0) || !lnW || !thr || jmax < 1 || jmax > OR_MAX_JMAX) return OR_ERR_ARG;
    int64_t V = (int64_t)L * L * L;
    if (e_min < 0 || e_max > V || e_min > e_max) return OR_ERR_ARG;
    double beta = 1.0 / T;
    int nE = e_max - e_min + 1, nj = 24 * jmax + 1;
    for (int e = 0; e < nE; ++e)
        for (int d = -1; d <= 1; ++d)
            for (int dej = -12 * jmax; dej <= 12 * jmax; ++dej) {
                uint32_t t;
                int en = e + d;
                if (en < 0 || en >= nE) {
                    t = 0u;
                } else {
                    double x = -(beta * (double)dej) + (lnW[en] - lnW[e]);
                    t = threshold_of(x);
                }
                thr[((int64_t)e * 3 + (d + 1)) * nj + (dej + 12 * jmax)] = t;
            }
    return OR_OK;
}

int or_sweeps_bonds(int L, const int8_t *J, int jmax, int e_min, int e_max, const uint32_t *thr,
                    uint32_t seed, uint32_t walker_id, uint64_t sweep0, int n_sweeps,
                    int8_t *spins, int32_t tallies[3], uint64_t *hist, int32_t *ts, int check)
{
    if (L < 2 || !thr || !spins || !tallies || n_sweeps < 0 || !bonds_ok(L, J, jmax))
        return OR_ERR_ARG;
    int nj = 24 * jmax + 1;
    int64_t ej = tallies[0], ed = tallies[1], m = tallies[2];
    if (ed < e_min || ed > e_max) return OR_ERR_WINDOW;
    for (int k = 0; k < n_sweeps; ++k) {
        uint64_t sweep = sweep0 + (uint64_t)k;
        for (int z = 0; z < L; ++z)
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) {
                    int64_t i = site_of(L, x, y, z);
                    uint32_t w = site_word(seed, walker_id, sweep, i, 0u);
                    uint32_t b = w >> 31;
                    uint32_t u = w & 0x7FFFFFFFu;
                    int s = spins[i];
                    int other[2], n = 0;
                    for (int v = -1; v <= 1; ++v)
                        if (v != s) other[n++] = v;
                    int sp = other[b];
                    int h = bond_field(L, spins, J, x, y, z);
                    int dej = -(sp - s) * h;
                    int d = sp * sp - s * s;
                    int64_t en = ed + d;
                    if (en < e_min || en > e_max) continue;
                    uint32_t t = thr[((ed - e_min) * 3 + (d + 1)) * nj + (dej + 12 * jmax)];
                    if (u < t) {
                        spins[i] = (int8_t)sp;
                        ej += dej;
                        ed = en;
                        m += sp - s;
                    }
                }
        if (hist) hist[ed - e_min] += 1;
        if (ts) {
            ts[3 * (int64_t)k + 0] = (int32_t)ej;
            ts[3 * (int64_t)k + 1] = (int32_t)ed;
            ts[3 * (int64_t)k + 2] = (int32_t)m;
        }
        if (check) {
            int64_t e[3];
            or_energies_bonds(L, spins, J, e);
            if (e[0] != ej || e[1] != ed || e[2] != m) return OR_ERR_TALLY;
        }
    }
    tallies[0] = (int32_t)ej;
    tallies[1] = (int32_t)ed;
    tallies[2] = (int32_t)m;
    return OR_OK;
}

int or_update_lnW(int nE, const uint64_t *H, double *lnW)
{
    if (nE <= 0 || !H || !lnW) return OR_ERR_ARG;
    for (int e = 0; e < nE; ++e)
        if (H[e] > 0) lnW[e] -= log((double)H[e]);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Accumulated, error-weighted weight recursion (reading R13).  Sec. II      */
/* adapts W iteratively by the recursion of the multicanonical method that   */
/* it cites (Berg and Neuhaus; Janke); this is that recursion's accumulated  */
/* form, restated from its published definition.  Iteration n estimates the  */
/* ratio of neighbouring weights r(E) = lnW(E+1) - lnW(E) from its histogram */
/* H, and the estimates of all iterations so far are averaged with weights   */
/* equal to their inverse variances:                                         */
/*   est(E) = r(E) + ln H(E) - ln H(E+1)      this iteration's estimate       */
/*   p(E)   = H(E) H(E+1) / (H(E) + H(E+1))   1 / variance of est(E)          */
/*   acc(E) <- acc(E) + p(E)                  accumulated weight              */
/*   r(E)   <- r(E) + (p(E) / acc(E)) (ln H(E) - ln H(E+1))                   */
/* so r stays the p-weighted mean of every estimate so far, taken over the  */
/* iterations that hit both bins of the pair.  A pair with an empty bin      */
/* takes the plain recursion's step instead, with the empty bin counted as 1 */
/* (r(E) += ln max(H(E), 1) - ln max(H(E+1), 1), what lnW -= ln H for H > 0  */
/* does to the ratio), and adds nothing to acc: the weights keep pushing     */
/* into unvisited bins as fast as the plain recursion, no pseudo-count       */
/* dilutes the first real estimates there, and the first iteration           */
/* (acc = 0) is exactly the plain step.                                       */
/* lnW at the first bin of the window is kept and lnW(E+1) = lnW(E) + r(E).  */
/* acc has nE - 1 entries (one per neighbouring pair), zero at the start.    */
/* ------------------------------------------------------------------------ */
int or_update_lnW_acc(int nE, const uint64_t *H, double *lnW, double *acc)
{
    if (nE <= 0 || !H || !lnW || (nE > 1 && !acc)) return OR_ERR_ARG;
    if (nE == 1) return OR_OK;
    double *r = (double *)malloc((size_t)(nE - 1) * sizeof(double));
    if (!r) return OR_ERR_NOMEM;
    for (int e = 0; e + 1 < nE; ++e) {
        const double h0 = (double)H[e], h1 = (double)H[e + 1];
        double re = lnW[e + 1] - lnW[e];
        if (H[e] > 0 && H[e + 1] > 0) {
            const double p = h0 * h1 / (h0 + h1);
            acc[e] = acc[e] + p;
            re = re + (p / acc[e]) * (log(h0) - log(h1));
        } else {
            re = re + (log(h0 > 1.0 ? h0 : 1.0) - log(h1 > 1.0 ? h1 : 1.0));
        }
        r[e] = re;
    }
    for (int e = 0; e + 1 < nE; ++e) lnW[e + 1] = lnW[e] + r[e];
    free(r);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* A whole run of one group: walkers are independent given the table, so the */
/* walkers of an iteration are split over threads; histograms are summed.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int L, e_min, e_max, check;
    const int8_t *J; /* couplings of the disordered model (R16), or NULL */
    int jmax;
    const uint32_t *thr;
    uint32_t seed, walker_id0;
    uint64_t sweep0;
    int n_sweeps;
    int w_begin, w_end;
    int8_t *spins;       /* [n_walkers][V] */
    int32_t *tallies;    /* [n_walkers][3] */
    uint64_t *hist;      /* [nE], private to the job */
    int32_t *ts;         /* [n_walkers][n_sweeps][3] or NULL */
    int status;
} sweep_job;

static void *sweep_job_run(void *arg)
{
    sweep_job *j = (sweep_job *)arg;
    int64_t V = (int64_t)j->L * j->L * j->L;
    j->status = OR_OK;
    for (int w = j->w_begin; w < j->w_end; ++w) {
        int8_t *sp = j->spins + (int64_t)w * V;
        int32_t *tl = j->tallies + 3 * (int64_t)w;
        int32_t *ts = j->ts ? j->ts + (int64_t)w * j->n_sweeps * 3 : NULL;
        uint32_t id = j->walker_id0 + (uint32_t)w;
        int rc = j->J ? or_sweeps_bonds(j->L, j->J, j->jmax, j->e_min, j->e_max, j->thr, j->seed,
                                        id, j->sweep0, j->n_sweeps, sp, tl, j->hist, ts, j->check)
                      : or_sweeps(j->L, j->e_min, j->e_max, j->thr, j->seed, id, j->sweep0,
                                  j->n_sweeps, sp, tl, j->hist, ts, j->check);
        if (rc != OR_OK) {
            j->status = rc;
            return NULL;
        }
    }
    return NULL;
}

static int sweep_all(int n_walkers, int n_threads, int nE, sweep_job proto, uint64_t *hist_sum)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_walkers) n_threads = n_walkers;
    sweep_job *jobs = (sweep_job *)calloc((size_t)n_threads, sizeof(sweep_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    uint64_t *h = (uint64_t *)calloc((size_t)n_threads * (size_t)nE, sizeof(uint64_t));
    if (!jobs || !tid || !h) {
        free(jobs);
        free(tid);
        free(h);
        return OR_ERR_NOMEM;
    }
    for (int t = 0; t < n_threads; ++t) {
        jobs[t] = proto;
        jobs[t].w_begin = (int)((int64_t)n_walkers * t / n_threads);
        jobs[t].w_end = (int)((int64_t)n_walkers * (t + 1) / n_threads);
        jobs[t].hist = h + (size_t)t * nE;
    }
    for (int t = 1; t < n_threads; ++t) pthread_create(&tid[t], NULL, sweep_job_run, &jobs[t]);
    sweep_job_run(&jobs[0]);
    for (int t = 1; t < n_threads; ++t) pthread_join(tid[t], NULL);
    int status = OR_OK;
    for (int t = 0; t < n_threads; ++t) {
        if (jobs[t].status != OR_OK) status = jobs[t].status;
        if (hist_sum)
            for (int e = 0; e < nE; ++e) hist_sum[e] += h[(size_t)t * nE + e];
    }
    free(jobs);
    free(tid);
    free(h);
    return status;
}

int or_muca_run(int L, double T, int n_walkers, int e_min, int e_max, uint32_t seed,
                uint32_t walker_id0, int n_iter, int sweeps_per_iter, int n_meas,
                double *lnW, uint64_t *hist_iter, int8_t *spins_out,
                int32_t *tallies_out, int32_t *ts, int check, int n_threads)
{
    return or_muca_run_rec(L, T, n_walkers, e_min, e_max, seed, walker_id0, n_iter,
                           sweeps_per_iter, n_meas, lnW, hist_iter, spins_out, tallies_out, ts,
                           check, n_threads, 0, NULL);
}

int or_muca_run_rec(int L, double T, int n_walkers, int e_min, int e_max, uint32_t seed,
                    uint32_t walker_id0, int n_iter, int sweeps_per_iter, int n_meas,
                    double *lnW, uint64_t *hist_iter, int8_t *spins_out,
                    int32_t *tallies_out, int32_t *ts, int check, int n_threads,
                    int recursion, double *acc)
{
    return or_muca_run_win(L, T, n_walkers, e_min, e_max, seed, walker_id0, n_iter,
                           sweeps_per_iter, n_meas, lnW, hist_iter, spins_out, tallies_out, ts,
                           check, n_threads, recursion, acc, e_min, e_max, 0.0, 0, NULL);
}

/* Reading R15, the adaptive E_Delta window (the paper samples one range,
 * [0, V], and gives no rule for moving a window; the weight iterations of the
 * recursions it cites start from where the walkers are).  The walkers move in
 * an active window [a, b] inside [e_min, e_max]: a proposal whose E_Delta + d
 * leaves [a, b] is rejected, as R4 rejects one leaving [e_min, e_max].  After
 * the iteration's merge and weight update (over all of [e_min, e_max]), if
 * grow_flat > 0 and the merged histogram over [a, b] has
 * min H / mean H >= grow_flat (mean H = sum H / (b - a + 1)), the window grows
 * by grow_step bins on each side, clamped to [e_min, e_max].  A new bin starts
 * from the weight of the old edge next to it (lnW copied outward from a and
 * from b), and the accumulated pair weights (R13) of the pairs that contain a
 * new bin start from 0: nothing has been measured there. */
static double window_flatness(const uint64_t *H, int a, int b)
{
    uint64_t lo = H[a], sum = 0;
    for (int e = a; e <= b; ++e) {
        if (H[e] < lo) lo = H[e];
        sum += H[e];
    }
    if (sum == 0) return 0.0;
    const double mean = (double)sum / (double)(b - a + 1);
    return (double)lo / mean;
}

int or_muca_run_win(int L, double T, int n_walkers, int e_min, int e_max, uint32_t seed,
                    uint32_t walker_id0, int n_iter, int sweeps_per_iter, int n_meas,
                    double *lnW, uint64_t *hist_iter, int8_t *spins_out,
                    int32_t *tallies_out, int32_t *ts, int check, int n_threads,
                    int recursion, double *acc, int win_lo, int win_hi, double grow_flat,
                    int grow_step, int32_t *win_iter)
{
    return or_muca_run_bonds(L, T, n_walkers, e_min, e_max, seed, walker_id0, n_iter,
                             sweeps_per_iter, n_meas, lnW, hist_iter, spins_out, tallies_out, ts,
                             check, n_threads, recursion, acc, win_lo, win_hi, grow_flat,
                             grow_step, win_iter, NULL, 0);
}

/* The table of the run: the clean one (R4) or the disordered one (R16). */
static void run_table(int L, double T, const int8_t *J, int jmax, int lo, int hi,
                      const double *lnW, uint32_t *thr)
{
    if (J)
        or_build_table_bonds(L, T, jmax, lo, hi, lnW, thr);
    else
        or_build_table(L, T, lo, hi, lnW, thr);
}

int or_muca_run_bonds(int L, double T, int n_walkers, int e_min, int e_max, uint32_t seed,
                      uint32_t walker_id0, int n_iter, int sweeps_per_iter, int n_meas,
                      double *lnW, uint64_t *hist_iter, int8_t *spins_out,
                      int32_t *tallies_out, int32_t *ts, int check, int n_threads,
                      int recursion, double *acc, int win_lo, int win_hi, double grow_flat,
                      int grow_step, int32_t *win_iter, const int8_t *J, int jmax)
{
    if (L < 2 || !(T > 0.0) || n_walkers < 1 || n_iter < 0 || sweeps_per_iter < 0 ||
        n_meas < 0 || !lnW || recursion < 0 || recursion > 1 || (recursion == 1 && !acc))
        return OR_ERR_ARG;
    if (J && !bonds_ok(L, J, jmax)) return OR_ERR_ARG;
    int64_t V = (int64_t)L * L * L;
    if (e_min < 0 || e_max > V || e_min > e_max) return OR_ERR_ARG;
    if (win_lo < e_min || win_hi > e_max || win_lo > win_hi) return OR_ERR_ARG;
    if (grow_flat < 0.0 || (grow_flat > 0.0 && grow_step < 1)) return OR_ERR_ARG;
    int nE = e_max - e_min + 1;
    /* the active window [a, b], relative to e_min */
    int a = win_lo - e_min, b = win_hi - e_min;
    int8_t *spins = (int8_t *)malloc((size_t)n_walkers * (size_t)V);
    int32_t *tal = (int32_t *)malloc((size_t)n_walkers * 3 * sizeof(int32_t));
    const int nk = J ? 24 * jmax + 1 : OR_NK;
    uint32_t *thr = (uint32_t *)malloc((size_t)nE * 3 * (size_t)nk * sizeof(uint32_t));
    uint64_t *hist = (uint64_t *)malloc((size_t)nE * sizeof(uint64_t));
    int rc = OR_OK;
    if (!spins || !tal || !thr || !hist) {
        rc = OR_ERR_NOMEM;
        goto done;
    }
    for (int w = 0; w < n_walkers; ++w) {
        int8_t *s = spins + (int64_t)w * V;
        or_init_spins(L, seed, walker_id0 + (uint32_t)w, s);
        int64_t e[3];
        if (J)
            or_energies_bonds(L, s, J, e);
        else
            or_energies(L, s, e);
        if (e[1] < e_min + a || e[1] > e_min + b) {
            rc = OR_ERR_WINDOW;
            goto done;
        }
        tal[3 * w + 0] = (int32_t)e[0];
        tal[3 * w + 1] = (int32_t)e[1];
        tal[3 * w + 2] = (int32_t)e[2];
    }
    uint64_t sweep = 0;
    sweep_job proto;
    memset(&proto, 0, sizeof proto);
    proto.L = L;
    proto.check = check;
    proto.J = J;
    proto.jmax = jmax;
    proto.thr = thr;
    proto.seed = seed;
    proto.walker_id0 = walker_id0;
    proto.spins = spins;
    proto.tallies = tal;
    /* the sweeps see the window [a, b] only: its table rows, built from its
     * slice of lnW, and its slice of the histogram */
    proto.e_min = e_min + a;
    proto.e_max = e_min + b;
    run_table(L, T, J, jmax, e_min + a, e_min + b, lnW + a, thr);
    for (int it = 0; it < n_iter; ++it) {
        memset(hist, 0, (size_t)nE * sizeof(uint64_t));
        proto.sweep0 = sweep;
        proto.n_sweeps = sweeps_per_iter;
        proto.ts = NULL;
        rc = sweep_all(n_walkers, n_threads, b - a + 1, proto, hist + a);
        if (rc != OR_OK) goto done;
        sweep += (uint64_t)sweeps_per_iter;
        if (hist_iter) memcpy(hist_iter + (size_t)it * nE, hist, (size_t)nE * sizeof(uint64_t));
        const double flat = window_flatness(hist, a, b);
        if (recursion == 1) {
            rc = or_update_lnW_acc(nE, hist, lnW, acc);
            if (rc != OR_OK) goto done;
        } else {
            or_update_lnW(nE, hist, lnW);
        }
        if (grow_flat > 0.0 && flat >= grow_flat && (a > 0 || b < nE - 1)) {
            const int na = a - grow_step > 0 ? a - grow_step : 0;
            const int nb = b + grow_step < nE - 1 ? b + grow_step : nE - 1;
            for (int e = na; e < a; ++e) lnW[e] = lnW[a];
            for (int e = b + 1; e <= nb; ++e) lnW[e] = lnW[b];
            if (recursion == 1) {
                for (int e = na; e < a; ++e) acc[e] = 0.0;
                for (int e = b; e < nb; ++e) acc[e] = 0.0;
            }
            a = na;
            b = nb;
            proto.e_min = e_min + a;
            proto.e_max = e_min + b;
        }
        if (win_iter) {
            win_iter[2 * it + 0] = e_min + a;
            win_iter[2 * it + 1] = e_min + b;
        }
        run_table(L, T, J, jmax, e_min + a, e_min + b, lnW + a, thr);
    }
    if (n_meas > 0) {
        proto.sweep0 = sweep;
        proto.n_sweeps = n_meas;
        proto.ts = ts;
        rc = sweep_all(n_walkers, n_threads, b - a + 1, proto, NULL);
        if (rc != OR_OK) goto done;
    }
    if (spins_out) memcpy(spins_out, spins, (size_t)n_walkers * (size_t)V);
    if (tallies_out) memcpy(tallies_out, tal, (size_t)n_walkers * 3 * sizeof(int32_t));
done:
    free(spins);
    free(tal);
    free(thr);
    free(hist);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Time-series reweighting (Eq. 3) and the observables (Eq. 6, reading R8).   */
/* The weight of sample s at Delta_k is exp(a_s) with                         */
/* a_s = -beta Delta_k E_Delta,s - lnW(E_Delta,s); Eq. 3 only needs it up to a */
/* common factor, so it is normalised by the largest one, exp(a_s - a_max).   */
/* Reading R9: a_s - a_max is evaluated as                                    */
/*   -beta Delta_k (E_s - E*) - (lnW(E_s) - lnW(E*)),  E* the sample of a_max, */
/* the same number without subtracting two O(beta Delta V) terms (they carry */
/* ~1e-11 absolute rounding at V = 32768).  All sums are compensated         */
/* (Neumaier).                                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    double s, c;
} nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_get(const nsum *a) { return a->s + a->c; }

typedef struct {
    const int32_t *e_j, *e_d, *m;
    int64_t n;
    const double *lnW;
    int e_min, nE, V;
    double beta;
    const double *grid;
    int k_begin, k_end;
    double *out;
} rw_job;

static void reweight_one(const rw_job *j, int k)
{
    double c = j->beta * j->grid[k];
    double amax = -INFINITY;
    int32_t estar = j->e_d[0];
    for (int64_t s = 0; s < j->n; ++s) {
        double a = -(c * (double)j->e_d[s]) - j->lnW[j->e_d[s] - j->e_min];
        if (a > amax) {
            amax = a;
            estar = j->e_d[s];
        }
    }
    double lstar = j->lnW[estar - j->e_min];
    nsum z = {0, 0}, sj = {0, 0}, sd = {0, 0}, sm1 = {0, 0}, sm2 = {0, 0}, sm4 = {0, 0};
    for (int64_t s = 0; s < j->n; ++s) {
        double a = -(c * (double)(j->e_d[s] - estar)) - (j->lnW[j->e_d[s] - j->e_min] - lstar);
        double w = exp(a);
        double ej = (double)j->e_j[s], ed = (double)j->e_d[s];
        double mm = (double)j->m[s] / (double)j->V;
        nsum_add(&z, w);
        nsum_add(&sj, w * ej);
        nsum_add(&sd, w * ed);
        nsum_add(&sm1, w * fabs(mm));
        nsum_add(&sm2, w * (mm * mm));
        nsum_add(&sm4, w * ((mm * mm) * (mm * mm)));
    }
    double Z = nsum_get(&z);
    double mj = nsum_get(&sj) / Z, md = nsum_get(&sd) / Z;
    double m1 = nsum_get(&sm1) / Z, m2 = nsum_get(&sm2) / Z, m4 = nsum_get(&sm4) / Z;
    /* reading R10: the covariance of Eq. 6 and the variance in chi are summed
     * in their centred forms <(E_J - <E_J>)(E_Delta - <E_Delta>)> and
     * <(|m| - <|m|>)^2> (equal in exact arithmetic; the uncentred forms cancel
     * about four digits at L = 32) */
    nsum sc = {0, 0}, sx = {0, 0};
    for (int64_t s = 0; s < j->n; ++s) {
        double a = -(c * (double)(j->e_d[s] - estar)) - (j->lnW[j->e_d[s] - j->e_min] - lstar);
        double w = exp(a);
        double dj = (double)j->e_j[s] - mj, dd = (double)j->e_d[s] - md;
        double dm = fabs((double)j->m[s] / (double)j->V) - m1;
        nsum_add(&sc, w * (dj * dd));
        nsum_add(&sx, w * (dm * dm));
    }
    double *o = j->out + 5 * (int64_t)k;
    o[0] = mj;
    o[1] = md;
    o[2] = -j->beta * (nsum_get(&sc) / Z);
    o[3] = j->beta * (double)j->V * (nsum_get(&sx) / Z);
    o[4] = 1.0 - m4 / (3.0 * m2 * m2);
}

static void *rw_job_run(void *arg)
{
    rw_job *j = (rw_job *)arg;
    for (int k = j->k_begin; k < j->k_end; ++k) reweight_one(j, k);
    return NULL;
}

static int rw_check(const int32_t *e_j, const int32_t *e_d, const int32_t *m, int64_t n,
                    const double *lnW, int e_min, int nE, int V, const double *grid,
                    int n_grid, const double *out)
{
    if (!e_j || !e_d || !m || n < 1 || !lnW || nE < 1 || V < 1 || !grid || n_grid < 0 || !out)
        return OR_ERR_ARG;
    for (int64_t s = 0; s < n; ++s)
        if (e_d[s] < e_min || e_d[s] >= e_min + nE) return OR_ERR_WINDOW;
    return OR_OK;
}

int or_reweight(const int32_t *e_j, const int32_t *e_d, const int32_t *m, int64_t n,
                const double *lnW, int e_min, int nE, double beta, int V,
                const double *grid, int n_grid, int n_threads, double *out)
{
    int rc = rw_check(e_j, e_d, m, n, lnW, e_min, nE, V, grid, n_grid, out);
    if (rc != OR_OK) return rc;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_grid) n_threads = n_grid > 0 ? n_grid : 1;
    rw_job *jobs = (rw_job *)calloc((size_t)n_threads, sizeof(rw_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !tid) {
        free(jobs);
        free(tid);
        return OR_ERR_NOMEM;
    }
    for (int t = 0; t < n_threads; ++t) {
        rw_job j = {e_j, e_d, m, n, lnW, e_min, nE, V, beta, grid,
                    (int)((int64_t)n_grid * t / n_threads),
                    (int)((int64_t)n_grid * (t + 1) / n_threads), out};
        jobs[t] = j;
    }
    for (int t = 1; t < n_threads; ++t) pthread_create(&tid[t], NULL, rw_job_run, &jobs[t]);
    rw_job_run(&jobs[0]);
    for (int t = 1; t < n_threads; ++t) pthread_join(tid[t], NULL);
    free(jobs);
    free(tid);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* binary128 variant: Eq. 3 and Eq. 6 evaluated literally (uncentred moments) */
/* with 113-bit mantissas; it pins the FP64 oracle's own rounding.            */
/* ------------------------------------------------------------------------ */
#if defined(__aarch64__) || defined(__powerpc64__)
typedef long double qreal;
#define QEXP expl
#define QFABS fabsl
#else
#include <quadmath.h>
typedef __float128 qreal;
#define QEXP expq
#define QFABS fabsq
#endif

static void reweight_one_q(const rw_job *j, int k)
{
    qreal c = (qreal)j->beta * (qreal)j->grid[k];
    qreal amax = 0;
    int32_t estar = j->e_d[0];
    int first = 1;
    for (int64_t s = 0; s < j->n; ++s) {
        qreal a = -(c * (qreal)j->e_d[s]) - (qreal)j->lnW[j->e_d[s] - j->e_min];
        if (first || a > amax) {
            amax = a;
            estar = j->e_d[s];
        }
        first = 0;
    }
    qreal lstar = (qreal)j->lnW[estar - j->e_min];
    qreal z = 0, sj = 0, sd = 0, sjd = 0, sm1 = 0, sm2 = 0, sm4 = 0;
    for (int64_t s = 0; s < j->n; ++s) {
        qreal a = -(c * (qreal)(j->e_d[s] - estar)) - ((qreal)j->lnW[j->e_d[s] - j->e_min] - lstar);
        qreal w = QEXP(a);
        qreal ej = (qreal)j->e_j[s], ed = (qreal)j->e_d[s];
        qreal mm = (qreal)j->m[s] / (qreal)j->V;
        z += w;
        sj += w * ej;
        sd += w * ed;
        sjd += w * (ej * ed);
        sm1 += w * QFABS(mm);
        sm2 += w * (mm * mm);
        sm4 += w * ((mm * mm) * (mm * mm));
    }
    qreal mj = sj / z, md = sd / z, mjd = sjd / z, m1 = sm1 / z, m2 = sm2 / z, m4 = sm4 / z;
    qreal beta = (qreal)j->beta;
    double *o = j->out + 5 * (int64_t)k;
    o[0] = (double)mj;
    o[1] = (double)md;
    o[2] = (double)(-beta * (mjd - mj * md));
    o[3] = (double)(beta * (qreal)j->V * (m2 - m1 * m1));
    o[4] = (double)(1 - m4 / (3 * m2 * m2));
}

static void *rw_job_run_q(void *arg)
{
    rw_job *j = (rw_job *)arg;
    for (int k = j->k_begin; k < j->k_end; ++k) reweight_one_q(j, k);
    return NULL;
}

int or_reweight_q(const int32_t *e_j, const int32_t *e_d, const int32_t *m, int64_t n,
                  const double *lnW, int e_min, int nE, double beta, int V,
                  const double *grid, int n_grid, int n_threads, double *out)
{
    int rc = rw_check(e_j, e_d, m, n, lnW, e_min, nE, V, grid, n_grid, out);
    if (rc != OR_OK) return rc;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_grid) n_threads = n_grid > 0 ? n_grid : 1;
    rw_job *jobs = (rw_job *)calloc((size_t)n_threads, sizeof(rw_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !tid) {
        free(jobs);
        free(tid);
        return OR_ERR_NOMEM;
    }
    for (int t = 0; t < n_threads; ++t) {
        rw_job j = {e_j, e_d, m, n, lnW, e_min, nE, V, beta, grid,
                    (int)((int64_t)n_grid * t / n_threads),
                    (int)((int64_t)n_grid * (t + 1) / n_threads), out};
        jobs[t] = j;
    }
    for (int t = 1; t < n_threads; ++t) pthread_create(&tid[t], NULL, rw_job_run_q, &jobs[t]);
    rw_job_run_q(&jobs[0]);
    for (int t = 1; t < n_threads; ++t) pthread_join(tid[t], NULL);
    free(jobs);
    free(tid);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Pseudo-transition point (Sec. III): Delta*_L is the field where C(Delta)   */
/* of Eq. 6 is largest, found as the zero crossing of its derivative by       */
/* bisection with time-series reweighting (Eq. 3), for the full series and    */
/* for w subsets that each leave out 1/w of the measurements (jackknife);     */
/* C*_L = C(Delta*_L).  Differentiating a reweighted mean,                    */
/*   d<O>/dDelta = -beta (<O E_Delta> - <O><E_Delta>),                         */
/* applied to Eq. 6 gives                                                      */
/*   dC/dDelta = beta^2 <(E_J - <E_J>)(E_Delta - <E_Delta>)^2>.                */
/* Readings: the series is n_rows rows of row_len samples (one row per sweep),*/
/* subset b leaves out rows [b n_rows / w, (b+1) n_rows / w); the interval     */
/* [lo, hi] must bracket the maximum (dC/dDelta > 0 at lo, < 0 at hi); each   */
/* of n_iter steps keeps the half whose ends still bracket it                  */
/* (mid = lo + (hi - lo) / 2; dC/dDelta(mid) > 0 moves lo, else hi), and the   */
/* result is the midpoint of the last interval.                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    const int32_t *e_j, *e_d;
    int64_t n_rows;
    int32_t row_len;
    int64_t skip0, skip1; /* rows left out */
    const double *lnW;
    int e_min;
    double beta;
} pk_set;

/* <E_J>, <E_Delta>, the covariance and the third mixed moment at Delta,
 * centred exponents (reading R9) and centred sums (reading R10). */
static void pk_moments(const pk_set *p, double delta, double *cov, double *third)
{
    const double c = p->beta * delta;
    double amax = -INFINITY;
    int32_t estar = 0;
    for (int64_t r = 0; r < p->n_rows; ++r) {
        if (r >= p->skip0 && r < p->skip1) continue;
        for (int32_t k = 0; k < p->row_len; ++k) {
            const int32_t e = p->e_d[r * p->row_len + k];
            const double a = -(c * (double)e) - p->lnW[e - p->e_min];
            if (a > amax) {
                amax = a;
                estar = e;
            }
        }
    }
    const double lstar = p->lnW[estar - p->e_min];
    nsum z = {0, 0}, sj = {0, 0}, sd = {0, 0};
    for (int64_t r = 0; r < p->n_rows; ++r) {
        if (r >= p->skip0 && r < p->skip1) continue;
        for (int32_t k = 0; k < p->row_len; ++k) {
            const int64_t s = r * p->row_len + k;
            const int32_t e = p->e_d[s];
            const double w = exp(-(c * (double)(e - estar)) - (p->lnW[e - p->e_min] - lstar));
            nsum_add(&z, w);
            nsum_add(&sj, w * (double)p->e_j[s]);
            nsum_add(&sd, w * (double)e);
        }
    }
    const double Z = nsum_get(&z), mj = nsum_get(&sj) / Z, md = nsum_get(&sd) / Z;
    nsum s2 = {0, 0}, s3 = {0, 0};
    for (int64_t r = 0; r < p->n_rows; ++r) {
        if (r >= p->skip0 && r < p->skip1) continue;
        for (int32_t k = 0; k < p->row_len; ++k) {
            const int64_t s = r * p->row_len + k;
            const int32_t e = p->e_d[s];
            const double w = exp(-(c * (double)(e - estar)) - (p->lnW[e - p->e_min] - lstar));
            const double dj = (double)p->e_j[s] - mj, dd = (double)e - md;
            nsum_add(&s2, w * (dj * dd));
            nsum_add(&s3, w * (dj * dd * dd));
        }
    }
    *cov = nsum_get(&s2) / Z;
    *third = nsum_get(&s3) / Z;
}

typedef struct {
    pk_set set;
    double lo, hi;
    int n_iter;
    double *out; /* Delta*, C* */
    int rc;
} pk_job;

static void *pk_job_run(void *arg)
{
    pk_job *j = (pk_job *)arg;
    double cov, t_lo, t_hi;
    pk_moments(&j->set, j->lo, &cov, &t_lo);
    pk_moments(&j->set, j->hi, &cov, &t_hi);
    if (!(t_lo > 0.0 && t_hi < 0.0)) {
        j->rc = OR_ERR_ARG;
        return NULL;
    }
    double lo = j->lo, hi = j->hi;
    for (int i = 0; i < j->n_iter; ++i) {
        const double mid = lo + 0.5 * (hi - lo);
        double t;
        pk_moments(&j->set, mid, &cov, &t);
        if (t > 0.0) lo = mid;
        else hi = mid;
    }
    const double ds = lo + 0.5 * (hi - lo);
    double t;
    pk_moments(&j->set, ds, &cov, &t);
    j->out[0] = ds;
    j->out[1] = -j->set.beta * cov;
    j->rc = OR_OK;
    return NULL;
}

int or_find_peak(const int32_t *e_j, const int32_t *e_d, int64_t n_rows, int32_t row_len,
                 const double *lnW, int e_min, int nE, double beta, double lo, double hi,
                 int n_iter, int n_jack, int n_threads, double *out)
{
    if (!e_j || !e_d || !lnW || !out || n_rows < 1 || row_len < 1 || nE < 1 || !(beta > 0.0) ||
        !(lo < hi) || n_iter < 0 || n_jack < 0 || n_jack == 1 || n_jack > n_rows)
        return OR_ERR_ARG;
    for (int64_t s = 0; s < n_rows * (int64_t)row_len; ++s)
        if (e_d[s] < e_min || e_d[s] >= e_min + nE) return OR_ERR_WINDOW;
    const int n_sets = 1 + n_jack;
    pk_job *jobs = (pk_job *)calloc((size_t)n_sets, sizeof(pk_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)n_sets, sizeof(pthread_t));
    if (!jobs || !tid) {
        free(jobs);
        free(tid);
        return OR_ERR_NOMEM;
    }
    for (int b = 0; b < n_sets; ++b) {
        pk_set st = {e_j, e_d, n_rows, row_len, 0, 0, lnW, e_min, beta};
        if (b > 0) {
            st.skip0 = (int64_t)(b - 1) * n_rows / n_jack;
            st.skip1 = (int64_t)b * n_rows / n_jack;
        }
        pk_job j = {st, lo, hi, n_iter, out + 2 * b, OR_OK};
        jobs[b] = j;
    }
    /* data sets in parallel, at most n_threads at a time */
    if (n_threads < 1) n_threads = 1;
    for (int b0 = 0; b0 < n_sets; b0 += n_threads) {
        const int b1 = b0 + n_threads < n_sets ? b0 + n_threads : n_sets;
        for (int b = b0 + 1; b < b1; ++b) pthread_create(&tid[b], NULL, pk_job_run, &jobs[b]);
        pk_job_run(&jobs[b0]);
        for (int b = b0 + 1; b < b1; ++b) pthread_join(tid[b], NULL);
    }
    int rc = OR_OK;
    for (int b = 0; b < n_sets; ++b)
        if (jobs[b].rc != OR_OK) rc = jobs[b].rc;
    free(jobs);
    free(tid);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Equal-height field and barrier (Sec. II and the barrier of Sec. IV): the    */
/* reweighted E_Delta distribution of the series at field Delta is            */
/*   P(E) ~ n(E) exp(-beta Delta E) / W(E),  n(E) the samples in bin E.        */
/* Delta_eqh is where its two peaks have equal height, and                     */
/*   B = ln(P_max / P_min)_eqh / (2 beta Delta_eqh)                            */
/* with P_max the (common) peak height and P_min the lowest value between the */
/* peaks.  Readings: the peaks are the highest occupied bins below and at or   */
/* above a split E_split; raising Delta tilts ln P towards small E, so         */
/* g = ln P_left,max - ln P_right,max grows with Delta and the caller's         */
/* [lo, hi] must have g(lo) < 0 < g(hi); each of n_iter steps halves it (g(mid) */
/* < 0 moves lo, else hi) and Delta_eqh is the last midpoint; ties between     */
/* bins go to the smaller E; P_min is the smallest ln P over occupied bins     */
/* between the two peak bins; jackknife subsets as in or_find_peak.            */
/* ------------------------------------------------------------------------ */
typedef struct {
    const int32_t *e_d;
    int64_t n_rows;
    int32_t row_len;
    int64_t skip0, skip1;
    const double *lnW;
    int e_min, nE, split;
    double beta, lo, hi;
    int n_iter;
    double *out; /* Delta_eqh, B, E of the left peak, E of the right peak, E of the minimum */
    int rc;
} eqh_job;

/* the two peak bins (relative to e_min) of ln P at Delta; returns g */
static double eqh_peaks(const eqh_job *j, const double *ln_n, double delta, int *pl, int *pr)
{
    double vl = -INFINITY, vr = -INFINITY;
    int al = -1, ar = -1;
    for (int e = 0; e < j->nE; ++e) {
        if (ln_n[e] == -INFINITY) continue;
        const double v = ln_n[e] - j->beta * delta * (double)(j->e_min + e) - j->lnW[e];
        if (j->e_min + e < j->split) {
            if (v > vl) { vl = v; al = e; }
        } else {
            if (v > vr) { vr = v; ar = e; }
        }
    }
    *pl = al;
    *pr = ar;
    return vl - vr;
}

static void *eqh_job_run(void *arg)
{
    eqh_job *j = (eqh_job *)arg;
    double *ln_n = (double *)malloc((size_t)j->nE * sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)j->nE, sizeof(int64_t));
    if (!ln_n || !cnt) {
        free(ln_n);
        free(cnt);
        j->rc = OR_ERR_NOMEM;
        return NULL;
    }
    for (int64_t r = 0; r < j->n_rows; ++r) {
        if (r >= j->skip0 && r < j->skip1) continue;
        for (int32_t k = 0; k < j->row_len; ++k) ++cnt[j->e_d[r * j->row_len + k] - j->e_min];
    }
    for (int e = 0; e < j->nE; ++e) ln_n[e] = cnt[e] > 0 ? log((double)cnt[e]) : -INFINITY;
    int pl, pr;
    const double g_lo = eqh_peaks(j, ln_n, j->lo, &pl, &pr);
    const int ok_lo = pl >= 0 && pr >= 0;
    const double g_hi = eqh_peaks(j, ln_n, j->hi, &pl, &pr);
    if (!ok_lo || pl < 0 || pr < 0 || !(g_lo < 0.0 && g_hi > 0.0)) {
        free(ln_n);
        free(cnt);
        j->rc = OR_ERR_ARG;
        return NULL;
    }
    double lo = j->lo, hi = j->hi;
    for (int i = 0; i < j->n_iter; ++i) {
        const double mid = lo + 0.5 * (hi - lo);
        if (eqh_peaks(j, ln_n, mid, &pl, &pr) < 0.0) lo = mid;
        else hi = mid;
    }
    const double d = lo + 0.5 * (hi - lo);
    eqh_peaks(j, ln_n, d, &pl, &pr);
    const double vl = ln_n[pl] - j->beta * d * (double)(j->e_min + pl) - j->lnW[pl];
    const double vr = ln_n[pr] - j->beta * d * (double)(j->e_min + pr) - j->lnW[pr];
    const double vmax = vl > vr ? vl : vr;
    double vmin = INFINITY;
    int pm = pl;
    for (int e = pl; e <= pr; ++e) {
        if (ln_n[e] == -INFINITY) continue;
        const double v = ln_n[e] - j->beta * d * (double)(j->e_min + e) - j->lnW[e];
        if (v < vmin) { vmin = v; pm = e; }
    }
    j->out[0] = d;
    j->out[1] = (vmax - vmin) / (2.0 * j->beta * d);
    j->out[2] = (double)(j->e_min + pl);
    j->out[3] = (double)(j->e_min + pr);
    j->out[4] = (double)(j->e_min + pm);
    free(ln_n);
    free(cnt);
    j->rc = OR_OK;
    return NULL;
}

int or_equal_height(const int32_t *e_d, int64_t n_rows, int32_t row_len, const double *lnW,
                    int e_min, int nE, double beta, int split, double lo, double hi, int n_iter,
                    int n_jack, int n_threads, double *out)
{
    if (!e_d || !lnW || !out || n_rows < 1 || row_len < 1 || nE < 1 || !(beta > 0.0) ||
        !(lo < hi) || n_iter < 0 || n_jack < 0 || n_jack == 1 || n_jack > n_rows)
        return OR_ERR_ARG;
    for (int64_t s = 0; s < n_rows * (int64_t)row_len; ++s)
        if (e_d[s] < e_min || e_d[s] >= e_min + nE) return OR_ERR_WINDOW;
    const int n_sets = 1 + n_jack;
    eqh_job *jobs = (eqh_job *)calloc((size_t)n_sets, sizeof(eqh_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)n_sets, sizeof(pthread_t));
    if (!jobs || !tid) {
        free(jobs);
        free(tid);
        return OR_ERR_NOMEM;
    }
    for (int b = 0; b < n_sets; ++b) {
        eqh_job j = {e_d, n_rows, row_len, 0, 0, lnW, e_min, nE, split, beta, lo, hi, n_iter,
                     out + 5 * b, OR_OK};
        if (b > 0) {
            j.skip0 = (int64_t)(b - 1) * n_rows / n_jack;
            j.skip1 = (int64_t)b * n_rows / n_jack;
        }
        jobs[b] = j;
    }
    if (n_threads < 1) n_threads = 1;
    for (int b0 = 0; b0 < n_sets; b0 += n_threads) {
        const int b1 = b0 + n_threads < n_sets ? b0 + n_threads : n_sets;
        for (int b = b0 + 1; b < b1; ++b) pthread_create(&tid[b], NULL, eqh_job_run, &jobs[b]);
        eqh_job_run(&jobs[b0]);
        for (int b = b0 + 1; b < b1; ++b) pthread_join(tid[b], NULL);
    }
    int rc = OR_OK;
    for (int b = 0; b < n_sets; ++b)
        if (jobs[b].rc != OR_OK) rc = jobs[b].rc;
    free(jobs);
    free(tid);
    return rc;
}
