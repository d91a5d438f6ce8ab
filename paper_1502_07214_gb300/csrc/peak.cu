// peak.cu -- the pseudo-transition point Delta*_L of Sec. III: the crystal
// field where C(Delta) of Eq. 6 is largest, found as the zero crossing of
// dC/dDelta by bisection with time-series reweighting (Eq. 3), for the full
// series and for w jackknife subsets that each leave out one block of
// consecutive measurements; C*_L = C(Delta*_L).
//
// Differentiating a reweighted mean, d<O>/dDelta = -beta (<O E_Delta> - <O><E_Delta>);
// applied to Eq. 6,
//   dC/dDelta = beta^2 <(E_J - <E_J>)(E_Delta - <E_Delta>)^2>.
// A sample enters C and dC/dDelta only through its E_Delta bin and its E_J,
// and (E_Delta - <E_Delta>) is constant within a bin, so both need per bin
// only the number of samples n and their mean E_J:
//   C = -beta / Z sum_E w(E) n(E) (mj(E) - <E_J>)(E - <E_Delta>),
//   dC/dDelta / beta^2 = 1 / Z sum_E w(E) n(E) (mj(E) - <E_J>)(E - <E_Delta>)^2,
// with w(E) = exp(-beta Delta E - lnW(E)) taken relative to its largest value.
//
// GPU layout: one pass over the series forms exact integer sums (count, sum
// E_J) per bin and per jackknife block; each data set's sums are all blocks'
// sums minus the left-out block's (integers, exact); one thread-block cluster
// per data set then runs the whole bisection, each step three FP64 passes over
// the bins (largest weight, weighted means, centred moments), every CTA of the
// cluster over its own slice of the bins, the CTAs' partial results combined
// through distributed shared memory in rank order (so that every CTA holds
// the same numbers and takes the same bisection step).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/muca.h"
#include "muca_internal.h"

namespace {

namespace cg = cooperative_groups;

// Integer sums per jackknife block: cnt[b][E], sej[b][E].  bnd[i] is the first
// row of block i (bnd[n_blocks] = n_rows).
template <bool SEJ>
__global__ void jk_bin_kernel(const int32_t *__restrict__ ej, const int32_t *__restrict__ ed,
                              int64_t n_rows, int row_len, int64_t row_stride, int e_min, int nE,
                              const int64_t *__restrict__ bnd, int n_blocks,
                              unsigned long long *cnt, unsigned long long *sej, int *err)
{
    for (int64_t r = blockIdx.y; r < n_rows; r += gridDim.y) {
        int b = 0;
        while (b + 1 < n_blocks && bnd[b + 1] <= r) ++b;
        unsigned long long *cb = cnt + (size_t)b * nE, *sb = sej + (size_t)b * nE;
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < row_len;
             c += gridDim.x * blockDim.x) {
            const int64_t o = r * row_stride + c;
            const int e = (int)((unsigned)__ldg(ed + o) - (unsigned)e_min);
            if ((unsigned)e >= (unsigned)nE) {
                atomicOr(err, 1);
                continue;
            }
            atomicAdd(cb + e, 1ull);
            if (SEJ) atomicAdd(sb + e, (unsigned long long)(long long)__ldg(ej + o));
        }
    }
}

// Per data set d (0: every block; 1 + i: every block but i) and bin: the
// sample count and the mean E_J.
__global__ void jk_stats_kernel(const unsigned long long *__restrict__ cnt,
                                const unsigned long long *__restrict__ sej, int n_blocks, int nE,
                                double *n_out, double *mj_out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (e >= nE) return;
    unsigned long long n = 0, s = 0;
    for (int b = 0; b < n_blocks; ++b) {
        n += cnt[(size_t)b * nE + e];
        s += sej[(size_t)b * nE + e];
    }
    if (d > 0) {
        n -= cnt[(size_t)(d - 1) * nE + e];
        s -= sej[(size_t)(d - 1) * nE + e];
    }
    n_out[(size_t)d * nE + e] = (double)n;
    mj_out[(size_t)d * nE + e] = n ? (double)(long long)s / (double)n : 0.0;
}

struct KS {  // Kahan-compensated FP64 sum
    double s = 0.0, c = 0.0;
    __device__ void add(double x)
    {
        const double y = x - c;
        const double t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

constexpr int kPkThreads = 256;

// Sum over the block of K compensated sums: every thread gets each sum as a
// pair (tot, cc) whose value is tot - cc.
template <int K>
__device__ void pk_block_sum(KS (&a)[K], double (&tot)[K], double (&cc)[K], double *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = a[k].s, c = -a[k].c;
        for (int o = 16; o > 0; o >>= 1) {
            const double s2 = __shfl_xor_sync(0xFFFFFFFFu, s, o);
            const double c2 = __shfl_xor_sync(0xFFFFFFFFu, c, o);
            const double t = s + s2;
            const double bp = t - s;
            const double err = (s - (t - bp)) + (s2 - bp);
            s = t;
            c = c + c2 + err;
        }
        __syncthreads();
        if (lane == 0) {
            sh[2 * wid] = s;
            sh[2 * wid + 1] = c;
        }
        __syncthreads();
        double T = 0.0, C = 0.0;
        for (int i = 0; i < nw; ++i) {
            const double y = sh[2 * i] - C;
            const double t = T + y;
            C = (t - T) - y;
            T = t;
            C -= sh[2 * i + 1];
        }
        tot[k] = T;
        cc[k] = C;
    }
}

// Partial results of one CTA of a cluster, read by every CTA of the cluster.
struct PkPart {
    double av;    // largest exponent over the CTA's bins
    int aa;       // its bin
    double s[6];  // weighted sums, (tot, cc) pairs
    double t[4];  // centred sums, (tot, cc) pairs
};

// The cluster's sums from its CTAs' (tot, cc) pairs at offset `off` of
// PkPart (K sums), combined in rank order.
template <int K>
__device__ void pk_cluster_sum(cg::cluster_group &cl, PkPart *part, int which, double (&out)[K])
{
    const int ncta = (int)cl.num_blocks();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double T = 0.0, C = 0.0;
        for (int r = 0; r < ncta; ++r) {
            const PkPart *pr = cl.map_shared_rank(part, r);
            const double *v = which ? pr->t : pr->s;
            const double y = v[2 * k] - C;
            const double t = T + y;
            C = (t - T) - y;
            T = t;
            C += v[2 * k + 1];
        }
        out[k] = T - C;
    }
}

// The bin E* of the largest weight exp(-c E - lnW(E)) among occupied bins
// (ties to the smaller bin).
__device__ int pk_argmax(const double *n, const double *lnW, int e0, int e1, int e_min, double c,
                         double *sh, int *shi, double &vout)
{
    double v = -INFINITY;
    int arg = 0x7FFFFFFF;
    for (int e = e0 + (int)threadIdx.x; e < e1; e += blockDim.x)
        if (n[e] > 0.0) {
            const double a = __dsub_rn(-__dmul_rn(c, (double)(e_min + e)), lnW[e]);
            if (a > v) {
                v = a;
                arg = e;
            }
        }
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        const int a2 = __shfl_xor_sync(0xFFFFFFFFu, arg, o);
        if (v2 > v || (v2 == v && a2 < arg)) {
            v = v2;
            arg = a2;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[wid] = v;
        shi[wid] = arg;
    }
    __syncthreads();
    v = sh[0];
    arg = shi[0];
    for (int i = 1; i < nw; ++i)
        if (sh[i] > v || (sh[i] == v && shi[i] < arg)) {
            v = sh[i];
            arg = shi[i];
        }
    vout = v;
    return arg;
}

// Covariance <(E_J - <E_J>)(E_Delta - <E_Delta>)> and third moment
// <(E_J - <E_J>)(E_Delta - <E_Delta>)^2> of the data set at field Delta.  This
// CTA takes bins [e0, e1); the cluster combines the CTAs' partial results
// (three cluster barriers).  wb: the data set's scratch of nE weights; each
// thread reads back only the weights it wrote.
__device__ void pk_moments(cg::cluster_group &cl, PkPart *part, const double *n, const double *mj,
                           const double *lnW, int nE, int e0, int e1, int e_min, double beta,
                           double delta, double *sh, int *shi, double *wb, double &cov,
                           double &third)
{
    const double c = beta * delta;
    double av;
    int aa = pk_argmax(n, lnW, e0, e1, e_min, c, sh, shi, av);
    if (threadIdx.x == 0) {
        part->av = av;
        part->aa = aa;
    }
    cl.sync();
    double v = -INFINITY;
    int es = 0x7FFFFFFF;
    for (int r = 0; r < (int)cl.num_blocks(); ++r) {
        const PkPart *pr = cl.map_shared_rank(part, r);
        const double rv = pr->av;
        const int ra = pr->aa;
        if (rv > v || (rv == v && ra < es)) {
            v = rv;
            es = ra;
        }
    }
    if (es >= nE) es = 0;  // no occupied bin: nothing to weigh
    const double lstar = lnW[es];
    KS a[3];
    for (int e = e0 + (int)threadIdx.x; e < e1; e += blockDim.x) {
        const double ne = n[e];
        if (ne <= 0.0) continue;
        const double w =
            exp(__dsub_rn(-__dmul_rn(c, (double)(e - es)), __dsub_rn(lnW[e], lstar))) * ne;
        wb[e] = w;
        a[0].add(w);
        a[1].add(w * mj[e]);
        a[2].add(w * (double)(e_min + e));
    }
    {
        double tot[3], cc[3];
        pk_block_sum<3>(a, tot, cc, sh);
        if (threadIdx.x == 0)
            for (int k = 0; k < 3; ++k) {
                part->s[2 * k] = tot[k];
                part->s[2 * k + 1] = cc[k];
            }
    }
    cl.sync();
    double S[3];
    pk_cluster_sum<3>(cl, part, 0, S);
    const double jbar = S[1] / S[0], dbar = S[2] / S[0];
    KS b[2];
    for (int e = e0 + (int)threadIdx.x; e < e1; e += blockDim.x) {
        const double ne = n[e];
        if (ne <= 0.0) continue;
        const double w = wb[e];
        const double dj = mj[e] - jbar, dd = (double)(e_min + e) - dbar;
        b[0].add(w * (dj * dd));
        b[1].add(w * (dj * dd * dd));
    }
    {
        double tot[2], cc[2];
        pk_block_sum<2>(b, tot, cc, sh);
        if (threadIdx.x == 0)
            for (int k = 0; k < 2; ++k) {
                part->t[2 * k] = tot[k];
                part->t[2 * k + 1] = cc[k];
            }
    }
    cl.sync();
    double T[2];
    pk_cluster_sum<2>(cl, part, 1, T);
    cov = T[0] / S[0];
    third = T[1] / S[0];
}

// One cluster per data set: bisection on the sign of dC/dDelta in [lo, hi].
// Every CTA of a cluster holds the same combined sums, so all take the same
// steps; a final cluster barrier keeps each CTA's shared memory alive until
// the others have read it.
__global__ void __launch_bounds__(kPkThreads)
peak_kernel(const double *__restrict__ n_all, const double *__restrict__ mj_all,
            const double *__restrict__ lnW, int nE, int e_min, double beta, double lo, double hi,
            int n_iter, double *res, int *bad, double *wscr)
{
    __shared__ double sh[64];
    __shared__ int shi[32];
    __shared__ PkPart part;
    cg::cluster_group cl = cg::this_cluster();
    const int ncta = (int)cl.num_blocks(), q = (int)cl.block_rank();
    const int d = blockIdx.x / ncta;
    const int e0 = (int)((int64_t)nE * q / ncta), e1 = (int)((int64_t)nE * (q + 1) / ncta);
    const double *n = n_all + (size_t)d * nE, *mj = mj_all + (size_t)d * nE;
    double *wb = wscr + (size_t)d * nE;
    double cov, t_lo, t_hi;
    pk_moments(cl, &part, n, mj, lnW, nE, e0, e1, e_min, beta, lo, sh, shi, wb, cov, t_lo);
    pk_moments(cl, &part, n, mj, lnW, nE, e0, e1, e_min, beta, hi, sh, shi, wb, cov, t_hi);
    if (!(t_lo > 0.0 && t_hi < 0.0)) {
        if (q == 0 && threadIdx.x == 0) bad[d] = 1;
        cl.sync();
        return;
    }
    for (int i = 0; i < n_iter; ++i) {
        const double mid = lo + 0.5 * (hi - lo);
        double t;
        pk_moments(cl, &part, n, mj, lnW, nE, e0, e1, e_min, beta, mid, sh, shi, wb, cov, t);
        if (t > 0.0) lo = mid;
        else hi = mid;
    }
    const double ds = lo + 0.5 * (hi - lo);
    double t;
    pk_moments(cl, &part, n, mj, lnW, nE, e0, e1, e_min, beta, ds, sh, shi, wb, cov, t);
    if (q == 0 && threadIdx.x == 0) {
        res[2 * d] = ds;
        res[2 * d + 1] = -beta * cov;
    }
    cl.sync();
}

// ---------------------------------------------------- equal height, barrier
// The reweighted E_Delta distribution at field Delta, from the series' count
// n(E) per bin: ln P(E) = ln n(E) - beta Delta E - lnW(E) (+ const).  Delta_eqh
// is where its highest bins below and at or above split are equally high;
// B = ln(P_max / P_min) / (2 beta Delta_eqh), P_min the lowest occupied bin
// between the two peaks.

// Per data set d and bin: ln of the sample count (-inf when empty).
__global__ void jk_lncount_kernel(const unsigned long long *__restrict__ cnt, int n_blocks, int nE,
                                  double *lnn)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (e >= nE) return;
    unsigned long long n = 0;
    for (int b = 0; b < n_blocks; ++b) n += cnt[(size_t)b * nE + e];
    if (d > 0) n -= cnt[(size_t)(d - 1) * nE + e];
    lnn[(size_t)d * nE + e] = n ? log((double)n) : -INFINITY;
}

// ln P(E) at Delta, evaluated in the order (ln n - (beta Delta) E) - lnW.
__device__ __forceinline__ double eqh_lnp(double lnn, double bd, int E, double lnw)
{
    return __dsub_rn(__dsub_rn(lnn, __dmul_rn(bd, (double)E)), lnw);
}

// Block-wide best (value, bin): larger value wins when want_max, smaller when
// not; ties go to the smaller bin.  Every thread gets the result.
__device__ void eqh_best(double &v, int &a, bool want_max, double *sh, int *shi)
{
    auto better = [&](double v2, int a2) {
        if (a2 < 0) return false;
        if (a < 0) return true;
        if (want_max ? v2 > v : v2 < v) return true;
        return v2 == v && a2 < a;
    };
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        const int a2 = __shfl_xor_sync(0xFFFFFFFFu, a, o);
        if (better(v2, a2)) {
            v = v2;
            a = a2;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[wid] = v;
        shi[wid] = a;
    }
    __syncthreads();
    v = sh[0];
    a = shi[0];
    for (int i = 1; i < nw; ++i)
        if (better(sh[i], shi[i])) {
            v = sh[i];
            a = shi[i];
        }
}

// The two peak bins at Delta among bins [e0, e1) (relative to e_min, -1 when a
// side is empty); returns g.
__device__ double eqh_peaks(const double *lnn, const double *lnW, int e0, int e1, int e_min,
                            int split, double bd, int &pl, int &pr, double &vl, double &vr,
                            double *sh, int *shi)
{
    vl = -INFINITY;
    vr = -INFINITY;
    pl = -1;
    pr = -1;
    for (int e = e0 + (int)threadIdx.x; e < e1; e += blockDim.x) {
        if (lnn[e] == -INFINITY) continue;
        const double v = eqh_lnp(lnn[e], bd, e_min + e, lnW[e]);
        if (e_min + e < split) {
            if (pl < 0 || v > vl) {
                vl = v;
                pl = e;
            }
        } else if (pr < 0 || v > vr) {
            vr = v;
            pr = e;
        }
    }
    eqh_best(vl, pl, true, sh, shi);
    eqh_best(vr, pr, true, sh, shi);
    return vl - vr;
}

// One CTA's best (value, bin) pairs for the two peaks, or its lowest bin.
struct EqPart {
    double vl, vr;
    int pl, pr;
};

// Larger (want_max) or smaller value wins, ties to the smaller bin, bin -1 is empty.
__device__ __forceinline__ bool eqh_better(double v2, int a2, double v, int a, bool want_max)
{
    if (a2 < 0) return false;
    if (a < 0) return true;
    if (want_max ? v2 > v : v2 < v) return true;
    return v2 == v && a2 < a;
}

// The cluster's peaks from its CTAs' block results, combined in rank order
// through the slot `slot` of every CTA's parts (slots alternate, so one
// cluster barrier per combination suffices).
__device__ double eqh_cluster_peaks(cg::cluster_group &cl, EqPart *part, int &slot, int &pl, int &pr,
                                    double &vl, double &vr)
{
    if (threadIdx.x == 0) part[slot] = EqPart{vl, vr, pl, pr};
    cl.sync();
    double bl = -INFINITY, br = -INFINITY;
    int al = -1, ar = -1;
    for (int r = 0; r < (int)cl.num_blocks(); ++r) {
        const EqPart q = cl.map_shared_rank(part, r)[slot];
        if (eqh_better(q.vl, q.pl, bl, al, true)) {
            bl = q.vl;
            al = q.pl;
        }
        if (eqh_better(q.vr, q.pr, br, ar, true)) {
            br = q.vr;
            ar = q.pr;
        }
    }
    slot ^= 1;
    vl = bl;
    vr = br;
    pl = al;
    pr = ar;
    return vl - vr;
}

// One cluster per data set (each CTA over its slice [e0, e1) of the bins):
// bisection on g = ln P_low - ln P_high, then the barrier at Delta_eqh.
__global__ void __launch_bounds__(kPkThreads)
eqh_kernel(const double *__restrict__ lnn_all, const double *__restrict__ lnW, int nE, int e_min,
           int split, double beta, double lo, double hi, int n_iter, double *res, int *bad)
{
    __shared__ double sh[32];
    __shared__ int shi[32];
    __shared__ EqPart part[2];
    cg::cluster_group cl = cg::this_cluster();
    const int ncta = (int)cl.num_blocks(), q = (int)cl.block_rank();
    const int d = blockIdx.x / ncta;
    const int e0 = (int)((int64_t)nE * q / ncta), e1 = (int)((int64_t)nE * (q + 1) / ncta);
    const double *lnn = lnn_all + (size_t)d * nE;
    int slot = 0;
    auto peaks = [&](double bd, int &pl, int &pr, double &vl, double &vr) {
        eqh_peaks(lnn, lnW, e0, e1, e_min, split, bd, pl, pr, vl, vr, sh, shi);
        return eqh_cluster_peaks(cl, part, slot, pl, pr, vl, vr);
    };
    int pl, pr;
    double vl, vr;
    const double g_lo = peaks(beta * lo, pl, pr, vl, vr);
    const bool ok_lo = pl >= 0 && pr >= 0;
    const double g_hi = peaks(beta * hi, pl, pr, vl, vr);
    if (!ok_lo || pl < 0 || pr < 0 || !(g_lo < 0.0 && g_hi > 0.0)) {
        if (q == 0 && threadIdx.x == 0) bad[d] = 1;
        cl.sync();
        return;
    }
    for (int i = 0; i < n_iter; ++i) {
        const double mid = lo + 0.5 * (hi - lo);
        if (peaks(beta * mid, pl, pr, vl, vr) < 0.0) lo = mid;
        else hi = mid;
    }
    const double dq = lo + 0.5 * (hi - lo);
    const double bd = beta * dq;
    peaks(bd, pl, pr, vl, vr);
    const double vmax = vl > vr ? vl : vr;
    double vmin = INFINITY;
    int pm = -1;
    for (int e = max(pl, e0) + (int)threadIdx.x; e <= min(pr, e1 - 1); e += blockDim.x) {
        if (lnn[e] == -INFINITY) continue;
        const double v = eqh_lnp(lnn[e], bd, e_min + e, lnW[e]);
        if (pm < 0 || v < vmin) {
            vmin = v;
            pm = e;
        }
    }
    eqh_best(vmin, pm, false, sh, shi);
    if (threadIdx.x == 0) part[slot] = EqPart{vmin, 0.0, pm, -1};
    cl.sync();
    double bm = INFINITY;
    int am = -1;
    for (int r = 0; r < ncta; ++r) {
        const EqPart qq = cl.map_shared_rank(part, r)[slot];
        if (eqh_better(qq.vl, qq.pl, bm, am, false)) {
            bm = qq.vl;
            am = qq.pl;
        }
    }
    vmin = bm;
    pm = am;
    if (q == 0 && threadIdx.x == 0) {
        double *o = res + 5 * (size_t)d;
        o[0] = dq;
        o[1] = (vmax - vmin) / (2.0 * beta * dq);
        o[2] = (double)(e_min + pl);
        o[3] = (double)(e_min + pr);
        o[4] = (double)(e_min + pm);
    }
    cl.sync();
}

int pk_fail(int code, const std::string &msg)
{
    muca::set_last_error(msg.c_str());
    return code;
}

}  // namespace

// Launch configuration of a per-data-set cluster kernel: one cluster per data
// set and one CTA per SM (the CTAs reserve unused dynamic shared memory above
// half an SM's); the cluster size is the largest of 8 .. 1 for which every
// data set's cluster can be resident at once (clusters live within a GPC, so
// the SM count alone does not tell).  attr must outlive cfg.
static cudaError_t cluster_config(const void *kernel, int n_sets, cudaStream_t st,
                                  cudaLaunchConfig_t &cfg, cudaLaunchAttribute (&attr)[1])
{
    int dev = 0, nsm = 152, smem_sm = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return ce;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const size_t one_per_sm = smem_sm > 0 ? (size_t)smem_sm / 2 + 1024 : 0;
    ce = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)one_per_sm);
    if (ce != cudaSuccess) return ce;
    cfg = cudaLaunchConfig_t{};
    cfg.blockDim = dim3(kPkThreads);
    cfg.dynamicSmemBytes = one_per_sm;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncta = std::max(1, std::min(8, nsm / std::max(n_sets, 1)));
    for (; ncta > 1; --ncta) {
        attr[0].val.clusterDim.x = (unsigned)ncta;
        cfg.gridDim = dim3((unsigned)(n_sets * ncta));
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, kernel, &cfg) == cudaSuccess && nc >= n_sets) break;
    }
    (void)cudaGetLastError();
    attr[0].val.clusterDim.x = (unsigned)ncta;
    cfg.gridDim = dim3((unsigned)(n_sets * ncta));
    return cudaSuccess;
}

extern "C" int muca_find_peak(const int32_t *e_j, const int32_t *e_d, int64_t n_rows,
                              int32_t row_len, int64_t row_stride, const double *lnW,
                              int32_t e_min, int32_t n_e, double beta, double delta_lo,
                              double delta_hi, int32_t n_iter, int32_t n_jack, double *out,
                              void *stream)
{
    if (!e_j || !e_d || !lnW || !out)
        return pk_fail(MUCA_ERR_INVALID_ARG, "muca_find_peak: null pointer");
    if (n_rows < 1 || row_len < 1 || (n_rows > 1 && row_stride < row_len) || n_e < 1 ||
        n_iter < 0 || n_iter > 200 || n_jack < 0 || n_jack == 1 || n_jack > n_rows ||
        n_jack > 1024)
        return pk_fail(MUCA_ERR_INVALID_ARG, "muca_find_peak: bad sizes");
    if ((int64_t)e_min + n_e - 1 > INT32_MAX)
        return pk_fail(MUCA_ERR_INVALID_ARG, "muca_find_peak: e_min + n_e - 1 exceeds int32");
    if (!(beta > 0.0) || !std::isfinite(beta) || !std::isfinite(delta_lo) ||
        !std::isfinite(delta_hi) || !(delta_lo < delta_hi))
        return pk_fail(MUCA_ERR_INVALID_ARG, "muca_find_peak: need beta > 0 and delta_lo < delta_hi");
    for (int e = 0; e < n_e; ++e)
        if (!std::isfinite(lnW[e])) return pk_fail(MUCA_ERR_INVALID_ARG, "muca_find_peak: lnW not finite");
    cudaStream_t st = (cudaStream_t)stream;
    const int n_blocks = n_jack > 0 ? n_jack : 1, n_sets = 1 + n_jack;
    std::vector<int64_t> bnd(n_blocks + 1);
    for (int i = 0; i <= n_blocks; ++i) bnd[i] = (int64_t)i * n_rows / n_blocks;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_sums = al((size_t)2 * n_blocks * n_e * sizeof(unsigned long long));
    const size_t b_sets = al((size_t)2 * n_sets * n_e * sizeof(double));
    const size_t b_lnw = al((size_t)n_e * sizeof(double));
    const size_t b_bnd = al(bnd.size() * sizeof(int64_t));
    const size_t b_res = al((size_t)2 * n_sets * sizeof(double));
    const size_t b_bad = al((size_t)(n_sets + 1) * sizeof(int));
    const size_t b_w = al((size_t)n_sets * n_e * sizeof(double));
    char *p = nullptr;
    cudaError_t ce =
        cudaMallocAsync((void **)&p, b_sums + b_sets + b_lnw + b_bnd + b_res + b_bad + b_w, st);
    if (ce != cudaSuccess)
        return pk_fail(ce == cudaErrorMemoryAllocation ? MUCA_ERR_OOM : MUCA_ERR_CUDA,
                       std::string("cudaMallocAsync: ") + cudaGetErrorString(ce));
    unsigned long long *cnt = (unsigned long long *)p, *sej = cnt + (size_t)n_blocks * n_e;
    double *n_all = (double *)(p + b_sums), *mj_all = n_all + (size_t)n_sets * n_e;
    double *d_lnW = (double *)(p + b_sums + b_sets);
    int64_t *d_bnd = (int64_t *)(p + b_sums + b_sets + b_lnw);
    double *d_res = (double *)(p + b_sums + b_sets + b_lnw + b_bnd);
    int *d_bad = (int *)(p + b_sums + b_sets + b_lnw + b_bnd + b_res);  // [0]: window, [1 + d]
    double *d_w = (double *)(p + b_sums + b_sets + b_lnw + b_bnd + b_res + b_bad);
    std::vector<double> res(2 * (size_t)n_sets, 0.0);
    std::vector<int> bad(n_sets + 1, 0);
    int rc = MUCA_OK;
#define PCK(call)                                                                         \
    do {                                                                                  \
        ce = (call);                                                                      \
        if (ce != cudaSuccess) {                                                          \
            rc = pk_fail(MUCA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(ce)); \
            goto done;                                                                    \
        }                                                                                 \
    } while (0)
    PCK(cudaMemsetAsync(p, 0, b_sums, st));
    PCK(cudaMemsetAsync(d_bad, 0, b_bad, st));
    PCK(cudaMemcpyAsync(d_lnW, lnW, (size_t)n_e * sizeof(double), cudaMemcpyHostToDevice, st));
    PCK(cudaMemcpyAsync(d_bnd, bnd.data(), bnd.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    {
        dim3 g((unsigned)std::min<int64_t>((row_len + 255) / 256, 1024),
               (unsigned)std::min<int64_t>(n_rows, 4096));
        jk_bin_kernel<true><<<g, 256, 0, st>>>(e_j, e_d, n_rows, row_len, row_stride, e_min, n_e,
                                               d_bnd, n_blocks, cnt, sej, d_bad);
        PCK(cudaGetLastError());
        dim3 g2((unsigned)((n_e + 255) / 256), (unsigned)n_sets);
        jk_stats_kernel<<<g2, 256, 0, st>>>(cnt, sej, n_blocks, n_e, n_all, mj_all);
        PCK(cudaGetLastError());
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute attr[1];
        PCK(cluster_config((const void *)peak_kernel, n_sets, st, cfg, attr));
        PCK(cudaLaunchKernelEx(&cfg, peak_kernel, (const double *)n_all, (const double *)mj_all,
                               (const double *)d_lnW, (int)n_e, (int)e_min, beta, delta_lo,
                               delta_hi, (int)n_iter, d_res, d_bad + 1, d_w));
    }
    PCK(cudaMemcpyAsync(res.data(), d_res, res.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    PCK(cudaMemcpyAsync(bad.data(), d_bad, bad.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
#undef PCK
    if (bad[0]) {
        rc = pk_fail(MUCA_ERR_WINDOW, "a sample's E_Delta lies outside [e_min, e_min + n_e)");
        goto done;
    }
    for (int d = 0; d < n_sets; ++d)
        if (bad[1 + d]) {
            rc = pk_fail(MUCA_ERR_INVALID_ARG,
                         "muca_find_peak: [delta_lo, delta_hi] does not bracket the maximum of C "
                         "for data set " + std::to_string(d) +
                         " (dC/dDelta must be > 0 at delta_lo and < 0 at delta_hi)");
            goto done;
        }
    {
        // jackknife errors: var = (w - 1) / w sum_i (x_i - mean_i x_i)^2
        double err[2] = {0.0, 0.0};
        if (n_jack > 0) {
            for (int q = 0; q < 2; ++q) {
                double mean = 0.0;
                for (int i = 0; i < n_jack; ++i) mean += res[2 * (1 + i) + q];
                mean /= n_jack;
                double ss = 0.0;
                for (int i = 0; i < n_jack; ++i) {
                    const double dv = res[2 * (1 + i) + q] - mean;
                    ss += dv * dv;
                }
                err[q] = std::sqrt((double)(n_jack - 1) / n_jack * ss);
            }
        }
        out[0] = res[0];
        out[1] = err[0];
        out[2] = res[1];
        out[3] = err[1];
        for (int i = 0; i < n_jack; ++i) {
            out[4 + 2 * i] = res[2 * (1 + i)];
            out[5 + 2 * i] = res[2 * (1 + i) + 1];
        }
    }
done:
    cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
    return rc;
}

extern "C" int muca_equal_height(const int32_t *e_d, int64_t n_rows, int32_t row_len,
                                 int64_t row_stride, const double *lnW, int32_t e_min,
                                 int32_t n_e, double beta, int32_t split, double delta_lo,
                                 double delta_hi, int32_t n_iter, int32_t n_jack, double *out,
                                 void *stream)
{
    if (!e_d || !lnW || !out) return pk_fail(MUCA_ERR_INVALID_ARG, "muca_equal_height: null pointer");
    if (n_rows < 1 || row_len < 1 || (n_rows > 1 && row_stride < row_len) || n_e < 1 ||
        n_iter < 0 || n_iter > 200 || n_jack < 0 || n_jack == 1 || n_jack > n_rows ||
        n_jack > 1024)
        return pk_fail(MUCA_ERR_INVALID_ARG, "muca_equal_height: bad sizes");
    if ((int64_t)e_min + n_e - 1 > INT32_MAX)
        return pk_fail(MUCA_ERR_INVALID_ARG, "muca_equal_height: e_min + n_e - 1 exceeds int32");
    if (!(beta > 0.0) || !std::isfinite(beta) || !std::isfinite(delta_lo) ||
        !std::isfinite(delta_hi) || !(delta_lo < delta_hi))
        return pk_fail(MUCA_ERR_INVALID_ARG,
                       "muca_equal_height: need beta > 0 and delta_lo < delta_hi");
    for (int e = 0; e < n_e; ++e)
        if (!std::isfinite(lnW[e]))
            return pk_fail(MUCA_ERR_INVALID_ARG, "muca_equal_height: lnW not finite");
    cudaStream_t st = (cudaStream_t)stream;
    const int n_blocks = n_jack > 0 ? n_jack : 1, n_sets = 1 + n_jack;
    std::vector<int64_t> bnd(n_blocks + 1);
    for (int i = 0; i <= n_blocks; ++i) bnd[i] = (int64_t)i * n_rows / n_blocks;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_cnt = al((size_t)n_blocks * n_e * sizeof(unsigned long long));
    const size_t b_lnn = al((size_t)n_sets * n_e * sizeof(double));
    const size_t b_lnw = al((size_t)n_e * sizeof(double));
    const size_t b_bnd = al(bnd.size() * sizeof(int64_t));
    const size_t b_res = al((size_t)5 * n_sets * sizeof(double));
    const size_t b_bad = al((size_t)(n_sets + 1) * sizeof(int));
    char *p = nullptr;
    cudaError_t ce = cudaMallocAsync((void **)&p, b_cnt + b_lnn + b_lnw + b_bnd + b_res + b_bad, st);
    if (ce != cudaSuccess)
        return pk_fail(ce == cudaErrorMemoryAllocation ? MUCA_ERR_OOM : MUCA_ERR_CUDA,
                       std::string("cudaMallocAsync: ") + cudaGetErrorString(ce));
    unsigned long long *cnt = (unsigned long long *)p;
    double *lnn = (double *)(p + b_cnt);
    double *d_lnW = (double *)(p + b_cnt + b_lnn);
    int64_t *d_bnd = (int64_t *)(p + b_cnt + b_lnn + b_lnw);
    double *d_res = (double *)(p + b_cnt + b_lnn + b_lnw + b_bnd);
    int *d_bad = (int *)(p + b_cnt + b_lnn + b_lnw + b_bnd + b_res);
    std::vector<double> res(5 * (size_t)n_sets, 0.0);
    std::vector<int> bad(n_sets + 1, 0);
    int rc = MUCA_OK;
#define PCK(call)                                                                         \
    do {                                                                                  \
        ce = (call);                                                                      \
        if (ce != cudaSuccess) {                                                          \
            rc = pk_fail(MUCA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(ce)); \
            goto done;                                                                    \
        }                                                                                 \
    } while (0)
    PCK(cudaMemsetAsync(p, 0, b_cnt, st));
    PCK(cudaMemsetAsync(d_bad, 0, b_bad, st));
    PCK(cudaMemcpyAsync(d_lnW, lnW, (size_t)n_e * sizeof(double), cudaMemcpyHostToDevice, st));
    PCK(cudaMemcpyAsync(d_bnd, bnd.data(), bnd.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    {
        dim3 g((unsigned)std::min<int64_t>((row_len + 255) / 256, 1024),
               (unsigned)std::min<int64_t>(n_rows, 4096));
        jk_bin_kernel<false><<<g, 256, 0, st>>>(e_d, e_d, n_rows, row_len, row_stride, e_min, n_e,
                                                d_bnd, n_blocks, cnt, nullptr, d_bad);
        PCK(cudaGetLastError());
        dim3 g2((unsigned)((n_e + 255) / 256), (unsigned)n_sets);
        jk_lncount_kernel<<<g2, 256, 0, st>>>(cnt, n_blocks, n_e, lnn);
        PCK(cudaGetLastError());
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute attr[1];
        PCK(cluster_config((const void *)eqh_kernel, n_sets, st, cfg, attr));
        PCK(cudaLaunchKernelEx(&cfg, eqh_kernel, (const double *)lnn, (const double *)d_lnW,
                               (int)n_e, (int)e_min, (int)split, beta, delta_lo, delta_hi,
                               (int)n_iter, d_res, d_bad + 1));
    }
    PCK(cudaMemcpyAsync(res.data(), d_res, res.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    PCK(cudaMemcpyAsync(bad.data(), d_bad, bad.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
#undef PCK
    if (bad[0]) {
        rc = pk_fail(MUCA_ERR_WINDOW, "a sample's E_Delta lies outside [e_min, e_min + n_e)");
        goto done;
    }
    for (int d = 0; d < n_sets; ++d)
        if (bad[1 + d]) {
            rc = pk_fail(MUCA_ERR_INVALID_ARG,
                         "muca_equal_height: [delta_lo, delta_hi] does not bracket the equal-height "
                         "field for data set " + std::to_string(d) +
                         " (the peak below split must be lower at delta_lo and higher at delta_hi)");
            goto done;
        }
    {
        double err[2] = {0.0, 0.0};
        if (n_jack > 0) {
            for (int q = 0; q < 2; ++q) {
                double mean = 0.0;
                for (int i = 0; i < n_jack; ++i) mean += res[5 * (1 + i) + q];
                mean /= n_jack;
                double ss = 0.0;
                for (int i = 0; i < n_jack; ++i) {
                    const double dv = res[5 * (1 + i) + q] - mean;
                    ss += dv * dv;
                }
                err[q] = std::sqrt((double)(n_jack - 1) / n_jack * ss);
            }
        }
        out[0] = res[0];
        out[1] = err[0];
        out[2] = res[1];
        out[3] = err[1];
        out[4] = res[2];
        out[5] = res[3];
        out[6] = res[4];
        for (int i = 0; i < n_jack; ++i) {
            out[7 + 2 * i] = res[5 * (1 + i)];
            out[8 + 2 * i] = res[5 * (1 + i) + 1];
        }
    }
done:
    cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
    return rc;
}
