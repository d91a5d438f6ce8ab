// reweight.cu -- time-series reweighting of a multicanonical run to a grid of
// crystal fields Delta_k (Eq. 3), with C(Delta) from Eq. 6, chi and U4.
//
// The multicanonical weight of a sample depends on the sample only through its
// E_Delta (Eq. 3: exp(-beta Delta E_Delta) / W(E_Delta)).  The GPU path therefore
// works in two stages:
//   A. one streaming pass over the samples accumulates, per E_Delta bin, exact
//      integer sums: count, sum E_J, sum |M|, sum M^2 and sum M^4 (128-bit);
//   B. for every Delta_k, a pass over the occupied bins: shift the exponents by
//      their maximum, exponentiate, and form the weighted sums; C and chi are
//      taken as centred second passes, so no difference of large moments is
//      ever formed.
// Stage B runs in FP64, or in FP32 where the exponent -beta Delta_k E - lnW(E)
// is carried as a float pair (hi + lo, error-free products and sums) so that
// its O(10^5) magnitude does not eat the 24-bit mantissa, and all sums are
// Kahan-compensated.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/muca.h"
#include "muca_internal.h"

namespace {

int rw_fail(int code, const std::string &msg)
{
    muca::set_last_error(msg.c_str());
    return code;
}

// Integer bin sums of stage A (device scratch).
struct Bins {
    unsigned long long *cnt;   // samples per bin
    unsigned long long *sej;   // sum E_J (two's complement)
    unsigned long long *sam;   // sum |M|
    unsigned long long *sm2;   // sum M^2
    unsigned long long *sm4lo; // sum M^4, low 64 bits
    unsigned long long *sm4hi; // sum M^4, high 64 bits
};

// Per-bin statistics consumed by stage B.
template <typename F>
struct BinStats {
    F *n;    // count
    F *mej;  // mean E_J in the bin
    F *cm;   // mean |m| in the bin, m = M / V
    F *vb;   // sum over the bin of (|m| - cm)^2
    F *q2;   // sum m^2
    F *q4;   // sum m^4
    F *lw;   // lnW (FP64) or its high float (FP32)
    F *lwlo; // FP32 only: lnW - hi
};

// Offset of a sample's E_Delta from the window start, formed in unsigned
// arithmetic so that it is defined for every int32 value; a sample lies in the
// window iff (unsigned)offset < nE (the argument check keeps e_min + nE - 1
// inside int32, so the window does not wrap).
__device__ __forceinline__ int bin_offset(int v, int e_min)
{
    return (int)((unsigned)v - (unsigned)e_min);
}

// Stage A, one sample at a time: every sum of every sample is a 64-bit
// atomic add into the global bin sums; M^4 is a 128-bit sum whose low word's
// returned old value gives the carry into the high word.
__global__ void bin_kernel(const int32_t *__restrict__ ej, const int32_t *__restrict__ ed,
                           const int32_t *__restrict__ m, int64_t n_rows, int row_len,
                           int64_t row_stride, int e_min, int nE, Bins b, int *err)
{
    for (int64_t r = blockIdx.y; r < n_rows; r += gridDim.y) {
        const int64_t base = r * row_stride;
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < row_len;
             c += gridDim.x * blockDim.x) {
            const int64_t o = base + c;
            const int e = bin_offset(__ldg(ed + o), e_min);
            if ((unsigned)e >= (unsigned)nE) {
                atomicOr(err, 1);
                continue;
            }
            const long long j = __ldg(ej + o);
            const long long mm = __ldg(m + o);
            const unsigned long long am = (unsigned long long)(mm < 0 ? -mm : mm);
            const unsigned long long m2 = am * am;
            const unsigned long long m4lo = m2 * m2, m4hi = __umul64hi(m2, m2);
            atomicAdd(b.cnt + e, 1ull);
            atomicAdd(b.sej + e, (unsigned long long)j);
            atomicAdd(b.sam + e, am);
            atomicAdd(b.sm2 + e, m2);
            const unsigned long long old = atomicAdd(b.sm4lo + e, m4lo);
            const unsigned long long carry = (old + m4lo < old) ? 1ull : 0ull;
            if (m4hi + carry) atomicAdd(b.sm4hi + e, m4hi + carry);
        }
    }
}

// ------------------------------------------------- stage A through buckets
// The same integer bin sums, formed without one global atomic per sample and
// without one shared atomic per sum.  Bins are grouped into buckets of kBkt
// consecutive bins.  Four launches per pass:
//   1. count: each block counts its samples per bucket and writes one counter
//      per (bucket, block);
//   2. scan: one block gives every (bucket, block) segment two places: where
//      its records are stored (block-major: a block's records of every bucket
//      in one region, so that a block writes to one neighbourhood of memory)
//      and where they stand in bucket order (bucket-major), the order the sums
//      walk in;
//   3. scatter: each block re-reads the same samples, takes places from its
//      own shared cursors and writes 8-byte records;
//   4. sums: each block takes an equal share of the records in bucket order,
//      gathering a bucket's segments through a table in shared memory,
//      counting-sorts tiles of them by bin in shared memory (one 32-bit shared
//      atomic per record), and every thread sums the run of its own bin in
//      registers; a bucket's sums go to the global bins once per block.
// A record holds the bin offset, E_J (|E_J| < 2^20) and |M| (<= 2^18, so
// M^4 <= 2^72); a sample outside those ranges is added straight to the global
// sums instead and leaves a null record.  Every sum stays an exact integer, so
// the result does not depend on the order in which records are summed.
constexpr int kBktBits = 10;
constexpr int kBkt = 1 << kBktBits;
constexpr unsigned kNullRec = 0xFFFFFFFFu;
constexpr int kMaxBk = 1024;      // buckets of the bucketed path (n_e <= 2^20)
constexpr int kMaxG = 1024;       // blocks of the count and scatter launches
constexpr int kCsThreads = 1024;  // threads of a count or scatter block
constexpr int kCsPer = 4;         // samples per thread and chunk
constexpr int kChunk = kCsThreads * kCsPer;  // samples of one row per chunk

__device__ __forceinline__ void direct_add(const Bins &b, int e, long long j, unsigned long long am)
{
    const unsigned long long m2 = am * am;
    const unsigned long long m4lo = m2 * m2, m4hi = __umul64hi(m2, m2);
    atomicAdd(b.cnt + e, 1ull);
    atomicAdd(b.sej + e, (unsigned long long)j);
    atomicAdd(b.sam + e, am);
    atomicAdd(b.sm2 + e, m2);
    const unsigned long long old = atomicAdd(b.sm4lo + e, m4lo);
    const unsigned long long carry = (old + m4lo < old) ? 1ull : 0ull;
    if (m4hi + carry) atomicAdd(b.sm4hi + e, m4hi + carry);
}

__device__ __forceinline__ unsigned warp_incl_scan(unsigned v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += u;
    }
    return v;
}

// Chunks of one block: chunk t is columns [(t % cpr) kChunk, + kChunk) of row
// t / cpr, and block i takes chunks [n i / G, n (i+1) / G) of the n = rows x
// cpr chunks.  The count and scatter launches share this partition; a block
// walks its chunks as (row, chunk of the row) without dividing per chunk.
struct ChunkWalk {
    int64_t t, t1, row;
    int ci;
    __device__ __forceinline__ ChunkWalk(int64_t n_rows, int cpr)
    {
        const int64_t n = n_rows * cpr;
        t = n * blockIdx.x / gridDim.x;
        t1 = n * (blockIdx.x + 1) / gridDim.x;
        row = t / cpr;
        ci = (int)(t - row * cpr);
    }
    __device__ __forceinline__ void next(int cpr)
    {
        ++t;
        if (++ci == cpr) {
            ci = 0;
            ++row;
        }
    }
};

// This thread's kCsPer values of one column in columns [col0, col0 + kChunk)
// of a row (0 past the row's end).
__device__ __forceinline__ void load_chunk(const int32_t *__restrict__ row, int col0, int row_len,
                                           int (&v)[kCsPer])
{
#pragma unroll
    for (int q = 0; q < kCsPer; ++q) {
        const int c = col0 + q * kCsThreads + threadIdx.x;
        v[q] = c < row_len ? __ldg(row + c) : 0;
    }
}

// Samples per (bucket, block), written to cnt[bucket * gridDim.x + block];
// flags a sample outside [e_min, e_min + nE).
__global__ void __launch_bounds__(kCsThreads)
bucket_count_kernel(const int32_t *__restrict__ ed, int64_t n_rows, int row_len,
                    int64_t row_stride, int e_min, int nE, int nbk, int cpr,
                    unsigned *__restrict__ cnt, int *err)
{
    __shared__ unsigned sc[kMaxBk];
    for (int i = threadIdx.x; i < nbk; i += blockDim.x) sc[i] = 0u;
    __syncthreads();
    // two chunks per step, so that twice the loads are in flight
    for (ChunkWalk w(n_rows, cpr); w.t < w.t1;) {
        int col[2];
        int v[2][kCsPer];
        col[0] = w.ci * kChunk;
        load_chunk(ed + w.row * row_stride, col[0], row_len, v[0]);
        w.next(cpr);
        const bool two = w.t < w.t1;
        col[1] = two ? w.ci * kChunk : row_len;
        if (two) {
            load_chunk(ed + w.row * row_stride, col[1], row_len, v[1]);
            w.next(cpr);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int q = 0; q < kCsPer; ++q) {
                const int c = col[h] + q * kCsThreads + threadIdx.x;
                const int e = bin_offset(v[h][q], e_min);
                const bool in = c < row_len, ok = in && (unsigned)e < (unsigned)nE;
                if (in && !ok) atomicOr(err, 1);
                if (ok) atomicAdd(&sc[(unsigned)e >> kBktBits], 1u);
            }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbk; i += blockDim.x) cnt[(size_t)i * gridDim.x + blockIdx.x] = sc[i];
}

// One block of 1024 threads.  In: cnt[k * g + b], the samples of bucket k in
// count block b (g <= 1024 blocks).  Out: lst[k * g + b], the segment's first
// place in bucket order; cnt[k * g + b] (in place), its first place in the
// record buffer (block b's segments of buckets 0, 1, ... one after another,
// after those of blocks 0 .. b-1); bstart / bcnt, each bucket's first place in
// bucket order and its size.
__global__ void __launch_bounds__(1024)
bucket_scan_kernel(unsigned *cnt, unsigned *lst, int nbk, int g, unsigned *bstart, unsigned *bcnt)
{
    __shared__ unsigned tot[kMaxBk];
    __shared__ unsigned ws[32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = w; k < nbk; k += 32) {
        unsigned s = 0u;
        for (int b = lane; b < g; b += 32) s += cnt[(size_t)k * g + b];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) tot[k] = s;
    }
    __syncthreads();
    // bucket order: exclusive scan of the bucket totals
    {
        const unsigned v = (int)threadIdx.x < nbk ? tot[threadIdx.x] : 0u;
        const unsigned incl = warp_incl_scan(v);
        if (lane == 31) ws[w] = incl;
        __syncthreads();
        const unsigned wv = ws[lane];
        const unsigned wi = warp_incl_scan(wv);
        const unsigned wex = __shfl_sync(0xffffffffu, wi - wv, w);
        __syncthreads();
        if ((int)threadIdx.x < nbk) {
            tot[threadIdx.x] = wex + incl - v;
            bstart[threadIdx.x] = wex + incl - v;
            bcnt[threadIdx.x] = v;
        }
        __syncthreads();
    }
    for (int k = w; k < nbk; k += 32) {
        unsigned run = tot[k];
        for (int b0 = 0; b0 < g; b0 += 32) {
            const int b = b0 + lane;
            const unsigned x = b < g ? cnt[(size_t)k * g + b] : 0u;
            const unsigned xi = warp_incl_scan(x);
            if (b < g) lst[(size_t)k * g + b] = run + xi - x;
            run += __shfl_sync(0xffffffffu, xi, 31);
        }
    }
    // storage order: thread b sums its block's counts, scans them over the
    // blocks, then lays its segments out bucket after bucket
    const int b = threadIdx.x;
    unsigned bt = 0u;
    if (b < g)
        for (int k = 0; k < nbk; ++k) bt += cnt[(size_t)k * g + b];
    const unsigned incl = warp_incl_scan(bt);
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    const unsigned wv = ws[lane];
    const unsigned wi = warp_incl_scan(wv);
    unsigned run = __shfl_sync(0xffffffffu, wi - wv, w) + incl - bt;
    if (b < g)
        for (int k = 0; k < nbk; ++k) {
            const unsigned x = cnt[(size_t)k * g + b];
            cnt[(size_t)k * g + b] = run;
            run += x;
        }
}

// Records: the block's samples of bucket k take places off[k * gridDim.x +
// block], +1, ... (the scan's storage places), handed out by shared cursors.
// A record is
// (bin offset in its bucket | (E_J + 2^20) << kBktBits, |M|).
__global__ void __launch_bounds__(kCsThreads)
bucket_scatter_kernel(const int32_t *__restrict__ ej, const int32_t *__restrict__ ed,
                      const int32_t *__restrict__ m, int64_t n_rows, int row_len,
                      int64_t row_stride, int e_min, int nE, int nbk, int cpr,
                      const unsigned *__restrict__ off, uint2 *__restrict__ rec, Bins b)
{
    __shared__ unsigned cur[kMaxBk];
    for (int i = threadIdx.x; i < nbk; i += blockDim.x)
        cur[i] = off[(size_t)i * gridDim.x + blockIdx.x];
    __syncthreads();
    for (ChunkWalk w(n_rows, cpr); w.t < w.t1; w.next(cpr)) {
        const int col0 = w.ci * kChunk;
        const int64_t base = w.row * row_stride;
        int vd[kCsPer], vj[kCsPer], vm[kCsPer];
        load_chunk(ed + base, col0, row_len, vd);
        load_chunk(ej + base, col0, row_len, vj);
        load_chunk(m + base, col0, row_len, vm);
#pragma unroll
        for (int q = 0; q < kCsPer; ++q) {
            const int c = col0 + q * kCsThreads + threadIdx.x;
            const int e = bin_offset(vd[q], e_min);
            const bool ok = c < row_len && (unsigned)e < (unsigned)nE;
            if (!ok) continue;
            const unsigned pos = atomicAdd(&cur[(unsigned)e >> kBktBits], 1u);
            const int j = vj[q], mm = vm[q];
            const unsigned am = mm < 0 ? 0u - (unsigned)mm : (unsigned)mm;
            uint2 rr;
            if (j > -(1 << 20) && j < (1 << 20) && am <= (1u << 18)) {
                rr.x = ((unsigned)e & (kBkt - 1)) | ((unsigned)(j + (1 << 20)) << kBktBits);
                rr.y = am;
            } else {
                direct_add(b, e, j, am);
                rr.x = 0u;
                rr.y = kNullRec;
            }
            rec[pos] = rr;
        }
    }
}

// Stage A sums.  Block i takes places [total i / G, total (i+1) / G) of
// bucket order; within each bucket it gathers tiles of kHS records through the
// bucket's segment table (place in bucket order -> place in the buffer), sorts
// each tile by bin in shared memory, and thread t sums bin t of the bucket in
// registers (count, E_J + 2^20, |M|, M^2 and M^4), which go to the global sums
// at the end of the bucket.  The sort buffers are double buffered, so a tile
// needs four barriers.
constexpr int kHT = kBkt;
constexpr int kHS = 8192;
constexpr int kHRpt = kHS / kHT;
constexpr size_t kHistSmem = 2 * (size_t)kHS * sizeof(uint2) + 3 * (size_t)kBkt * sizeof(unsigned) +
                             32 * sizeof(unsigned) + (2 * (size_t)kMaxG + 1) * sizeof(unsigned);

// Sums of one bin.  M^4 is kept as three 64-bit sums of 36-bit products: with
// M^2 = h 2^18 + l (h, l < 2^18), M^4 = h^2 2^36 + 2 h l 2^18 + l^2, exact for
// up to 2^28 records; the 128-bit value is formed once, at the flush.
struct BinAcc {
    unsigned n = 0u;
    unsigned long long j = 0ull, a = 0ull, q = 0ull, s0 = 0ull, s1 = 0ull, s2 = 0ull;
    __device__ __forceinline__ void add(uint2 r)
    {
        const unsigned am = r.y;
        const unsigned long long m2 = (unsigned long long)am * am;
        const unsigned h = (unsigned)(m2 >> 18), l = (unsigned)m2 & 0x3FFFFu;
        n += 1u;
        j += r.x >> kBktBits;
        a += am;
        q += m2;
        s0 += (unsigned long long)l * l;
        s1 += (unsigned long long)h * l;
        s2 += (unsigned long long)h * h;
    }
    __device__ __forceinline__ void flush(const Bins &b, int e)
    {
        if (!n) return;
        atomicAdd(b.cnt + e, (unsigned long long)n);
        atomicAdd(b.sej + e, j - ((unsigned long long)n << 20));
        atomicAdd(b.sam + e, a);
        atomicAdd(b.sm2 + e, q);
        const unsigned __int128 m4 = ((unsigned __int128)s2 << 36) + ((unsigned __int128)s1 << 19) + s0;
        const unsigned long long lo = (unsigned long long)m4, hi = (unsigned long long)(m4 >> 64);
        const unsigned long long old = atomicAdd(b.sm4lo + e, lo);
        const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
        if (hi + carry) atomicAdd(b.sm4hi + e, hi + carry);
        n = 0u;
        j = a = q = s0 = s1 = s2 = 0ull;
    }
};

__global__ void __launch_bounds__(kHT, 1)
bucket_hist_kernel(const uint2 *__restrict__ rec, const unsigned *__restrict__ pst,
                   const unsigned *__restrict__ lst, int g, const unsigned *__restrict__ bstart,
                   const unsigned *__restrict__ bcnt, int nbk, unsigned total, Bins b)
{
    extern __shared__ __align__(16) unsigned char hsm[];
    uint2 *srt0 = (uint2 *)hsm;                                  // [2][kHS]
    unsigned *scnt0 = (unsigned *)(hsm + 2 * kHS * sizeof(uint2)); // [2][kBkt]
    unsigned *soff = scnt0 + 2 * kBkt;                           // [kBkt]
    unsigned *wsum = soff + kBkt;                                // [32]
    unsigned *segL = wsum + 32;                                  // [g + 1] bucket order
    unsigned *segP = segL + kMaxG + 1;                           // [g] buffer
    const unsigned lo = (unsigned)((unsigned long long)total * blockIdx.x / gridDim.x);
    const unsigned hi = (unsigned)((unsigned long long)total * (blockIdx.x + 1) / gridDim.x);
    if (lo >= hi) return;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 2 * kBkt; i += kHT) scnt0[i] = 0u;
    int k = 0;
    while (k < nbk && bstart[k] + bcnt[k] <= lo) ++k;
    BinAcc acc;
    int buf = 0;
    for (; k < nbk && bstart[k] < hi; ++k) {
        const unsigned s_lo = max(lo, bstart[k]), s_hi = min(hi, bstart[k] + bcnt[k]);
        // the bucket's segment table (the previous bucket's last reads are done)
        __syncthreads();
        for (int i = tid; i < g; i += kHT) {
            segL[i] = lst[(size_t)k * g + i];
            segP[i] = pst[(size_t)k * g + i];
        }
        if (tid == 0) segL[g] = bstart[k] + bcnt[k];
        __syncthreads();
        // record j of the tile at s0: place s0 + j kHT + tid in bucket order,
        // in segment sg (segL[sg] <= place < segL[sg + 1]); places only grow
        // (the segment's end in bucket order and its buffer offset are kept in
        // registers; unsigned wrap-around makes i + dlt the buffer place)
        int sg = 0;
        unsigned send = segL[1], dlt = segP[0] - segL[0];
        auto load = [&](unsigned s0, uint2 (&r)[kHRpt]) {
#pragma unroll
            for (int q = 0; q < kHRpt; ++q) {
                const unsigned i = s0 + q * kHT + tid;
                if (i < s_hi) {
                    while (send <= i) {
                        ++sg;
                        send = segL[sg + 1];
                        dlt = segP[sg] - segL[sg];
                    }
                    r[q] = rec[i + dlt];
                } else {
                    r[q] = make_uint2(0u, kNullRec);
                }
            }
        };
        uint2 r[kHRpt];
        load(s_lo, r);
        for (unsigned s0 = s_lo; s0 < s_hi; s0 += kHS) {
            unsigned *scnt = scnt0 + buf * kBkt;
            uint2 *srt = srt0 + buf * kHS;
            unsigned rk[kHRpt];
#pragma unroll
            for (int q = 0; q < kHRpt; ++q)
                rk[q] = r[q].y != kNullRec ? atomicAdd(&scnt[r[q].x & (kBkt - 1)], 1u) : 0u;
            __syncthreads();
            const unsigned c = scnt[tid];
            const unsigned incl = warp_incl_scan(c);
            if (lane == 31) wsum[w] = incl;
            __syncthreads();
            const unsigned wv = wsum[lane];
            const unsigned wi = warp_incl_scan(wv);
            const unsigned o = __shfl_sync(0xffffffffu, wi - wv, w) + incl - c;
            soff[tid] = o;
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kHRpt; ++q)
                if (r[q].y != kNullRec) srt[soff[r[q].x & (kBkt - 1)] + rk[q]] = r[q];
            // the next tile's records, loaded while this tile is summed
            load(s0 + kHS, r);
            __syncthreads();
            unsigned i = o;
            for (; i + 1 < o + c; i += 2) {
                const uint2 x = srt[i], y = srt[i + 1];
                acc.add(x);
                acc.add(y);
            }
            if (i < o + c) acc.add(srt[i]);
            scnt[tid] = 0u;
            buf ^= 1;
        }
        acc.flush(b, k * kBkt + tid);
    }
}

__device__ __forceinline__ double u128_to_double(unsigned long long hi, unsigned long long lo)
{
    return (double)hi * 18446744073709551616.0 + (double)lo;
}

__device__ __forceinline__ float u128_to_float(unsigned long long hi, unsigned long long lo)
{
    return (float)hi * 18446744073709551616.0f + (float)lo;
}

// Stage A2: integer sums -> per-bin statistics.  vb uses the exact integer
// n sum M^2 - (sum |M|)^2 (128-bit) before any rounding.
__global__ void stats_kernel_f64(Bins b, int nE, int V, const double *__restrict__ lnW,
                                 BinStats<double> s)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    const unsigned long long n = b.cnt[e];
    s.lw[e] = lnW[e];
    if (n == 0) {
        s.n[e] = 0;
        return;
    }
    const double dn = (double)n, dV = (double)V;
    const long long sej = (long long)b.sej[e];
    const unsigned long long sam = b.sam[e], sm2 = b.sm2[e];
    const unsigned __int128 a = (unsigned __int128)n * sm2;
    const unsigned __int128 c = (unsigned __int128)sam * sam;
    const unsigned __int128 v = a - c;
    s.n[e] = dn;
    s.mej[e] = (double)sej / dn;
    s.cm[e] = (double)sam / dn / dV;
    s.vb[e] = u128_to_double((unsigned long long)(v >> 64), (unsigned long long)v) / dn / dV / dV;
    s.q2[e] = (double)sm2 / dV / dV;
    s.q4[e] = u128_to_double(b.sm4hi[e], b.sm4lo[e]) / dV / dV / dV / dV;
}

__global__ void stats_kernel_f32(Bins b, int nE, int V, const float *__restrict__ lw_hi,
                                 const float *__restrict__ lw_lo, BinStats<float> s)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    const unsigned long long n = b.cnt[e];
    s.lw[e] = lw_hi[e];
    s.lwlo[e] = lw_lo[e];
    if (n == 0) {
        s.n[e] = 0.f;
        return;
    }
    const float fn = (float)n, fV = (float)V;
    const long long sej = (long long)b.sej[e];
    const unsigned long long sam = b.sam[e], sm2 = b.sm2[e];
    const unsigned __int128 a = (unsigned __int128)n * sm2;
    const unsigned __int128 c = (unsigned __int128)sam * sam;
    const unsigned __int128 v = a - c;
    s.n[e] = fn;
    s.mej[e] = (float)sej / fn;
    s.cm[e] = (float)sam / fn / fV;
    s.vb[e] = u128_to_float((unsigned long long)(v >> 64), (unsigned long long)v) / fn / fV / fV;
    s.q2[e] = (float)sm2 / fV / fV;
    s.q4[e] = u128_to_float(b.sm4hi[e], b.sm4lo[e]) / fV / fV / fV / fV;
}

// ---------------------------------------------------------------- reductions
template <typename F>
struct KSum {  // Kahan-compensated accumulator
    F s, c;
    __device__ void init() { s = c = F(0); }
    __device__ void add(F x)
    {
        const F y = x - c;
        const F t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

template <typename F>
__device__ __forceinline__ F block_max(F v, F *sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    F r = sh[0];
    for (int i = 1; i < nw; ++i) r = fmax(r, sh[i]);
    return r;
}

// Sum of K compensated accumulators over the block; every thread gets the sums.
template <typename F, int K>
__device__ __forceinline__ void block_sum(KSum<F> (&a)[K], F (&out)[K], F *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        F s = a[k].s, c = -a[k].c;
        for (int o = 16; o > 0; o >>= 1) {
            const F s2 = __shfl_xor_sync(0xFFFFFFFFu, s, o);
            const F c2 = __shfl_xor_sync(0xFFFFFFFFu, c, o);
            // two-sum of s and s2 keeps the rounding error in c
            const F t = s + s2;
            const F bp = t - s;
            const F err = (s - (t - bp)) + (s2 - bp);
            s = t;
            c = c + c2 + err;
        }
        __syncthreads();
        if (lane == 0) {
            sh[2 * wid] = s;
            sh[2 * wid + 1] = c;
        }
        __syncthreads();
        KSum<F> tot;
        tot.init();
        F cc = F(0);
        for (int i = 0; i < nw; ++i) {
            tot.add(sh[2 * i]);
            cc += sh[2 * i + 1];
        }
        out[k] = tot.s + (cc - tot.c);
    }
}

// ------------------------------------------------------------ FP64 stage B
// Exponent of Eq. 3: a = -(c E) - lnW(E), c = beta Delta_k.  It is used to
// find the bin E* of the largest weight; the normalised exponents are then
// formed as -c (E - E*) - (lnW(E) - lnW(E*)) so that two O(beta Delta V) numbers
// are never subtracted.
__device__ __forceinline__ double expo64(double c, int E, double lw)
{
    return __dsub_rn(-__dmul_rn(c, (double)E), lw);
}

__device__ __forceinline__ double rel64(double c, int dE, double lw, double lstar)
{
    return __dsub_rn(-__dmul_rn(c, (double)dE), __dsub_rn(lw, lstar));
}

// Block-wide argmax of (value, bin); ties go to the smaller bin.
__device__ __forceinline__ void block_argmax(double &v, int &e, double *shv, int *she)
{
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xFFFFFFFFu, v, o);
        const int e2 = __shfl_xor_sync(0xFFFFFFFFu, e, o);
        if (v2 > v || (v2 == v && e2 < e)) {
            v = v2;
            e = e2;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        shv[wid] = v;
        she[wid] = e;
    }
    __syncthreads();
    v = shv[0];
    e = she[0];
    for (int i = 1; i < nw; ++i)
        if (shv[i] > v || (shv[i] == v && she[i] < e)) {
            v = shv[i];
            e = she[i];
        }
}

__global__ void __launch_bounds__(256)
grid_kernel_f64(BinStats<double> s, int nE, int e_min, double beta, int V,
                const double *__restrict__ cgrid, double *__restrict__ out)
{
    __shared__ double sh[64];
    __shared__ int she[32];
    const int k = blockIdx.x;
    const double c = cgrid[k];
    double amax = -INFINITY;
    int estar = 0x7FFFFFFF;
    for (int e = threadIdx.x; e < nE; e += blockDim.x)
        if (s.n[e] > 0) {
            const double a = expo64(c, e_min + e, s.lw[e]);
            if (a > amax) {
                amax = a;
                estar = e;
            }
        }
    block_argmax(amax, estar, sh, she);
    const double lstar = s.lw[estar];
    KSum<double> acc[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[i].init();
    for (int e = threadIdx.x; e < nE; e += blockDim.x) {
        const double n = s.n[e];
        if (n <= 0) continue;
        const double d = rel64(c, e - estar, s.lw[e], lstar);
        if (d < -800.0) continue;
        const double w = exp(d);
        const double wn = w * n;
        acc[0].add(wn);
        acc[1].add(wn * (double)(e_min + e));
        acc[2].add(wn * s.mej[e]);
        acc[3].add(wn * s.cm[e]);
        acc[4].add(w * s.q2[e]);
        acc[5].add(w * s.q4[e]);
    }
    double S[6];
    block_sum<double, 6>(acc, S, sh);
    const double Z = S[0], mE = S[1] / Z, mJ = S[2] / Z, mu = S[3] / Z;
    KSum<double> acc2[2];
    acc2[0].init();
    acc2[1].init();
    for (int e = threadIdx.x; e < nE; e += blockDim.x) {
        const double n = s.n[e];
        if (n <= 0) continue;
        const double d = rel64(c, e - estar, s.lw[e], lstar);
        if (d < -800.0) continue;
        const double w = exp(d);
        const double wn = w * n;
        acc2[0].add(wn * ((s.mej[e] - mJ) * ((double)(e_min + e) - mE)));
        const double dm = s.cm[e] - mu;
        acc2[1].add(w * s.vb[e] + wn * (dm * dm));
    }
    double S2[2];
    block_sum<double, 2>(acc2, S2, sh);
    if (threadIdx.x == 0) {
        double *o = out + 5 * (int64_t)k;
        o[0] = mJ;
        o[1] = mE;
        o[2] = -beta * (S2[0] / Z);
        o[3] = beta * (double)V * (S2[1] / Z);
        const double m2 = S[4] / Z, m4 = S[5] / Z;
        o[4] = 1.0 - m4 / (3.0 * m2 * m2);
    }
}

// ------------------------------------------------------------ FP32 stage B
// a = -(c_hi + c_lo) E - (lw_hi + lw_lo) as an unevaluated float pair.
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 expo32(float chi, float clo, int E, float lwh, float lwl)
{
    const float fe = (float)E;                  // exact: E < 2^24
    // the _rn intrinsics keep the compiler from fusing the error-free steps
    const float p = __fmul_rn(chi, fe);         // two-product: p + pe = chi E exactly
    const float pe = fmaf(chi, fe, -p);
    const float s = __fsub_rn(-p, lwh);         // two-sum of -p and -lwh
    const float bp = __fadd_rn(s, p);
    const float se = __fadd_rn(__fsub_rn(-p, __fsub_rn(s, bp)), __fsub_rn(-lwh, bp));
    const float lo = se - pe - fmaf(clo, fe, lwl);
    return {s, lo};
}

// One block serves kGridD consecutive Delta points, so that every bin's
// statistics are read once per kGridD points; per point, the arithmetic and the
// order of every sum are those of a block serving that point alone.
constexpr int kGridD = 4;

template <int D>
__global__ void __launch_bounds__(256, 4)  // four blocks per SM: more warps hide the latencies
grid_kernel_f32(BinStats<float> s, int nE, int e_min, float beta, int V,
                const float *__restrict__ c_hi, const float *__restrict__ c_lo, int n_grid,
                double *__restrict__ out)
{
    __shared__ float sh[64];
    const int k0 = blockIdx.x * D;
    float ch[D], cl[D], amax[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int k = min(k0 + d, n_grid - 1);
        ch[d] = c_hi[k];
        cl[d] = c_lo[k];
        amax[d] = -INFINITY;
    }
    for (int e = threadIdx.x; e < nE; e += blockDim.x)
        if (s.n[e] > 0.f) {
            const float lh = s.lw[e], ll = s.lwlo[e];
#pragma unroll
            for (int d = 0; d < D; ++d)
                amax[d] = fmaxf(amax[d], expo32(ch[d], cl[d], e_min + e, lh, ll).hi);
        }
#pragma unroll
    for (int d = 0; d < D; ++d) amax[d] = block_max(amax[d], sh);
    KSum<float> acc[D][6];
#pragma unroll
    for (int d = 0; d < D; ++d)
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[d][i].init();
    for (int e = threadIdx.x; e < nE; e += blockDim.x) {
        const float n = s.n[e];
        if (n <= 0.f) continue;
        const float lh = s.lw[e], ll = s.lwlo[e], mej = s.mej[e], cm = s.cm[e], q2 = s.q2[e],
                    q4 = s.q4[e];
        const float fe = (float)(e_min + e);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const F2 a = expo32(ch[d], cl[d], e_min + e, lh, ll);
            const float x = (a.hi - amax[d]) + a.lo;
            if (x < -104.f) continue;
            const float w = expf(x);
            const float wn = w * n;
            acc[d][0].add(wn);
            acc[d][1].add(wn * fe);
            acc[d][2].add(wn * mej);
            acc[d][3].add(wn * cm);
            acc[d][4].add(w * q2);
            acc[d][5].add(w * q4);
        }
    }
    float Z[D], mE[D], mJ[D], mu[D], m2[D], m4[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        float S[6];
        block_sum<float, 6>(acc[d], S, sh);
        Z[d] = S[0];
        mE[d] = S[1] / Z[d];
        mJ[d] = S[2] / Z[d];
        mu[d] = S[3] / Z[d];
        m2[d] = S[4] / Z[d];
        m4[d] = S[5] / Z[d];
    }
    KSum<float> acc2[D][2];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        acc2[d][0].init();
        acc2[d][1].init();
    }
    for (int e = threadIdx.x; e < nE; e += blockDim.x) {
        const float n = s.n[e];
        if (n <= 0.f) continue;
        const float lh = s.lw[e], ll = s.lwlo[e], mej = s.mej[e], cm = s.cm[e], vb = s.vb[e];
        const float fe = (float)(e_min + e);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const F2 a = expo32(ch[d], cl[d], e_min + e, lh, ll);
            const float x = (a.hi - amax[d]) + a.lo;
            if (x < -104.f) continue;
            const float w = expf(x);
            const float wn = w * n;
            acc2[d][0].add(wn * ((mej - mJ[d]) * (fe - mE[d])));
            const float dm = cm - mu[d];
            acc2[d][1].add(w * vb + wn * (dm * dm));
        }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
        float S2[2];
        block_sum<float, 2>(acc2[d], S2, sh);
        if (threadIdx.x == 0 && k0 + d < n_grid) {
            double *o = out + 5 * (int64_t)(k0 + d);
            o[0] = mJ[d];
            o[1] = mE[d];
            o[2] = -beta * (S2[0] / Z[d]);
            o[3] = beta * (float)V * (S2[1] / Z[d]);
            o[4] = 1.f - m4[d] / (3.f * m2[d] * m2[d]);
        }
    }
}

// Scratch layout of one call (bytes), all 256-byte aligned.
struct Scratch {
    size_t bins, stats, grid, out, err, total;
};

Scratch scratch_layout(int nE, int n_grid, int precision)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    Scratch s{};
    s.bins = al((size_t)6 * nE * sizeof(unsigned long long));
    s.stats = al((size_t)8 * nE * (precision == 32 ? sizeof(float) : sizeof(double)) +
                 (precision == 32 ? 2 * (size_t)nE * sizeof(float) : (size_t)nE * sizeof(double)));
    s.grid = al((size_t)2 * n_grid * sizeof(double));
    s.out = al((size_t)5 * n_grid * sizeof(double));
    s.err = al(sizeof(int));
    s.total = s.bins + s.stats + s.grid + s.out + s.err;
    return s;
}

// Buckets of a window of nE bins.
int bucket_count_of(int nE) { return (int)(((int64_t)nE + kBkt - 1) >> kBktBits); }

// Bytes of the bucket counters at the start of a record buffer (256-byte
// aligned): [nbk][kMaxG] storage places, [nbk][kMaxG] places in bucket order,
// then each bucket's start and size.
size_t bucket_counter_bytes(int nE)
{
    const size_t nbk = (size_t)bucket_count_of(nE);
    return ((2 * nbk * kMaxG + 2 * nbk) * sizeof(unsigned) + 255) & ~(size_t)255;
}

}  // namespace

namespace muca {

size_t reweight_record_bytes(int32_t n_e, int64_t n_samples)
{
    // windows of more than kMaxBk buckets take the direct path: no records
    if (bucket_count_of(n_e) > kMaxBk) return 0;
    const int64_t cap = std::min<int64_t>(n_samples, (int64_t)1 << 26);
    return bucket_counter_bytes(n_e) + (size_t)std::max<int64_t>(cap, 0) * sizeof(uint2);
}


// The whole reweighting on a caller-provided scratch region of
// scratch_layout(...).total bytes (device memory).
int reweight_on_scratch(const int32_t *e_j, const int32_t *e_d, const int32_t *m, int64_t n_rows,
                        int32_t row_len, int64_t row_stride, const double *lnW, int32_t e_min,
                        int32_t n_e, double beta, int32_t V, const double *delta_grid,
                        int32_t n_grid, int32_t precision, double *out, cudaStream_t st,
                        char *scratch, char *records, size_t records_bytes)
{
    const Scratch L = scratch_layout(n_e, n_grid, precision);
    char *p = scratch;
    Bins b;
    b.cnt = (unsigned long long *)p;
    b.sej = b.cnt + n_e;
    b.sam = b.sej + n_e;
    b.sm2 = b.sam + n_e;
    b.sm4lo = b.sm2 + n_e;
    b.sm4hi = b.sm4lo + n_e;
    char *ps = p + L.bins;
    char *pg = ps + L.stats;
    double *d_out = (double *)(pg + L.grid);
    int *d_err = (int *)((char *)d_out + L.out);
    cudaError_t ce;
#define RCK(call)                                                                   \
    do {                                                                            \
        ce = (call);                                                                \
        if (ce != cudaSuccess)                                                      \
            return rw_fail(MUCA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(ce)); \
    } while (0)
    RCK(cudaMemsetAsync(p, 0, L.bins, st));
    RCK(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    const int nbk = bucket_count_of(n_e);
    const size_t rec_cap =
        (records && nbk <= kMaxBk)
            ? (records_bytes - std::min(records_bytes, bucket_counter_bytes(n_e))) / sizeof(uint2)
            : 0;
    if (n_rows > 0 && row_len > 0 && (size_t)row_len <= rec_cap) {
        // stage A through buckets, a pass of at most rec_cap samples at a time
        unsigned *d_cnt = (unsigned *)records;  // [nbk][g], g <= kMaxG
        unsigned *d_lst = d_cnt + (size_t)nbk * kMaxG;
        unsigned *d_bstart = d_lst + (size_t)nbk * kMaxG, *d_bcnt = d_bstart + nbk;
        uint2 *d_rec = (uint2 *)(records + bucket_counter_bytes(n_e));
        int dev = 0, nsm = 152;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        RCK(cudaFuncSetAttribute(bucket_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kHistSmem));
        const int cpr = (int)(((int64_t)row_len + kChunk - 1) / kChunk);
        const int64_t rows_pass = std::min<int64_t>(n_rows, (int64_t)(rec_cap / (size_t)row_len));
        for (int64_t r0 = 0; r0 < n_rows; r0 += rows_pass) {
            const int64_t nr = std::min(rows_pass, n_rows - r0);
            const int64_t off = r0 * row_stride;
            // one 1024-thread block per SM
            const int g = (int)std::min<int64_t>(nr * cpr, std::min(nsm, kMaxG));
            bucket_count_kernel<<<g, kCsThreads, 0, st>>>(e_d + off, nr, row_len, row_stride,
                                                          e_min, n_e, nbk, cpr, d_cnt,
                                                          d_err);
            RCK(cudaGetLastError());
            bucket_scan_kernel<<<1, 1024, 0, st>>>(d_cnt, d_lst, nbk, g, d_bstart, d_bcnt);
            RCK(cudaGetLastError());
            bucket_scatter_kernel<<<g, kCsThreads, 0, st>>>(
                e_j + off, e_d + off, m + off, nr, row_len, row_stride, e_min, n_e, nbk, cpr,
                d_cnt, d_rec, b);
            RCK(cudaGetLastError());
            bucket_hist_kernel<<<nsm, kHT, kHistSmem, st>>>(d_rec, d_cnt, d_lst, g, d_bstart,
                                                           d_bcnt, nbk, (unsigned)(nr * row_len),
                                                           b);
            RCK(cudaGetLastError());
        }
    } else if (n_rows > 0 && row_len > 0) {
        dim3 grid((unsigned)std::min<int64_t>((row_len + 255) / 256, 1024),
                  (unsigned)std::min<int64_t>(n_rows, 4096));
        bin_kernel<<<grid, 256, 0, st>>>(e_j, e_d, m, n_rows, row_len, row_stride, e_min, n_e, b,
                                         d_err);
        RCK(cudaGetLastError());
    }
    const int sb = (n_e + 255) / 256;
    if (precision == 64) {
        BinStats<double> s;
        double *q = (double *)ps;
        s.n = q;
        s.mej = q + n_e;
        s.cm = q + 2 * (size_t)n_e;
        s.vb = q + 3 * (size_t)n_e;
        s.q2 = q + 4 * (size_t)n_e;
        s.q4 = q + 5 * (size_t)n_e;
        s.lw = q + 6 * (size_t)n_e;
        s.lwlo = nullptr;
        double *d_lnW = q + 7 * (size_t)n_e;
        double *d_c = (double *)pg;
        std::vector<double> c(n_grid);
        for (int k = 0; k < n_grid; ++k) c[k] = beta * delta_grid[k];
        RCK(cudaMemcpyAsync(d_lnW, lnW, (size_t)n_e * sizeof(double), cudaMemcpyHostToDevice, st));
        RCK(cudaMemcpyAsync(d_c, c.data(), (size_t)n_grid * sizeof(double),
                            cudaMemcpyHostToDevice, st));
        stats_kernel_f64<<<sb, 256, 0, st>>>(b, n_e, V, d_lnW, s);
        RCK(cudaGetLastError());
        if (n_grid > 0) grid_kernel_f64<<<n_grid, 256, 0, st>>>(s, n_e, e_min, beta, V, d_c, d_out);
        RCK(cudaGetLastError());
        // keep the host vectors alive until the copies are done
        RCK(cudaStreamSynchronize(st));
    } else {
        BinStats<float> s;
        float *q = (float *)ps;
        s.n = q;
        s.mej = q + n_e;
        s.cm = q + 2 * (size_t)n_e;
        s.vb = q + 3 * (size_t)n_e;
        s.q2 = q + 4 * (size_t)n_e;
        s.q4 = q + 5 * (size_t)n_e;
        s.lw = q + 6 * (size_t)n_e;
        s.lwlo = q + 7 * (size_t)n_e;
        float *d_lh = q + 8 * (size_t)n_e, *d_ll = q + 9 * (size_t)n_e;
        float *d_ch = (float *)pg, *d_cl = d_ch + n_grid;
        // inputs handed to the FP32 path as float pairs (hi + lo)
        std::vector<float> lh(n_e), ll(n_e), ch(n_grid), cl(n_grid);
        for (int e = 0; e < n_e; ++e) {
            lh[e] = (float)lnW[e];
            ll[e] = (float)(lnW[e] - (double)lh[e]);
        }
        for (int k = 0; k < n_grid; ++k) {
            const double c = beta * delta_grid[k];
            ch[k] = (float)c;
            cl[k] = (float)(c - (double)ch[k]);
        }
        RCK(cudaMemcpyAsync(d_lh, lh.data(), n_e * sizeof(float), cudaMemcpyHostToDevice, st));
        RCK(cudaMemcpyAsync(d_ll, ll.data(), n_e * sizeof(float), cudaMemcpyHostToDevice, st));
        RCK(cudaMemcpyAsync(d_ch, ch.data(), n_grid * sizeof(float), cudaMemcpyHostToDevice, st));
        RCK(cudaMemcpyAsync(d_cl, cl.data(), n_grid * sizeof(float), cudaMemcpyHostToDevice, st));
        stats_kernel_f32<<<sb, 256, 0, st>>>(b, n_e, V, d_lh, d_ll, s);
        RCK(cudaGetLastError());
        if (n_grid > 0)
            grid_kernel_f32<kGridD><<<(n_grid + kGridD - 1) / kGridD, 256, 0, st>>>(
                s, n_e, e_min, (float)beta, V, d_ch, d_cl, n_grid, d_out);
        RCK(cudaGetLastError());
        RCK(cudaStreamSynchronize(st));
    }
    int h_err = 0;
    RCK(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RCK(cudaMemcpyAsync(out, d_out, (size_t)5 * n_grid * sizeof(double), cudaMemcpyDeviceToHost,
                        st));
    RCK(cudaStreamSynchronize(st));
#undef RCK
    if (h_err) return rw_fail(MUCA_ERR_WINDOW, "a sample's E_Delta lies outside [e_min, e_min + n_e)");
    return MUCA_OK;
}

size_t reweight_scratch_bytes(int32_t n_e, int32_t n_grid, int32_t precision)
{
    return scratch_layout(n_e, n_grid, precision).total;
}

int reweight_check_args(const int32_t *e_j, const int32_t *e_d, const int32_t *m, int64_t n_rows,
                        int32_t row_len, int64_t row_stride, const double *lnW, int32_t e_min,
                        int32_t n_e,
                        double beta, int32_t V, const double *delta_grid, int32_t n_grid,
                        int32_t precision, double *out)
{
    if (!e_j || !e_d || !m || !lnW || !out || (n_grid > 0 && !delta_grid))
        return rw_fail(MUCA_ERR_INVALID_ARG, "muca_reweight: null pointer");
    if (n_rows < 0 || row_len < 0 || (n_rows > 1 && row_stride < row_len) || n_e < 1 || V < 1 ||
        n_grid < 0)
        return rw_fail(MUCA_ERR_INVALID_ARG, "muca_reweight: bad sizes");
    if (n_rows * (int64_t)row_len < 1)
        return rw_fail(MUCA_ERR_INVALID_ARG, "muca_reweight: no samples");
    if ((int64_t)e_min + n_e - 1 > INT32_MAX)
        return rw_fail(MUCA_ERR_INVALID_ARG, "muca_reweight: e_min + n_e - 1 exceeds int32");
    if (precision != 32 && precision != 64)
        return rw_fail(MUCA_ERR_INVALID_ARG, "muca_reweight: precision must be 32 or 64");
    if (!(beta > 0.0) || !std::isfinite(beta))
        return rw_fail(MUCA_ERR_INVALID_ARG, "muca_reweight: beta must be > 0");
    for (int e = 0; e < n_e; ++e)
        if (!std::isfinite(lnW[e])) return rw_fail(MUCA_ERR_INVALID_ARG, "muca_reweight: lnW not finite");
    for (int k = 0; k < n_grid; ++k)
        if (!std::isfinite(delta_grid[k]))
            return rw_fail(MUCA_ERR_INVALID_ARG, "muca_reweight: Delta grid not finite");
    return MUCA_OK;
}

}  // namespace muca

// Device memory pool of the reweighting on the current device, created on
// first use.  It keeps what it has once held (release threshold: all), so that
// repeated calls do not map and unmap their working memory each time.
static int reweight_pool(cudaMemPool_t *out)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = -1;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess)
        return rw_fail(MUCA_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
    if (dev < 0 || dev >= 64) return rw_fail(MUCA_ERR_NOT_SUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        ce = cudaMemPoolCreate(&p, &props);
        if (ce != cudaSuccess)
            return rw_fail(MUCA_ERR_CUDA, std::string("cudaMemPoolCreate: ") + cudaGetErrorString(ce));
        uint64_t keep = ~0ull;
        ce = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (ce != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return rw_fail(MUCA_ERR_CUDA, std::string("cudaMemPoolSetAttribute: ") +
                                              cudaGetErrorString(ce));
        }
        pools[dev] = p;
    }
    *out = pools[dev];
    return MUCA_OK;
}

extern "C" int muca_reweight(const int32_t *e_j, const int32_t *e_d, const int32_t *m,
                             int64_t n_rows, int32_t row_len, int64_t row_stride,
                             const double *lnW, int32_t e_min, int32_t n_e, double beta, int32_t V,
                             const double *delta_grid, int32_t n_grid, int32_t precision,
                             double *out, void *stream)
{
    int rc = muca::reweight_check_args(e_j, e_d, m, n_rows, row_len, row_stride, lnW, e_min, n_e,
                                       beta, V, delta_grid, n_grid, precision, out);
    if (rc != MUCA_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = muca::reweight_scratch_bytes(n_e, n_grid, precision);
    const size_t rbytes = muca::reweight_record_bytes(n_e, n_rows * (int64_t)row_len);
    cudaMemPool_t pool = nullptr;
    rc = reweight_pool(&pool);
    if (rc != MUCA_OK) return rc;
    void *scratch = nullptr;
    cudaError_t ce = cudaMallocFromPoolAsync(&scratch, bytes + rbytes, pool, st);
    if (ce != cudaSuccess)
        return rw_fail(ce == cudaErrorMemoryAllocation ? MUCA_ERR_OOM : MUCA_ERR_CUDA,
                       std::string("cudaMallocAsync: ") + cudaGetErrorString(ce));
    rc = muca::reweight_on_scratch(e_j, e_d, m, n_rows, row_len, row_stride, lnW, e_min, n_e, beta,
                                   V, delta_grid, n_grid, precision, out, st, (char *)scratch,
                                   (char *)scratch + bytes, rbytes);
    cudaFreeAsync(scratch, st);
    cudaStreamSynchronize(st);
    return rc;
}
