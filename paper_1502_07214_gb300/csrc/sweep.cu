// sweep.cu -- initial spins, energy tallies and the typewriter Metropolis sweep
// of the parallel multicanonical Blume-Capel simulation.
//
// Model: Eq. 1 of the paper, H = E_J + Delta E_Delta with E_J = -sum_<ij> s_i s_j
// and E_Delta = sum_i s_i^2 on an L^3 periodic simple-cubic lattice.  Update:
// single-site Metropolis with the multicanonical weight exp(-beta E_J) W(E_Delta)
// (Sec. II), visiting sites in typewriter order i = x + L (y + L z).
//
// GPU design.  Every walker is a strict serial chain: site x+1 sees the
// E_Delta and the spin that site x left behind.  Throughput is therefore
// (number of walkers) / (latency of one chain step), and the kernel is built
// to make that step short and to keep everything else off it.  The threshold
// a step reads depends on the walker's current E_Delta, so a dependent load
// sits on the chain; from L2 that load costs hundreds of cycles, from shared
// memory a few tens.  Each walker therefore keeps a window of kRing table
// rows around its E_Delta in shared memory (a ring indexed by row mod kRing),
// re-centred between rows with cp.async.  A row's chain reads only the window,
// without asking whether a row is there, and records the lowest and highest
// row it read; a walker whose row read outside the rows valid during it runs
// the row again from the global table.
//
// Two kernel designs share these pieces.  In the lane kernels (below), P lanes
// of a warp serve one walker (walker slot t / P, lane h = t % P) and do every
// phase of a row themselves; the warp-specialised kernel (further below) gives
// the chain a warp of its own and the other phases to helper warps.  In the
// lane kernels a row (fixed y, z) of L sites goes through these phases, staged
// in shared memory:
//   1. cp.async (L2 -> shared) of the NEXT row's old spins and of its four y/z
//      neighbour rows, and of the table rows that re-centre the window;
//   2. the Philox blocks of the row, split over the P lanes;
//   3. per-site descriptors, split over the P lanes: for site x the table
//      columns it can need (site x-1 accepted or rejected), the row shift of
//      site x-1's move, and site x's own move;
//   4. the chain, unrolled over the row: compare u with the threshold in
//      flight, select the next site's address, issue its load, record the
//      new spin - nothing else depends on the previous step;
//   5. the new spins of the row stored, and the energy
//      tallies from byte dot products of old and new spins:
//        dM = sum (N - O), dE_Delta = sum (N^2 - O^2),
//        dE_J = -sum (N - O) H - sum_cyclic (N_x N_{x+1} - O_x O_{x+1}),
//      which equals the sum of the per-site energy changes;
//   6. the next row's old spins and neighbour sums from the prefetched rows
//      (its y-1 neighbour is the row just finished).
// Sizes with L % 4 == 0 up to 48 use this path; any other L uses a plain
// per-site path with the same results.
#include <map>
#include <mutex>
#include <utility>
#include <cstdint>

#include "muca_internal.h"
#include "philox.cuh"

namespace muca {

namespace {

__device__ __forceinline__ int sbyte(uint32_t w, int q)
{
    return (int)(int8_t)(uint8_t)(w >> (8 * q));
}

// Warp-aggregated histogram increment: lanes holding the same bin elect one
// leader that adds the count of its peers (kernel (b) of the hot path).
__device__ __forceinline__ void hist_add(unsigned long long *hist, int bin, unsigned amask)
{
    const unsigned peers = __match_any_sync(amask, bin);
    const int leader = __ffs(peers) - 1;
    if ((int)(threadIdx.x & 31) == leader)
        atomicAdd(hist + bin, (unsigned long long)__popc(peers));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Running state of one walker between sweeps.
struct Chain {
    int EJ, ED, M;
};

// The proposal: bit 31 of the site's Philox word picks the smaller (0) or the
// larger (1) of the two values different from s.
__device__ __forceinline__ int proposal(int s, uint32_t word)
{
    const int lo = (s == -1) ? 0 : -1;
    const int hi = (s == 1) ? 0 : 1;
    return (word >> 31) ? hi : lo;
}

// ---------------------------------------------------------------------------
// Plain per-site path for any L >= 2 (neighbours read from the lattice).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int8_t *site_ptr(uint32_t *lat, ptrdiff_t st, int Lw, int row, int x)
{
    return reinterpret_cast<int8_t *>(lat + ((ptrdiff_t)row * Lw + (x >> 2)) * st) + (x & 3);
}

__device__ void sweep_sites(uint32_t *__restrict__ lat, ptrdiff_t st, int L, int Lw,
                            const uint32_t *__restrict__ thrE, int e_min, uint32_t key0,
                            uint32_t key1, uint64_t sw, Chain &c)
{
    const uint32_t slo = (uint32_t)sw, shi = (uint32_t)(sw >> 32);
    uint32_t r0 = 0, r1 = 0, r2 = 0, r3 = 0;
    int i = 0;
    for (int z = 0; z < L; ++z) {
        const int zm = z == 0 ? L - 1 : z - 1, zp = z + 1 == L ? 0 : z + 1;
        for (int y = 0; y < L; ++y) {
            const int ym = y == 0 ? L - 1 : y - 1, yp = y + 1 == L ? 0 : y + 1;
            const int row = z * L + y;
            for (int x = 0; x < L; ++x, ++i) {
                if ((i & 3) == 0) {
                    const uint4 r = philox4x32_10(make_uint4((uint32_t)(i >> 2), slo, shi, 0u),
                                                  key0, key1);
                    r0 = r.x;
                    r1 = r.y;
                    r2 = r.z;
                    r3 = r.w;
                }
                const uint32_t word = r0;
                r0 = r1;
                r1 = r2;
                r2 = r3;
                const int xm = x == 0 ? L - 1 : x - 1, xp = x + 1 == L ? 0 : x + 1;
                int8_t *p = site_ptr(lat, st, Lw, row, x);
                const int h = *site_ptr(lat, st, Lw, row, xm) + *site_ptr(lat, st, Lw, row, xp) +
                              *site_ptr(lat, st, Lw, z * L + ym, x) +
                              *site_ptr(lat, st, Lw, z * L + yp, x) +
                              *site_ptr(lat, st, Lw, zm * L + y, x) +
                              *site_ptr(lat, st, Lw, zp * L + y, x);
                const int s = *p;
                const int sp = proposal(s, word);
                const int d = sp * sp - s * s;
                const int dEJ = -(sp - s) * h;
                const int col = kBlk * (d + 1) + (d == 0 ? (dEJ + 12) >> 1 : dEJ + 6);
                const uint32_t t = __ldg(thrE + (ptrdiff_t)(c.ED - e_min) * kRow + col);
                if ((word & 0x7FFFFFFFu) < t) {
                    *p = (int8_t)sp;
                    c.EJ += dEJ;
                    c.ED += d;
                    c.M += sp - s;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Shared memory of a block, per walker slot (S slots):
//   staging fields laid out [field][index][slot] (lanes of different slots
//   touch consecutive words);
//   the table window: kRing rows of kRow words per slot, slot-major, slots
//   kRingStride words apart (16-byte aligned, padded to spread the banks).
// ---------------------------------------------------------------------------
constexpr int kMaxL = 48;
constexpr int kMaxLw = kMaxL / 4;
constexpr int kStageWords = 8 * kMaxLw + 4 * kMaxL;  // per slot
constexpr int kRing = 32;                            // table rows per walker window
constexpr int kRingStride = kRing * kRow + 4;        // words per slot
constexpr int kMargin = 14;                          // re-centre when this close to an edge

struct Stage {
    uint32_t *base;  // staging fields
    uint32_t *ring;  // table windows
    int S;
    // prefetched rows of the next row: f = 0 y-1, 1 y+1, 2 z-1, 3 z+1, 4 itself
    __device__ uint32_t *pf(int f, int j) const { return base + (f * kMaxLw + j) * S; }
    __device__ uint32_t *O(int j) const { return base + (5 * kMaxLw + j) * S; }
    __device__ uint32_t *H(int j) const { return base + (6 * kMaxLw + j) * S; }
    __device__ uint32_t *N(int j) const { return base + (7 * kMaxLw + j) * S; }
    __device__ uint32_t *rnd(int x) const { return base + (8 * kMaxLw + x) * S; }
    __device__ uint32_t *AUX(int x) const { return base + (8 * kMaxLw + kMaxL + x) * S; }
    __device__ uint32_t *win(int slot) const { return ring + (size_t)slot * kRingStride; }
};

// Where the block's walkers' lattices live: a [L*L][Lw][stride] word array
// (global: stride Wpad, shared tile: stride S), starting at the block's first walker.
struct BlockLattice {
    uint32_t *base;
    ptrdiff_t stride;
};

// The table window of one walker: rows [lo, lo + kRing) are (or, after the
// pending copies complete, will be) in the ring; [vlo, vhi) may be read now.
struct Window {
    int lo, vlo, vhi;
};

// Copy table rows [a, b) into the walker's ring (cp.async, 16-byte chunks,
// split over the walker's P lanes).
__device__ __forceinline__ void window_fill(uint32_t *win, const uint32_t *__restrict__ thrE,
                                            int a, int b, int P, int h)
{
    constexpr int kChunks = kRow / 4;
    const int n = (b - a) * kChunks;
    for (int c = h; c < n; c += P) {
        const int row = a + c / kChunks, k = c - (c / kChunks) * kChunks;
        cp_async16(win + (row & (kRing - 1)) * kRow + 4 * k, thrE + (ptrdiff_t)row * kRow + 4 * k);
    }
}

// The window position for table row e when the window is at lo: lo while e
// stays kMargin rows away from both edges, else the position that centres e,
// kept inside the table allocation [-kGuard, nE + kGuard).
__device__ __forceinline__ int window_target(int lo, int e, int nE)
{
    if (e >= lo + kMargin && e < lo + kRing - kMargin) return lo;
    int n = e - kRing / 2;
    n = max(n, -kGuard);
    return min(n, nE + kGuard - kRing);
}

// Rows [a, b) that enter the window when it moves from lo to n.
__device__ __forceinline__ void window_delta(int lo, int n, int &a, int &b)
{
    if (n > lo) {
        a = max(lo + kRing, n);
        b = n + kRing;
    } else if (n < lo) {
        a = n;
        b = min(lo, n + kRing);
    } else {
        a = b = 0;
    }
}

// Re-centre the window on row e if e came within kMargin rows of an edge:
// start the copies of the rows that enter it; [vlo, vhi) becomes the rows in
// both the old and the new window.
__device__ __forceinline__ void window_recentre(Window &wd, uint32_t *win,
                                                const uint32_t *__restrict__ thrE, int e, int nE,
                                                int P, int h)
{
    const int lo = window_target(wd.lo, e, nE);
    if (lo == wd.lo) return;
    int a, b;
    window_delta(wd.lo, lo, a, b);
    window_fill(win, thrE, a, b, P, h);
    wd.vlo = max(wd.lo, lo);
    wd.vhi = min(wd.lo, lo) + kRing;
    wd.lo = lo;
}

// Phase 1: copy the five rows around row (y1, z1) of all the block's walkers
// into the staging area.  In global memory the words of 4 consecutive walkers
// form one 16-byte chunk, copied with cp.async (completion awaited before
// phase 6); from a shared tile they are copied directly.
template <int L, bool GLOBAL>
__device__ __forceinline__ void stage_rows(const BlockLattice &bl, const Stage &sg, int y1,
                                           int z1, int nw, int tid, int nthreads)
{
    constexpr int Lw = L / 4;
    const int r_ym = z1 * L + (y1 == 0 ? L - 1 : y1 - 1), r_yp = z1 * L + (y1 + 1 == L ? 0 : y1 + 1);
    const int r_zm = (z1 == 0 ? L - 1 : z1 - 1) * L + y1, r_zp = (z1 + 1 == L ? 0 : z1 + 1) * L + y1;
    const int r_self = z1 * L + y1;
    auto row_of = [&](int f) {
        return f == 0 ? r_ym : f == 1 ? r_yp : f == 2 ? r_zm : f == 3 ? r_zp : r_self;
    };
    if (GLOBAL) {
        const int nch = (sg.S + 3) >> 2;  // 16-byte chunks per word
        for (int c = tid; c < 5 * Lw * nch; c += nthreads) {
            const int f = c / (Lw * nch), rem = c - f * (Lw * nch);
            const int j = rem / nch, k = rem - j * nch;
            cp_async16(sg.pf(f, j) + 4 * k,
                       bl.base + ((ptrdiff_t)row_of(f) * Lw + j) * bl.stride + 4 * k);
        }
    } else {
        for (int c = tid; c < 5 * Lw * nw; c += nthreads) {
            const int f = c / (Lw * nw), rem = c - f * (Lw * nw);
            const int j = rem / nw, k = rem - j * nw;
            sg.pf(f, j)[k] = bl.base[((ptrdiff_t)row_of(f) * Lw + j) * bl.stride + k];
        }
    }
}

// Phase 6: old spins and y/z neighbour sums of the row whose neighbourhood was
// staged; ym_is_new: its y-1 neighbour is the row just finished (N), not the
// staged copy.
template <int L>
__device__ __forceinline__ void build_row(const Stage &sg, int slot, int P, int h, bool ym_is_new)
{
    constexpr int Lw = L / 4;
    for (int j = h; j < Lw; j += P) {
        const uint32_t ym = ym_is_new ? sg.N(j)[slot] : sg.pf(0, j)[slot];
        sg.O(j)[slot] = sg.pf(4, j)[slot];
        sg.H(j)[slot] = __vadd4(__vadd4(ym, sg.pf(1, j)[slot]),
                                __vadd4(sg.pf(2, j)[slot], sg.pf(3, j)[slot]));
    }
}

// Descriptor of site x (phase 3), one word:
//   bits 0..5   column if site x-1 was accepted, 6..11 if it was rejected
//   bits 12..13 row shift of site x-1's move, plus 1
//   bits 14..15 d = s'^2 - s^2 of site x's move, plus 1
//   bits 16..17 s' + 1, bits 18..19 s + 1, bit 20 set iff s' > s
__device__ __forceinline__ int dsc_colA(uint32_t a) { return (int)(a & 63u); }
__device__ __forceinline__ int dsc_colR(uint32_t a) { return (int)((a >> 6) & 63u); }
__device__ __forceinline__ int dsc_dprev(uint32_t a) { return (int)((a >> 12) & 3u) - 1; }
__device__ __forceinline__ int dsc_d(uint32_t a) { return (int)((a >> 14) & 3u) - 1; }
__device__ __forceinline__ int dsc_sp(uint32_t a) { return (int)((a >> 16) & 3u) - 1; }
__device__ __forceinline__ int dsc_s(uint32_t a) { return (int)((a >> 18) & 3u) - 1; }
__device__ __forceinline__ int dsc_k(uint32_t a) { return (a >> 20) & 1u ? 1 : -1; }

// The chain of one walker over one row (phase 4), fully unrolled.  Inputs:
// the site descriptors and random words of the row (dsc[x * stride],
// rn[x * stride]); np: the packed new spins of the row's y-1 neighbour, added
// to the columns when ycorr (the split kernel leaves that neighbour out of the
// descriptors); e: the table row of E_Delta at the row start.  Returns the
// row of E_Delta at the row end and the row's new spins, packed (nn).
// It reads every threshold from the walker's window ring (row e at ring row
// e mod kRing) without asking whether row e is there; lo_e and hi_e return
// the lowest and highest row it read, so that the caller can check
// afterwards that all of them were in the window and otherwise run the row
// again with row_chain_global.  Nothing that depends on the previous step
// sits on the chain but the compare, the select of the next address and the
// load.
template <int L>
__device__ __forceinline__ int row_chain_fast(const uint32_t *dsc, const uint32_t *rn, int stride,
                                              const uint32_t (&np)[L / 4], bool ycorr, int e,
                                              const uint32_t *win, uint32_t (&nn)[L / 4],
                                              int &lo_e, int &hi_e)
{
    constexpr int Lw = L / 4;
    uint32_t ny[Lw];
#pragma unroll
    for (int j = 0; j < Lw; ++j) {
        ny[j] = ycorr ? np[j] : 0u;
        nn[j] = 0u;
    }
    const int kL = dsc_k(dsc[(L - 1) * stride]);
    uint32_t a = dsc[0];
    uint32_t u = rn[0] & 0x7FFFFFFFu;
    int ce = e, lo = e, hi = e;
    uint32_t t = win[(ce & (kRing - 1)) * kRow + dsc_colR(a) - dsc_k(a) * sbyte(ny[0], 0)];
    int corr = 0;  // column correction of site L-1: its x+1 is the new site 0
#pragma unroll
    for (int x = 0; x < L; ++x) {
        uint32_t a1 = 0u, u1 = 0u;
        int iA = 0, iR = 0;
        if (x + 1 < L) {
            a1 = dsc[(x + 1) * stride];
            u1 = rn[(x + 1) * stride] & 0x7FFFFFFFu;
            int cc = -dsc_k(a1) * sbyte(ny[(x + 1) >> 2], (x + 1) & 3);
            if (x + 1 == L - 1) cc += corr;
            iA = ((ce + dsc_dprev(a1)) & (kRing - 1)) * kRow + dsc_colA(a1) + cc;
            iR = (ce & (kRing - 1)) * kRow + dsc_colR(a1) + cc;
        }
        const bool acc = u < t;
        if (x + 1 < L) t = win[acc ? iA : iR];
        if (acc) ce += dsc_d(a);
        lo = min(lo, ce);
        hi = max(hi, ce);
        nn[x >> 2] |= (uint32_t)((acc ? dsc_sp(a) : dsc_s(a)) & 0xFF) << (8 * (x & 3));
        if (x == 0) corr = acc ? -kL * (dsc_sp(a) - dsc_s(a)) : 0;
        a = a1;
        u = u1;
    }
    lo_e = lo;
    hi_e = hi;
    return ce;
}

// The same row, every threshold read from the global table (rows -kGuard ..
// nE + kGuard - 1 are all there): the path of rows whose E_Delta left the
// window.  Site by site, not unrolled; np is nullptr when the row has no y-1
// correction.  Writes the row's packed new spins to nout[j * stride].
template <int L>
__device__ __noinline__ int row_chain_global(const uint32_t *dsc, const uint32_t *rn, int stride,
                                             const uint32_t *np, int e,
                                             const uint32_t *__restrict__ thrE, uint32_t *nout)
{
    const int kL = dsc_k(dsc[(L - 1) * stride]);
    bool prev = false;  // site x-1 accepted
    int corr = 0;
    uint32_t word = 0u;
#pragma unroll 1
    for (int x = 0; x < L; ++x) {
        const uint32_t a = dsc[x * stride];
        const uint32_t u = rn[x * stride] & 0x7FFFFFFFu;
        int col = prev ? dsc_colA(a) : dsc_colR(a);
        if (np) col -= dsc_k(a) * sbyte(np[(x >> 2) * stride], x & 3);
        if (x == L - 1) col += corr;
        const bool acc = u < __ldg(thrE + (ptrdiff_t)e * kRow + col);
        if (acc) e += dsc_d(a);
        word |= (uint32_t)((acc ? dsc_sp(a) : dsc_s(a)) & 0xFF) << (8 * (x & 3));
        if ((x & 3) == 3) {
            nout[(x >> 2) * stride] = word;
            word = 0u;
        }
        if (x == 0) corr = acc ? -kL * (dsc_sp(a) - dsc_s(a)) : 0;
        prev = acc;
    }
    return e;
}

// The unrolled row path (L % 4 == 0).  Threads of the block run this in lock
// step: all P lanes of a walker execute the chain on the same data.
template <int L, bool GLOBAL>
__device__ __forceinline__ void sweep_rows(const BlockLattice &bl, const Stage &sg,
                                           const uint32_t *__restrict__ thrE, int nE,
                                           uint32_t key0, uint32_t key1, uint64_t sw, int &e,
                                           Window &wd, Chain &c, int slot, int P, int h, int nw,
                                           int tid, int nthreads, unsigned amask)
{
    static_assert(L % 4 == 0 && L <= kMaxL, "row path needs L % 4 == 0, L <= 48");
    constexpr int Lw = L / 4, R = L * L;
    const uint32_t slo = (uint32_t)sw, shi = (uint32_t)(sw >> 32);
    uint32_t *const own = bl.base + slot;  // this walker's word 0
    uint32_t *const win = sg.win(slot);
    // the neighbourhood of row 0
    stage_rows<L, GLOBAL>(bl, sg, 0, 0, nw, tid, nthreads);
    window_recentre(wd, win, thrE, e, nE, P, h);
    cp_async_commit();
    cp_async_wait_all();
    wd.vlo = wd.lo;
    wd.vhi = wd.lo + kRing;
    __syncwarp(amask);
    build_row<L>(sg, slot, P, h, false);
    __syncwarp(amask);
    int y = 0, z = 0;
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        int y1 = y + 1, z1 = z;
        const bool wrap = (y1 == L);
        if (wrap) {
            y1 = 0;
            z1 = z + 1;
        }
        const bool more = r + 1 < R;
        // 1. the next row's neighbourhood; the table window
        if (more) stage_rows<L, GLOBAL>(bl, sg, y1, z1, nw, tid, nthreads);
        window_recentre(wd, win, thrE, e, nE, P, h);
        cp_async_commit();
        // 2. Philox blocks of this row (site i = r L + 4 j is block r Lw + j)
        for (int j = h; j < Lw; j += P) {
            const uint4 v =
                philox4x32_10(make_uint4((uint32_t)(r * Lw + j), slo, shi, 0u), key0, key1);
            sg.rnd(4 * j)[slot] = v.x;
            sg.rnd(4 * j + 1)[slot] = v.y;
            sg.rnd(4 * j + 2)[slot] = v.z;
            sg.rnd(4 * j + 3)[slot] = v.w;
        }
        __syncwarp(amask);
        // 3. descriptors of the row's sites
        for (int x = h; x < L; x += P) {
            const int s = sbyte(sg.O(x >> 2)[slot], x & 3);
            const int xr = (x + 1 == L) ? 0 : x + 1;  // old value of x = 0 for x = L-1;
            const int right = sbyte(sg.O(xr >> 2)[slot], xr & 3);  // corrected in the chain
            const int base = sbyte(sg.H(x >> 2)[slot], x & 3) + right;
            const int sp = proposal(s, sg.rnd(x)[slot]);
            const int d = sp * sp - s * s;
            const int k = sp > s ? 1 : -1;
            const int c0 = kBlk * (d + 1) + 6 - k * base;
            int ps, psp;
            if (x == 0) {
                ps = psp = sbyte(sg.O(Lw - 1)[slot], 3);  // x - 1 of x = 0: old x = L - 1
            } else {
                ps = sbyte(sg.O((x - 1) >> 2)[slot], (x - 1) & 3);
                psp = proposal(ps, sg.rnd(x - 1)[slot]);
            }
            const int pd = (x == 0) ? 0 : psp * psp - ps * ps;
            sg.AUX(x)[slot] = (uint32_t)(c0 - k * psp) | ((uint32_t)(c0 - k * ps) << 6) |
                              ((uint32_t)(pd + 1) << 12) | ((uint32_t)(d + 1) << 14) |
                              ((uint32_t)(sp + 1) << 16) | ((uint32_t)(s + 1) << 18) |
                              (k > 0 ? (1u << 20) : 0u);
        }
        __syncwarp(amask);
        // 4. the chain (every lane of the walker runs it on the same data),
        //    checked against the window that was complete while it ran
        uint32_t nn[Lw], np0[Lw];
#pragma unroll
        for (int j = 0; j < Lw; ++j) np0[j] = 0u;
        {
            int lo, hi;
            const int ce =
                row_chain_fast<L>(sg.AUX(0) + slot, sg.rnd(0) + slot, sg.S, np0, false, e, win, nn,
                                  lo, hi);
            if (lo >= wd.vlo && hi < wd.vhi) {
                e = ce;
            } else {
                e = row_chain_global<L>(sg.AUX(0) + slot, sg.rnd(0) + slot, sg.S, nullptr, e, thrE,
                                        sg.N(0) + slot);
#pragma unroll
                for (int j = 0; j < Lw; ++j) nn[j] = sg.N(j)[slot];
            }
        }
        // 5. new spins, their store, the tallies
#pragma unroll
        for (int j = 0; j < Lw; ++j) {
            if (j % P == h) {
                sg.N(j)[slot] = nn[j];
                own[((ptrdiff_t)r * Lw + j) * bl.stride] = nn[j];
            }
        }
        __syncwarp(amask);
        int dJ = 0, dM = 0, dD = 0;
        for (int j = h; j < Lw; j += P) {
            const uint32_t N0 = sg.N(j)[slot], O0 = sg.O(j)[slot];
            const int j1 = (j + 1 == Lw) ? 0 : j + 1;
            const uint32_t n1 = __funnelshift_r(N0, sg.N(j1)[slot], 8);
            const uint32_t o1 = __funnelshift_r(O0, sg.O(j1)[slot], 8);
            dJ -= __dp4a((int)__vsub4(N0, O0), (int)sg.H(j)[slot], 0);
            dJ -= __dp4a((int)N0, (int)n1, 0) - __dp4a((int)O0, (int)o1, 0);
            dM += __dp4a((int)N0, 0x01010101, 0) - __dp4a((int)O0, 0x01010101, 0);
            dD += __dp4a((int)N0, (int)N0, 0) - __dp4a((int)O0, (int)O0, 0);
        }
        for (int o = 1; o < P; o <<= 1) {
            dJ += __shfl_xor_sync(amask, dJ, o);
            dM += __shfl_xor_sync(amask, dM, o);
            dD += __shfl_xor_sync(amask, dD, o);
        }
        c.EJ += dJ;
        c.M += dM;
        c.ED += dD;
        // 6. the next row; the window copies are complete from here on
        cp_async_wait_all();
        wd.vlo = wd.lo;
        wd.vhi = wd.lo + kRing;
        __syncwarp(amask);
        if (more) build_row<L>(sg, slot, P, h, !wrap);
        __syncwarp(amask);
        y = y1;
        z = z1;
    }
}

template <bool RECORD, bool GLOBAL>
__device__ __forceinline__ void run_block(const GroupDev &g, const BlockDesc &bd,
                                          uint32_t *__restrict__ lat_block, ptrdiff_t st,
                                          uint32_t *__restrict__ stage, uint32_t *__restrict__ ring,
                                          uint32_t seed, uint64_t sweep0, int n_sweeps,
                                          int64_t ts_pos)
{
    const int P = bd.P, tid = (int)threadIdx.x, slot = tid / P, h = tid - slot * P;
    const bool active = slot < bd.nw;
    // lanes without a walker leave now; every warp-collective below names
    // only the lanes that stay
    const unsigned amask = __ballot_sync(0xFFFFFFFFu, active);
    const unsigned lead_mask = __ballot_sync(0xFFFFFFFFu, active && h == 0);
    if (!active) return;
    const int w = bd.w0 + slot;
    const uint32_t key0 = g.walker0 + (uint32_t)w;
    Chain c;
    c.EJ = g.tal[w];
    c.ED = g.tal[g.Wpad + w];
    c.M = g.tal[2 * g.Wpad + w];
    const BlockLattice bl{lat_block, st};
    const Stage sg{stage, ring, bd.S};
    const int nthreads = bd.nw * P;
    // an empty window: the first re-centre fills it completely
    Window wd{-(1 << 20), 0, 0};
    for (int k = 0; k < n_sweeps; ++k) {
        const uint64_t sw = sweep0 + (uint64_t)k;
        int e = c.ED - g.e_min;
        // the row path needs a table of at least one window
        switch (g.nE + 2 * kGuard >= kRing ? g.L : 0) {
#define MUCA_ROWS(LL)                                                                           \
    case LL:                                                                                    \
        sweep_rows<LL, GLOBAL>(bl, sg, g.thrE, g.nE, key0, seed, sw, e, wd, c, slot, P, h,    \
                               bd.nw, tid, nthreads, amask);                                    \
        break;
            MUCA_ROWS(4)
            MUCA_ROWS(8)
            MUCA_ROWS(12)
            MUCA_ROWS(16)
            MUCA_ROWS(20)
            MUCA_ROWS(24)
            MUCA_ROWS(28)
            MUCA_ROWS(32)
            MUCA_ROWS(48)
#undef MUCA_ROWS
            default:
                sweep_sites(lat_block + slot, st, g.L, g.Lw, g.thrE, g.e_min, key0, seed, sw, c);
                break;
        }
        if (h == 0) {
            hist_add(g.hist, c.ED - g.e_min, lead_mask);
            if (RECORD) {
                int32_t *o = g.ts + (ts_pos + k) * 3 * (int64_t)g.W + w;
                o[0] = c.EJ;
                o[g.W] = c.ED;
                o[2 * g.W] = c.M;
            }
        }
    }
    if (h == 0) {
        g.tal[w] = c.EJ;
        g.tal[g.Wpad + w] = c.ED;
        g.tal[2 * g.Wpad + w] = c.M;
    }
}

// A block is one warp; thread t serves walker slot t / P as lane t % P.
// Dynamic shared memory: the staging area of S slots, then their table windows.
template <bool RECORD>
__global__ void __launch_bounds__(32)
sweep_global_kernel(const GroupDev *__restrict__ groups, const BlockDesc *__restrict__ blocks,
                    uint32_t seed, uint64_t sweep0, int n_sweeps, int64_t ts_pos)
{
    extern __shared__ __align__(16) uint32_t s_dyn[];
    const BlockDesc bd = blocks[blockIdx.x];
    const GroupDev g = groups[bd.group];
    uint32_t *ring = s_dyn + (size_t)bd.S * kStageWords;
    run_block<RECORD, true>(g, bd, g.spins + bd.w0, g.Wpad, s_dyn, ring, seed, sweep0, n_sweeps,
                            ts_pos);
}

// Shared-memory-resident variant: the block's walkers keep their lattices in
// shared memory as a [L * L][Lw][S] word tile for the whole launch, read from
// and written back to the global array at the start and the end; the staging
// area and the table windows follow the tile.  A block is one warp.
template <bool RECORD>
__global__ void __launch_bounds__(32)
sweep_smem_kernel(const GroupDev *__restrict__ groups, const BlockDesc *__restrict__ blocks,
                  uint32_t seed, uint64_t sweep0, int n_sweeps, int64_t ts_pos)
{
    extern __shared__ __align__(16) uint32_t s_lat[];
    const BlockDesc bd = blocks[blockIdx.x];
    const GroupDev g = groups[bd.group];
    const int S = bd.S;
    const int nwords = g.L * g.L * g.Lw;
    for (int idx = threadIdx.x; idx < nwords * S; idx += blockDim.x) {
        const int wd = idx / S, c = idx - wd * S;
        s_lat[idx] = (c < bd.nw) ? g.spins[(ptrdiff_t)wd * g.Wpad + bd.w0 + c] : 0u;
    }
    __syncthreads();
    // the tile is padded to a 16-byte boundary
    uint32_t *stage = s_lat + (((size_t)nwords * S + 3) & ~(size_t)3);
    uint32_t *ring = stage + (size_t)S * kStageWords;
    run_block<RECORD, false>(g, bd, s_lat, S, stage, ring, seed, sweep0, n_sweeps, ts_pos);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nwords * S; idx += blockDim.x) {
        const int wd = idx / S, c = idx - wd * S;
        if (c < bd.nw) g.spins[(ptrdiff_t)wd * g.Wpad + bd.w0 + c] = s_lat[idx];
    }
}

// ---------------------------------------------------------------------------
// Warp-specialised variant (global lattice, L % 4 == 0 up to 48).  A block is
// kWsWarps warps: warp 0 runs the chains of the block's G walkers (one lane
// each) and nothing else; the other warps ("helpers") prepare the next row, finish
// the previous one and keep the chains' table windows filled, so that the
// per-row work overlaps the chain instead of adding to it:
//   helpers, iteration i:  wait until the chain finished row i-2; form its new
//     spins from its acceptance bits, store them and accumulate its energy
//     changes; copy the table rows the chain asked for at the end of row i-2
//     into its window; build the old spins and neighbour sums of row i from
//     the staged rows, draw its Philox words and proposals, write its site
//     descriptors; release row i to the chain; stage the neighbourhood of row
//     i+1 (cp.async).
//   chain, row r:  wait for row r; run the chain from the window; write the
//     row's acceptance bits; choose the window position for the rows to
//     come; release the row's buffers.
// The only input of row r+1 that depends on row r's outcome is the y-1
// neighbour.  The helpers form the columns of row r+1 with its old spins and
// store, per site, the column change if it was accepted; the chain applies it
// from the acceptance bits of row r, which it keeps in registers.  Likewise
// for site L-1, whose x+1 neighbour is site 0 of the same row.
// Window protocol: the rows asked for at the end of row r are copied by the
// helpers while the chain runs row r+1 and are complete when row r+2 starts
// (the helpers wait for their copies before they release a row), so row r+1
// may trust only rows that are in both the previous and the new window.
// Buffers: descriptors, random words, proposals, acceptance bits and window
// requests double-buffered by row parity; old spins, neighbour sums and new
// spins triple-buffered by row mod 3.  Descriptors and random words keep the
// four sites of a packed word together (16 bytes per walker slot), so a
// helper writes a word's four with one store and the chain reads a row's
// 2 L inputs with L / 2 loads: fewer shared-memory instructions beside the
// chain's dependent loads made the 48-site sweep 6 % faster.  Named barriers: ready[b] (helpers arrive, chain waits), free[b]
// (chain arrives, helpers wait), and one among the helpers.  Helper thread ht
// serves walker slot ht mod G and the words j = ht / G, ht / G + kWsHelp / G, ...
// of each row, so that its share of the energy changes belongs to one walker
// and is summed in registers over the sweep.
// ---------------------------------------------------------------------------
constexpr int kWsWarps = 8;
constexpr int kWsThreads = 32 * kWsWarps;
// Warp w of a block issues from scheduler w mod 4 of its SM.  Warp kWsIdle
// shares the chain warp's scheduler and only waits at the sweep barriers, so
// that no helper instruction competes with the chain for issue slots.
constexpr int kWsIdle = 4;
constexpr int kWsHelp = kWsThreads - 64;  // helper threads
constexpr int kWsSync = 32 + kWsHelp;     // threads of the ready / free barriers
// words of a row per helper thread: Lw <= kMaxLw words over at least
// kWsHelp / 32 helpers per walker slot
constexpr int kWsItems = (kMaxLw + kWsHelp / 32 - 1) / (kWsHelp / 32);
constexpr int kBarReady = 1, kBarFree = 3, kBarHelp = 5;
// shared words per walker slot: window, descriptors and random words x2, the
// packed-word buffers (O, H, N x3, staged rows x5, proposals x2), acceptance
// bits x2, window requests x2, tallies
constexpr int kWsWords = kRingStride + 4 * kMaxL + 16 * kMaxLw + 4 + 4 + 2;

__device__ __forceinline__ void bar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void bar_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

struct WsSmem {
    uint32_t *base;
    int G;
    __device__ uint32_t *win(int slot) const { return base + (size_t)slot * kRingStride; }
    __device__ uint32_t *rest() const { return base + (size_t)G * kRingStride; }
    // descriptors and random words of buffer b: site x of slot s at word
    // (x / 4) 4G + 4 s + x % 4, so that the four sites of a packed word are
    // one 16-byte unit (one store by a helper, one load by the chain)
    __device__ uint32_t *descq(int b) const { return rest() + b * kMaxL * G; }
    __device__ uint32_t *rndq(int b) const { return rest() + (2 + b) * kMaxL * G; }
    __device__ uint32_t *words(int k, int j) const
    {
        return rest() + 4 * kMaxL * G + (k * kMaxLw + j) * G;
    }
    __device__ uint32_t *O(int b, int j) const { return words(b, j); }
    __device__ uint32_t *H(int b, int j) const { return words(3 + b, j); }
    __device__ uint32_t *N(int b, int j) const { return words(6 + b, j); }
    __device__ uint32_t *pf(int f, int j) const { return words(9 + f, j); }
    __device__ uint32_t *SP(int b, int j) const { return words(14 + b, j); }
    __device__ uint32_t *ints() const { return rest() + 4 * kMaxL * G + 16 * kMaxLw * G; }
    // acceptance bits of a row: word q (sites 32 q ..) of slot s
    __device__ uint32_t *ACC(int b, int q, int slot) const { return ints() + (2 * b + q) * G + slot; }
    __device__ int *req(int b, int slot) const { return (int *)ints() + 4 * G + 2 * (b * G + slot); }
    __device__ int *tal(int slot) const { return (int *)ints() + 8 * G + 2 * slot; }
};

// Helpers: the five rows around row (y1, z1) of the block's walkers into pf.
template <int L>
__device__ __forceinline__ void ws_stage(const WsSmem &sm, const uint32_t *lat, ptrdiff_t st,
                                         int y1, int z1, int ht)
{
    constexpr int Lw = L / 4;
    const int r_ym = z1 * L + (y1 == 0 ? L - 1 : y1 - 1), r_yp = z1 * L + (y1 + 1 == L ? 0 : y1 + 1);
    const int r_zm = (z1 == 0 ? L - 1 : z1 - 1) * L + y1, r_zp = (z1 + 1 == L ? 0 : z1 + 1) * L + y1;
    const int r_self = z1 * L + y1;
    const int lg = __ffs(sm.G >> 2) - 1;  // chunks of 4 walkers per word: G / 4 (a power of 2)
    const int nch = sm.G >> 2;
    // the y-1 row is read only by rows with y = 0 (the others take the old
    // spins of the row before, already in shared memory)
    const int f0 = (y1 == 0) ? 0 : 1;
    for (int c = ht; c < (5 - f0) * Lw * nch; c += kWsHelp) {
        const int fj = c >> lg, k = c & (nch - 1);
        const int f = f0 + fj / Lw, j = fj - (fj / Lw) * Lw;
        const int row = f == 0 ? r_ym : f == 1 ? r_yp : f == 2 ? r_zm : f == 3 ? r_zp : r_self;
        cp_async16(sm.pf(f, j) + 4 * k, lat + ((ptrdiff_t)row * Lw + j) * st + 4 * k);
    }
    cp_async_commit();
}

// Site descriptor of the split kernel (written by the helpers), one word:
//   bits 0..5   column if site x-1 was accepted, 6..11 if it was rejected,
//               both with the old spin of the y-1 neighbour in the sum
//   bits 12..13 d = s'^2 - s^2 of site x's move, plus 1
//   bits 14..16 q + 2: the column change when the y-1 neighbour (row r-1,
//               same x) was accepted, -k (s'_y-1 - s_y-1); 0 on rows y = 0
//   bits 17..19 (site L-1 only) Q + 2: its column change when site 0 of the
//               same row was accepted
// Random words are stored with bit 31 cleared (the chain's u).
__device__ __forceinline__ int dw_colA(uint32_t a) { return (int)(a & 63u); }
__device__ __forceinline__ int dw_colR(uint32_t a) { return (int)((a >> 6) & 63u); }
__device__ __forceinline__ int dw_d(uint32_t a) { return (int)((a >> 12) & 3u) - 1; }
__device__ __forceinline__ int dw_q(uint32_t a) { return (int)((a >> 14) & 7u) - 2; }
__device__ __forceinline__ int dw_Q(uint32_t a) { return (int)((a >> 17) & 7u) - 2; }

// The chain of the split kernel over one row, fully unrolled, from the
// window (as row_chain_fast).  pacc: the acceptance bits of the y-1 row
// (zero when it gives no correction); returns E_Delta's row at the row end
// and the row's acceptance bits; lo_e / hi_e: the rows it read.
template <int L>
__device__ __forceinline__ int ws_chain_fast(const uint32_t *dsc, const uint32_t *rn, int stride,
                                             const uint32_t (&pacc)[(L + 31) / 32], int e,
                                             const uint32_t *win, uint32_t (&accb)[(L + 31) / 32],
                                             int &lo_e, int &hi_e)
{
    constexpr int NB = (L + 31) / 32;
    uint32_t A[L], U[L];
#pragma unroll
    for (int j = 0; j < L / 4; ++j) {
        const uint4 a = *reinterpret_cast<const uint4 *>(dsc + j * stride);
        const uint4 u = *reinterpret_cast<const uint4 *>(rn + j * stride);
        A[4 * j] = a.x;
        A[4 * j + 1] = a.y;
        A[4 * j + 2] = a.z;
        A[4 * j + 3] = a.w;
        U[4 * j] = u.x;
        U[4 * j + 1] = u.y;
        U[4 * j + 2] = u.z;
        U[4 * j + 3] = u.w;
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) accb[q] = 0u;
    auto ycc = [&](int x) { return ((pacc[x >> 5] >> (x & 31)) & 1u) ? dw_q(A[x]) : 0; };
    int ce = e, lo = e, hi = e;
    uint32_t t = win[(ce & (kRing - 1)) * kRow + dw_colR(A[0]) + ycc(0)];
    int corr = 0;  // column change of site L-1: its x+1 is the new site 0
#pragma unroll
    for (int x = 0; x < L; ++x) {
        int iA = 0, iR = 0;
        if (x + 1 < L) {
            int cc = ycc(x + 1);
            if (x + 1 == L - 1) cc += corr;
            iA = ((ce + dw_d(A[x])) & (kRing - 1)) * kRow + dw_colA(A[x + 1]) + cc;
            iR = (ce & (kRing - 1)) * kRow + dw_colR(A[x + 1]) + cc;
        }
        const bool acc = U[x] < t;
        if (x + 1 < L) t = win[acc ? iA : iR];
        if (acc) {
            ce += dw_d(A[x]);
            accb[x >> 5] |= 1u << (x & 31);
        }
        lo = min(lo, ce);
        hi = max(hi, ce);
        if (x == 0) corr = acc ? dw_Q(A[L - 1]) : 0;
    }
    lo_e = lo;
    hi_e = hi;
    return ce;
}

// The same row from the global table, site by site (rows whose E_Delta left
// the window).  pacc points to the y-1 row's acceptance bits (word q at
// pacc[q * G]) or is nullptr; the row's bits go to accb[q * G].
template <int L>
__device__ __noinline__ int ws_chain_global(const uint32_t *dsc, const uint32_t *rn, int stride,
                                            const uint32_t *pacc, int e,
                                            const uint32_t *__restrict__ thrE, uint32_t *accb,
                                            int G)
{
    bool prev = false;  // site x-1 accepted
    int corr = 0;
    uint32_t bits = 0u;
#pragma unroll 1
    for (int x = 0; x < L; ++x) {
        const uint32_t a = dsc[(x >> 2) * stride + (x & 3)];
        int col = prev ? dw_colA(a) : dw_colR(a);
        if (pacc && ((pacc[(x >> 5) * G] >> (x & 31)) & 1u)) col += dw_q(a);
        if (x == L - 1) col += corr;
        const bool acc = rn[(x >> 2) * stride + (x & 3)] < __ldg(thrE + (ptrdiff_t)e * kRow + col);
        if (acc) {
            e += dw_d(a);
            bits |= 1u << (x & 31);
        }
        if ((x & 31) == 31 || x == L - 1) {
            accb[(x >> 5) * G] = bits;
            bits = 0u;
        }
        if (x == 0) corr = acc ? dw_Q(dsc[((L - 1) >> 2) * stride + ((L - 1) & 3)]) : 0;
        prev = acc;
    }
    return e;
}

// Bytes of word j of a row's new spins: the proposal where the site's
// acceptance bit is set, else the old spin.
__device__ __forceinline__ uint32_t new_word(uint32_t old, uint32_t prop, uint32_t bits4)
{
    const uint32_t m = ((bits4 * 0x00204081u) & 0x01010101u) * 0xFFu;
    return (prop & m) | (old & ~m);
}

template <int L, bool RECORD>
__device__ __forceinline__ void ws_sweeps(const GroupDev &g, const BlockDesc &bd,
                                          const WsSmem &sm, uint32_t seed, uint64_t sweep0,
                                          int n_sweeps, int64_t ts_pos)
{
    constexpr int Lw = L / 4, R = L * L;
    const int tid = (int)threadIdx.x;
    const int G = sm.G, nw = bd.nw;
    uint32_t *const lat = g.spins + bd.w0;  // word (row, j) of slot s: lat[(row Lw + j) Wpad + s]
    const ptrdiff_t st = g.Wpad;
    const uint32_t *__restrict__ thrE = g.thrE;
    if (tid < 32) {
        // ------------------------------------------------------------ chain warp
        const int slot = tid;
        const bool active = slot < nw;
        const unsigned amask = __ballot_sync(0xFFFFFFFFu, active);
        const int w = bd.w0 + slot;
        Chain c{0, 0, 0};
        uint32_t *const win = sm.win(slot < G ? slot : 0);
        // lo_a: the window once every copy asked for so far is complete;
        // lo_b: the window before the last request
        int lo_a = 0, lo_b = 0;
        if (active) {
            c.EJ = g.tal[w];
            c.ED = g.tal[g.Wpad + w];
            c.M = g.tal[2 * g.Wpad + w];
            lo_a = window_target(-(1 << 20), c.ED - g.e_min, g.nE);
            window_fill(win, thrE, lo_a, lo_a + kRing, 1, 0);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp();
        for (int k = 0; k < n_sweeps; ++k) {
            int e = c.ED - g.e_min;
            lo_b = lo_a;  // the requests of the last sweep are complete when row 0 starts
            constexpr int NB = (L + 31) / 32;
            uint32_t pacc[NB];  // acceptance bits of the previous row
#pragma unroll
            for (int q = 0; q < NB; ++q) pacc[q] = 0u;
#pragma unroll 1
            for (int r = 0; r < R; ++r) {
                bar_sync(kBarReady + (r & 1), kWsSync);
                if (active) {
                    const int b = r & 1;
                    const int vlo = max(lo_a, lo_b), vhi = min(lo_a, lo_b) + kRing;
                    uint32_t accb[NB];
                    int lo, hi;
                    const int ce = ws_chain_fast<L>(sm.descq(b) + 4 * slot, sm.rndq(b) + 4 * slot, 4 * G,
                                                    pacc, e, win, accb, lo, hi);
                    if (lo >= vlo && hi < vhi) {
                        e = ce;
#pragma unroll
                        for (int q = 0; q < NB; ++q) sm.ACC(b, q, slot)[0] = accb[q];
                    } else {
                        e = ws_chain_global<L>(sm.descq(b) + 4 * slot, sm.rndq(b) + 4 * slot, 4 * G,
                                               sm.ACC(b ^ 1, 0, slot), e, thrE, sm.ACC(b, 0, slot),
                                               G);
#pragma unroll
                        for (int q = 0; q < NB; ++q) accb[q] = sm.ACC(b, q, slot)[0];
                    }
#pragma unroll
                    for (int q = 0; q < NB; ++q) pacc[q] = accb[q];
                    // the window for the rows to come
                    const int lo_c = window_target(lo_a, e, g.nE);
                    int ra, rb;
                    window_delta(lo_a, lo_c, ra, rb);
                    sm.req(b, slot)[0] = ra;
                    sm.req(b, slot)[1] = rb;
                    lo_b = lo_a;
                    lo_a = lo_c;
                }
                __syncwarp();
                bar_arrive(kBarFree + (r & 1), kWsSync);
            }
            c.ED = e + g.e_min;
            __syncthreads();  // the helpers' tallies of this sweep are complete
            if (active) {
                c.EJ += sm.tal(slot)[0];
                c.M += sm.tal(slot)[1];
                sm.tal(slot)[0] = 0;
                sm.tal(slot)[1] = 0;
                hist_add(g.hist, c.ED - g.e_min, amask);
                if (RECORD) {
                    int32_t *o = g.ts + (ts_pos + k) * 3 * (int64_t)g.W + w;
                    o[0] = c.EJ;
                    o[g.W] = c.ED;
                    o[2 * g.W] = c.M;
                }
            }
            __syncthreads();  // tallies cleared before the helpers add again
        }
        if (active) {
            g.tal[w] = c.EJ;
            g.tal[g.Wpad + w] = c.ED;
            g.tal[2 * g.Wpad + w] = c.M;
        }
    } else if ((tid >> 5) == kWsIdle) {
        for (int k = 0; k < n_sweeps; ++k) {
            __syncthreads();
            __syncthreads();
        }
    } else {
        // ------------------------------------------------------------ helpers
        const int ht = tid - ((tid >> 5) > kWsIdle ? 64 : 32);
        const int lgG = __ffs(G) - 1;
        const int hs = ht & (G - 1);       // walker slot
        const int hj0 = ht >> lgG;         // first word of the slot's rows
        const int hstep = kWsHelp >> lgG;  // helpers per slot
        const bool hact = hs < nw;
        const uint32_t key0 = g.walker0 + (uint32_t)(bd.w0 + hs);
        uint32_t *const hwin = sm.win(hs);
        // CARRY (rows of up to 32 sites): the thread's words j = hj0 + t hstep
        // (t < kWsItems) keep their old spins, proposals and neighbour sums in
        // registers for the two rows in flight (c*: the row prepared last, p*:
        // the row before) and pN the new spins of the row finished last; only
        // neighbouring words are read from shared memory.  Without CARRY every
        // word goes through shared memory (measured faster for L = 48, slower
        // for L <= 32).
        constexpr bool CARRY = L <= 32;
        uint32_t cO[kWsItems], cS[kWsItems], cH[kWsItems];
        uint32_t pO[kWsItems], pS[kWsItems], pH[kWsItems], pN[kWsItems];
#pragma unroll
        for (int t = 0; t < kWsItems; ++t) cO[t] = cS[t] = cH[t] = pO[t] = pS[t] = pH[t] = pN[t] = 0u;
        for (int k = 0; k < n_sweeps; ++k) {
            const uint64_t sw = sweep0 + (uint64_t)k;
            const uint32_t slo = (uint32_t)sw, shi = (uint32_t)(sw >> 32);
            int dJ = 0, dM = 0;
            ws_stage<L>(sm, lat, st, 0, 0, ht);
#pragma unroll 1
            for (int i = 0; i < R + 2; ++i) {
                if (i >= 2) {
                    bar_sync(kBarFree + (i & 1), kWsSync);
                    // finish row jr = i - 2: store its new spins, add its energy changes
                    const int jr = i - 2;
                    const bool nonwrap = (jr % L != 0);
                    const int bj = jr % 3, bp = (jr + 2) % 3, ba = jr & 1;
                    if (hact) {
                        // new spins of word jj of row jr from its acceptance bits
                        auto nword = [&](int jj, uint32_t o, uint32_t sp) {
                            const uint32_t bits4 =
                                (sm.ACC(ba, (4 * jj) >> 5, hs)[0] >> ((4 * jj) & 31)) & 15u;
                            return new_word(o, sp, bits4);
                        };
                        if constexpr (CARRY) {
#pragma unroll
                            for (int t = 0; t < kWsItems; ++t) {
                                const int j = hj0 + t * hstep;
                                if (j >= Lw) break;
                                const int j1 = (j + 1 == Lw) ? 0 : j + 1;
                                const uint32_t O0 = pO[t], O1 = sm.O(bj, j1)[hs];
                                const uint32_t N0 = nword(j, O0, pS[t]);
                                const uint32_t n1 =
                                    __funnelshift_r(N0, nword(j1, O1, sm.SP(ba, j1)[hs]), 8);
                                const uint32_t o1 = __funnelshift_r(O0, O1, 8);
                                const uint32_t Hw = nonwrap ? __vadd4(pH[t], pN[t]) : pH[t];
                                dJ -= __dp4a((int)__vsub4(N0, O0), (int)Hw, 0);
                                dJ -= __dp4a((int)N0, (int)n1, 0) - __dp4a((int)O0, (int)o1, 0);
                                dM += __dp4a((int)N0, 0x01010101, 0) -
                                      __dp4a((int)O0, 0x01010101, 0);
                                lat[((ptrdiff_t)jr * Lw + j) * st + hs] = N0;
                                pN[t] = N0;
                            }
                        } else {
                            for (int j = hj0; j < Lw; j += hstep) {
                                const uint32_t O0 = sm.O(bj, j)[hs];
                                const uint32_t N0 = nword(j, O0, sm.SP(ba, j)[hs]);
                                sm.N(bj, j)[hs] = N0;
                                const int j1 = (j + 1 == Lw) ? 0 : j + 1;
                                const uint32_t O1 = sm.O(bj, j1)[hs];
                                const uint32_t n1 =
                                    __funnelshift_r(N0, nword(j1, O1, sm.SP(ba, j1)[hs]), 8);
                                const uint32_t o1 = __funnelshift_r(O0, O1, 8);
                                uint32_t Hw = sm.H(bj, j)[hs];
                                if (nonwrap) Hw = __vadd4(Hw, sm.N(bp, j)[hs]);
                                dJ -= __dp4a((int)__vsub4(N0, O0), (int)Hw, 0);
                                dJ -= __dp4a((int)N0, (int)n1, 0) - __dp4a((int)O0, (int)o1, 0);
                                dM += __dp4a((int)N0, 0x01010101, 0) -
                                      __dp4a((int)O0, 0x01010101, 0);
                                lat[((ptrdiff_t)jr * Lw + j) * st + hs] = N0;
                            }
                        }
                        // the table rows the chain asked for at the end of row jr
                        const int ra = sm.req(jr & 1, hs)[0], rb = sm.req(jr & 1, hs)[1];
                        constexpr int kChunks = kRow / 4;
                        for (int q = hj0; q < (rb - ra) * kChunks; q += hstep) {
                            const int row = ra + q / kChunks, part = q - (q / kChunks) * kChunks;
                            cp_async16(hwin + (row & (kRing - 1)) * kRow + 4 * part,
                                       thrE + (ptrdiff_t)row * kRow + 4 * part);
                        }
                    }
                    cp_async_commit();
                }
                if constexpr (CARRY) {
                    // the row prepared last becomes the row before
#pragma unroll
                    for (int t = 0; t < kWsItems; ++t) {
                        pO[t] = cO[t];
                        pS[t] = cS[t];
                        pH[t] = cH[t];
                    }
                }
                if (i < R) {
                    // prepare row i
                    const bool wrap = (i % L == 0);
                    const int bo = i % 3, b = i & 1;
                    cp_async_wait_all();
                    bar_sync(kBarHelp, kWsHelp);
                    if (hact) {
                        // old spins, neighbour sums, Philox words, proposals (the
                        // words unrolled only with CARRY: for 48-site rows the
                        // unrolled helpers slowed the chain down)
#pragma unroll(CARRY ? kWsItems : 1)
                        for (int t = 0; t < kWsItems; ++t) {
                            const int j = hj0 + t * hstep;
                            if (j >= Lw) break;
                            const uint32_t o = sm.pf(4, j)[hs];
                            uint32_t Hw =
                                __vadd4(sm.pf(1, j)[hs], __vadd4(sm.pf(2, j)[hs], sm.pf(3, j)[hs]));
                            if (wrap) Hw = __vadd4(Hw, sm.pf(0, j)[hs]);
                            sm.O(bo, j)[hs] = o;
                            if constexpr (CARRY) {
                                cO[t] = o;
                                cH[t] = Hw;
                            } else {
                                sm.H(bo, j)[hs] = Hw;
                            }
                            const uint4 v = philox4x32_10(
                                make_uint4((uint32_t)(i * Lw + j), slo, shi, 0u), key0, seed);
                            *reinterpret_cast<uint4 *>(sm.rndq(b) + j * 4 * G + 4 * hs) =
                                make_uint4(v.x & 0x7FFFFFFFu, v.y & 0x7FFFFFFFu, v.z & 0x7FFFFFFFu,
                                           v.w & 0x7FFFFFFFu);
                            const uint32_t spw =
                                ((uint32_t)proposal(sbyte(o, 0), v.x) & 0xFFu) |
                                (((uint32_t)proposal(sbyte(o, 1), v.y) & 0xFFu) << 8) |
                                (((uint32_t)proposal(sbyte(o, 2), v.z) & 0xFFu) << 16) |
                                (((uint32_t)proposal(sbyte(o, 3), v.w) & 0xFFu) << 24);
                            if constexpr (CARRY) cS[t] = spw;
                            sm.SP(b, j)[hs] = spw;
                        }
                    }
                    bar_sync(kBarHelp, kWsHelp);
                    if (hact) {
                        // descriptors of the four sites of each word
                        const int bq = (i + 2) % 3;  // row i-1: its old spins
                        const int s0 = sbyte(sm.O(bo, 0)[hs], 0), sp0 = sbyte(sm.SP(b, 0)[hs], 0);
#pragma unroll(CARRY ? kWsItems : 1)
                        for (int t = 0; t < kWsItems; ++t) {
                            const int j = hj0 + t * hstep;
                            if (j >= Lw) break;
                            const int jl = (j == 0) ? Lw - 1 : j - 1, jn = (j + 1 == Lw) ? 0 : j + 1;
                            uint32_t o, spw, Hw, yo = 0u, yp = 0u;
                            if constexpr (CARRY) {
                                o = cO[t];
                                spw = cS[t];
                                Hw = cH[t];
                            } else {
                                o = sm.O(bo, j)[hs];
                                spw = sm.SP(b, j)[hs];
                                Hw = sm.H(bo, j)[hs];
                            }
                            const uint32_t ol = sm.O(bo, jl)[hs], spl = sm.SP(b, jl)[hs];
                            const uint32_t on = sm.O(bo, jn)[hs];
                            // neighbour sums with the old y-1 row; its changes: yo -> yp
                            if (!wrap) {
                                if constexpr (CARRY) {
                                    yo = pO[t];
                                    yp = pS[t];
                                } else {
                                    yo = sm.O(bq, j)[hs];
                                    yp = sm.SP(b ^ 1, j)[hs];
                                }
                                Hw = __vadd4(Hw, yo);
                            }
                            uint32_t dq[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int s = sbyte(o, q), sp = sbyte(spw, q);
                                // right neighbour: for x = L-1 the old site 0, corrected in the chain
                                const int right = (q < 3) ? sbyte(o, q + 1) : sbyte(on, 0);
                                const int base = sbyte(Hw, q) + right;
                                const int d = sp * sp - s * s;
                                const int kk = sp > s ? 1 : -1;
                                const int c0 = kBlk * (d + 1) + 6 - kk * base;
                                // left neighbour: site x-1 (for x = 0 the old site L-1)
                                int ps, psp;
                                if (q > 0) {
                                    ps = sbyte(o, q - 1);
                                    psp = sbyte(spw, q - 1);
                                } else {
                                    ps = sbyte(ol, 3);
                                    psp = (j == 0) ? ps : sbyte(spl, 3);
                                }
                                const int qy = -kk * (sbyte(yp, q) - sbyte(yo, q));
                                const int qL = (4 * j + q == L - 1) ? -kk * (sp0 - s0) : 0;
                                dq[q] =
                                    (uint32_t)(c0 - kk * psp) | ((uint32_t)(c0 - kk * ps) << 6) |
                                    ((uint32_t)(d + 1) << 12) | ((uint32_t)(qy + 2) << 14) |
                                    ((uint32_t)(qL + 2) << 17);
                            }
                            *reinterpret_cast<uint4 *>(sm.descq(b) + j * 4 * G + 4 * hs) =
                                make_uint4(dq[0], dq[1], dq[2], dq[3]);
                        }
                    }
                    bar_arrive(kBarReady + b, kWsSync);
                }
                if (i + 1 < R) {
                    // the neighbourhood of row i + 1 (all stores of finished rows are done)
                    bar_sync(kBarHelp, kWsHelp);
                    ws_stage<L>(sm, lat, st, (i + 1) % L, (i + 1) / L, ht);
                }
            }
            if (hact) {
                if (dJ) atomicAdd(sm.tal(hs), dJ);
                if (dM) atomicAdd(sm.tal(hs) + 1, dM);
            }
            __syncthreads();
            __syncthreads();
        }
        cp_async_wait_all();
    }
}

// WIDE: rows longer than kWsNarrowMaxL sites.  The two classes are separate
// kernels: compiled together, the register-carrying helpers of the narrow
// rows made the 48-site rows measurably slower.
template <bool RECORD, bool WIDE>
__global__ void __launch_bounds__(kWsThreads, 1)
sweep_ws_kernel(const GroupDev *__restrict__ groups, const BlockDesc *__restrict__ blocks,
                uint32_t seed, uint64_t sweep0, int n_sweeps, int64_t ts_pos)
{
    extern __shared__ __align__(16) uint32_t s_ws[];
    const BlockDesc bd = blocks[blockIdx.x];
    const GroupDev g = groups[bd.group];
    const WsSmem sm{s_ws, bd.S};
    if (threadIdx.x < (unsigned)bd.S) {
        sm.tal(threadIdx.x)[0] = 0;
        sm.tal(threadIdx.x)[1] = 0;
    }
    __syncthreads();
#define MUCA_WS(LL)                                                           \
    case LL: ws_sweeps<LL, RECORD>(g, bd, sm, seed, sweep0, n_sweeps, ts_pos); \
        break;
    if constexpr (WIDE) {
        switch (g.L) {
            MUCA_WS(48)
            default: break;
        }
    } else {
        switch (g.L) {
            MUCA_WS(8)
            MUCA_WS(12)
            MUCA_WS(16)
            MUCA_WS(20)
            MUCA_WS(24)
            MUCA_WS(28)
            MUCA_WS(32)
            default: break;
        }
    }
#undef MUCA_WS
}

// Initial spins i.i.d. uniform on {-1, 0, +1} from Philox stream 1; thread
// (word, walker) fills the (up to) four sites of one packed word.
__global__ void init_spins_kernel(GroupDev g, uint32_t seed)
{
    const int64_t nwords = (int64_t)g.L * g.L * g.Lw;
    const int64_t total = nwords * g.W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t wd = t / g.W;
        const int w = (int)(t - wd * g.W);
        const int row = (int)(wd / g.Lw), j = (int)(wd - (int64_t)row * g.Lw);
        uint32_t word = 0;
        for (int q = 0; q < 4; ++q) {
            const int x = 4 * j + q;
            if (x >= g.L) break;
            const int64_t i = (int64_t)row * g.L + x;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)(i >> 2), 0u, 0u, 1u),
                                          g.walker0 + (uint32_t)w, seed);
            const uint32_t rq = (i & 3) == 0 ? r.x : (i & 3) == 1 ? r.y : (i & 3) == 2 ? r.z : r.w;
            const int v = (int)(((uint64_t)rq * 3u) >> 32) - 1;
            word |= (uint32_t)(v & 0xFF) << (8 * q);
        }
        g.spins[wd * g.Wpad + w] = word;
    }
}

// E_J (three forward bonds per site, each weighted by its coupling when the
// group has couplings), E_Delta and M of every walker, one thread per walker.
// mode 0 stores them as the running tallies, mode 1 compares them with the
// running tallies and sets *err on a mismatch.
__global__ void energies_kernel(GroupDev g, int mode, int *err)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= g.W) return;
    const int L = g.L, Lw = g.Lw;
    uint32_t *lat = g.spins + w;
    const ptrdiff_t st = g.Wpad;
    int ej = 0, ed = 0, m = 0;
    for (int z = 0; z < L; ++z) {
        const int zp = (z + 1 == L) ? 0 : z + 1;
        for (int y = 0; y < L; ++y) {
            const int yp = (y + 1 == L) ? 0 : y + 1;
            for (int x = 0; x < L; ++x) {
                const int xp = (x + 1 == L) ? 0 : x + 1;
                const int s = *site_ptr(lat, st, Lw, z * L + y, x);
                const int i = x + L * (y + L * z);
                const int jx = g.J ? g.J[3 * i + 0] : 1, jy = g.J ? g.J[3 * i + 1] : 1,
                          jz = g.J ? g.J[3 * i + 2] : 1;
                ej -= s * (jx * *site_ptr(lat, st, Lw, z * L + y, xp) +
                           jy * *site_ptr(lat, st, Lw, z * L + yp, x) +
                           jz * *site_ptr(lat, st, Lw, zp * L + y, x));
                ed += s * s;
                m += s;
            }
        }
    }
    if (mode == 0) {
        g.tal[w] = ej;
        g.tal[g.Wpad + w] = ed;
        g.tal[2 * g.Wpad + w] = m;
    } else if (g.tal[w] != ej || g.tal[g.Wpad + w] != ed || g.tal[2 * g.Wpad + w] != m) {
        atomicOr(err, 1);
    }
}

}  // namespace

cudaError_t launch_init_spins(const GroupDev &g, uint32_t seed, cudaStream_t st)
{
    const int64_t total = (int64_t)g.L * g.L * g.Lw * g.W;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 64) blocks = 152 * 64;
    init_spins_kernel<<<blocks, 256, 0, st>>>(g, seed);
    return cudaGetLastError();
}

cudaError_t launch_energies(const GroupDev &g, int mode, int *err, cudaStream_t st)
{
    energies_kernel<<<(g.W + 127) / 128, 128, 0, st>>>(g, mode, err);
    return cudaGetLastError();
}

size_t lattice_bytes(int L) { return (size_t)L * L * ((L + 3) / 4) * 4; }

size_t stage_bytes_for(int slots)
{
    return (size_t)slots * (kStageWords + kRingStride) * sizeof(uint32_t);
}

size_t smem_bytes_for(int L, int walkers)
{
    return ((lattice_bytes(L) * (size_t)walkers + 15) / 16) * 16;
}

int max_smem_per_block()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    return v;
}

// A kernel's dynamic shared-memory limit belongs to the process (per device),
// not to a context: every context that launches the kernel needs a limit at
// least as large as its own blocks use, so the limit is only ever raised.
cudaError_t raise_smem_limit(const void *func, size_t smem_bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> set;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = set[{dev, func}];
    if (smem_bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e == cudaSuccess) cur = smem_bytes;
    return e;
}

cudaError_t prepare_smem_kernel(size_t smem_bytes)
{
    cudaError_t e = raise_smem_limit((const void *)sweep_smem_kernel<true>, smem_bytes);
    if (e != cudaSuccess) return e;
    return raise_smem_limit((const void *)sweep_smem_kernel<false>, smem_bytes);
}

cudaError_t prepare_global_kernel(size_t smem_bytes)
{
    cudaError_t e = raise_smem_limit((const void *)sweep_global_kernel<true>, smem_bytes);
    if (e != cudaSuccess) return e;
    return raise_smem_limit((const void *)sweep_global_kernel<false>, smem_bytes);
}

size_t ws_bytes_for(int slots) { return (size_t)slots * kWsWords * sizeof(uint32_t); }

cudaError_t prepare_ws_kernel(size_t smem_bytes, bool wide)
{
    cudaError_t e = raise_smem_limit(
        wide ? (const void *)sweep_ws_kernel<true, true> : (const void *)sweep_ws_kernel<true, false>,
        smem_bytes);
    if (e != cudaSuccess) return e;
    return raise_smem_limit(wide ? (const void *)sweep_ws_kernel<false, true>
                                 : (const void *)sweep_ws_kernel<false, false>,
                            smem_bytes);
}

cudaError_t launch_sweeps_ws(const GroupDev *groups_dev, const BlockDesc *blocks_dev, int n_blocks,
                             size_t smem_bytes, uint32_t seed, uint64_t sweep0, int n_sweeps,
                             int64_t ts_pos, bool record, bool wide, cudaStream_t st)
{
    if (n_blocks <= 0 || n_sweeps <= 0) return cudaSuccess;
    auto k = record ? (wide ? sweep_ws_kernel<true, true> : sweep_ws_kernel<true, false>)
                    : (wide ? sweep_ws_kernel<false, true> : sweep_ws_kernel<false, false>);
    k<<<n_blocks, kWsThreads, smem_bytes, st>>>(groups_dev, blocks_dev, seed, sweep0, n_sweeps,
                                                ts_pos);
    return cudaGetLastError();
}

cudaError_t launch_sweeps(const GroupDev *groups_dev, const BlockDesc *blocks_dev, int n_blocks,
                          int threads, size_t smem_bytes, bool smem_kernel, uint32_t seed,
                          uint64_t sweep0, int n_sweeps, int64_t ts_pos, bool record,
                          cudaStream_t st)
{
    if (n_blocks <= 0 || n_sweeps <= 0) return cudaSuccess;
    if (smem_kernel) {
        if (record)
            sweep_smem_kernel<true><<<n_blocks, threads, smem_bytes, st>>>(
                groups_dev, blocks_dev, seed, sweep0, n_sweeps, ts_pos);
        else
            sweep_smem_kernel<false><<<n_blocks, threads, smem_bytes, st>>>(
                groups_dev, blocks_dev, seed, sweep0, n_sweeps, ts_pos);
    } else {
        if (record)
            sweep_global_kernel<true><<<n_blocks, threads, smem_bytes, st>>>(
                groups_dev, blocks_dev, seed, sweep0, n_sweeps, ts_pos);
        else
            sweep_global_kernel<false><<<n_blocks, threads, smem_bytes, st>>>(
                groups_dev, blocks_dev, seed, sweep0, n_sweeps, ts_pos);
    }
    return cudaGetLastError();
}

}  // namespace muca
