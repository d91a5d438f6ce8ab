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
// to make that step short and to keep everything else off it.  P lanes of a
// warp serve one walker (walker slot t / P, lane h = t % P).  A row (fixed
// y, z) of L sites goes through these phases, staged in shared memory:
//   1. cp.async (L2 -> shared, bypassing L1) of the NEXT row's old spins and
//      of its four y/z neighbour rows, completing behind the current row;
//   2. the Philox blocks of the row, split over the P lanes;
//   3. per-site descriptors, split over the P lanes: for site x the two table
//      offsets it can need (site x-1 accepted or rejected) relative to the
//      E_Delta row of the state before site x-1, the row shift dK of its own
//      move, and its old spin and proposal;
//   4. the chain, unrolled over the row: compare u with the threshold in
//      flight, select the next site's offset, issue its load - nothing else
//      depends on the previous step - and record the acceptance bit;
//   5. the new spins of the row from the acceptance bits, and the energy
//      tallies from byte dot products of old and new spins:
//        dM = sum (N - O), dE_Delta = sum (N^2 - O^2),
//        dE_J = -sum (N - O) H - sum_cyclic (N_x N_{x+1} - O_x O_{x+1}),
//      which equals the sum of the per-site energy changes;
//   6. the next row's old spins and neighbour sums from the prefetched rows
//      (its y-1 neighbour is the row just finished).
// The threshold table (L2-resident, rows of 128 bytes) is the only memory the
// chain touches.  Sizes with L % 4 == 0 up to 48 use this path; any other L
// uses a plain per-site path with the same results.
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
                            const uint32_t *__restrict__ thr0, const uint32_t *__restrict__ thrE,
                            int e_min, uint32_t key0, uint32_t key1, uint64_t sw, Chain &c)
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
                const uint32_t t =
                    d == 0 ? __ldg(thr0 + ((dEJ + 12) >> 1))
                           : __ldg(thrE + (ptrdiff_t)(c.ED - e_min) * kRow + (d > 0 ? kPlus : 0) +
                                   dEJ + 6);
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
// Staging area of a block in shared memory: for every walker slot (S slots),
// fields laid out [field][index][slot] so that the lanes of different slots
// touch consecutive words.
// ---------------------------------------------------------------------------
constexpr int kMaxL = 48;
constexpr int kMaxLw = kMaxL / 4;
constexpr int kStageWords = 8 * kMaxLw + 4 * kMaxL;  // per slot

struct Stage {
    uint32_t *base;
    int S;
    // prefetched rows of the next row: f = 0 y-1, 1 y+1, 2 z-1, 3 z+1, 4 itself
    __device__ uint32_t *pf(int f, int j) const { return base + (f * kMaxLw + j) * S; }
    __device__ uint32_t *O(int j) const { return base + (5 * kMaxLw + j) * S; }
    __device__ uint32_t *H(int j) const { return base + (6 * kMaxLw + j) * S; }
    __device__ uint32_t *N(int j) const { return base + (7 * kMaxLw + j) * S; }
    __device__ uint32_t *rnd(int x) const { return base + (8 * kMaxLw + x) * S; }
    __device__ int *GA(int x) const { return (int *)base + (8 * kMaxLw + kMaxL + x) * S; }
    __device__ int *GR(int x) const { return (int *)base + (8 * kMaxLw + 2 * kMaxL + x) * S; }
    __device__ uint32_t *AUX(int x) const { return base + (8 * kMaxLw + 3 * kMaxL + x) * S; }
};

// Where the block's walkers' lattices live: a [L*L][Lw][stride] word array
// (global: stride Wpad, shared tile: stride S), starting at the block's first walker.
struct BlockLattice {
    uint32_t *base;
    ptrdiff_t stride;
};

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
        cp_async_commit();
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

// The unrolled row path (L % 4 == 0).  Threads of the block run this in lock
// step: all P lanes of a walker execute the chain on the same data.
template <int L, bool GLOBAL>
__device__ __forceinline__ void sweep_rows(const BlockLattice &bl, const Stage &sg,
                                           const uint32_t *__restrict__ thrE, int off0,
                                           uint32_t key0, uint32_t key1, uint64_t sw, int &rowoff,
                                           Chain &c, int slot, int P, int h, int nw, int tid,
                                           int nthreads, unsigned amask)
{
    static_assert(L % 4 == 0 && L <= kMaxL, "row path needs L % 4 == 0, L <= 48");
    constexpr int Lw = L / 4, R = L * L, NB = (L + 31) / 32;
    const uint32_t slo = (uint32_t)sw, shi = (uint32_t)(sw >> 32);
    uint32_t *const own = bl.base + slot;  // this walker's word 0
    // the neighbourhood of row 0
    stage_rows<L, GLOBAL>(bl, sg, 0, 0, nw, tid, nthreads);
    if (GLOBAL) cp_async_wait_all();
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
        // 1. the next row's neighbourhood
        if (more) stage_rows<L, GLOBAL>(bl, sg, y1, z1, nw, tid, nthreads);
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
            const uint32_t word = sg.rnd(x)[slot];
            const int sp = proposal(s, word);
            const int d = sp * sp - s * s;
            const int k = sp > s ? 1 : -1;
            const bool m = (d != 0);  // the threshold sits in the E_Delta row
            const int c0 = (d > 0 ? kPlus + 6 : 6) - k * base;
            int ps, psp, pdK;
            if (x == 0) {
                ps = psp = sbyte(sg.O(Lw - 1)[slot], 3);  // x - 1 of x = 0: old x = L - 1
                pdK = 0;
            } else {
                ps = sbyte(sg.O((x - 1) >> 2)[slot], (x - 1) & 3);
                psp = proposal(ps, sg.rnd(x - 1)[slot]);
                pdK = (psp * psp - ps * ps) * kRow;
            }
            sg.GA(x)[slot] = (m ? pdK : off0) + c0 - k * psp;
            sg.GR(x)[slot] = (m ? 0 : off0) + c0 - k * ps;
            sg.AUX(x)[slot] = (m ? 1u : 0u) | (k > 0 ? 4u : 0u) | ((uint32_t)(d * kRow & 0xFF) << 8) |
                              ((uint32_t)(sp & 0xFF) << 16) | ((uint32_t)(s & 0xFF) << 24);
        }
        __syncwarp(amask);
        // 4. the chain
        uint32_t accb[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) accb[b] = 0u;
        {
            uint32_t aux = sg.AUX(0)[slot];
            uint32_t t = __ldg(thrE + ((aux & 1u) ? rowoff : 0) + sg.GR(0)[slot]);
            uint32_t u = sg.rnd(0)[slot] & 0x7FFFFFFFu;
            int corr = 0;
#pragma unroll
            for (int x = 0; x < L; ++x) {
                const int dK = sbyte(aux, 1);
                uint32_t aux1 = 0u, u1 = 0u;
                int IA = 0, IR = 0;
                if (x + 1 < L) {
                    aux1 = sg.AUX(x + 1)[slot];
                    const int mo = (aux1 & 1u) ? rowoff : 0;
                    IA = mo + sg.GA(x + 1)[slot];
                    IR = mo + sg.GR(x + 1)[slot];
                    if (x + 1 == L - 1) {
                        IA += corr;
                        IR += corr;
                    }
                    u1 = sg.rnd(x + 1)[slot] & 0x7FFFFFFFu;
                }
                const bool acc = u < t;
                if (x + 1 < L) t = __ldg(thrE + (acc ? IA : IR));
                if (acc) {
                    rowoff += dK;
                    accb[x >> 5] |= 1u << (x & 31);
                }
                if (x == 0) {
                    // x + 1 of x = L - 1 is the new value of x = 0
                    const int kL = (sg.AUX(L - 1)[slot] & 4u) ? 1 : -1;
                    corr = acc ? -kL * (sbyte(aux, 2) - sbyte(aux, 3)) : 0;
                }
                aux = aux1;
                u = u1;
            }
        }
        // 5. new spins, their store, the tallies
        for (int j = h; j < Lw; j += P) {
            uint32_t nwd = 0u;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int x = 4 * j + q;
                const uint32_t a = sg.AUX(x)[slot];
                const uint32_t bits = (NB == 1 || x < 32) ? accb[0] : accb[NB - 1];
                const int sn = ((bits >> (x & 31)) & 1u) ? sbyte(a, 2) : sbyte(a, 3);
                nwd |= (uint32_t)(sn & 0xFF) << (8 * q);
            }
            sg.N(j)[slot] = nwd;
            own[((ptrdiff_t)r * Lw + j) * bl.stride] = nwd;
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
        // 6. the next row
        if (more) {
            if (GLOBAL) cp_async_wait_all();
            __syncwarp(amask);
            build_row<L>(sg, slot, P, h, !wrap);
        }
        __syncwarp(amask);
        y = y1;
        z = z1;
    }
}

template <bool RECORD, bool GLOBAL>
__device__ __forceinline__ void run_block(const GroupDev &g, const BlockDesc &bd,
                                          uint32_t *__restrict__ lat_block, ptrdiff_t st,
                                          uint32_t *__restrict__ stage, uint32_t seed,
                                          uint64_t sweep0, int n_sweeps, int64_t ts_pos)
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
    const Stage sg{stage, bd.S};
    const int nthreads = bd.nw * P;
    const int off0 = (int)(g.thr0 - g.thrE);
    for (int k = 0; k < n_sweeps; ++k) {
        const uint64_t sw = sweep0 + (uint64_t)k;
        int rowoff = (c.ED - g.e_min) * kRow;
        switch (g.L) {
#define MUCA_ROWS(LL)                                                                          \
    case LL:                                                                                   \
        sweep_rows<LL, GLOBAL>(bl, sg, g.thrE, off0, key0, seed, sw, rowoff, c, slot, P, h,  \
                               bd.nw, tid, nthreads, amask);                                   \
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
                sweep_sites(lat_block + slot, st, g.L, g.Lw, g.thr0, g.thrE, g.e_min, key0, seed,
                            sw, c);
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

// Thread t of a block serves walker slot t / P as lane t % P.
template <bool RECORD>
__global__ void __launch_bounds__(128)
sweep_global_kernel(const GroupDev *__restrict__ groups, const BlockDesc *__restrict__ blocks,
                    uint32_t seed, uint64_t sweep0, int n_sweeps, int64_t ts_pos)
{
    extern __shared__ __align__(16) uint32_t s_stage[];
    const BlockDesc bd = blocks[blockIdx.x];
    const GroupDev g = groups[bd.group];
    run_block<RECORD, true>(g, bd, g.spins + bd.w0, g.Wpad, s_stage, seed, sweep0, n_sweeps,
                            ts_pos);
}

// Shared-memory-resident variant: the block's walkers keep their lattices in
// shared memory as a [L * L][Lw][S] word tile for the whole launch, read from
// and written back to the global array at the start and the end; the staging
// area follows the tile.
template <bool RECORD>
__global__ void __launch_bounds__(128)
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
    run_block<RECORD, false>(g, bd, s_lat, S, s_lat + (size_t)nwords * S, seed, sweep0, n_sweeps,
                             ts_pos);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nwords * S; idx += blockDim.x) {
        const int wd = idx / S, c = idx - wd * S;
        if (c < bd.nw) g.spins[(ptrdiff_t)wd * g.Wpad + bd.w0 + c] = s_lat[idx];
    }
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

// E_J (three forward bonds per site), E_Delta and M of every walker, one
// thread per walker.  mode 0 stores them as the running tallies, mode 1
// compares them with the running tallies and sets *err on a mismatch.
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
                ej -= s * (*site_ptr(lat, st, Lw, z * L + y, xp) +
                           *site_ptr(lat, st, Lw, z * L + yp, x) +
                           *site_ptr(lat, st, Lw, zp * L + y, x));
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

size_t stage_bytes_for(int slots) { return (size_t)slots * kStageWords * sizeof(uint32_t); }

size_t smem_bytes_for(int L, int walkers) { return lattice_bytes(L) * (size_t)walkers; }

int max_smem_per_block()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    return v;
}

cudaError_t prepare_smem_kernel(size_t smem_bytes)
{
    cudaError_t e = cudaFuncSetAttribute(sweep_smem_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_smem_kernel<false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
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
