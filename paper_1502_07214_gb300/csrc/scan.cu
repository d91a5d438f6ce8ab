// scan.cu -- the row-scan sweep kernel: the typewriter Metropolis sweep of
// Sec. II (single-site updates in the order i = x + L (y + L z), acceptance
// exp(-beta dE_J) W(E_Delta') / W(E_Delta) through the threshold table)
// with each row of L sites resolved by a prefix scan instead of site by site.
//
// The other sweep kernels (sweep.cu) follow every walker's chain one site
// at a time, so a walker costs one dependent table load per site and the
// throughput is (walkers) / (latency of a step).  Here the chain is cut into
// its two kinds of links (scan_core.cuh): the left neighbour's acceptance,
// a linear recurrence over GF(2) that a bit-mask scan resolves for a whole
// row, and E_Delta, which moves only at accepted moves with d != 0 and
// splits a row into a few segments resolved one after the other.  Every
// site's two thresholds are independent loads, so the work becomes
// throughput-bound integer arithmetic.
//
// Layout of the work.  A block is one warp of 32 / S walkers of one group;
// a walker's L / 4 packed words of a row are split into runs of M
// consecutive words, one run per lane of its segment of S lanes (scan_seg,
// scan_words in muca_internal.h).  Per row, every lane forms its run's move
// descriptors byte-parallel (scan_core.cuh), loads the two thresholds of
// each of its sites from the walker's table row E0, and scans its own
// sites' acceptance bits for an unknown input; the lanes' maps are then
// composed through two ballots, and the first accepted move that changes
// E_Delta is found through three.  New spins, their store and the energy
// changes follow from the final acceptance bits of each lane.
// Table rows: each walker keeps a ring of R table rows around its E_Delta
// in shared memory, re-centred after a row with cp.async; a row whose E0 is
// not among the rows known to be complete reads the global table instead.
#include <cstdint>
#include <type_traits>

#include "muca_internal.h"
#include "philox.cuh"
#include "scan_core.cuh"

namespace muca {

namespace {

using scan::fshl;
using scan::perm;

__device__ __forceinline__ void cp16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Lanes holding the same bin elect one leader that adds their count.
__device__ __forceinline__ void hist_add_leaders(unsigned long long *hist, int bin, unsigned mask)
{
    const unsigned peers = __match_any_sync(mask, bin);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1)
        atomicAdd(hist + bin, (unsigned long long)__popc(peers));
}

// Window of R table rows of one walker: rows [lo, lo + R) at ring row
// (row mod R).  Re-centred on E when E comes within R / 2 - 2 rows of an
// edge, kept inside the table allocation [-kGuard, nE + kGuard).
template <int R>
__device__ __forceinline__ int ring_target(int lo, int e, int nE)
{
    constexpr int kMarg = R / 2 - 2;
    if (e >= lo + kMarg && e < lo + R - kMarg) return lo;
    return min(max(e - R / 2, -kGuard), nE + kGuard - R);
}

// Copy table rows [a, b) into the ring, 16-byte chunks over the P lanes.
template <int R>
__device__ __forceinline__ void ring_copy(uint32_t *ring, const uint32_t *__restrict__ thrE, int a,
                                          int b, int P, int h)
{
    constexpr int kChunks = kRow / 4;
    const int n = (b - a) * kChunks;
    for (int c = h; c < n; c += P) {
        const int row = a + c / kChunks, part = c - (c / kChunks) * kChunks;
        cp16(ring + (row & (R - 1)) * kRow + 4 * part, thrE + (ptrdiff_t)row * kRow + 4 * part);
    }
}

// Sum of a value over the n lanes [base, base + n) of one walker.
__device__ __forceinline__ int lanes_sum(int v, unsigned live, int base, int h, int n)
{
    int s = v;
    for (int o = 1; o < n; ++o) s += __shfl_sync(live, v, base + (h + o) % n);
    return s;
}

// The move descriptors of one lane's run of M words of a row (scan_core.cuh):
// biased old spins U, y / z neighbour sums HYZ, columns CR (left neighbour
// rejected) and CA (accepted, plus 2), k masks KM, biased proposals PR,
// deltas DL (+2), the sites' u, and the run's d != 0 / d = +1 site masks.
template <int M>
struct RunDesc {
    uint32_t U[M], HYZ[M], CR[M], CA[M], KM[M], PR[M], DL[M], UQ[M][4];
    uint32_t dml, dpl;
};

// One warp's walkers: walker slot t of the warp is walker w_first + t; lane
// h < L / (4 M) of its segment of S lanes holds the M packed words
// j = h M .. h M + M - 1 of every row (sites 4 h M .. 4 (h + 1) M - 1), so a
// warp's load of word t of a run covers 32 / S >= 8 walkers: whole 32-byte
// sectors for segments of up to 4 lanes.
//
// The rows are software-pipelined: while row r is resolved, the lane draws
// the Philox words of row r + 1 and forms its descriptors with the old spins
// of row r as its y-1 neighbour, and loads the words of row r + 2.  Row r's
// outcome then reaches row r + 1 as one byte-parallel correction: where site
// x of row r was accepted, the neighbour sum of site x of row r + 1 moves by
// delta_x, and its columns by -k delta_x.  Only the resolution of a row (its
// table loads, scans and breaks) and that correction stay on the walker's
// serial path.
template <int L>
__device__ __forceinline__ void scan_sweeps(const GroupDev &g, int w_first, int nw, uint32_t *rings,
                                         uint32_t seed, uint64_t sweep0, int n_sweeps,
                                         int64_t ts_pos, int record)
{
    constexpr int Lw = L / 4, S = scan_seg(L), M = scan_words(L), A = Lw / M;
    constexpr int R = scan_ring(L), NR = L * L, NB = 4 * M;  // NB: sites per lane
    constexpr uint32_t kLane = NB == 32 ? ~0u : (1u << NB) - 1u;
    static_assert(S > 0 && M > 0 && Lw % M == 0 && A <= S && 32 % S == 0, "row-scan shape");
    const int lane = (int)(threadIdx.x & 31), slot = lane / S, h = lane - slot * S;
    const bool active = slot < nw && h < A;
    // lanes without a run leave now; every collective below names the rest
    const unsigned amask = __ballot_sync(0xFFFFFFFFu, active);
    const unsigned lmask = __ballot_sync(0xFFFFFFFFu, active && h == 0);
    if (!active) return;
    const int sbase = slot * S;
    const int srcL = sbase + (h == 0 ? A - 1 : h - 1), srcR = sbase + (h == A - 1 ? 0 : h + 1);
    const bool last = (h == A - 1);
    const int w = w_first + slot;
    uint32_t *const ring = rings + (size_t)slot * (R * kRow + 4);
    const uint32_t *__restrict__ thrE = g.thrE;
    const ptrdiff_t st = g.Wpad;
    // word (row, h M + t) at lat[(row Lw + t) Wpad]
    uint32_t *const lat = g.spins + w + (ptrdiff_t)h * M * st;
    auto wp = [&](int row, int t) { return lat + ((ptrdiff_t)row * Lw + t) * st; };
    // row index of (y, z), both taken mod L
    auto rowi = [&](int y, int z) {
        y = y < 0 ? y + L : (y >= L ? y - L : y);
        z = z < 0 ? z + L : (z >= L ? z - L : z);
        return z * L + y;
    };
    const PhiloxKeys keys = philox_keys(g.walker0 + (uint32_t)w, seed);
    int E = g.tal[g.Wpad + w] - g.e_min;
    int EJ = g.tal[w], Mg = g.tal[2 * g.Wpad + w];
    // lo_a: the window once every copy asked for is complete; lo_b: before
    // the last request (the rows of both are valid while it is pending)
    int lo_a = ring_target<R>(-(1 << 20), E, g.nE), lo_b = lo_a;
    ring_copy<R>(ring, thrE, lo_a, lo_a + R, A, h);
    cp_commit();
    cp_wait_all();
    __syncwarp(amask);

    // descriptors of row `row` from its old words O, its y / z neighbour words
    auto describe = [&](int row, const uint32_t (&O)[M], const uint32_t (&YM)[M],
                        const uint32_t (&YP)[M], const uint32_t (&ZM)[M], const uint32_t (&ZP)[M],
                        uint32_t slo, uint32_t shi, RunDesc<M> &D) {
        uint4 rn[M];
#pragma unroll
        for (int t = 0; t < M; ++t) {
            rn[t] = philox4x32_10(make_uint4((uint32_t)(row * Lw + h * M + t), slo, shi, 0u), keys);
            D.U[t] = scan::to_biased(O[t]);
        }
        const uint32_t uL = __shfl_sync(amask, D.U[M - 1], srcL);
        const uint32_t uR = __shfl_sync(amask, D.U[0], srcR);
        D.dml = D.dpl = 0u;
#pragma unroll
        for (int t = 0; t < M; ++t) {
            D.HYZ[t] = scan::sum4_biased(YM[t], YP[t], ZM[t], ZP[t]);
            const scan::WordDesc d = scan::word_desc(
                D.U[t], t ? D.U[t ? t - 1 : 0] : uL, t + 1 < M ? D.U[t + 1 < M ? t + 1 : t] : uR,
                D.HYZ[t], rn[t].x, rn[t].y, rn[t].z, rn[t].w);
            D.CR[t] = d.colR;
            D.KM[t] = d.km;
            D.PR[t] = d.prop;
            D.DL[t] = d.dl;
            D.dml |= d.dm4 << (4 * t);
            D.dpl |= d.dp4 << (4 * t);
            D.UQ[t][0] = rn[t].x & 0x7FFFFFFFu;
            D.UQ[t][1] = rn[t].y & 0x7FFFFFFFu;
            D.UQ[t][2] = rn[t].z & 0x7FFFFFFFu;
            D.UQ[t][3] = rn[t].w & 0x7FFFFFFFu;
        }
        const uint32_t dlL = __shfl_sync(amask, D.DL[M - 1], srcL);
#pragma unroll
        for (int t = 0; t < M; ++t) {
            // delta + 2 of each site's left neighbour; site 0 has none (2)
            const uint32_t prev = t ? D.DL[t ? t - 1 : 0] : (h == 0 ? 0x02000000u : dlL);
            D.CA[t] = scan::col_accepted2(D.CR[t], D.KM[t], fshl(prev, D.DL[t], 8));
        }
    };

    for (int k = 0; k < n_sweeps; ++k) {
        const uint64_t sw = sweep0 + (uint64_t)k;
        const uint32_t slo = (uint32_t)sw, shi = (uint32_t)(sw >> 32);
        int dJ = 0, dM = 0;
        // row 0 = (y 0, z 0): its descriptors; the old words of rows 0 and 1;
        // the neighbour words of row 1
        uint32_t Oc[M], O1[M], YM1[M], YP1[M], ZM1[M], ZP1[M];
        RunDesc<M> Dc;
        {
            uint32_t YM[M], ZM[M], ZP[M];
#pragma unroll
            for (int t = 0; t < M; ++t) {
                Oc[t] = *wp(0, t);
                O1[t] = *wp(rowi(1, 0), t);
                YM[t] = *wp(rowi(-1, 0), t);
                ZM[t] = *wp(rowi(0, -1), t);
                ZP[t] = *wp(rowi(0, 1), t);
                YM1[t] = Oc[t];
                YP1[t] = *wp(rowi(2, 0), t);
                ZM1[t] = *wp(rowi(1, -1), t);
                ZP1[t] = *wp(rowi(1, 1), t);
            }
            describe(0, Oc, YM, O1, ZM, ZP, slo, shi, Dc);
        }
        uint32_t a_prev = 0u, DLp[M];
#pragma unroll
        for (int t = 0; t < M; ++t) DLp[t] = 0x02020202u;
        int y = 0, z = 0;
#pragma unroll 1
        for (int r = 0; r < NR; ++r) {
            // ---- row r's outcome-independent part was formed with the old
            // spins of row r-1 as its y-1 neighbour: apply row r-1's changes
            if (y != 0) {
#pragma unroll
                for (int t = 0; t < M; ++t) {
                    const uint32_t m = scan::bits_bytes((a_prev >> (4 * t)) & 15u);
                    const uint32_t dy = (DLp[t] & m) | (0x02020202u & ~m);  // change + 2
                    const uint32_t x = (Dc.KM[t] & (0x04040404u - dy)) | (~Dc.KM[t] & dy);
                    Dc.HYZ[t] = Dc.HYZ[t] + dy - 0x02020202u;
                    Dc.CR[t] = Dc.CR[t] + x - 0x02020202u;
                    Dc.CA[t] = Dc.CA[t] + x - 0x02020202u;
                }
            }
            // site 0 as seen by the last lane: its column, u and delta
            const uint32_t s0 = __shfl_sync(amask, (Dc.CR[0] & 0xFFu) | (Dc.DL[0] << 8), sbase);
            const uint32_t s0u = __shfl_sync(amask, Dc.UQ[0][0], sbase);
            // site L-1 if site 0 (its x+1 neighbour) is accepted: the column
            // moves by -k_{L-1} delta_0
            int cRa = 0, cAa = 0;
            if (last) {
                const int d0 = (int)((s0 >> 8) & 0xFFu) - 2;
                const int corr = (Dc.KM[M - 1] >> 31) ? -d0 : d0;
                cRa = (int)(Dc.CR[M - 1] >> 24) + corr;
                cAa = (int)(Dc.CA[M - 1] >> 24) + corr - 2;
            }
            // the window copies asked for before the last row are complete
            cp_wait_prev();
            __syncwarp(amask);
            const int vlo = max(lo_a, lo_b), vhi = min(lo_a, lo_b) + R;
            // ---- one pass over the row from table row E0: the acceptance
            // bits of the sites that are not yet final, their lane scan, the
            // lanes' maps composed left to right, and the first accepted move
            // that changes E_Delta (sites up to it are final).  Branch-free:
            // every lane runs every step (the last lane's extra columns are
            // clamped into the row on the others), so that the first pass and
            // the next row's work form one block of straight-line code.
            uint32_t a = 0u, fixed = 0u, a0 = 0u;
            bool a0_known = false;
            int E0 = E;
            const unsigned seg = ((1u << A) - 1u) << sbase;  // this walker's lanes
            const uint32_t cRs = (uint32_t)min(max(cRa, 0), kRow - 1);
            const uint32_t cAs = (uint32_t)min(max(cAa, 0), kRow - 1);
            // one pass reading thresholds through thr(column); returns whether
            // the walker needs another pass
            auto pass = [&](auto thr, unsigned live) -> bool {
                // acceptance bits if the left neighbour is rejected (lr) or
                // accepted (la); the sign of u - t is u < t (u < 2^31, t <= 2^31)
                uint32_t lr = 0u, la = 0u;
#pragma unroll
                for (int t = 0; t < M; ++t) {
                    uint32_t wr = 0u, wa = 0u;
#pragma unroll
                    for (int q = 3; q >= 0; --q) {
                        wr = fshl(Dc.UQ[t][q] - thr(perm(Dc.CR[t], 0u, 0x4440u | (uint32_t)q)), wr, 1);
                        wa = fshl(Dc.UQ[t][q] - thr(perm(Dc.CA[t], 0u, 0x4440u | (uint32_t)q) - 2u),
                                  wa, 1);
                    }
                    lr |= (wr & 15u) << (4 * t);
                    la |= (wa & 15u) << (4 * t);
                }
                // site L-1 (last lane) if site 0 was accepted; site 0 sees only
                // old spins, so its acceptance is final in the first pass
                const uint32_t b0 = (s0u - thr(s0 & 0xFFu)) >> 31;
                a0 = a0_known ? a0 : b0;
                a0_known = true;
                const uint32_t ar = (Dc.UQ[M - 1][3] - thr(cRs)) >> 31;
                const uint32_t aa = (Dc.UQ[M - 1][3] - thr(cAs)) >> 31;
                constexpr uint32_t top = 1u << (NB - 1);
                const bool swap = last && a0;
                lr = swap ? (lr & ~top) | (ar << (NB - 1)) : lr;
                la = swap ? (la & ~top) | (aa << (NB - 1)) : la;
                uint32_t G, Pp;
                scan::scan_bits<NB>((a & fixed) | (lr & ~fixed),
                                    (la ^ lr) & ~fixed & (h == 0 ? ~1u : ~0u), G, Pp);
                // each lane's map of its run (a_out = g xor (p and a_in)), the
                // maps of the walker's lanes collected by two ballots and scanned
                // as bits: a_in of lane h is a_out of lane h - 1
                const unsigned bg = __ballot_sync(live, (G >> (NB - 1)) & 1u);
                const unsigned bp = __ballot_sync(live, (Pp >> (NB - 1)) & 1u);
                uint32_t lg, lp;
                scan::scan_bits<S>((bg & seg) >> sbase, ((bp & seg) >> sbase) & ~1u, lg, lp);
                const uint32_t ain = h ? (lg >> (h - 1)) & 1u : 0u;
                a = (G ^ (Pp & (0u - ain))) & kLane;
                // the first break: lane f (first lane with one), its site Kl, the
                // sign of its d and whether it is the row's last site
                const uint32_t brk = a & Dc.dml & ~fixed;
                const int kl = __ffs((int)brk) - 1;
                const unsigned bb = __ballot_sync(live, brk != 0u);
                const unsigned bs = __ballot_sync(live, brk != 0u && ((Dc.dpl >> kl) & 1u));
                const unsigned bt = __ballot_sync(live, brk != 0u && kl == NB - 1);
                const unsigned mine = (bb & seg) >> sbase;
                const int f = __ffs((int)mine) - 1;
                const bool any = mine != 0u;
                E0 += any ? (((bs >> (sbase + f)) & 1u) ? 1 : -1) : 0;
                const bool more = any && !(f == A - 1 && ((bt >> (sbase + f)) & 1u));
                fixed |= more ? (h < f ? kLane : h == f ? (2u << kl) - 1u : 0u) : 0u;
                return more;
            };
            auto thr_ring = [&](uint32_t c) { return ring[(E0 & (R - 1)) * kRow + (int)c]; };
            auto thr_glob = [&](uint32_t c) { return __ldg(thrE + (ptrdiff_t)E0 * kRow + (int)c); };
            // ---- rows r+1 and r+2 (independent of row r's outcome, placed
            // before the first pass so that the two interleave): the
            // descriptors of row r+1, with the old spins of row r as its y-1
            // neighbour unless it starts a plane; the words of row r+2
            int y1 = y + 1, z1 = z;
            if (y1 == L) {
                y1 = 0;
                z1 = (z + 1 == L) ? 0 : z + 1;
            }
            int y2 = y1 + 1, z2 = z1;
            if (y2 == L) {
                y2 = 0;
                z2 = (z1 + 1 == L) ? 0 : z1 + 1;
            }
            RunDesc<M> Dn;
            uint32_t O2[M], YM2[M], YP2[M], ZM2[M], ZP2[M];
            {
                const int r4 = r + 4 < NR ? r + 4 : r + 4 - NR;
#pragma unroll
                for (int t = 0; t < M; ++t) {
                    YP2[t] = *wp(rowi(y2 + 1, z2), t);
                    ZM2[t] = *wp(rowi(y2, z2 - 1), t);
                    ZP2[t] = *wp(rowi(y2, z2 + 1), t);
                    // a row that starts a plane has no earlier row of its plane
                    // in registers
                    O2[t] = y2 == 0 ? *wp(rowi(0, z2), t) : 0u;
                    YM2[t] = y2 == 0 ? *wp(rowi(-1, z2), t) : 0u;
                    // the z+1 rows, first read from DRAM in a sweep, four rows ahead into L2
                    prefetch_l2(wp(rowi(r4 % L, r4 / L + 1), t));
                }
                uint32_t YMn[M];
#pragma unroll
                for (int t = 0; t < M; ++t) YMn[t] = y1 == 0 ? YM1[t] : Oc[t];
                describe(z1 * L + y1, O1, YMn, YP1, ZM1, ZP1, slo, shi, Dn);
            }
            // the first pass reads the ring without asking; if row E0 was not
            // among its complete rows, nothing of it is kept and the row is
            // resolved from the global table below
            const bool ring_ok = (E0 >= vlo && E0 < vhi);
            bool again;
            {
                const uint32_t sa = a, sf = fixed;
                const int sE = E0;
                again = pass(thr_ring, amask);
                if (!ring_ok) {
                    a = sa;
                    fixed = sf;
                    E0 = sE;
                    a0_known = false;
                    again = true;
                }
            }
            // ---- further passes for walkers whose E_Delta changed in the row
            unsigned live = __ballot_sync(amask, again);
            while (live & (1u << lane)) {
                if (E0 >= vlo && E0 < vhi)
                    again = pass(thr_ring, live);
                else
                    again = pass(thr_glob, live);
                live = __ballot_sync(live, again);
            }
            __syncwarp(amask);
            E = E0;
            // ---- new spins, their store, the energy changes
            uint32_t NBW[M];
#pragma unroll
            for (int t = 0; t < M; ++t) {
                const uint32_t m = scan::bits_bytes((a >> (4 * t)) & 15u);
                NBW[t] = (Dc.PR[t] & m) | (Dc.U[t] & ~m);
            }
            const uint32_t nbR = __shfl_sync(amask, NBW[0], srcR);
            const uint32_t uR = __shfl_sync(amask, Dc.U[0], srcR);
#pragma unroll
            for (int t = 0; t < M; ++t) {
                const int tn = t + 1 < M ? t + 1 : t;
                scan::word_energy(NBW[t], Dc.U[t], Dc.HYZ[t], t + 1 < M ? NBW[tn] : nbR,
                                  t + 1 < M ? Dc.U[tn] : uR, dJ, dM);
                *wp(r, t) = scan::to_raw(NBW[t]);
            }
            // ---- the window for the rows to come
            const int lo_c = ring_target<R>(lo_a, E, g.nE);
            if (lo_c != lo_a) {
                const int ra = lo_c > lo_a ? max(lo_a + R, lo_c) : lo_c;
                const int rb = lo_c > lo_a ? lo_c + R : min(lo_a, lo_c + R);
                ring_copy<R>(ring, thrE, ra, rb, A, h);
            }
            cp_commit();
            lo_b = lo_a;
            lo_a = lo_c;
            // ---- advance: row r+1 becomes the current row
            a_prev = a;
#pragma unroll
            for (int t = 0; t < M; ++t) {
                DLp[t] = Dc.DL[t];
                Oc[t] = O1[t];
                O1[t] = y2 == 0 ? O2[t] : YP1[t];
                YM1[t] = YM2[t];
                YP1[t] = YP2[t];
                ZM1[t] = ZM2[t];
                ZP1[t] = ZP2[t];
            }
            Dc = Dn;
            y = y1;
            z = z1;
        }
        EJ += lanes_sum(dJ, amask, sbase, h, A);
        Mg += lanes_sum(dM, amask, sbase, h, A);
        if (h == 0) {
            hist_add_leaders(g.hist, E, lmask);
            if (record) {
                int32_t *o = g.ts + (ts_pos + k) * 3 * (int64_t)g.W + w;
                o[0] = EJ;
                o[g.W] = E + g.e_min;
                o[2 * g.W] = Mg;
            }
        }
    }
    if (h == 0) {
        g.tal[w] = EJ;
        g.tal[g.Wpad + w] = E + g.e_min;
        g.tal[2 * g.Wpad + w] = Mg;
    }
    cp_wait_all();
}

// A block is one warp of 32 / scan_seg(L) consecutive walkers of one group of
// row length L.  Dynamic shared memory: the table rings of the warp's walkers.
template <int L>
__global__ void __launch_bounds__(32)
sweep_scan_kernel(const GroupDev *__restrict__ groups, const BlockDesc *__restrict__ blocks,
                  uint32_t seed, uint64_t sweep0, int n_sweeps, int64_t ts_pos, int record)
{
    extern __shared__ __align__(16) uint32_t s_scan[];
    const BlockDesc bd = blocks[blockIdx.x];
    const GroupDev g = groups[bd.group];
    scan_sweeps<L>(g, bd.w0, bd.nw, s_scan, seed, sweep0, n_sweeps, ts_pos, record);
}

// The kernel of row length L as a function pointer (nullptr outside the range).
using ScanKernel = void (*)(const GroupDev *, const BlockDesc *, uint32_t, uint64_t, int,
                            int64_t, int);
ScanKernel scan_kernel_of(int L)
{
    switch (L) {
#define MUCA_SCAN(LL) \
    case LL: return sweep_scan_kernel<LL>;
        MUCA_SCAN(4)
        MUCA_SCAN(8)
        MUCA_SCAN(12)
        MUCA_SCAN(16)
        MUCA_SCAN(20)
        MUCA_SCAN(24)
        MUCA_SCAN(28)
        MUCA_SCAN(32)
        MUCA_SCAN(36)
        MUCA_SCAN(40)
        MUCA_SCAN(44)
        MUCA_SCAN(48)
        MUCA_SCAN(52)
        MUCA_SCAN(56)
        MUCA_SCAN(60)
        MUCA_SCAN(64)
#undef MUCA_SCAN
        default: return nullptr;
    }
}

}  // namespace

bool scan_supported(int L, int nE) { return scan_seg(L) > 0 && nE + 2 * kGuard >= scan_ring(L); }

int scan_block_walkers(int L)
{
    const int s = scan_seg(L);
    return s > 0 ? 32 / s : 0;
}

size_t scan_bytes_for(int L)
{
    if (scan_seg(L) <= 0) return 0;
    return (size_t)scan_block_walkers(L) * (scan_ring(L) * kRow + 4) * sizeof(uint32_t);
}

cudaError_t prepare_scan_kernel(int L, size_t smem_bytes)
{
    const ScanKernel k = scan_kernel_of(L);
    if (!k) return cudaErrorInvalidValue;
    return raise_smem_limit((const void *)k, smem_bytes);
}

cudaError_t launch_sweeps_scan(int L, const GroupDev *groups_dev, const BlockDesc *blocks_dev,
                               int n_blocks, size_t smem_bytes, uint32_t seed, uint64_t sweep0,
                               int n_sweeps, int64_t ts_pos, bool record, cudaStream_t st)
{
    if (n_blocks <= 0 || n_sweeps <= 0) return cudaSuccess;
    const ScanKernel k = scan_kernel_of(L);
    if (!k) return cudaErrorInvalidValue;
    k<<<n_blocks, 32, smem_bytes, st>>>(groups_dev, blocks_dev, seed, sweep0, n_sweeps, ts_pos,
                                        record ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace muca
