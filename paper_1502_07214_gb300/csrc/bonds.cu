// bonds.cu -- typewriter Metropolis sweeps of the disordered model: the
// Blume-Capel model with one quenched integer coupling per bond (the bond
// disorder that the paper's outlook applies the method to), in the same
// multicanonical ensemble in E_Delta (Sec. II).
//
// E_J = -sum over the forward bonds (i, mu) of J[3 i + mu] s_i s_{i+mu}; the
// local field of site i weights each of its six neighbours by the coupling of
// the bond between them (its own forward bonds and the forward bonds of its
// three backward neighbours).  Couplings are integers in [-jmax, jmax], so
// dE_J = -(s' - s) h is an integer in [-12 jmax, 12 jmax] and the acceptance
// table of the group has rows of 24 jmax + 1 thresholds per (E_Delta, d):
//   thrJ[((E_Delta - e_min) * 3 + d + 1) * (24 jmax + 1) + dE_J + 12 jmax].
// Everything else (Philox words per site, proposals, the rejection of moves
// that leave the window through zero thresholds, the histogram after every
// sweep, the recorded series) is the clean model's.
//
// One thread per walker, a warp of 8 to 32 walkers (about four warps per SM);
// the walkers of a warp read whole 32-byte sectors per packed spin word.  One
// kernel per row length: for L % 4 == 0 a walker's row lives in registers
// (bonds_rows: x neighbours are byte extracts, the y / z neighbour words are
// loaded once per packed word, a site's six couplings are one load of its
// pack), for other L every neighbour and coupling is read from global memory
// (bonds_sites).  Each site keeps one dependent chain: its left neighbour,
// the field, the threshold load from the table, the compare.
#include <cuda_runtime.h>

#include <cstdint>

#include "muca_internal.h"
#include "philox.cuh"

namespace muca {
namespace {

__device__ __forceinline__ int8_t *spin_at(uint32_t *lat, ptrdiff_t st, int Lw, int row, int x)
{
    return reinterpret_cast<int8_t *>(lat + ((ptrdiff_t)row * Lw + (x >> 2)) * st) + (x & 3);
}

__device__ __forceinline__ void hist_inc(unsigned long long *hist, int bin, unsigned amask)
{
    const unsigned peers = __match_any_sync(amask, bin);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1)
        atomicAdd(hist + bin, (unsigned long long)__popc(peers));
}

// One sweep of one walker, site by site with every neighbour read from the
// lattice in global memory (any L).
__device__ __forceinline__ void bonds_sites(const GroupDev &g, uint32_t *lat, uint32_t key0,
                                            uint32_t seed, uint64_t sw, int &EJ, int &ED, int &M)
{
    const int L = g.L, Lw = g.Lw, nj = 24 * g.jmax + 1, off = 12 * g.jmax;
    const int8_t *__restrict__ J = g.J;
    const ptrdiff_t st = g.Wpad;
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
                    const uint4 r =
                        philox4x32_10(make_uint4((uint32_t)(i >> 2), slo, shi, 0u), key0, seed);
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
                // sites of the backward neighbours (their forward bonds end here)
                const int ixm = xm + L * row, iym = x + L * (z * L + ym), izm = x + L * (zm * L + y);
                const int h = J[3 * i + 0] * *spin_at(lat, st, Lw, row, xp) +
                              J[3 * ixm + 0] * *spin_at(lat, st, Lw, row, xm) +
                              J[3 * i + 1] * *spin_at(lat, st, Lw, z * L + yp, x) +
                              J[3 * iym + 1] * *spin_at(lat, st, Lw, z * L + ym, x) +
                              J[3 * i + 2] * *spin_at(lat, st, Lw, zp * L + y, x) +
                              J[3 * izm + 2] * *spin_at(lat, st, Lw, zm * L + y, x);
                int8_t *p = spin_at(lat, st, Lw, row, x);
                const int s = *p;
                const int lo = (s == -1) ? 0 : -1, hi = (s == 1) ? 0 : 1;
                const int sp = (word >> 31) ? hi : lo;
                const int d = sp * sp - s * s;
                const int dEJ = -(sp - s) * h;
                const uint32_t thr =
                    __ldg(g.thrJ + ((ptrdiff_t)(ED - g.e_min) * 3 + (d + 1)) * nj + dEJ + off);
                if ((word & 0x7FFFFFFFu) < thr) {
                    *p = (int8_t)sp;
                    EJ += dEJ;
                    ED += d;
                    M += sp - s;
                }
            }
        }
    }
}

__device__ __forceinline__ int sbyte(uint32_t w, int q) { return (int)(int8_t)(uint8_t)(w >> (8 * q)); }
__device__ __forceinline__ int jbyte(unsigned long long w, int k)
{
    return (int)(int8_t)(uint8_t)(w >> (8 * k));
}

// One sweep of one walker with rows of L = 4 LW sites: the row held in
// registers (every index a compile-time constant), the y / z neighbour words
// of each packed word loaded once for its four sites, the six couplings of a
// site from one load of its pack, the row stored once at its end.  Site
// order, Philox words and thresholds are those of bonds_sites: with
// L % 4 == 0 the block of site i = row L + 4 j + q is row LW + j and its
// word is q.
template <int LW>
__device__ __forceinline__ void bonds_rows(const GroupDev &g, uint32_t *lat, uint32_t key0,
                                           uint32_t seed, uint64_t sw, int &EJ, int &ED, int &M)
{
    constexpr int L = 4 * LW;
    const int nj = 24 * g.jmax + 1, off = 12 * g.jmax;
    const unsigned long long *__restrict__ J6 = g.J6;
    const uint32_t *__restrict__ thrJ = g.thrJ;
    const ptrdiff_t st = g.Wpad;
    const uint32_t slo = (uint32_t)sw, shi = (uint32_t)(sw >> 32);
    auto wp = [&](int row, int j) { return lat + ((ptrdiff_t)row * LW + j) * st; };
    for (int z = 0; z < L; ++z) {
        const int zm = z == 0 ? L - 1 : z - 1, zp = z + 1 == L ? 0 : z + 1;
        for (int y = 0; y < L; ++y) {
            const int ym = y == 0 ? L - 1 : y - 1, yp = y + 1 == L ? 0 : y + 1;
            const int row = z * L + y;
            uint32_t O[LW];
#pragma unroll
            for (int j = 0; j < LW; ++j) O[j] = *wp(row, j);
            const unsigned long long *jrow = J6 + (ptrdiff_t)row * L;
#pragma unroll
            for (int j = 0; j < LW; ++j) {
                // the y / z neighbour words of this word (not changed by the row)
                const uint32_t YMj = *wp(z * L + ym, j), YPj = *wp(z * L + yp, j);
                const uint32_t ZMj = *wp(zm * L + y, j), ZPj = *wp(zp * L + y, j);
                const uint4 rn =
                    philox4x32_10(make_uint4((uint32_t)(row * LW + j), slo, shi, 0u), key0, seed);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int x = 4 * j + q;
                    constexpr int kL = L;
                    const int xr = x + 1 == kL ? 0 : x + 1, xl = x == 0 ? kL - 1 : x - 1;
                    const uint32_t word = q == 0 ? rn.x : q == 1 ? rn.y : q == 2 ? rn.z : rn.w;
                    const unsigned long long jj = __ldg(jrow + x);
                    const int h = jbyte(jj, 0) * sbyte(O[xr >> 2], xr & 3) +
                                  jbyte(jj, 1) * sbyte(O[xl >> 2], xl & 3) +
                                  jbyte(jj, 2) * sbyte(YPj, q) + jbyte(jj, 3) * sbyte(YMj, q) +
                                  jbyte(jj, 4) * sbyte(ZPj, q) + jbyte(jj, 5) * sbyte(ZMj, q);
                    const int s = sbyte(O[j], q);
                    const int lo = (s == -1) ? 0 : -1, hi = (s == 1) ? 0 : 1;
                    const int sp = (word >> 31) ? hi : lo;
                    const int d = sp * sp - s * s;
                    const int dEJ = -(sp - s) * h;
                    const uint32_t thr =
                        __ldg(thrJ + ((ptrdiff_t)(ED - g.e_min) * 3 + (d + 1)) * nj + dEJ + off);
                    if ((word & 0x7FFFFFFFu) < thr) {
                        O[j] = (O[j] & ~(0xFFu << (8 * q))) | ((uint32_t)(uint8_t)sp << (8 * q));
                        EJ += dEJ;
                        ED += d;
                        M += sp - s;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < LW; ++j) *wp(row, j) = O[j];
        }
    }
}

// One kernel per row kind: LW > 0 the rows of L = 4 LW sites (bonds_rows),
// LW = 0 any L (bonds_sites); each gets its own register allocation.
template <int LW>
__global__ void __launch_bounds__(32)
sweep_bonds_kernel(const GroupDev *__restrict__ groups, const BlockDesc *__restrict__ blocks,
                   uint32_t seed, uint64_t sweep0, int n_sweeps, int64_t ts_pos, int record)
{
    const BlockDesc bd = blocks[blockIdx.x];
    const GroupDev &g = groups[bd.group];
    const int t = (int)threadIdx.x;
    const bool active = t < bd.nw;
    const unsigned amask = __ballot_sync(0xFFFFFFFFu, active);
    if (!active) return;
    const int w = bd.w0 + t;
    uint32_t *lat = g.spins + w;
    const uint32_t key0 = g.walker0 + (uint32_t)w;
    int EJ = g.tal[w], ED = g.tal[g.Wpad + w], M = g.tal[2 * g.Wpad + w];
    for (int k = 0; k < n_sweeps; ++k) {
        const uint64_t sw = sweep0 + (uint64_t)k;
        if constexpr (LW > 0)
            bonds_rows<LW>(g, lat, key0, seed, sw, EJ, ED, M);
        else
            bonds_sites(g, lat, key0, seed, sw, EJ, ED, M);
        hist_inc(g.hist, ED - g.e_min, amask);
        if (record) {
            int32_t *o = g.ts + (ts_pos + k) * 3 * (int64_t)g.W + w;
            o[0] = EJ;
            o[g.W] = ED;
            o[2 * g.W] = M;
        }
    }
    g.tal[w] = EJ;
    g.tal[g.Wpad + w] = ED;
    g.tal[2 * g.Wpad + w] = M;
}

}  // namespace

cudaError_t launch_sweeps_bonds(int L, const GroupDev *groups_dev, const BlockDesc *blocks_dev,
                                int n_blocks, uint32_t seed, uint64_t sweep0, int n_sweeps,
                                int64_t ts_pos, bool record, cudaStream_t st)
{
    if (n_blocks <= 0) return cudaSuccess;
    const int rec = record ? 1 : 0;
    switch (L % 4 == 0 ? L : 0) {
#define MUCA_BOND_LAUNCH(LL)                                                                 \
    case LL:                                                                                 \
        sweep_bonds_kernel<LL / 4><<<n_blocks, 32, 0, st>>>(groups_dev, blocks_dev, seed,     \
                                                            sweep0, n_sweeps, ts_pos, rec);  \
        break;
        MUCA_BOND_LAUNCH(4)
        MUCA_BOND_LAUNCH(8)
        MUCA_BOND_LAUNCH(12)
        MUCA_BOND_LAUNCH(16)
        MUCA_BOND_LAUNCH(20)
        MUCA_BOND_LAUNCH(24)
        MUCA_BOND_LAUNCH(28)
        MUCA_BOND_LAUNCH(32)
        MUCA_BOND_LAUNCH(36)
        MUCA_BOND_LAUNCH(40)
        MUCA_BOND_LAUNCH(44)
        MUCA_BOND_LAUNCH(48)
        MUCA_BOND_LAUNCH(52)
        MUCA_BOND_LAUNCH(56)
        MUCA_BOND_LAUNCH(60)
        MUCA_BOND_LAUNCH(64)
#undef MUCA_BOND_LAUNCH
        default:
            sweep_bonds_kernel<0><<<n_blocks, 32, 0, st>>>(groups_dev, blocks_dev, seed, sweep0,
                                                           n_sweeps, ts_pos, rec);
            break;
    }
    return cudaGetLastError();
}

}  // namespace muca
