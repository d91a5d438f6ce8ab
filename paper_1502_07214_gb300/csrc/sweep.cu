// sweep.cu -- initial spins, energy tallies and the typewriter Metropolis sweep
// of the parallel multicanonical Blume-Capel simulation.
//
// Model: Eq. 1 of the paper, H = E_J + Delta E_Delta with E_J = -sum_<ij> s_i s_j
// and E_Delta = sum_i s_i^2 on an L^3 periodic simple-cubic lattice.  Update:
// single-site Metropolis with the multicanonical weight exp(-beta E_J) W(E_Delta)
// (Sec. II), visiting sites in typewriter order i = x + L (y + L z).
//
// GPU design.  One thread owns one walker for the whole launch; the walkers of
// a warp advance in lock step through the same sites.  Each walker is a strict
// serial chain (site i+1 sees the E_Delta and the spin left behind by site i),
// so the kernel is organised around keeping that chain short:
//   - a row (fixed y, z) is processed as straight-line code with its L old
//     spins and the sums of their four y/z neighbours held in registers as
//     packed bytes; the words of the NEXT row and of its neighbour rows are
//     loaded at the start of the current row, so HBM/L2 latency is hidden
//     behind L Metropolis steps (the row just finished serves as the next
//     row's y-1 neighbour without a reload);
//   - the Philox block of four sites is independent of the chain and is
//     scheduled freely inside the unrolled row;
//   - each step reads one threshold from the L1/L2-resident table row of the
//     walker's current E_Delta (all three kinds of move live in one row, so
//     the lanes of a warp never diverge on the move kind).
// Sizes with L % 4 == 0 up to 48 use that unrolled path; any other L uses a
// plain per-site path with the same results.
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

// Running state of one walker.  rowoff = (E_Delta - e_min) * kRow selects the
// table row of the current E_Delta.
struct Chain {
    int EJ, ED, M, rowoff;
};

// One Metropolis step (Sec. II acceptance with the multicanonical weight).
//   word  the site's Philox word: bit 31 picks the proposal, bits 0..30 are u
//   s     the site's spin; base = sum of its neighbours except x - 1;
//   left  the current value of the x - 1 neighbour.
// The table column is 13 (d + 1) + (d == 0 ? (dE_J + 12) / 2 : dE_J + 6) with
// dE_J = -(s' - s)(base + left); written as c0 - k left with k = sign(s' - s)
// so that only one multiply-add separates `left` from the load.
__device__ __forceinline__ int metropolis(uint32_t word, int s, int base, int left,
                                          const uint32_t *__restrict__ thr, Chain &c)
{
    const int b = (int)(word >> 31);
    const uint32_t u = word & 0x7FFFFFFFu;
    const int lo = (s == -1) ? 0 : -1;
    const int hi = (s == 1) ? 0 : 1;
    const int sp = b ? hi : lo;
    const int diff = sp - s;
    const int d = sp * sp - s * s;
    const int k = diff > 0 ? 1 : -1;
    const int c0 = kBlk * (d + 1) + 6 - k * base;
    const uint32_t t = __ldg(thr + (c.rowoff + c0 - k * left));
    const bool acc = u < t;
    if (acc) {
        c.EJ -= diff * (base + left);
        c.ED += d;
        c.M += diff;
        c.rowoff += d * kRow;
    }
    return acc ? sp : s;
}

// ---------------------------------------------------------------------------
// Unrolled row path for L % 4 == 0.  lat points at word 0 of the walker;
// word (row, j) is lat[(row * Lw + j) * st].
// ---------------------------------------------------------------------------
template <int L>
__device__ __forceinline__ void sweep_rows(uint32_t *__restrict__ lat, ptrdiff_t st,
                                           const uint32_t *__restrict__ thr, uint32_t key0,
                                           uint32_t key1, uint64_t sw, Chain &c)
{
    static_assert(L % 4 == 0, "row path needs L % 4 == 0");
    constexpr int Lw = L / 4, R = L * L;
    const uint32_t slo = (uint32_t)sw, shi = (uint32_t)(sw >> 32);
    auto at = [&](int row, int j) -> uint32_t * { return lat + ((ptrdiff_t)row * Lw + j) * st; };
    uint32_t O[Lw], H[Lw];
    {
        // row 0 = (y 0, z 0): neighbours y-1 = (L-1, 0), y+1 = (1, 0), z-1 = (0, L-1), z+1 = (0, 1)
#pragma unroll
        for (int j = 0; j < Lw; ++j) {
            O[j] = *at(0, j);
            H[j] = __vadd4(__vadd4(*at(L - 1, j), *at(1, j)),
                           __vadd4(*at((L - 1) * L, j), *at(L, j)));
        }
    }
    int y = 0, z = 0;
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        // next row (y1, z1) and its neighbour rows; the last row loads row 0's
        // neighbourhood again (harmless: the values are not used)
        int y1 = y + 1, z1 = z;
        const bool wrap = (y1 == L);
        if (wrap) {
            y1 = 0;
            z1 = (z + 1 == L) ? 0 : z + 1;
        }
        const int rs = z1 * L + y1;
        const int ryp = z1 * L + (y1 + 1 == L ? 0 : y1 + 1);
        const int rym = z1 * L + (y1 == 0 ? L - 1 : y1 - 1);
        const int rzm = (z1 == 0 ? L - 1 : z1 - 1) * L + y1;
        const int rzp = (z1 + 1 == L ? 0 : z1 + 1) * L + y1;
        uint32_t Ps[Lw], Pyp[Lw], Pzm[Lw], Pzp[Lw], Pym[Lw];
#pragma unroll
        for (int j = 0; j < Lw; ++j) {
            Ps[j] = *at(rs, j);
            Pyp[j] = *at(ryp, j);
            Pzm[j] = *at(rzm, j);
            Pzp[j] = *at(rzp, j);
            Pym[j] = wrap ? *at(rym, j) : 0u;
        }
        // the row itself: Philox block of site i = r L + 4 j is r Lw + j
        int left = sbyte(O[Lw - 1], 3);  // x - 1 of x = 0: old value of x = L - 1
        int first = 0;                   // new value of x = 0 (x + 1 of x = L - 1)
        uint32_t N[Lw];
#pragma unroll
        for (int j = 0; j < Lw; ++j) {
            const uint4 rnd = philox4x32_10(make_uint4((uint32_t)(r * Lw + j), slo, shi, 0u),
                                            key0, key1);
            const uint32_t rw[4] = {rnd.x, rnd.y, rnd.z, rnd.w};
            uint32_t nw = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int x = 4 * j + q;
                const int s = sbyte(O[j], q);
                const int right = (x == L - 1) ? first
                                  : (q < 3)    ? sbyte(O[j], q + 1)
                                               : sbyte(O[(j + 1) % Lw], 0);
                const int base = sbyte(H[j], q) + right;
                const int sn = metropolis(rw[q], s, base, left, thr, c);
                nw |= (uint32_t)(sn & 0xFF) << (8 * q);
                if (x == 0) first = sn;
                left = sn;
            }
            N[j] = nw;
            *at(r, j) = nw;
        }
#pragma unroll
        for (int j = 0; j < Lw; ++j) {
            const uint32_t ym = wrap ? Pym[j] : N[j];
            H[j] = __vadd4(__vadd4(ym, Pyp[j]), __vadd4(Pzm[j], Pzp[j]));
            O[j] = Ps[j];
        }
        y = y1;
        z = z1;
    }
}

// ---------------------------------------------------------------------------
// Plain per-site path for any L >= 2 (neighbours read from the lattice).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int8_t *site_ptr(uint32_t *lat, ptrdiff_t st, int Lw, int row, int x)
{
    return reinterpret_cast<int8_t *>(lat + ((ptrdiff_t)row * Lw + (x >> 2)) * st) + (x & 3);
}

__device__ void sweep_sites(uint32_t *__restrict__ lat, ptrdiff_t st, int L, int Lw,
                            const uint32_t *__restrict__ thr, uint32_t key0, uint32_t key1,
                            uint64_t sw, Chain &c)
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
                *p = (int8_t)metropolis(word, *p, h, 0, thr, c);
            }
        }
    }
}

template <bool RECORD>
__device__ __forceinline__ void run_walker(uint32_t *__restrict__ lat, ptrdiff_t st,
                                           const GroupDev &g, uint32_t key0, uint32_t key1,
                                           uint64_t sweep0, int n_sweeps, int w, int64_t ts_pos,
                                           unsigned amask)
{
    Chain c;
    c.EJ = g.tal[w];
    c.ED = g.tal[g.Wpad + w];
    c.M = g.tal[2 * g.Wpad + w];
    c.rowoff = (c.ED - g.e_min) * kRow;
    const uint32_t *__restrict__ thr = g.thr;
    for (int k = 0; k < n_sweeps; ++k) {
        const uint64_t sw = sweep0 + (uint64_t)k;
        switch (g.L) {
            case 4: sweep_rows<4>(lat, st, thr, key0, key1, sw, c); break;
            case 8: sweep_rows<8>(lat, st, thr, key0, key1, sw, c); break;
            case 12: sweep_rows<12>(lat, st, thr, key0, key1, sw, c); break;
            case 16: sweep_rows<16>(lat, st, thr, key0, key1, sw, c); break;
            case 20: sweep_rows<20>(lat, st, thr, key0, key1, sw, c); break;
            case 24: sweep_rows<24>(lat, st, thr, key0, key1, sw, c); break;
            case 28: sweep_rows<28>(lat, st, thr, key0, key1, sw, c); break;
            case 32: sweep_rows<32>(lat, st, thr, key0, key1, sw, c); break;
            case 48: sweep_rows<48>(lat, st, thr, key0, key1, sw, c); break;
            default: sweep_sites(lat, st, g.L, g.Lw, thr, key0, key1, sw, c); break;
        }
        hist_add(g.hist, c.ED - g.e_min, amask);
        if (RECORD) {
            int32_t *o = g.ts + (ts_pos + k) * 3 * (int64_t)g.W + w;
            o[0] = c.EJ;
            o[g.W] = c.ED;
            o[2 * g.W] = c.M;
        }
    }
    g.tal[w] = c.EJ;
    g.tal[g.Wpad + w] = c.ED;
    g.tal[2 * g.Wpad + w] = c.M;
}

template <bool RECORD>
__global__ void __launch_bounds__(128)
sweep_global_kernel(const GroupDev *__restrict__ groups, const BlockDesc *__restrict__ blocks,
                    uint32_t seed, uint64_t sweep0, int n_sweeps, int64_t ts_pos)
{
    const BlockDesc bd = blocks[blockIdx.x];
    const GroupDev g = groups[bd.group];
    const int lw = (int)threadIdx.x;
    const bool active = lw < bd.nw;
    const unsigned amask = __ballot_sync(0xFFFFFFFFu, active);
    if (!active) return;
    const int w = bd.w0 + lw;
    run_walker<RECORD>(g.spins + w, g.Wpad, g, g.walker0 + (uint32_t)w, seed, sweep0, n_sweeps, w,
                       ts_pos, amask);
}

// Shared-memory-resident variant: the block's G lattices live in shared memory
// as a [L * L][Lw][G] word tile for the whole launch, read from and written
// back to the global array at the start and the end.
template <bool RECORD>
__global__ void __launch_bounds__(32)
sweep_smem_kernel(const GroupDev *__restrict__ groups, const BlockDesc *__restrict__ blocks,
                  uint32_t seed, uint64_t sweep0, int n_sweeps, int64_t ts_pos)
{
    extern __shared__ __align__(16) uint32_t s_lat[];
    const BlockDesc bd = blocks[blockIdx.x];
    const GroupDev g = groups[bd.group];
    const int G = bd.G;
    const int nwords = g.L * g.L * g.Lw;
    for (int idx = threadIdx.x; idx < nwords * G; idx += blockDim.x) {
        const int wd = idx / G, c = idx - wd * G;
        s_lat[idx] = (c < bd.nw) ? g.spins[(ptrdiff_t)wd * g.Wpad + bd.w0 + c] : 0u;
    }
    __syncthreads();
    const int lw = (int)threadIdx.x;
    const bool active = lw < bd.nw;
    const unsigned amask = __ballot_sync(0xFFFFFFFFu, active);
    if (active) {
        const int w = bd.w0 + lw;
        run_walker<RECORD>(s_lat + lw, G, g, g.walker0 + (uint32_t)w, seed, sweep0, n_sweeps, w,
                           ts_pos, amask);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nwords * G; idx += blockDim.x) {
        const int wd = idx / G, c = idx - wd * G;
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
                          int threads, size_t smem_bytes, uint32_t seed, uint64_t sweep0,
                          int n_sweeps, int64_t ts_pos, bool record, cudaStream_t st)
{
    if (n_blocks <= 0 || n_sweeps <= 0) return cudaSuccess;
    if (smem_bytes > 0) {
        if (record)
            sweep_smem_kernel<true><<<n_blocks, threads, smem_bytes, st>>>(
                groups_dev, blocks_dev, seed, sweep0, n_sweeps, ts_pos);
        else
            sweep_smem_kernel<false><<<n_blocks, threads, smem_bytes, st>>>(
                groups_dev, blocks_dev, seed, sweep0, n_sweeps, ts_pos);
    } else {
        if (record)
            sweep_global_kernel<true><<<n_blocks, threads, 0, st>>>(groups_dev, blocks_dev, seed,
                                                                    sweep0, n_sweeps, ts_pos);
        else
            sweep_global_kernel<false><<<n_blocks, threads, 0, st>>>(groups_dev, blocks_dev, seed,
                                                                     sweep0, n_sweeps, ts_pos);
    }
    return cudaGetLastError();
}

}  // namespace muca
