// sweep.cu -- initial spins, energy tallies and the typewriter Metropolis sweep
// of the parallel multicanonical Blume-Capel simulation.
//
// Model: Eq. 1 of the paper, H = E_J + Delta E_Delta with E_J = -sum_<ij> s_i s_j
// and E_Delta = sum_i s_i^2 on an L^3 periodic simple-cubic lattice.  Update:
// single-site Metropolis with the multicanonical weight exp(-beta E_J) W(E_Delta)
// (Sec. II), visiting sites in typewriter order i = x + L (y + L z).
//
// GPU layout: one thread owns one walker for the whole launch.  Spins are int8
// in a site-major, walker-minor array [V][Wpad], so the 32 lanes of a warp touch
// one contiguous 32-byte sector per site.  The acceptance decision compares the
// 31-bit Philox draw with a uint32 threshold from the group's packed table (see
// muca_internal.h); the table is L2-resident and built on the host in FP64.
#include <cstdint>

#include "muca_internal.h"
#include "philox.cuh"

namespace muca {

namespace {

// Warp-aggregated histogram increment: lanes holding the same bin elect one
// leader that adds the count of its peers (kernel (b) of the hot path).
__device__ __forceinline__ void hist_add(unsigned long long *hist, int bin, unsigned amask)
{
    const unsigned peers = __match_any_sync(amask, bin);
    const int leader = __ffs(peers) - 1;
    if ((int)(threadIdx.x & 31) == leader)
        atomicAdd(hist + bin, (unsigned long long)__popc(peers));
}

// n_sweeps typewriter sweeps of one walker whose lattice starts at `lat`, with
// consecutive sites `st` bytes apart.  EJ, ED, M are the running tallies.
template <bool RECORD>
__device__ __forceinline__ void run_sweeps(int8_t *__restrict__ lat, ptrdiff_t st,
                                           const GroupDev &g, uint32_t key0, uint32_t key1,
                                           uint64_t sweep0, int n_sweeps, int &EJ, int &ED,
                                           int &M, const uint32_t *__restrict__ s_thr0, int w,
                                           int64_t ts_pos, unsigned amask)
{
    const int L = g.L;
    const ptrdiff_t sx = st, sy = (ptrdiff_t)L * st, sz = (ptrdiff_t)L * L * st;
    // rows indexed directly by E_Delta
    const uint32_t *__restrict__ thrE = g.thrE - (ptrdiff_t)g.e_min * kRow;
    for (int k = 0; k < n_sweeps; ++k) {
        const uint64_t sw = sweep0 + (uint64_t)k;
        const uint32_t slo = (uint32_t)sw, shi = (uint32_t)(sw >> 32);
        uint32_t r0 = 0, r1 = 0, r2 = 0, r3 = 0;
        int i = 0;
        int8_t *pz = lat;
        for (int z = 0; z < L; ++z, pz += sz) {
            const ptrdiff_t ozm = (z == 0) ? (L - 1) * sz : -sz;
            const ptrdiff_t ozp = (z == L - 1) ? -(L - 1) * sz : sz;
            int8_t *py = pz;
            for (int y = 0; y < L; ++y, py += sy) {
                const ptrdiff_t oym = (y == 0) ? (L - 1) * sy : -sy;
                const ptrdiff_t oyp = (y == L - 1) ? -(L - 1) * sy : sy;
                int left = py[(L - 1) * sx];  // x - 1 of x = 0: old value of x = L - 1
                int cur = py[0];
                int8_t *q = py;
                for (int x = 0; x < L; ++x, ++i, q += sx) {
                    if ((i & 3) == 0) {
                        const uint4 r = philox4x32_10(
                            make_uint4((uint32_t)(i >> 2), slo, shi, 0u), key0, key1);
                        r0 = r.x;
                        r1 = r.y;
                        r2 = r.z;
                        r3 = r.w;
                    }
                    const uint32_t word = r0;
                    r0 = r1;
                    r1 = r2;
                    r2 = r3;
                    // x + 1 of x = L - 1 is x = 0 of this row, already updated
                    const int right = (x == L - 1) ? (int)py[0] : (int)q[sx];
                    const int h = left + right + q[oym] + q[oyp] + q[ozm] + q[ozp];
                    const int s = cur;
                    const int b = (int)(word >> 31);
                    const uint32_t u = word & 0x7FFFFFFFu;
                    const int lo = (s == -1) ? 0 : -1;
                    const int hi = (s == 1) ? 0 : 1;
                    const int sp = b ? hi : lo;
                    const int diff = sp - s;
                    const int dEJ = -diff * h;
                    const int d = sp * sp - s * s;
                    uint32_t t;
                    if (d == 0)
                        t = s_thr0[(dEJ + 12) >> 1];
                    else
                        t = __ldg(thrE + (ptrdiff_t)ED * kRow + (d > 0 ? kRowPlus : 0) + dEJ + 6);
                    const bool acc = u < t;
                    if (acc) {
                        *q = (int8_t)sp;
                        EJ += dEJ;
                        ED += d;
                        M += diff;
                    }
                    left = acc ? sp : s;
                    cur = right;
                }
            }
        }
        hist_add(g.hist, ED - g.e_min, amask);
        if (RECORD) {
            int32_t *o = g.ts + (ts_pos + k) * 3 * (int64_t)g.W + w;
            o[0] = EJ;
            o[g.W] = ED;
            o[2 * g.W] = M;
        }
    }
}

template <bool RECORD>
__global__ void __launch_bounds__(1024)
sweep_global_kernel(const GroupDev *__restrict__ groups, const BlockDesc *__restrict__ blocks,
                    uint32_t seed, uint64_t sweep0, int n_sweeps, int64_t ts_pos)
{
    __shared__ uint32_t s_thr0[kThr0];
    const BlockDesc bd = blocks[blockIdx.x];
    const GroupDev g = groups[bd.group];
    if (threadIdx.x < kThr0) s_thr0[threadIdx.x] = g.thr0[threadIdx.x];
    __syncthreads();
    const int lw = (int)threadIdx.x;
    const bool active = lw < bd.nw;
    const unsigned amask = __ballot_sync(0xFFFFFFFFu, active);
    if (!active) return;
    const int w = bd.w0 + lw;
    int EJ = g.tal[w], ED = g.tal[g.Wpad + w], M = g.tal[2 * g.Wpad + w];
    run_sweeps<RECORD>(g.spins + w, g.Wpad, g, g.walker0 + (uint32_t)w, seed, sweep0, n_sweeps,
                       EJ, ED, M, s_thr0, w, ts_pos, amask);
    g.tal[w] = EJ;
    g.tal[g.Wpad + w] = ED;
    g.tal[2 * g.Wpad + w] = M;
}

// Shared-memory-resident variant: the block's G lattices live in shared
// memory as [V][G] for the whole launch; spins are read from and written back
// to the global [V][Wpad] array at the start and the end.
template <bool RECORD>
__global__ void __launch_bounds__(1024)
sweep_smem_kernel(const GroupDev *__restrict__ groups, const BlockDesc *__restrict__ blocks,
                  uint32_t seed, uint64_t sweep0, int n_sweeps, int64_t ts_pos)
{
    extern __shared__ __align__(16) int8_t s_lat[];
    __shared__ uint32_t s_thr0[kThr0];
    const BlockDesc bd = blocks[blockIdx.x];
    const GroupDev g = groups[bd.group];
    const int G = bd.G;
    if (threadIdx.x < kThr0) s_thr0[threadIdx.x] = g.thr0[threadIdx.x];
    const int n = g.V * G;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        const int site = idx / G, c = idx - site * G;
        s_lat[idx] = (c < bd.nw) ? g.spins[(ptrdiff_t)site * g.Wpad + bd.w0 + c] : (int8_t)0;
    }
    __syncthreads();
    const int lw = (int)threadIdx.x;
    const bool active = lw < bd.nw;
    const unsigned amask = __ballot_sync(0xFFFFFFFFu, active);
    if (active) {
        const int w = bd.w0 + lw;
        int EJ = g.tal[w], ED = g.tal[g.Wpad + w], M = g.tal[2 * g.Wpad + w];
        run_sweeps<RECORD>(s_lat + lw, G, g, g.walker0 + (uint32_t)w, seed, sweep0, n_sweeps,
                           EJ, ED, M, s_thr0, w, ts_pos, amask);
        g.tal[w] = EJ;
        g.tal[g.Wpad + w] = ED;
        g.tal[2 * g.Wpad + w] = M;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        const int site = idx / G, c = idx - site * G;
        if (c < bd.nw) g.spins[(ptrdiff_t)site * g.Wpad + bd.w0 + c] = s_lat[idx];
    }
}

// Initial spins i.i.d. uniform on {-1, 0, +1} from Philox stream 1: thread
// (j, w) draws the four sites 4j .. 4j+3 of walker w.
__global__ void init_spins_kernel(GroupDev g, uint32_t seed)
{
    const int nb = (g.V + 3) >> 2;
    const int64_t total = (int64_t)nb * g.W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / g.W), w = (int)(t - (int64_t)j * g.W);
        const uint4 r =
            philox4x32_10(make_uint4((uint32_t)j, 0u, 0u, 1u), g.walker0 + (uint32_t)w, seed);
        const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int site = 4 * j + q;
            if (site < g.V)
                g.spins[(ptrdiff_t)site * g.Wpad + w] =
                    (int8_t)((int)(((uint64_t)rw[q] * 3u) >> 32) - 1);
        }
    }
}

// E_J (three forward bonds per site), E_Delta and M of every walker, one
// thread per walker.  mode 0 stores them as the running tallies, mode 1
// compares them with the running tallies and sets *err on a mismatch.
__global__ void energies_kernel(GroupDev g, int mode, int *err)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= g.W) return;
    const int L = g.L;
    const ptrdiff_t st = g.Wpad;
    const int8_t *p = g.spins + w;
    int ej = 0, ed = 0, m = 0;
    for (int z = 0; z < L; ++z) {
        const int zp = (z + 1 == L) ? 0 : z + 1;
        for (int y = 0; y < L; ++y) {
            const int yp = (y + 1 == L) ? 0 : y + 1;
            for (int x = 0; x < L; ++x) {
                const int xp = (x + 1 == L) ? 0 : x + 1;
                const int s = p[(x + L * (y + L * z)) * st];
                ej -= s * (p[(xp + L * (y + L * z)) * st] + p[(x + L * (yp + L * z)) * st] +
                           p[(x + L * (y + L * zp)) * st]);
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
    const int64_t total = (int64_t)((g.V + 3) >> 2) * g.W;
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

size_t smem_bytes_for(int V, int walkers) { return (size_t)V * (size_t)walkers; }

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
