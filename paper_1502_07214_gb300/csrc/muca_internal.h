// muca_internal.h -- types shared by the host runtime and the CUDA kernels of
// the multicanonical Blume-Capel library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace muca {

// Packed acceptance table of one group, as the sweep kernel reads it: one
// allocation of table_rows(nE) rows of kRow uint32 (160 bytes):
//   rows 0 .. kGuard-1     zero (guard)
//   row kGuard + e         E_Delta = e_min + e, e = 0 .. nE-1, every move kind:
//     column 13 (d + 1) + (d == 0 ? (dE_J + 12) / 2 : dE_J + 6),
//     d = -1: s = +-1 -> 0, d = 0: s = +-1 -> -+1, d = +1: s = 0 -> +-1
//   last kGuard rows       zero (guard)
// The d = 0 columns repeat in every row so that one index formula serves all
// moves.  The guard rows let the kernel read the rows E_Delta +- 1 and copy
// windows of rows without bounds checks; they are never compared against
// (moves that leave the window read 0 from the window's own rows).
constexpr int kRow = 40;
constexpr int kBlk = 13;
constexpr int kGuard = 2;
inline size_t table_rows(int nE) { return (size_t)nE + 2 * kGuard; }

// Spin layout of a group: int8 spins packed four consecutive sites of a row
// per 32-bit word, walker-minor: word (row, j) of walker w is at
//   spins[(row * Lw + j) * Wpad + w],  row = y + L z,  Lw = ceil(L / 4),
// and byte q of that word is site x = 4 j + q (bytes past x = L - 1 are 0).
// The 32 lanes of a warp thus read 128 contiguous bytes per word.

// Per-group parameters in device memory.
struct GroupDev {
    int L, V, W, Wpad, Lw;      // linear size, sites, walkers, padded walker stride, words/row
    int e_min, nE;              // E_Delta window start and number of bins
    uint32_t walker0;           // global id of walker 0 (Philox key word 0)
    uint32_t *spins;            // [L * L][Lw][Wpad] packed words
    int32_t *tal;               // [3][Wpad]: E_J, E_Delta, M
    unsigned long long *hist;   // [nE]
    const uint32_t *thrE;       // the row of E_Delta = e_min in the table allocation
    int32_t *ts;                // [cap][3][W] or nullptr
    // the disordered model (couplings per bond), or J = nullptr: couplings
    // J[3 i + mu] of the forward bonds, |J| <= jmax, and its table
    // [nE][3][24 jmax + 1], index dE_J + 12 jmax (bonds.cu)
    const int8_t *J;
    int jmax;
    const uint32_t *thrJ;
    // the six couplings of every site's bonds packed as int8 bytes of one
    // word: J[3 i], J[3 (i - x)], J[3 i + 1], J[3 (i - y) + 1], J[3 i + 2],
    // J[3 (i - z) + 2] (x+1, x-1, y+1, y-1, z+1, z-1 neighbours), bytes 6, 7 zero
    const unsigned long long *J6;
};

// A block of the sweep grid: which group, first walker, walkers in the block,
// walker slots S of the block (the stride of its staging area and, for
// shared-memory blocks, of its lattice tile; a multiple of 4 for global
// blocks), and the number P of lanes that serve one walker (thread t is lane
// t % P of walker slot t / P; P divides 32).
struct BlockDesc {
    int group;
    int w0;
    int nw;
    int S;
    int P;
};

// Launch helpers implemented in sweep.cu.  All return a cudaError_t.
cudaError_t launch_init_spins(const GroupDev &g, uint32_t seed, cudaStream_t st);
// mode 0: write the recomputed tallies; mode 1: compare and raise *err on mismatch.
cudaError_t launch_energies(const GroupDev &g, int mode, int *err, cudaStream_t st);
// One launch sweeping every block of `blocks` (n_blocks of them) with
// smem_bytes of dynamic shared memory; smem_kernel selects the
// shared-memory-resident kernel (prepare it once with prepare_smem_kernel
// outside any stream capture).
cudaError_t launch_sweeps(const GroupDev *groups_dev, const BlockDesc *blocks_dev, int n_blocks,
                          int threads, size_t smem_bytes, bool smem_kernel, uint32_t seed,
                          uint64_t sweep0, int n_sweeps, int64_t ts_pos, bool record,
                          cudaStream_t st);
// Raise the dynamic shared-memory limit of a kernel on the current device to
// at least smem_bytes; the limit is shared by every context of the process and
// never lowered.
cudaError_t raise_smem_limit(const void *func, size_t smem_bytes);
cudaError_t prepare_smem_kernel(size_t smem_bytes);
cudaError_t prepare_global_kernel(size_t smem_bytes);
// Warp-specialised launch (blocks of one chain warp and helper warps;
// BlockDesc.S walker slots, a power of 2 in [4, 32]).  Two instantiations:
// rows of up to kWsNarrowMaxL sites (wide = false) and longer rows.
constexpr int kWsNarrowMaxL = 32;
// kernel kinds: lanes, shared tile, split narrow, split wide, row scan,
// disordered model
constexpr int kKinds = 6;
cudaError_t launch_sweeps_ws(const GroupDev *groups_dev, const BlockDesc *blocks_dev, int n_blocks,
                             size_t smem_bytes, uint32_t seed, uint64_t sweep0, int n_sweeps,
                             int64_t ts_pos, bool record, bool wide, cudaStream_t st);
cudaError_t prepare_ws_kernel(size_t smem_bytes, bool wide);
size_t ws_bytes_for(int slots);
// Row-scan launch (scan.cu): a walker's packed words of a row are split
// into runs of scan_words(L) consecutive words, one run per lane of a segment
// of scan_seg(L) lanes (a power of 2; L / (4 scan_words(L)) of its lanes are
// used), so a warp serves 32 / scan_seg(L) walkers; blocks are one warp
// (BlockDesc.S = walkers per warp, BlockDesc.P = segment lanes), one kernel
// per row length; each walker
// keeps a ring of scan_ring(L) table rows in shared memory.  Windows shorter
// than a ring use other kernel kinds.
__host__ __device__ constexpr int scan_seg(int L)
{
    return (L < 4 || L > 64 || L % 4) ? 0
         : L == 4 ? 1 : L == 8 ? 2 : (L == 20 || L == 28 || L == 40 || L == 56 || L == 60) ? 8
         : (L == 44 || L == 52) ? 16 : 4;
}
__host__ __device__ constexpr int scan_words(int L)
{
    return scan_seg(L) == 0 ? 0
         : (L == 24 || L == 32 || L == 40 || L == 56) ? 2 : (L == 36 || L == 48 || L == 60) ? 3
         : L == 64 ? 4 : 1;
}
__host__ __device__ constexpr int scan_ring(int L) { return L <= 16 ? 16 : 32; }
bool scan_supported(int L, int nE);
int scan_block_walkers(int L);
size_t scan_bytes_for(int L);
// One kernel per row length L: prepare it (outside any stream capture) and
// launch it on blocks that all belong to groups of that L.
cudaError_t prepare_scan_kernel(int L, size_t smem_bytes);
cudaError_t launch_sweeps_scan(int L, const GroupDev *groups_dev, const BlockDesc *blocks_dev,
                               int n_blocks, size_t smem_bytes, uint32_t seed, uint64_t sweep0,
                               int n_sweeps, int64_t ts_pos, bool record, cudaStream_t st);
// Sweeps of groups with couplings per bond (bonds.cu): blocks of one warp,
// one thread per walker, BlockDesc.nw <= 32 walkers (P = 1); one launch per
// row length L, on blocks that all belong to groups of that L.
cudaError_t launch_sweeps_bonds(int L, const GroupDev *groups_dev, const BlockDesc *blocks_dev,
                                int n_blocks, uint32_t seed, uint64_t sweep0, int n_sweeps,
                                int64_t ts_pos, bool record, cudaStream_t st);
// Bytes of one walker's lattice (padded rows), of a shared-memory tile, and of
// the per-row staging area and table windows of `slots` walkers.
size_t lattice_bytes(int L);
size_t smem_bytes_for(int L, int walkers);
size_t stage_bytes_for(int slots);
int max_smem_per_block();

// Last-error text reported by muca_last_error(NULL) (thread-local).
void set_last_error(const char *msg);

// Reweighting on caller-provided device scratch (reweight.cu).
int reweight_check_args(const int32_t *e_j, const int32_t *e_d, const int32_t *m, int64_t n_rows,
                        int32_t row_len, int64_t row_stride, const double *lnW, int32_t e_min,
                        int32_t n_e,
                        double beta, int32_t V, const double *delta_grid, int32_t n_grid,
                        int32_t precision, double *out);
size_t reweight_scratch_bytes(int32_t n_e, int32_t n_grid, int32_t precision);
// records / records_bytes: an optional second device region (at most
// reweight_record_bytes(n_e, samples) bytes are used) that lets stage A sum
// the samples in shared memory per bucket of bins; without it (nullptr, 0)
// every sample adds to the global bin sums directly.
size_t reweight_record_bytes(int32_t n_e, int64_t n_samples);
int reweight_on_scratch(const int32_t *e_j, const int32_t *e_d, const int32_t *m, int64_t n_rows,
                        int32_t row_len, int64_t row_stride, const double *lnW, int32_t e_min,
                        int32_t n_e, double beta, int32_t V, const double *delta_grid,
                        int32_t n_grid, int32_t precision, double *out, cudaStream_t st,
                        char *scratch, char *records = nullptr, size_t records_bytes = 0);

}  // namespace muca
