// muca_internal.h -- types shared by the host runtime and the CUDA kernels of
// the multicanonical Blume-Capel library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace muca {

// Packed acceptance table of one group, as the sweep kernel reads it: one
// row of kRow uint32 per E_Delta in the window (row e <-> E_Delta = e_min + e):
//   [0 .. 12]   d = -1 (s = +-1 -> 0),   dE_J = -6 .. 6
//   [13 .. 25]  d =  0 (s = +-1 -> -+1), dE_J = -12, -10, .., 12
//   [26 .. 38]  d = +1 (s = 0 -> +-1),   dE_J = -6 .. 6
//   [39]        unused (0)
// Every proposal of a site therefore reads one entry of the row of the
// walker's current E_Delta: column 13 (d + 1) + (d == 0 ? (dE_J + 12) / 2 : dE_J + 6).
constexpr int kRow = 40;
constexpr int kBlk = 13;

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
    const uint32_t *thr;        // [nE][kRow]
    int32_t *ts;                // [cap][3][W] or nullptr
};

// A block of the sweep grid: which group, first walker, walkers in the block,
// and (shared-memory blocks) the walker stride G of the lattice tile.
struct BlockDesc {
    int group;
    int w0;
    int nw;
    int G;
};

// Launch helpers implemented in sweep.cu.  All return a cudaError_t.
cudaError_t launch_init_spins(const GroupDev &g, uint32_t seed, cudaStream_t st);
// mode 0: write the recomputed tallies; mode 1: compare and raise *err on mismatch.
cudaError_t launch_energies(const GroupDev &g, int mode, int *err, cudaStream_t st);
// One launch sweeping every block of `blocks` (n_blocks of them).  smem_bytes > 0
// selects the shared-memory-resident kernel (prepare it once with
// prepare_smem_kernel outside any stream capture).
cudaError_t launch_sweeps(const GroupDev *groups_dev, const BlockDesc *blocks_dev, int n_blocks,
                          int threads, size_t smem_bytes, uint32_t seed, uint64_t sweep0,
                          int n_sweeps, int64_t ts_pos, bool record, cudaStream_t st);
cudaError_t prepare_smem_kernel(size_t smem_bytes);
// Bytes of one walker's lattice (padded rows) and of a shared-memory tile.
size_t lattice_bytes(int L);
size_t smem_bytes_for(int L, int walkers);
int max_smem_per_block();

// Last-error text reported by muca_last_error(NULL) (thread-local).
void set_last_error(const char *msg);

// Reweighting on caller-provided device scratch (reweight.cu).
int reweight_check_args(const int32_t *e_j, const int32_t *e_d, const int32_t *m, int64_t n_rows,
                        int32_t row_len, int64_t row_stride, const double *lnW, int32_t n_e,
                        double beta, int32_t V, const double *delta_grid, int32_t n_grid,
                        int32_t precision, double *out);
size_t reweight_scratch_bytes(int32_t n_e, int32_t n_grid, int32_t precision);
int reweight_on_scratch(const int32_t *e_j, const int32_t *e_d, const int32_t *m, int64_t n_rows,
                        int32_t row_len, int64_t row_stride, const double *lnW, int32_t e_min,
                        int32_t n_e, double beta, int32_t V, const double *delta_grid,
                        int32_t n_grid, int32_t precision, double *out, cudaStream_t st,
                        char *scratch);

}  // namespace muca
