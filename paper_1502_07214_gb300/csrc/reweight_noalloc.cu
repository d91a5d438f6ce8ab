// reweight_noalloc.cu -- muca_reweight_noalloc: the time-series reweighting of
// muca_reweight with its working memory in a fixed array that the library
// carries in device memory, for callers that must not allocate.
//
// Who needs it: code that runs where a device allocation is off limits or
// unpredictable - a service that reserves all of its device memory up front
// and must not grow or fragment its pool afterwards, a real-time loop that
// cannot take the synchronisation an allocator may impose, or a binding from
// a language that reaches the library through plain pointers and has no
// device allocator of its own.
//
// The working memory is kScratchBytes of __device__ storage.  Every GPU that
// loads the library holds this array until the process exits.  All calls on a
// device share it and it keeps whatever the last call left in it; the
// reweighting clears the parts that must start at zero itself.  Two calls
// whose GPU work overlaps (for instance issued on different streams without
// ordering) race on the array and give wrong results: order them.  The call
// waits for its stream before it returns, like muca_reweight.
//
// The array's device address is looked up once per device and kept for the
// life of the process; after cudaDeviceReset the module, and with it the
// array, is loaded anew, so a process that resets a device must not call this
// entry point on that device again.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/muca.h"
#include "muca_internal.h"

namespace {

// 4 MiB: enough for n_e <= 32769 E_Delta bins (an L = 32 lattice) with
// n_grid <= 4096 Delta points in either precision.
constexpr size_t kScratchBytes = size_t(4) << 20;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  The first call on a
// device looks it up (cudaGetSymbolAddress) with that device current; later
// calls reuse it.
int scratch_address(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        muca::set_last_error((std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
        return MUCA_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        muca::set_last_error("muca_reweight_noalloc: device index out of range");
        return MUCA_ERR_NOT_SUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            muca::set_last_error(
                (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
            return MUCA_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return MUCA_OK;
}

}  // namespace

extern "C" int muca_reweight_noalloc(const int32_t *e_j, const int32_t *e_d, const int32_t *m,
                                     int64_t n_rows, int32_t row_len, int64_t row_stride,
                                     const double *lnW, int32_t e_min, int32_t n_e, double beta,
                                     int32_t V, const double *delta_grid, int32_t n_grid,
                                     int32_t precision, double *out, void *stream)
{
    int rc = muca::reweight_check_args(e_j, e_d, m, n_rows, row_len, row_stride, lnW, e_min, n_e,
                                       beta, V, delta_grid, n_grid, precision, out);
    if (rc != MUCA_OK) return rc;
    const size_t need = muca::reweight_scratch_bytes(n_e, n_grid, precision);
    if (need > kScratchBytes) {
        char msg[200];
        std::snprintf(msg, sizeof msg,
                      "muca_reweight_noalloc: n_e=%d, n_grid=%d need %zu bytes of working memory, "
                      "more than the fixed %zu",
                      n_e, n_grid, need, kScratchBytes);
        muca::set_last_error(msg);
        return MUCA_ERR_INVALID_ARG;
    }
    void *scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc != MUCA_OK) return rc;
    return muca::reweight_on_scratch(e_j, e_d, m, n_rows, row_len, row_stride, lnW, e_min, n_e,
                                     beta, V, delta_grid, n_grid, precision, out,
                                     (cudaStream_t)stream, (char *)scratch);
}
