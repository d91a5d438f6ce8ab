// runtime.cu -- host runtime behind the muca_* C ABI: context and device
// buffers, the FP64 weight recursion and acceptance-table build (Sec. II),
// kernel configuration (autotuned), CUDA-graph capture of the iteration loop,
// and checkpoint / restore.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/muca.h"
#include "muca_internal.h"

using namespace muca;

namespace {

thread_local std::string g_last_error = "no error";

struct Group {
    muca_group spec{};
    int L = 0, V = 0, W = 0, Wpad = 0, Lw = 0, e_min = 0, e_max = 0, nE = 0;
    double T = 0, beta = 0;
    uint32_t walker0 = 0;
    // device
    uint32_t *spins = nullptr;  // [L * L][Lw][Wpad] packed words
    int32_t *tal = nullptr;
    unsigned long long *hist = nullptr;
    uint32_t *thr = nullptr;    // table allocation, table_rows(nE) x kRow
    int32_t *ts = nullptr;
    // host
    std::vector<double> lnW;
    int recursion = MUCA_REC_PLAIN;  // weight recursion (muca_set_recursion)
    std::vector<double> acc;         // its accumulated pair weights, max(nE - 1, 1)
    double flat[3] = {0.0, 0.0, 0.0};  // flatness of the histogram of the last update
    // the active E_Delta window [win_lo, win_hi] (bins, relative to e_min) that
    // the walkers move in, and its growth rule (muca_set_window; grow_flat = 0:
    // fixed)
    int win_lo = 0, win_hi = 0, grow_step = 0;
    double grow_flat = 0.0;
    bool flat_full = false;  // the last update's histogram was taken over all nE bins
    std::vector<uint32_t> injected;  // logical table given by muca_set_table (empty if none)
    uint32_t *h_thr = nullptr;       // pinned copy of the table allocation
    unsigned long long *h_hist = nullptr;  // pinned [nE]
    // the disordered model (muca_set_bonds): couplings of the forward bonds on
    // the device, |J| <= jmax (0: the clean model), and its table
    // [nE][3][24 jmax + 1] on the device and pinned on the host
    int8_t *d_J = nullptr;
    unsigned long long *d_J6 = nullptr;  // per-site pack of the six couplings
    int jmax = 0;
    std::vector<int8_t> J;
    uint32_t *thrJ = nullptr, *h_thrJ = nullptr;
    // every walker's E_Delta lies in the active window (required before sweeping)
    bool in_window = false;
    // kernel configuration
    int residency = MUCA_RES_GLOBAL;
    int wpb = 32;  // walkers per block
    int P = 1;     // lanes per walker
};

struct GraphKey {
    int n_iters, sweeps;
    uint64_t sweep0;
};

}  // namespace

struct muca_ctx {
    std::vector<Group> g;
    uint32_t seed = 0;
    int debug = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side[kKinds] = {};  // one stream per kernel kind
    cudaStream_t cap = nullptr;   // stream the iteration graph is captured on
    cudaEvent_t ev_fork = nullptr, ev_join[kKinds] = {};
    uint64_t sweep = 0;
    int64_t ts_cap = 0, ts_len = 0;
    std::string err = "no error";
    int *d_err = nullptr;
    GroupDev *d_groups = nullptr;
    // one launch per kernel kind in use: 0 lanes-per-walker (global lattice),
    // 1 shared-memory lattice, 2 split warps (global lattice)
    BlockDesc *d_blocks[kKinds] = {};
    int n_blocks[kKinds] = {};
    size_t smem[kKinds] = {};
    // the row-scan kind (4) has one kernel per row length: its blocks are
    // sorted by L and launched per range, each on a stream of its own when
    // more than one launch is in use
    struct ScanRange {
        int L, first, count;
        size_t smem;
    };
    std::vector<ScanRange> scan_ranges;
    // the disordered model's blocks (kind 5), sorted by L: one launch per L
    std::vector<ScanRange> bond_ranges;
    std::vector<cudaStream_t> scan_streams;
    std::vector<cudaEvent_t> scan_events;
};

namespace {

int fail(muca_ctx *ctx, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    if (ctx) ctx->err = buf;
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MUCA_ERR_OOM : MUCA_ERR_CUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// ---------------------------------------------------------------------------
// Acceptance thresholds (Sec. II weights, built in FP64):
//   x = -beta dE_J + (lnW[E + d] - lnW[E]);  thr = 2^31 if x >= 0,
//   else floor(exp(x) 2^31); thr = 0 when E + d leaves the window (the
//   group's active window [lo, hi], bins relative to e_min).
// The arithmetic is written out exactly as it must round (the library is built
// with -ffp-contract=off, so no multiply-add is fused).
// ---------------------------------------------------------------------------
inline uint32_t thr_of(double x)
{
    if (x >= 0.0) return 0x80000000u;
    if (x < -21.5) return 0u;  // exp(x) 2^31 < 0.99: floor is 0
    const double t = std::floor(std::exp(x) * 2147483648.0);
    return t >= 2147483648.0 ? 0x80000000u : (uint32_t)t;
}

inline uint32_t table_entry(double beta, const double *lnW, int lo, int hi, int e, int d, int dej)
{
    const int en = e + d;
    if (en < lo || en > hi) return 0u;
    const double x = -(beta * (double)dej) + (lnW[en] - lnW[e]);
    return thr_of(x);
}

inline uint32_t thr_entry(const Group &g, int e, int d, int dej)
{
    return table_entry(g.beta, g.lnW.data(), g.win_lo, g.win_hi, e, d, dej);
}

template <class F>
void parallel_rows(int n, F f)
{
    const int min_rows = 4096;
    int nt = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 16u);
    if (n < 2 * min_rows || nt <= 1) {
        f(0, n);
        return;
    }
    nt = std::min(nt, n / min_rows);
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t)
        th.emplace_back(f, (int)((int64_t)n * t / nt), (int)((int64_t)n * (t + 1) / nt));
    f(0, (int)((int64_t)n / nt));
    for (auto &x : th) x.join();
}

// The disordered model's table [nE][3][24 jmax + 1] (index dE_J + 12 jmax)
// from lnW into its pinned host buffer: every entry of the formula, including
// dE_J that no move of the given couplings produces.
void build_bonds_table(Group &g)
{
    const int nj = 24 * g.jmax + 1, off = 12 * g.jmax;
    uint32_t *T = g.h_thrJ;
    parallel_rows(g.nE, [&g, T, nj, off](int b, int e_end) {
        for (int e = b; e < e_end; ++e)
            for (int d = -1; d <= 1; ++d)
                for (int dej = -off; dej <= off; ++dej)
                    T[((size_t)e * 3 + (d + 1)) * nj + (dej + off)] = thr_entry(g, e, d, dej);
    });
}

size_t bonds_table_words(const Group &g) { return (size_t)g.nE * 3 * (24 * g.jmax + 1); }

// The table a group's sweeps read: its bytes, host copy and device copy.
size_t table_bytes(const Group &g)
{
    return g.jmax ? bonds_table_words(g) * sizeof(uint32_t)
                  : table_rows(g.nE) * kRow * sizeof(uint32_t);
}
const uint32_t *table_host(const Group &g) { return g.jmax ? g.h_thrJ : g.h_thr; }
uint32_t *table_dev(const Group &g) { return g.jmax ? g.thrJ : g.thr; }

// Packed table of group g from its lnW into the pinned host buffer (the
// disordered model's table for a group with couplings).
void build_packed(Group &g)
{
    if (g.jmax) {
        build_bonds_table(g);
        return;
    }
    uint32_t *T = g.h_thr;
    std::memset(T, 0, table_rows(g.nE) * kRow * sizeof(uint32_t));
    uint32_t *E0 = T + (size_t)kGuard * kRow;
    uint32_t d0[kBlk];
    // d = 0 keeps E_Delta: the same entries in every row (taken in the window)
    for (int k = 0; k < kBlk; ++k) d0[k] = thr_entry(g, g.win_lo, 0, 2 * k - 12);
    parallel_rows(g.nE, [&g, E0, &d0](int b, int e_end) {
        for (int e = b; e < e_end; ++e) {
            uint32_t *row = E0 + (size_t)e * kRow;
            for (int dej = -6; dej <= 6; ++dej) {
                row[dej + 6] = thr_entry(g, e, -1, dej);
                row[2 * kBlk + dej + 6] = thr_entry(g, e, +1, dej);
            }
            for (int k = 0; k < kBlk; ++k) row[kBlk + k] = d0[k];
        }
    });
}

// Pack a logical [nE][3][25] table; its d = 0 entries must not depend on
// E_Delta (they never do for a table built from weights: lnW[E] - lnW[E] = 0).
int pack_logical(muca_ctx *ctx, Group &g, const uint32_t *lg)
{
    for (int e = 0; e < g.nE; ++e)
        for (int k = 0; k < kBlk; ++k)
            if (lg[((size_t)e * 3 + 1) * MUCA_NK + 2 * k] != lg[1 * MUCA_NK + 2 * k])
                return fail(ctx, MUCA_ERR_INVALID_ARG,
                            "set_table: d = 0 entries must not depend on E_Delta (row %d)", e);
    uint32_t *T = g.h_thr;
    std::memset(T, 0, table_rows(g.nE) * kRow * sizeof(uint32_t));
    uint32_t *E0 = T + (size_t)kGuard * kRow;
    for (int e = 0; e < g.nE; ++e) {
        const uint32_t *r = lg + (size_t)e * 3 * MUCA_NK;
        uint32_t *row = E0 + (size_t)e * kRow;
        for (int dej = -6; dej <= 6; ++dej) {
            row[dej + 6] = r[0 * MUCA_NK + dej + 12];
            row[2 * kBlk + dej + 6] = r[2 * MUCA_NK + dej + 12];
        }
        for (int k = 0; k < kBlk; ++k) row[kBlk + k] = r[1 * MUCA_NK + 2 * k];
    }
    return MUCA_OK;
}

int upload_table(muca_ctx *ctx, Group &g)
{
    CK(cudaMemcpyAsync(table_dev(g), table_host(g), table_bytes(g), cudaMemcpyHostToDevice,
                       ctx->stream));
    return MUCA_OK;
}

// One weight update (muca_weight_update).  Plain: lnW[E] -= ln H[E] where
// H[E] > 0.  Accumulated: the ratio r(E) = lnW[E+1] - lnW[E] of every pair
// with both bins hit moves by (p / acc) (ln H[E] - ln H[E+1]), p = H[E] H[E+1]
// / (H[E] + H[E+1]) added to acc first, which keeps r the inverse-variance
// mean of the estimates of every iteration that hit both bins; a pair with an
// empty bin takes the plain step (the empty bin counted as 1) and adds
// nothing to acc; lnW[0] stays and the weights are summed up from the new
// ratios.
void weight_update(int kind, int nE, const unsigned long long *H, double *lnW, double *acc)
{
    if (kind == MUCA_REC_PLAIN) {
        for (int e = 0; e < nE; ++e)
            if (H[e] > 0) lnW[e] -= std::log((double)H[e]);
        return;
    }
    if (nE < 2) return;
    std::vector<double> r((size_t)nE - 1);
    for (int e = 0; e + 1 < nE; ++e) {
        const double h0 = (double)H[e], h1 = (double)H[e + 1];
        double re = lnW[e + 1] - lnW[e];
        if (H[e] > 0 && H[e + 1] > 0) {
            const double p = h0 * h1 / (h0 + h1);
            acc[e] = acc[e] + p;
            re = re + (p / acc[e]) * (std::log(h0) - std::log(h1));
        } else {
            re = re + (std::log(h0 > 1.0 ? h0 : 1.0) - std::log(h1 > 1.0 ? h1 : 1.0));
        }
        r[e] = re;
    }
    for (int e = 0; e + 1 < nE; ++e) lnW[e + 1] = lnW[e] + r[e];
}

// The weight update of one iteration of group g on its merged histogram:
// the histogram's flatness over the active window is recorded, the weight
// recursion runs over all nE bins, and then the adaptive window grows when
// the histogram was flat over it.  Growth (the adaptive window of the weight
// iteration): by grow_step bins on each side, clamped to [e_min, e_max],
// after an iteration with min H / mean H >= grow_flat over the window
// (mean H = sum H / bins); a new bin starts from the weight of the old edge
// next to it, and the accumulated weights of the pairs that contain a new
// bin start from 0.
void update_lnW(Group &g)
{
    unsigned long long lo = ~0ull, hi = 0, sum = 0;
    int64_t hit = 0;
    for (int e = g.win_lo; e <= g.win_hi; ++e) {
        const unsigned long long h = g.h_hist[e];
        lo = std::min(lo, h);
        hi = std::max(hi, h);
        sum += h;
        hit += h > 0;
    }
    if (sum == 0) {
        g.flat[0] = g.flat[1] = g.flat[2] = 0.0;
    } else {
        const double mean = (double)sum / (double)(g.win_hi - g.win_lo + 1);
        g.flat[0] = (double)lo / mean;
        g.flat[1] = (double)hi / mean;
        g.flat[2] = (double)hit;
    }
    weight_update(g.recursion, g.nE, g.h_hist, g.lnW.data(), g.acc.data());
    const bool full = g.win_lo == 0 && g.win_hi == g.nE - 1;
    g.flat_full = full;
    if (g.grow_flat > 0.0 && !full && g.flat[0] >= g.grow_flat) {
        const int lo_new = std::max(0, g.win_lo - g.grow_step);
        const int hi_new = std::min(g.nE - 1, g.win_hi + g.grow_step);
        for (int e = lo_new; e < g.win_lo; ++e) g.lnW[e] = g.lnW[g.win_lo];
        for (int e = g.win_hi + 1; e <= hi_new; ++e) g.lnW[e] = g.lnW[g.win_hi];
        if (g.recursion == MUCA_REC_ACCUMULATED) {
            for (int e = lo_new; e < g.win_lo; ++e) g.acc[e] = 0.0;
            for (int e = g.win_hi; e < hi_new; ++e) g.acc[e] = 0.0;
        }
        g.win_lo = lo_new;
        g.win_hi = hi_new;
    }
}

GroupDev dev_of(const Group &g)
{
    GroupDev d{};
    d.L = g.L;
    d.V = g.V;
    d.W = g.W;
    d.Wpad = g.Wpad;
    d.Lw = g.Lw;
    d.e_min = g.e_min;
    d.nE = g.nE;
    d.walker0 = g.walker0;
    d.spins = g.spins;
    d.tal = g.tal;
    d.hist = g.hist;
    d.thrE = g.thr ? g.thr + (size_t)kGuard * kRow : nullptr;
    d.ts = g.ts;
    d.J = g.jmax ? g.d_J : nullptr;
    d.jmax = g.jmax;
    d.thrJ = g.jmax ? g.thrJ : nullptr;
    d.J6 = g.jmax ? g.d_J6 : nullptr;
    return d;
}

int upload_groups(muca_ctx *ctx)
{
    std::vector<GroupDev> gd;
    for (auto &g : ctx->g) gd.push_back(dev_of(g));
    CK(cudaMemcpy(ctx->d_groups, gd.data(), gd.size() * sizeof(GroupDev), cudaMemcpyHostToDevice));
    return MUCA_OK;
}

// Kernel kind of a group's configuration.
int kind_of(const Group &g)
{
    if (g.jmax) return 5;
    if (g.residency == MUCA_RES_SCAN) return 4;
    if (g.residency == MUCA_RES_SPLIT) return g.L > kWsNarrowMaxL ? 3 : 2;
    return g.residency == MUCA_RES_SMEM ? 1 : 0;
}

// Block lists of the launches.  A block of group g serves wpb_g walkers:
//   kind 0: one warp, P_g lanes per walker, staging area and table windows;
//   kind 1: one warp, the walkers' lattices as a [L*L][Lw][wpb_g] tile too;
//   kinds 2, 3: split kernel (chain warp + helpers), wpb_g a power of 2 in
//   [4, 32]; kind 2 for rows of up to kWsNarrowMaxL sites, kind 3 above;
//   kind 4: row-scan kernel, one warp of wpb_g = 32 / P_g walkers per block,
//   P_g = scan_seg(L) lanes per walker.
// Walkers per warp of the disordered model's kernel: the walkers are spread
// over about four warps per SM (a power of 2, at most 32; at least 8 keep
// whole 32-byte sectors per packed-word load).  Measured at 4096 walkers of
// L = 24 with the site-by-site kernel: 8 per warp 1.58e10 attempts/s, 32 per
// warp 1.45e10 (each warp's per-site chain is the limit either way).
int bonds_walkers_per_warp(int W)
{
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
        nsm = 1;
    int wpb = 8;
    while (wpb < 32 && (int64_t)W > (int64_t)wpb * nsm * 4) wpb *= 2;
    return wpb;
}

int build_blocks(muca_ctx *ctx)
{
    std::vector<BlockDesc> b[kKinds];
    size_t sm[kKinds] = {};
    for (size_t gi = 0; gi < ctx->g.size(); ++gi) {
        const Group &g = ctx->g[gi];
        const int k = kind_of(g);
        const size_t need = k == 0   ? stage_bytes_for(g.wpb)
                            : k == 1 ? smem_bytes_for(g.L, g.wpb) + stage_bytes_for(g.wpb)
                            : k == 4 ? scan_bytes_for(g.L)
                            : k == 5 ? 0
                                     : ws_bytes_for(g.wpb);
        sm[k] = std::max(sm[k], need);
        const int wpb = k == 5 ? bonds_walkers_per_warp(g.W) : g.wpb, P = k == 5 ? 1 : g.P;
        for (int w0 = 0; w0 < g.W; w0 += wpb)
            b[k].push_back(BlockDesc{(int)gi, w0, std::min(wpb, g.W - w0), wpb, P});
    }
    // Longest blocks first: when a launch needs more than one wave of blocks,
    // the blocks of the largest lattices (work per sweep: walkers x sites)
    // start first instead of forming the tail.  Row-scan blocks are grouped
    // by L first (one kernel per row length).
    for (int k = 0; k < kKinds; ++k)
        std::stable_sort(b[k].begin(), b[k].end(), [&](const BlockDesc &x, const BlockDesc &y) {
            const int lx = ctx->g[x.group].L, ly = ctx->g[y.group].L;
            if ((k == 4 || k == 5) && lx != ly) return lx > ly;
            return (int64_t)x.nw * ctx->g[x.group].V > (int64_t)y.nw * ctx->g[y.group].V;
        });
    ctx->bond_ranges.clear();
    for (int i = 0; i < (int)b[5].size(); ++i) {
        const int L = ctx->g[b[5][i].group].L;
        if (ctx->bond_ranges.empty() || ctx->bond_ranges.back().L != L)
            ctx->bond_ranges.push_back({L, i, 0, 0});
        ++ctx->bond_ranges.back().count;
    }
    ctx->scan_ranges.clear();
    for (int i = 0; i < (int)b[4].size(); ++i) {
        const int L = ctx->g[b[4][i].group].L;
        if (ctx->scan_ranges.empty() || ctx->scan_ranges.back().L != L)
            ctx->scan_ranges.push_back({L, i, 0, scan_bytes_for(L)});
        ++ctx->scan_ranges.back().count;
    }
    for (const auto &rg : ctx->scan_ranges) {
        if ((int64_t)rg.smem + 1024 > (int64_t)max_smem_per_block())
            return fail(ctx, MUCA_ERR_INVALID_ARG, "%zu bytes of shared memory per block do not fit",
                        rg.smem);
        CK(prepare_scan_kernel(rg.L, rg.smem));
    }
    while (ctx->scan_streams.size() < ctx->scan_ranges.size()) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        ctx->scan_streams.push_back(s);
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->scan_events.push_back(e);
    }
    for (int k = 0; k < kKinds; ++k) {
        if (sm[k] > 0 && (int64_t)sm[k] + 1024 > (int64_t)max_smem_per_block())
            return fail(ctx, MUCA_ERR_INVALID_ARG, "%zu bytes of shared memory per block do not fit",
                        sm[k]);
        if (!b[k].empty()) {
            if (k == 0) CK(prepare_global_kernel(sm[k]));
            if (k == 1) CK(prepare_smem_kernel(sm[k]));
            if (k == 2 || k == 3) CK(prepare_ws_kernel(sm[k], k == 3));
        }
        if (ctx->d_blocks[k]) cudaFree(ctx->d_blocks[k]);
        ctx->d_blocks[k] = nullptr;
        if (!b[k].empty()) {
            CK(cudaMalloc(&ctx->d_blocks[k], b[k].size() * sizeof(BlockDesc)));
            CK(cudaMemcpy(ctx->d_blocks[k], b[k].data(), b[k].size() * sizeof(BlockDesc),
                          cudaMemcpyHostToDevice));
        }
        ctx->n_blocks[k] = (int)b[k].size();
        ctx->smem[k] = sm[k];
    }
    return MUCA_OK;
}

// The launches of one sweep call: on the caller's stream when one launch is
// in use, otherwise forked over per-launch streams and joined.
int launch_all(muca_ctx *ctx, int n_sweeps, bool record, cudaStream_t st)
{
    int used = (int)ctx->scan_ranges.size();
    for (int k = 0; k < 4; ++k) used += ctx->n_blocks[k] > 0;
    used += ctx->n_blocks[5] > 0;
    const bool fork = used > 1;
    if (fork) CK(cudaEventRecord(ctx->ev_fork, st));
    for (size_t i = 0; i < ctx->scan_ranges.size(); ++i) {
        const auto &rg = ctx->scan_ranges[i];
        cudaStream_t s = fork ? ctx->scan_streams[i] : st;
        if (fork) CK(cudaStreamWaitEvent(s, ctx->ev_fork, 0));
        CK(launch_sweeps_scan(rg.L, ctx->d_groups, ctx->d_blocks[4] + rg.first, rg.count, rg.smem,
                              ctx->seed, ctx->sweep, n_sweeps, ctx->ts_len, record, s));
        if (fork) {
            CK(cudaEventRecord(ctx->scan_events[i], s));
            CK(cudaStreamWaitEvent(st, ctx->scan_events[i], 0));
        }
    }
    for (int k = 0; k < 4; ++k) {
        if (ctx->n_blocks[k] == 0) continue;
        cudaStream_t s = fork ? ctx->side[k] : st;
        if (fork) CK(cudaStreamWaitEvent(s, ctx->ev_fork, 0));
        if (k >= 2)
            CK(launch_sweeps_ws(ctx->d_groups, ctx->d_blocks[k], ctx->n_blocks[k], ctx->smem[k],
                                ctx->seed, ctx->sweep, n_sweeps, ctx->ts_len, record, k == 3, s));
        else
            CK(launch_sweeps(ctx->d_groups, ctx->d_blocks[k], ctx->n_blocks[k], 32, ctx->smem[k],
                             k == 1, ctx->seed, ctx->sweep, n_sweeps, ctx->ts_len, record, s));
        if (fork) {
            CK(cudaEventRecord(ctx->ev_join[k], s));
            CK(cudaStreamWaitEvent(st, ctx->ev_join[k], 0));
        }
    }
    if (ctx->n_blocks[5] > 0) {
        cudaStream_t s = fork ? ctx->side[5] : st;
        if (fork) CK(cudaStreamWaitEvent(s, ctx->ev_fork, 0));
        for (const auto &rg : ctx->bond_ranges)
            CK(launch_sweeps_bonds(rg.L, ctx->d_groups, ctx->d_blocks[5] + rg.first, rg.count,
                                   ctx->seed, ctx->sweep, n_sweeps, ctx->ts_len, record, s));
        if (fork) {
            CK(cudaEventRecord(ctx->ev_join[5], s));
            CK(cudaStreamWaitEvent(st, ctx->ev_join[5], 0));
        }
    }
    return MUCA_OK;
}

int check_group_index(muca_ctx *ctx, int group)
{
    if (!ctx) return fail(nullptr, MUCA_ERR_INVALID_ARG, "null context");
    if (group < 0 || group >= (int)ctx->g.size())
        return fail(ctx, MUCA_ERR_INVALID_ARG, "group %d out of range [0, %d)", group,
                    (int)ctx->g.size());
    return MUCA_OK;
}

int run_tally_check(muca_ctx *ctx)
{
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    for (auto &g : ctx->g) CK(launch_energies(dev_of(g), 1, ctx->d_err, ctx->stream));
    int h = 0;
    CK(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (h) return fail(ctx, MUCA_ERR_TALLY_MISMATCH, "running tallies differ from recomputed");
    return MUCA_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: for MUCA_RES_AUTO / walkers_per_block = 0, time a few sweeps of
// each candidate configuration on a scratch copy of the group's state (the
// real state is restored, so results never depend on the choice) and keep
// the fastest.  Choices are cached per (L, walkers) for the process.
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;

struct Cand {
    int res, wpb, P;
};

// The unrolled row path: L % 4 == 0 up to 48 (see sweep.cu) and a table at
// least as long as the per-walker window.
bool fixed_path(const Group &g)
{
    const bool size_ok = g.L % 4 == 0 && g.L <= 48 && g.L != 36 && g.L != 40 && g.L != 44;
    return size_ok && g.nE + 2 * kGuard >= 32;
}

// Candidate configurations: (residency, walkers per block, lanes per walker).
// A sweep block is one warp: walkers_per_block x lanes_per_walker <= 32.
// Fewer walkers per warp spread the chains over more SM sub-partitions and let
// the extra lanes share the per-row work; the autotuner measures.
std::vector<Cand> candidates(const Group &g, int residency, int wpb, int P, int smem_max)
{
    std::vector<Cand> c;
    const bool want_g = residency == MUCA_RES_AUTO || residency == MUCA_RES_GLOBAL;
    const bool want_s = residency == MUCA_RES_AUTO || residency == MUCA_RES_SMEM;
    const std::vector<int> Ps = !fixed_path(g) ? std::vector<int>{1}
                                : P > 0        ? std::vector<int>{P}
                                               : std::vector<int>{1, 2, 4, 8};
    if (want_g)
        for (int p : Ps) {
            if (wpb > 0) {
                if (wpb * p == 32) c.push_back({MUCA_RES_GLOBAL, wpb, p});
            } else {
                c.push_back({MUCA_RES_GLOBAL, 32 / p, p});
            }
        }
    const bool want_r = residency == MUCA_RES_AUTO || residency == MUCA_RES_SCAN;
    if (want_r && scan_supported(g.L, g.nE)) {
        const int G = scan_block_walkers(g.L), Ps = scan_seg(g.L);
        if ((wpb == 0 || wpb == G) && (P == 0 || P == Ps)) c.push_back({MUCA_RES_SCAN, G, Ps});
    } else if (residency == MUCA_RES_SCAN) {
        // sizes the row-scan kernel does not cover run on the lanes-per-walker kernel
        c.push_back({MUCA_RES_GLOBAL, 32, 1});
    }
    const bool want_w = residency == MUCA_RES_AUTO || residency == MUCA_RES_SPLIT;
    if (want_w && fixed_path(g) && g.L >= 8) {
        for (int G : {32, 16, 8}) {
            if (wpb > 0 && wpb != G) continue;
            if ((int64_t)ws_bytes_for(G) + 1024 <= (int64_t)smem_max)
                c.push_back({MUCA_RES_SPLIT, G, 0});
        }
    } else if (residency == MUCA_RES_SPLIT) {
        // sizes the split kernel does not cover run on the lanes-per-walker kernel
        c.push_back({MUCA_RES_GLOBAL, 32, 1});
    }
    if (want_s) {
        const int64_t per = (int64_t)lattice_bytes(g.L) + (int64_t)stage_bytes_for(1) + 16;
        const int fit = (int)std::min<int64_t>(32, (int64_t)(smem_max - 1024) / per);
        for (int p : Ps) {
            if (wpb > 0) {
                if (wpb <= fit && wpb * p <= 32) c.push_back({MUCA_RES_SMEM, wpb, p});
            } else {
                // fewer than 8 lattices per block leave most of the GPU idle
                const int G = std::min(fit, 32 / p);
                if (G >= 8 || (G >= 1 && G == 32 / p)) c.push_back({MUCA_RES_SMEM, G, p});
            }
        }
    }
    return c;
}

// choices of the autotuner per (L, walkers, requested residency, walkers per
// block, lanes per walker)
std::map<std::tuple<int, int, int, int, int>, Cand> g_tune_cache;

}  // namespace

static int tune_group(muca_ctx *ctx, size_t gi, int residency, int wpb, int P)
{
    Group &g = ctx->g[gi];
    const int smem_max = max_smem_per_block();
    std::vector<Cand> cands = candidates(g, residency, wpb, P, smem_max);
    if (cands.empty())
        return fail(ctx, MUCA_ERR_INVALID_ARG,
                    "no kernel configuration fits group %d (L=%d, residency %d, walkers per block "
                    "%d, lanes per walker %d)",
                    (int)gi, g.L, residency, wpb, P);
    // a group outside its window cannot be swept yet: take the first candidate
    if (cands.size() == 1 || !g.in_window) {
        g.residency = cands[0].res;
        g.wpb = cands[0].wpb;
        g.P = cands[0].P;
        return MUCA_OK;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(std::make_tuple(g.L, g.W, residency, wpb, P));
        if (it != g_tune_cache.end()) {
            g.residency = it->second.res;
            g.wpb = it->second.wpb;
            g.P = it->second.P;
            return MUCA_OK;
        }
    }
    // scratch copy of the state
    const size_t sb = (size_t)g.L * g.L * g.Lw * g.Wpad * sizeof(uint32_t), tb = (size_t)3 * g.Wpad * sizeof(int32_t),
                 hb = (size_t)g.nE * sizeof(unsigned long long);
    uint32_t *s0 = nullptr;
    int32_t *t0 = nullptr;
    unsigned long long *h0 = nullptr;
    CK(cudaMalloc(&s0, sb));
    CK(cudaMalloc(&t0, tb));
    CK(cudaMalloc(&h0, hb));
    CK(cudaMemcpyAsync(s0, g.spins, sb, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(t0, g.tal, tb, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(h0, g.hist, hb, cudaMemcpyDeviceToDevice, ctx->stream));
    // a one-group context view for the trial launches
    std::vector<Group> saved_groups;
    saved_groups.swap(ctx->g);
    ctx->g.push_back(saved_groups[gi]);
    GroupDev *saved_dg = ctx->d_groups;
    GroupDev *dg = nullptr;
    CK(cudaMalloc(&dg, sizeof(GroupDev)));
    ctx->d_groups = dg;
    int rc = upload_groups(ctx);
    // Trials start from a relaxed copy: the sweeps right after a random start
    // move E_Delta much faster than a running simulation does, and the
    // row-scan kernel's cost grows with the moves that change E_Delta, so a
    // short relaxation would favour the kernels whose cost does not (at
    // L = 48 it is slower than the split kernel after 37 sweeps and faster
    // after 150).  The relaxation runs on a row-scan or split candidate when
    // there is one.
    const int relax_sweeps = std::max(4, std::min(300, (1 << 25) / std::max(1, g.V)));
    const int trial_sweeps = std::max(2, std::min(8, (1 << 18) / std::max(1, g.V)));
    Cand relax_c = cands[0];
    for (const Cand &c : cands)
        if (c.res == MUCA_RES_SCAN || (c.res == MUCA_RES_SPLIT && relax_c.res != MUCA_RES_SCAN))
            relax_c = c;
    if (rc == MUCA_OK) {
        ctx->g[0].residency = relax_c.res;
        ctx->g[0].wpb = relax_c.wpb;
        ctx->g[0].P = relax_c.P;
        rc = build_blocks(ctx);
    }
    if (rc == MUCA_OK) rc = launch_all(ctx, relax_sweeps, false, ctx->stream);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    Cand pick = cands[0];
    for (const Cand &c : cands) {
        if (rc != MUCA_OK) break;
        ctx->g[0].residency = c.res;
        ctx->g[0].wpb = c.wpb;
        ctx->g[0].P = c.P;
        rc = build_blocks(ctx);
        if (rc != MUCA_OK) break;
        rc = launch_all(ctx, 1, false, ctx->stream);  // warm-up
        cudaEventRecord(a, ctx->stream);
        if (rc == MUCA_OK) rc = launch_all(ctx, trial_sweeps, false, ctx->stream);
        cudaEventRecord(b, ctx->stream);
        if (cudaEventSynchronize(b) != cudaSuccess) rc = MUCA_ERR_CUDA;
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (rc == MUCA_OK && ms < best) {
            best = ms;
            pick = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->g.swap(saved_groups);
    ctx->d_groups = saved_dg;
    cudaFree(dg);
    // restore the state
    cudaMemcpyAsync(g.spins, s0, sb, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(g.tal, t0, tb, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(g.hist, h0, hb, cudaMemcpyDeviceToDevice, ctx->stream);
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(s0);
    cudaFree(t0);
    cudaFree(h0);
    if (rc != MUCA_OK) return rc;
    g.residency = pick.res;
    g.wpb = pick.wpb;
    g.P = pick.P;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[std::make_tuple(g.L, g.W, residency, wpb, P)] = pick;
    return MUCA_OK;
}

// Joint choice for a context of several groups.  All groups' blocks of one
// kernel kind share a launch, and a launch gives every block the largest
// shared-memory size among them, so choices made one group at a time can
// leave an SM holding one block where it could hold two.  Times the whole
// batch with the per-group choices and with one common walkers-per-block for
// the split-kernel groups, on a relaxed copy of the state, and keeps the
// fastest.  The state is restored afterwards.
static int tune_batch(muca_ctx *ctx)
{
    const size_t n = ctx->g.size();
    std::vector<size_t> split;
    for (size_t i = 0; i < n; ++i)
        if (ctx->g[i].residency == MUCA_RES_SPLIT) split.push_back(i);
    if (split.size() < 2) return MUCA_OK;
    struct Backup {
        uint32_t *s = nullptr;
        int32_t *t = nullptr;
        unsigned long long *h = nullptr;
        size_t sb = 0, tb = 0, hb = 0;
    };
    std::vector<Backup> bk(n);
    int rc = MUCA_OK;
    for (size_t i = 0; i < n && rc == MUCA_OK; ++i) {
        const Group &g = ctx->g[i];
        Backup &b = bk[i];
        b.sb = (size_t)g.L * g.L * g.Lw * g.Wpad * sizeof(uint32_t);
        b.tb = (size_t)3 * g.Wpad * sizeof(int32_t);
        b.hb = (size_t)g.nE * sizeof(unsigned long long);
        if (cudaMalloc(&b.s, b.sb) != cudaSuccess || cudaMalloc(&b.t, b.tb) != cudaSuccess ||
            cudaMalloc(&b.h, b.hb) != cudaSuccess ||
            cudaMemcpyAsync(b.s, g.spins, b.sb, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(b.t, g.tal, b.tb, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(b.h, g.hist, b.hb, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
            rc = fail(ctx, MUCA_ERR_CUDA, "batch tuning: backup of the state failed");
    }
    std::vector<int> tuned(n);
    for (size_t i = 0; i < n; ++i) tuned[i] = ctx->g[i].wpb;
    const int smem_max = max_smem_per_block();
    auto apply = [&](int G) {
        for (size_t i : split) ctx->g[i].wpb = G ? G : tuned[i];
    };
    int best_G = 0;
    if (rc == MUCA_OK) {
        apply(0);
        rc = build_blocks(ctx);
        if (rc == MUCA_OK) rc = launch_all(ctx, 32, false, ctx->stream);  // relax the copy
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int G : {0, 32, 16, 8}) {
        if (rc != MUCA_OK) break;
        if (G && (int64_t)ws_bytes_for(G) + 1024 > (int64_t)smem_max) continue;
        apply(G);
        rc = build_blocks(ctx);
        if (rc == MUCA_OK) rc = launch_all(ctx, 1, false, ctx->stream);
        cudaEventRecord(a, ctx->stream);
        if (rc == MUCA_OK) rc = launch_all(ctx, 4, false, ctx->stream);
        cudaEventRecord(b, ctx->stream);
        if (cudaEventSynchronize(b) != cudaSuccess) rc = MUCA_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rc == MUCA_OK && ms < best) {
            best = ms;
            best_G = G;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    apply(best_G);
    for (size_t i = 0; i < n; ++i) {
        const Group &g = ctx->g[i];
        const Backup &k = bk[i];
        if (k.s) cudaMemcpyAsync(g.spins, k.s, k.sb, cudaMemcpyDeviceToDevice, ctx->stream);
        if (k.t) cudaMemcpyAsync(g.tal, k.t, k.tb, cudaMemcpyDeviceToDevice, ctx->stream);
        if (k.h) cudaMemcpyAsync(g.hist, k.h, k.hb, cudaMemcpyDeviceToDevice, ctx->stream);
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && rc == MUCA_OK)
        rc = fail(ctx, MUCA_ERR_CUDA, "batch tuning: restoring the state failed");
    for (Backup &k : bk) {
        cudaFree(k.s);
        cudaFree(k.t);
        cudaFree(k.h);
    }
    return rc;
}

static void free_group(Group &g)
{
    cudaFree(g.spins);
    cudaFree(g.tal);
    cudaFree(g.hist);
    cudaFree(g.thr);
    cudaFree(g.ts);
    cudaFreeHost(g.h_thr);
    cudaFreeHost(g.h_hist);
    cudaFree(g.d_J);
    cudaFree(g.d_J6);
    cudaFree(g.thrJ);
    cudaFreeHost(g.h_thrJ);
    g.d_J = nullptr;
    g.d_J6 = nullptr;
    g.thrJ = nullptr;
    g.h_thrJ = nullptr;
    g.jmax = 0;
    g.spins = nullptr;
    g.tal = nullptr;
    g.hist = nullptr;
    g.thr = nullptr;
    g.ts = nullptr;
    g.h_thr = nullptr;
    g.h_hist = nullptr;
}

namespace muca {
void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace muca

extern "C" {

const char *muca_last_error(const muca_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_last_error.c_str();
}

void muca_destroy(muca_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &g : ctx->g) free_group(g);
    cudaFree(ctx->d_err);
    cudaFree(ctx->d_groups);
    for (int k = 0; k < kKinds; ++k) {
        if (ctx->side[k]) cudaStreamDestroy(ctx->side[k]);
        if (ctx->ev_join[k]) cudaEventDestroy(ctx->ev_join[k]);
        cudaFree(ctx->d_blocks[k]);
    }
    for (auto s : ctx->scan_streams) cudaStreamDestroy(s);
    for (auto e : ctx->scan_events) cudaEventDestroy(e);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    delete ctx;
}

int muca_init(const muca_group *groups, int n_groups, const muca_options *opt, void *stream,
              muca_ctx **out)
{
    muca_ctx *ctx = nullptr;
    if (!out) return fail(nullptr, MUCA_ERR_INVALID_ARG, "muca_init: out is NULL");
    *out = nullptr;
    if (!groups || n_groups < 1 || !opt)
        return fail(nullptr, MUCA_ERR_INVALID_ARG, "muca_init: need >= 1 group and options");
    if (opt->residency < MUCA_RES_AUTO || opt->residency > MUCA_RES_SCAN)
        return fail(nullptr, MUCA_ERR_INVALID_ARG, "muca_init: bad residency %d", opt->residency);
    if (opt->walkers_per_block < 0 || opt->walkers_per_block > 32)
        return fail(nullptr, MUCA_ERR_INVALID_ARG, "muca_init: bad walkers_per_block %d",
                    opt->walkers_per_block);
    if (opt->lanes_per_walker != 0 && opt->lanes_per_walker != 1 && opt->lanes_per_walker != 2 &&
        opt->lanes_per_walker != 4 && opt->lanes_per_walker != 8 && opt->lanes_per_walker != 16)
        return fail(nullptr, MUCA_ERR_INVALID_ARG, "muca_init: bad lanes_per_walker %d",
                    opt->lanes_per_walker);
    const int shards = opt->shard_count > 1 ? opt->shard_count : 1;
    const int srank = opt->shard_count > 1 ? opt->shard_rank : 0;
    if (opt->shard_count < 0 || opt->shard_rank < 0 || (opt->shard_count <= 1 && opt->shard_rank) ||
        srank >= shards)
        return fail(nullptr, MUCA_ERR_INVALID_ARG, "muca_init: bad shard %d of %d",
                    opt->shard_rank, opt->shard_count);
    int64_t total_w = 0;
    for (int i = 0; i < n_groups; ++i) {
        const muca_group &s = groups[i];
        if (s.L < 2 || s.L > MUCA_MAX_L)
            return fail(nullptr, MUCA_ERR_INVALID_ARG, "group %d: L=%d outside [2, %d]", i, s.L,
                        MUCA_MAX_L);
        if (!(s.T > 0.0) || !std::isfinite(s.T))
            return fail(nullptr, MUCA_ERR_INVALID_ARG, "group %d: T must be > 0", i);
        if (s.n_walkers < 1)
            return fail(nullptr, MUCA_ERR_INVALID_ARG, "group %d: n_walkers < 1", i);
        if ((int64_t)s.n_walkers * (srank + 1) / shards - (int64_t)s.n_walkers * srank / shards < 1)
            return fail(nullptr, MUCA_ERR_INVALID_ARG,
                        "group %d: %d walkers leave shard %d of %d empty", i, s.n_walkers, srank,
                        shards);
        const int V = s.L * s.L * s.L;
        const int emax = s.e_max < 0 ? V : s.e_max;
        if (s.e_min < 0 || emax > V || s.e_min > emax)
            return fail(nullptr, MUCA_ERR_INVALID_ARG, "group %d: window [%d, %d] not in [0, %d]",
                        i, s.e_min, emax, V);
        total_w += s.n_walkers;
    }
    if (total_w > 0x7FFFFFFF)
        return fail(nullptr, MUCA_ERR_INVALID_ARG, "too many walkers");
    ctx = new muca_ctx();
    ctx->seed = opt->seed;
    ctx->debug = opt->debug_flags;
    ctx->stream = (cudaStream_t)stream;
    int rc = MUCA_OK;
#define CKI(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            rc = fail(ctx, e_ == cudaErrorMemoryAllocation ? MUCA_ERR_OOM : MUCA_ERR_CUDA, \
                      "%s: %s", #call, cudaGetErrorString(e_));                            \
            goto bad;                                                                      \
        }                                                                                  \
    } while (0)
    {
        for (int k = 0; k < kKinds; ++k) {
            CKI(cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking));
            CKI(cudaEventCreateWithFlags(&ctx->ev_join[k], cudaEventDisableTiming));
        }
        CKI(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
        CKI(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
        CKI(cudaMalloc(&ctx->d_err, sizeof(int)));
        CKI(cudaMalloc(&ctx->d_groups, n_groups * sizeof(GroupDev)));
        uint32_t w0 = 0;
        ctx->g.resize(n_groups);
        for (int i = 0; i < n_groups; ++i) {
            Group &g = ctx->g[i];
            g.spec = groups[i];
            g.L = groups[i].L;
            g.V = g.L * g.L * g.L;
            // this context's shard of the group's walkers, numbered as in the
            // unsharded context
            const int64_t tot = groups[i].n_walkers;
            const int64_t lo = tot * srank / shards, hi = tot * (srank + 1) / shards;
            g.W = (int)(hi - lo);
            g.Wpad = ((g.W + 31) / 32) * 32;
            g.Lw = (g.L + 3) / 4;
            g.e_min = groups[i].e_min;
            g.e_max = groups[i].e_max < 0 ? g.V : groups[i].e_max;
            g.spec.e_max = g.e_max;
            g.nE = g.e_max - g.e_min + 1;
            g.win_lo = 0;
            g.win_hi = g.nE - 1;
            g.T = groups[i].T;
            g.beta = 1.0 / g.T;
            g.walker0 = w0 + (uint32_t)lo;
            w0 += (uint32_t)tot;
            g.lnW.assign(g.nE, 0.0);
            g.acc.assign((size_t)std::max(g.nE - 1, 1), 0.0);
            const size_t sbytes = (size_t)g.L * g.L * g.Lw * g.Wpad * sizeof(uint32_t);
            CKI(cudaMalloc(&g.spins, sbytes));
            CKI(cudaMemsetAsync(g.spins, 0, sbytes, ctx->stream));
            CKI(cudaMalloc(&g.tal, (size_t)3 * g.Wpad * sizeof(int32_t)));
            CKI(cudaMemsetAsync(g.tal, 0, (size_t)3 * g.Wpad * sizeof(int32_t), ctx->stream));
            CKI(cudaMalloc(&g.hist, (size_t)g.nE * sizeof(unsigned long long)));
            CKI(cudaMemsetAsync(g.hist, 0, (size_t)g.nE * sizeof(unsigned long long), ctx->stream));
            CKI(cudaMalloc(&g.thr, table_rows(g.nE) * kRow * sizeof(uint32_t)));
            CKI(cudaMallocHost(&g.h_thr, table_rows(g.nE) * kRow * sizeof(uint32_t)));
            CKI(cudaMallocHost(&g.h_hist, (size_t)g.nE * sizeof(unsigned long long)));
            CKI(launch_init_spins(dev_of(g), ctx->seed, ctx->stream));
            CKI(launch_energies(dev_of(g), 0, ctx->d_err, ctx->stream));
            build_packed(g);
            if ((rc = upload_table(ctx, g)) != MUCA_OK) goto bad;
        }
        if ((rc = upload_groups(ctx)) != MUCA_OK) goto bad;
        CKI(cudaStreamSynchronize(ctx->stream));
        // a group whose initial E_Delta values leave its window must get a
        // state through muca_set_state before it can be swept
        for (int i = 0; i < n_groups; ++i) {
            Group &g = ctx->g[i];
            std::vector<int32_t> ed(g.W);
            CKI(cudaMemcpy(ed.data(), g.tal + g.Wpad, g.W * sizeof(int32_t),
                           cudaMemcpyDeviceToHost));
            g.in_window = true;
            for (int w = 0; w < g.W; ++w)
                if (ed[w] < g.e_min || ed[w] > g.e_max) g.in_window = false;
        }
        for (int i = 0; i < n_groups; ++i)
            if ((rc = tune_group(ctx, i, opt->residency, opt->walkers_per_block,
                                 opt->lanes_per_walker)) != MUCA_OK)
                goto bad;
        if (n_groups > 1 && opt->residency == MUCA_RES_AUTO && opt->walkers_per_block == 0) {
            bool all_in = true;
            for (int i = 0; i < n_groups; ++i) all_in = all_in && ctx->g[i].in_window;
            if (all_in && (rc = tune_batch(ctx)) != MUCA_OK) goto bad;
        }
        if ((rc = build_blocks(ctx)) != MUCA_OK) goto bad;
        CKI(cudaStreamSynchronize(ctx->stream));
    }
#undef CKI
    *out = ctx;
    return MUCA_OK;
bad:
    g_last_error = ctx->err;
    muca_destroy(ctx);
    return rc;
}

int muca_sync(muca_ctx *ctx)
{
    if (!ctx) return fail(nullptr, MUCA_ERR_INVALID_ARG, "null context");
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCA_OK;
}

int muca_sweep_iter(muca_ctx *ctx, int n_sweeps, int record)
{
    if (!ctx) return fail(nullptr, MUCA_ERR_INVALID_ARG, "null context");
    if (n_sweeps < 0) return fail(ctx, MUCA_ERR_INVALID_ARG, "n_sweeps < 0");
    if (n_sweeps == 0) return MUCA_OK;
    for (size_t i = 0; i < ctx->g.size(); ++i)
        if (!ctx->g[i].in_window)
            return fail(ctx, MUCA_ERR_WINDOW,
                        "group %d has walkers outside its E_Delta window: set a state first",
                        (int)i);
    if (record && ctx->ts_len + n_sweeps > ctx->ts_cap)
        return fail(ctx, MUCA_ERR_INVALID_ARG,
                    "time series full: %lld recorded + %d > capacity %lld (muca_reserve_timeseries)",
                    (long long)ctx->ts_len, n_sweeps, (long long)ctx->ts_cap);
    int rc = launch_all(ctx, n_sweeps, record != 0, ctx->stream);
    if (rc != MUCA_OK) return rc;
    ctx->sweep += (uint64_t)n_sweeps;
    if (record) ctx->ts_len += n_sweeps;
    if (ctx->debug & MUCA_DEBUG_TALLY_CHECK) return run_tally_check(ctx);
    return MUCA_OK;
}

int muca_merge_update(muca_ctx *ctx)
{
    if (!ctx) return fail(nullptr, MUCA_ERR_INVALID_ARG, "null context");
    for (auto &g : ctx->g)
        CK(cudaMemcpyAsync(g.h_hist, g.hist, (size_t)g.nE * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (auto &g : ctx->g) {
        update_lnW(g);
        g.injected.clear();
        build_packed(g);
        int rc = upload_table(ctx, g);
        if (rc != MUCA_OK) return rc;
        CK(cudaMemsetAsync(g.hist, 0, (size_t)g.nE * sizeof(unsigned long long), ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCA_OK;
}

int muca_weight_update(int32_t kind, int32_t n_e, const uint64_t *hist, double *lnW, double *acc)
{
    if (kind != MUCA_REC_PLAIN && kind != MUCA_REC_ACCUMULATED)
        return fail(nullptr, MUCA_ERR_INVALID_ARG, "unknown weight recursion %d", kind);
    if (n_e < 1 || !hist || !lnW || (kind == MUCA_REC_ACCUMULATED && n_e > 1 && !acc))
        return fail(nullptr, MUCA_ERR_INVALID_ARG, "weight update: n_e < 1 or a NULL array");
    static_assert(sizeof(uint64_t) == sizeof(unsigned long long), "64-bit histogram counts");
    weight_update(kind, n_e, reinterpret_cast<const unsigned long long *>(hist), lnW, acc);
    return MUCA_OK;
}

int muca_set_recursion(muca_ctx *ctx, int32_t kind)
{
    if (!ctx) return fail(nullptr, MUCA_ERR_INVALID_ARG, "null context");
    if (kind != MUCA_REC_PLAIN && kind != MUCA_REC_ACCUMULATED)
        return fail(ctx, MUCA_ERR_INVALID_ARG, "unknown weight recursion %d", kind);
    CK(cudaStreamSynchronize(ctx->stream));  // a graph's host node may still update
    for (auto &g : ctx->g) {
        g.recursion = kind;
        std::fill(g.acc.begin(), g.acc.end(), 0.0);
    }
    return MUCA_OK;
}

int muca_get_flatness(muca_ctx *ctx, int group, double *out)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!out) return fail(ctx, MUCA_ERR_INVALID_ARG, "out is NULL");
    CK(cudaStreamSynchronize(ctx->stream));
    const Group &g = ctx->g[group];
    for (int k = 0; k < 3; ++k) out[k] = g.flat[k];
    return MUCA_OK;
}

int muca_set_window(muca_ctx *ctx, int group, int32_t lo, int32_t hi, double grow_flat,
                    int32_t grow_step)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    Group &g = ctx->g[group];
    if (lo < g.e_min || hi > g.e_max || lo > hi)
        return fail(ctx, MUCA_ERR_INVALID_ARG, "set_window: [%d, %d] not inside [%d, %d]", lo, hi,
                    g.e_min, g.e_max);
    if (!(grow_flat >= 0.0) || !std::isfinite(grow_flat) || (grow_flat > 0.0 && grow_step < 1))
        return fail(ctx, MUCA_ERR_INVALID_ARG, "set_window: grow_flat %g, grow_step %d", grow_flat,
                    grow_step);
    std::vector<int32_t> t((size_t)3 * g.Wpad);
    CK(cudaStreamSynchronize(ctx->stream));  // a graph's host node may still update
    CK(cudaMemcpy(t.data(), g.tal, t.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int w = 0; w < g.W; ++w) {
        const int ed = t[(size_t)g.Wpad + w];
        if (ed < lo || ed > hi)
            return fail(ctx, MUCA_ERR_WINDOW, "set_window: walker %d has E_Delta=%d outside [%d, %d]",
                        w, ed, lo, hi);
    }
    g.win_lo = lo - g.e_min;
    g.win_hi = hi - g.e_min;
    g.grow_flat = grow_flat;
    g.grow_step = grow_flat > 0.0 ? grow_step : 0;
    g.in_window = true;
    g.injected.clear();
    build_packed(g);
    rc = upload_table(ctx, g);
    if (rc != MUCA_OK) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCA_OK;
}

int muca_get_window(muca_ctx *ctx, int group, int32_t *out)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!out) return fail(ctx, MUCA_ERR_INVALID_ARG, "out is NULL");
    CK(cudaStreamSynchronize(ctx->stream));
    const Group &g = ctx->g[group];
    out[0] = g.e_min + g.win_lo;
    out[1] = g.e_min + g.win_hi;
    return MUCA_OK;
}

}  // extern "C"

namespace {

// Give group g the couplings J (host int8 [V][3]) with table width jmax, or
// take them away (J == nullptr): device copies, the table, the kernel kind;
// the tallies are recomputed from the current spins when `retally`.
int apply_bonds(muca_ctx *ctx, int group, const int8_t *J, int jmax, bool retally)
{
    Group &g = ctx->g[group];
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(g.d_J);
    cudaFree(g.d_J6);
    cudaFree(g.thrJ);
    cudaFreeHost(g.h_thrJ);
    g.d_J = nullptr;
    g.d_J6 = nullptr;
    g.thrJ = nullptr;
    g.h_thrJ = nullptr;
    g.jmax = 0;
    g.J.clear();
    if (J) {
        g.jmax = jmax;
        g.J.assign(J, J + (size_t)3 * g.V);
        CK(cudaMalloc(&g.d_J, (size_t)3 * g.V));
        CK(cudaMemcpy(g.d_J, J, (size_t)3 * g.V, cudaMemcpyHostToDevice));
        // the per-site pack: byte 2 mu + 0 the forward bond of the site, byte
        // 2 mu + 1 the forward bond of its backward neighbour in direction mu
        std::vector<unsigned long long> j6((size_t)g.V, 0ull);
        const int L = g.L;
        for (int z = 0; z < L; ++z)
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) {
                    const int i = x + L * (y + L * z);
                    const int back[3] = {(x + L - 1) % L + L * (y + L * z),
                                         x + L * ((y + L - 1) % L + L * z),
                                         x + L * (y + L * ((z + L - 1) % L))};
                    unsigned long long w = 0ull;
                    for (int mu = 0; mu < 3; ++mu) {
                        w |= (unsigned long long)(uint8_t)J[3 * i + mu] << (16 * mu);
                        w |= (unsigned long long)(uint8_t)J[3 * back[mu] + mu] << (16 * mu + 8);
                    }
                    j6[(size_t)i] = w;
                }
        CK(cudaMalloc(&g.d_J6, j6.size() * sizeof(unsigned long long)));
        CK(cudaMemcpy(g.d_J6, j6.data(), j6.size() * sizeof(unsigned long long),
                      cudaMemcpyHostToDevice));
        CK(cudaMalloc(&g.thrJ, bonds_table_words(g) * sizeof(uint32_t)));
        CK(cudaMallocHost(&g.h_thrJ, bonds_table_words(g) * sizeof(uint32_t)));
    }
    g.injected.clear();
    int rc = upload_groups(ctx);
    if (rc != MUCA_OK) return rc;
    rc = build_blocks(ctx);
    if (rc != MUCA_OK) return rc;
    if (retally) CK(launch_energies(dev_of(g), 0, ctx->d_err, ctx->stream));
    build_packed(g);
    rc = upload_table(ctx, g);
    if (rc != MUCA_OK) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCA_OK;
}

int check_bonds(muca_ctx *ctx, const Group &g, const int8_t *J, int jmax)
{
    if (jmax < 1 || jmax > MUCA_MAX_JMAX)
        return fail(ctx, MUCA_ERR_INVALID_ARG, "set_bonds: jmax %d outside [1, %d]", jmax,
                    MUCA_MAX_JMAX);
    for (size_t k = 0; k < (size_t)3 * g.V; ++k)
        if (J[k] < -jmax || J[k] > jmax)
            return fail(ctx, MUCA_ERR_INVALID_ARG, "set_bonds: coupling %d of bond %zu outside "
                        "[-%d, %d]", (int)J[k], k, jmax, jmax);
    return MUCA_OK;
}

}  // namespace

extern "C" {

int muca_set_bonds(muca_ctx *ctx, int group, const int8_t *J, int32_t jmax)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (J) {
        rc = check_bonds(ctx, ctx->g[group], J, jmax);
        if (rc) return rc;
    }
    return apply_bonds(ctx, group, J, J ? jmax : 0, true);
}

int muca_iterate(muca_ctx *ctx, int32_t max_iters, int32_t sweeps_per_iter, double flat_min,
                 int32_t *n_done)
{
    if (!ctx) return fail(nullptr, MUCA_ERR_INVALID_ARG, "null context");
    if (!n_done) return fail(ctx, MUCA_ERR_INVALID_ARG, "n_done is NULL");
    *n_done = 0;
    if (max_iters < 0 || sweeps_per_iter < 1 || !std::isfinite(flat_min))
        return fail(ctx, MUCA_ERR_INVALID_ARG,
                    "iterate: max_iters %d, sweeps_per_iter %d, flat_min %g", max_iters,
                    sweeps_per_iter, flat_min);
    for (int it = 0; it < max_iters; ++it) {
        int rc = muca_sweep_iter(ctx, sweeps_per_iter, 0);
        if (rc != MUCA_OK) return rc;
        rc = muca_merge_update(ctx);
        if (rc != MUCA_OK) return rc;
        *n_done = it + 1;
        bool flat = true;
        for (const auto &g : ctx->g) flat = flat && g.flat[0] >= flat_min && g.flat_full;
        if (flat) break;
    }
    return MUCA_OK;
}

}  // extern "C"

namespace {

struct HostUpdateArg {
    Group *g;
};

void CUDART_CB host_update(void *p)
{
    Group &g = *static_cast<Group *>(p);
    update_lnW(g);
    g.injected.clear();
    build_packed(g);
}

}  // namespace

extern "C" int muca_run_graph(muca_ctx *ctx, int n_iters, int sweeps_per_iter)
{
    if (!ctx) return fail(nullptr, MUCA_ERR_INVALID_ARG, "null context");
    if (n_iters < 0 || sweeps_per_iter < 0)
        return fail(ctx, MUCA_ERR_INVALID_ARG, "negative n_iters or sweeps_per_iter");
    if (n_iters == 0) return MUCA_OK;
    for (size_t i = 0; i < ctx->g.size(); ++i)
        if (!ctx->g[i].in_window)
            return fail(ctx, MUCA_ERR_WINDOW,
                        "group %d has walkers outside its E_Delta window: set a state first",
                        (int)i);
    CK(cudaStreamSynchronize(ctx->stream));
    // captured on the context's own non-blocking stream (the caller's stream
    // may be the legacy default stream, which cannot be captured), launched on
    // the caller's stream
    cudaStream_t cs = ctx->cap;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const uint64_t sweep_start = ctx->sweep;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = MUCA_OK;
    for (int it = 0; it < n_iters && rc == MUCA_OK; ++it) {
        rc = launch_all(ctx, sweeps_per_iter, false, cs);
        ctx->sweep += (uint64_t)sweeps_per_iter;
        for (auto &g : ctx->g) {
            if (rc != MUCA_OK) break;
            if (cudaMemcpyAsync(g.h_hist, g.hist, (size_t)g.nE * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
                cudaLaunchHostFunc(cs, host_update, &g) != cudaSuccess ||
                cudaMemcpyAsync(table_dev(g), table_host(g), table_bytes(g),
                                cudaMemcpyHostToDevice, cs) != cudaSuccess ||
                cudaMemsetAsync(g.hist, 0, (size_t)g.nE * sizeof(unsigned long long), cs) !=
                    cudaSuccess)
                rc = fail(ctx, MUCA_ERR_CUDA, "graph capture of the merge failed");
        }
    }
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (rc == MUCA_OK && ce != cudaSuccess)
        rc = fail(ctx, MUCA_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ce));
    if (rc == MUCA_OK) {
        ce = cudaGraphInstantiate(&exec, graph, 0);
        if (ce != cudaSuccess)
            rc = fail(ctx, MUCA_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ce));
    }
    if (rc == MUCA_OK) {
        ce = cudaGraphLaunch(exec, ctx->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
        if (ce != cudaSuccess)
            rc = fail(ctx, MUCA_ERR_CUDA, "graph launch: %s", cudaGetErrorString(ce));
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (rc != MUCA_OK) ctx->sweep = sweep_start;
    return rc;
}

extern "C" {

int muca_reserve_timeseries(muca_ctx *ctx, int64_t n_samples)
{
    if (!ctx) return fail(nullptr, MUCA_ERR_INVALID_ARG, "null context");
    if (n_samples < 0) return fail(ctx, MUCA_ERR_INVALID_ARG, "n_samples < 0");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->ts_len = 0;
    if (n_samples == ctx->ts_cap) return MUCA_OK;  // same capacity: only rewind
    for (auto &g : ctx->g) {
        cudaFree(g.ts);
        g.ts = nullptr;
    }
    ctx->ts_cap = 0;
    for (auto &g : ctx->g)
        if (n_samples > 0) CK(cudaMalloc(&g.ts, (size_t)n_samples * 3 * g.W * sizeof(int32_t)));
    ctx->ts_cap = n_samples;
    return upload_groups(ctx);
}

int muca_timeseries_device(muca_ctx *ctx, int group, const int32_t **dev, int64_t *n_samples)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (dev) *dev = ctx->g[group].ts;
    if (n_samples) *n_samples = ctx->ts_len;
    return MUCA_OK;
}

int muca_get_timeseries(muca_ctx *ctx, int group, int32_t *out)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!out) return fail(ctx, MUCA_ERR_INVALID_ARG, "out is NULL");
    Group &g = ctx->g[group];
    if (ctx->ts_len > 0)
        CK(cudaMemcpyAsync(out, g.ts, (size_t)ctx->ts_len * 3 * g.W * sizeof(int32_t),
                           cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCA_OK;
}

int muca_get_sweep_count(muca_ctx *ctx, int group, uint64_t *out)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!out) return fail(ctx, MUCA_ERR_INVALID_ARG, "out is NULL");
    *out = ctx->sweep;
    return MUCA_OK;
}

int muca_get_lnW(muca_ctx *ctx, int group, double *out)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!out) return fail(ctx, MUCA_ERR_INVALID_ARG, "out is NULL");
    const Group &g = ctx->g[group];
    std::memcpy(out, g.lnW.data(), g.nE * sizeof(double));
    return MUCA_OK;
}

int muca_set_lnW(muca_ctx *ctx, int group, const double *in)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!in) return fail(ctx, MUCA_ERR_INVALID_ARG, "in is NULL");
    Group &g = ctx->g[group];
    for (int e = 0; e < g.nE; ++e)
        if (!std::isfinite(in[e])) return fail(ctx, MUCA_ERR_INVALID_ARG, "lnW[%d] not finite", e);
    CK(cudaStreamSynchronize(ctx->stream));  // the pinned table may still be in flight
    std::memcpy(g.lnW.data(), in, g.nE * sizeof(double));
    std::fill(g.acc.begin(), g.acc.end(), 0.0);
    g.injected.clear();
    build_packed(g);
    rc = upload_table(ctx, g);
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCA_OK;
}

int muca_get_table(muca_ctx *ctx, int group, uint32_t *out)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!out) return fail(ctx, MUCA_ERR_INVALID_ARG, "out is NULL");
    const Group &g = ctx->g[group];
    if (g.jmax)
        return fail(ctx, MUCA_ERR_INVALID_ARG,
                    "get_table: group %d has couplings per bond (its table is muca_build_table_bonds')",
                    group);
    if (!g.injected.empty()) {
        std::memcpy(out, g.injected.data(), g.injected.size() * sizeof(uint32_t));
        return MUCA_OK;
    }
    for (int e = 0; e < g.nE; ++e)
        for (int d = -1; d <= 1; ++d)
            for (int dej = -12; dej <= 12; ++dej)
                out[((size_t)e * 3 + (d + 1)) * MUCA_NK + (dej + 12)] = thr_entry(g, e, d, dej);
    return MUCA_OK;
}

int muca_set_table(muca_ctx *ctx, int group, const uint32_t *in)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!in) return fail(ctx, MUCA_ERR_INVALID_ARG, "in is NULL");
    Group &g = ctx->g[group];
    if (g.jmax)
        return fail(ctx, MUCA_ERR_INVALID_ARG, "set_table: group %d has couplings per bond", group);
    CK(cudaStreamSynchronize(ctx->stream));
    rc = pack_logical(ctx, g, in);
    if (rc) return rc;
    g.injected.assign(in, in + (size_t)g.nE * 3 * MUCA_NK);
    rc = upload_table(ctx, g);
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCA_OK;
}

int muca_get_hist(muca_ctx *ctx, int group, uint64_t *out)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!out) return fail(ctx, MUCA_ERR_INVALID_ARG, "out is NULL");
    Group &g = ctx->g[group];
    CK(cudaMemcpyAsync(out, g.hist, (size_t)g.nE * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCA_OK;
}

int muca_set_hist(muca_ctx *ctx, int group, const uint64_t *in)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!in) return fail(ctx, MUCA_ERR_INVALID_ARG, "in is NULL");
    Group &g = ctx->g[group];
    CK(cudaMemcpyAsync(g.hist, in, (size_t)g.nE * sizeof(uint64_t), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCA_OK;
}

int muca_get_hist_device(muca_ctx *ctx, int group, uint64_t *dev_out)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!dev_out) return fail(ctx, MUCA_ERR_INVALID_ARG, "dev_out is NULL");
    Group &g = ctx->g[group];
    CK(cudaMemcpyAsync(dev_out, g.hist, (size_t)g.nE * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCA_OK;
}

int muca_set_hist_device(muca_ctx *ctx, int group, const uint64_t *dev_in)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!dev_in) return fail(ctx, MUCA_ERR_INVALID_ARG, "dev_in is NULL");
    Group &g = ctx->g[group];
    CK(cudaMemcpyAsync(g.hist, dev_in, (size_t)g.nE * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                       ctx->stream));
    return MUCA_OK;
}

int muca_get_walkers(muca_ctx *ctx, int group, int32_t *n_local, uint32_t *first_id)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (n_local) *n_local = ctx->g[group].W;
    if (first_id) *first_id = ctx->g[group].walker0;
    return MUCA_OK;
}

int muca_build_table(int32_t L, double T, int32_t e_min, int32_t e_max, const double *lnW,
                     uint32_t *out)
{
    if (L < 2 || L > MUCA_MAX_L || !(T > 0.0) || !std::isfinite(T))
        return fail(nullptr, MUCA_ERR_INVALID_ARG, "build_table: L=%d, T=%g", L, T);
    if (e_min < 0 || e_max < e_min || e_max > L * L * L || !lnW || !out)
        return fail(nullptr, MUCA_ERR_INVALID_ARG, "build_table: window [%d, %d] or NULL array",
                    e_min, e_max);
    const int nE = e_max - e_min + 1;
    const double beta = 1.0 / T;
    for (int e = 0; e < nE; ++e)
        for (int d = -1; d <= 1; ++d)
            for (int dej = -12; dej <= 12; ++dej)
                out[((size_t)e * 3 + (d + 1)) * MUCA_NK + (dej + 12)] =
                    table_entry(beta, lnW, 0, nE - 1, e, d, dej);
    return MUCA_OK;
}

int muca_build_table_bonds(int32_t L, double T, int32_t jmax, int32_t e_min, int32_t e_max,
                           const double *lnW, uint32_t *out)
{
    if (L < 2 || L > MUCA_MAX_L || !(T > 0.0) || !std::isfinite(T) || jmax < 1 ||
        jmax > MUCA_MAX_JMAX)
        return fail(nullptr, MUCA_ERR_INVALID_ARG, "build_table_bonds: L=%d, T=%g, jmax=%d", L, T,
                    jmax);
    if (e_min < 0 || e_max < e_min || e_max > L * L * L || !lnW || !out)
        return fail(nullptr, MUCA_ERR_INVALID_ARG,
                    "build_table_bonds: window [%d, %d] or NULL array", e_min, e_max);
    const int nE = e_max - e_min + 1, nj = 24 * jmax + 1, off = 12 * jmax;
    const double beta = 1.0 / T;
    for (int e = 0; e < nE; ++e)
        for (int d = -1; d <= 1; ++d)
            for (int dej = -off; dej <= off; ++dej)
                out[((size_t)e * 3 + (d + 1)) * nj + (dej + off)] =
                    table_entry(beta, lnW, 0, nE - 1, e, d, dej);
    return MUCA_OK;
}

int muca_get_state(muca_ctx *ctx, int group, int8_t *spins, int32_t *tallies)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    Group &g = ctx->g[group];
    if (spins) {
        const size_t nwords = (size_t)g.L * g.L * g.Lw;
        std::vector<uint32_t> dev(nwords * g.Wpad);
        CK(cudaMemcpyAsync(dev.data(), g.spins, dev.size() * sizeof(uint32_t),
                           cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        for (int w = 0; w < g.W; ++w)
            for (int row = 0; row < g.L * g.L; ++row)
                for (int x = 0; x < g.L; ++x) {
                    const uint32_t word = dev[((size_t)row * g.Lw + (x >> 2)) * g.Wpad + w];
                    spins[(size_t)w * g.V + (size_t)row * g.L + x] =
                        (int8_t)(uint8_t)(word >> (8 * (x & 3)));
                }
    }
    if (tallies) {
        std::vector<int32_t> t((size_t)3 * g.Wpad);
        CK(cudaMemcpyAsync(t.data(), g.tal, t.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        for (int w = 0; w < g.W; ++w)
            for (int f = 0; f < 3; ++f) tallies[3 * w + f] = t[(size_t)f * g.Wpad + w];
    }
    return MUCA_OK;
}

int muca_set_state(muca_ctx *ctx, int group, const int8_t *spins)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    if (!spins) return fail(ctx, MUCA_ERR_INVALID_ARG, "spins is NULL");
    Group &g = ctx->g[group];
    const size_t nwords = (size_t)g.L * g.L * g.Lw;
    std::vector<uint32_t> dev(nwords * g.Wpad, 0u);
    for (int w = 0; w < g.W; ++w)
        for (int row = 0; row < g.L * g.L; ++row)
            for (int x = 0; x < g.L; ++x) {
                const int8_t s = spins[(size_t)w * g.V + (size_t)row * g.L + x];
                if (s < -1 || s > 1)
                    return fail(ctx, MUCA_ERR_INVALID_ARG, "walker %d site %d: spin %d", w,
                                row * g.L + x, s);
                dev[((size_t)row * g.Lw + (x >> 2)) * g.Wpad + w] |=
                    (uint32_t)(uint8_t)s << (8 * (x & 3));
            }
    std::vector<int32_t> old((size_t)3 * g.Wpad);
    std::vector<uint32_t> old_spins(dev.size());
    CK(cudaMemcpyAsync(old.data(), g.tal, old.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(old_spins.data(), g.spins, dev.size() * sizeof(uint32_t),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(g.spins, dev.data(), dev.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(launch_energies(dev_of(g), 0, ctx->d_err, ctx->stream));
    std::vector<int32_t> t((size_t)3 * g.Wpad);
    CK(cudaMemcpyAsync(t.data(), g.tal, t.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int w = 0; w < g.W; ++w) {
        const int ed = t[(size_t)g.Wpad + w];
        if (ed < g.e_min + g.win_lo || ed > g.e_min + g.win_hi) {
            // put the previous state back
            CK(cudaMemcpyAsync(g.spins, old_spins.data(), old_spins.size() * sizeof(uint32_t),
                               cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaMemcpyAsync(g.tal, old.data(), old.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            return fail(ctx, MUCA_ERR_WINDOW, "walker %d: E_Delta=%d outside [%d, %d]", w, ed,
                        g.e_min + g.win_lo, g.e_min + g.win_hi);
        }
    }
    g.in_window = true;
    return MUCA_OK;
}

int muca_check_tallies(muca_ctx *ctx)
{
    if (!ctx) return fail(nullptr, MUCA_ERR_INVALID_ARG, "null context");
    return run_tally_check(ctx);
}

int muca_get_config(muca_ctx *ctx, int group, int32_t *residency, int32_t *walkers_per_block,
                    int32_t *lanes_per_walker)
{
    int rc = check_group_index(ctx, group);
    if (rc) return rc;
    const Group &g = ctx->g[group];
    if (residency) *residency = g.jmax ? MUCA_RES_BONDS : g.residency;
    if (walkers_per_block) *walkers_per_block = g.jmax ? bonds_walkers_per_warp(g.W) : g.wpb;
    if (lanes_per_walker) *lanes_per_walker = g.jmax ? 1 : g.P;
    return MUCA_OK;
}

// Checkpoint file: magic with the format version, seed, sweep, n_groups, per
// group the spec, per group the weight recursion (int32), per group the
// global id of its first walker and the walkers held (int32 x 2, the shard),
// per group the active window and its growth rule (int32 x 3 + FP64), per
// group the couplings (int32 jmax, then int8 [V][3] if jmax > 0), then per
// group lnW[nE], acc[max(nE - 1, 1)], hist[nE], tallies[3][Wpad],
// spins[V][Wpad].  Formats 04 (no couplings: the clean model), 03 (no
// window record), 02 (no shard record: every walker of the group) and 01
// (neither the shard, the recursion nor acc) are still read.
static const char kMagic[8] = {'M', 'U', 'C', 'A', 'B', 'C', '0', '5'};
static const char kMagic04[8] = {'M', 'U', 'C', 'A', 'B', 'C', '0', '4'};
static const char kMagic03[8] = {'M', 'U', 'C', 'A', 'B', 'C', '0', '3'};
static const char kMagic02[8] = {'M', 'U', 'C', 'A', 'B', 'C', '0', '2'};
static const char kMagic01[8] = {'M', 'U', 'C', 'A', 'B', 'C', '0', '1'};

int muca_checkpoint(muca_ctx *ctx, const char *path)
{
    if (!ctx) return fail(nullptr, MUCA_ERR_INVALID_ARG, "null context");
    if (!path) return fail(ctx, MUCA_ERR_INVALID_ARG, "path is NULL");
    CK(cudaStreamSynchronize(ctx->stream));
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(ctx, MUCA_ERR_IO, "cannot open %s for writing", path);
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8;
    const int32_t ng = (int32_t)ctx->g.size();
    ok = ok && std::fwrite(&ctx->seed, sizeof ctx->seed, 1, f) == 1;
    ok = ok && std::fwrite(&ctx->sweep, sizeof ctx->sweep, 1, f) == 1;
    ok = ok && std::fwrite(&ng, sizeof ng, 1, f) == 1;
    for (auto &g : ctx->g) ok = ok && std::fwrite(&g.spec, sizeof g.spec, 1, f) == 1;
    for (auto &g : ctx->g) {
        const int32_t rec = g.recursion;
        ok = ok && std::fwrite(&rec, sizeof rec, 1, f) == 1;
    }
    for (auto &g : ctx->g) {
        const int32_t shard[2] = {(int32_t)g.walker0, g.W};
        ok = ok && std::fwrite(shard, sizeof shard, 1, f) == 1;
    }
    for (auto &g : ctx->g) {
        const int32_t win[3] = {g.e_min + g.win_lo, g.e_min + g.win_hi, g.grow_step};
        ok = ok && std::fwrite(win, sizeof win, 1, f) == 1;
        ok = ok && std::fwrite(&g.grow_flat, sizeof g.grow_flat, 1, f) == 1;
    }
    for (auto &g : ctx->g) {
        const int32_t jm = g.jmax;
        ok = ok && std::fwrite(&jm, sizeof jm, 1, f) == 1;
        if (jm) ok = ok && std::fwrite(g.J.data(), 1, g.J.size(), f) == g.J.size();
    }
    for (auto &g : ctx->g) {
        if (!ok) break;
        std::vector<unsigned long long> h(g.nE);
        std::vector<int32_t> t((size_t)3 * g.Wpad);
        std::vector<uint32_t> s((size_t)g.L * g.L * g.Lw * g.Wpad);
        if (cudaMemcpy(h.data(), g.hist, h.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(t.data(), g.tal, t.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(s.data(), g.spins, s.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
            std::fclose(f);
            return fail(ctx, MUCA_ERR_CUDA, "checkpoint: device read failed");
        }
        ok = ok && std::fwrite(g.lnW.data(), 8, g.nE, f) == (size_t)g.nE;
        ok = ok && std::fwrite(g.acc.data(), 8, g.acc.size(), f) == g.acc.size();
        ok = ok && std::fwrite(h.data(), 8, h.size(), f) == h.size();
        ok = ok && std::fwrite(t.data(), 4, t.size(), f) == t.size();
        ok = ok && std::fwrite(s.data(), 4, s.size(), f) == s.size();
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(ctx, MUCA_ERR_IO, "checkpoint: write to %s failed", path);
    return MUCA_OK;
}

int muca_restore(muca_ctx *ctx, const char *path)
{
    if (!ctx) return fail(nullptr, MUCA_ERR_INVALID_ARG, "null context");
    if (!path) return fail(ctx, MUCA_ERR_INVALID_ARG, "path is NULL");
    CK(cudaStreamSynchronize(ctx->stream));
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(ctx, MUCA_ERR_IO, "cannot open %s", path);
    char magic[8];
    uint32_t seed = 0;
    uint64_t sweep = 0;
    int32_t ng = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8;
    const bool v5 = ok && std::memcmp(magic, kMagic, 8) == 0;
    const bool v4 = v5 || (ok && std::memcmp(magic, kMagic04, 8) == 0);
    const bool v3 = v4 || (ok && std::memcmp(magic, kMagic03, 8) == 0);
    const bool v2 = v3 || (ok && std::memcmp(magic, kMagic02, 8) == 0);
    ok = ok && (v2 || std::memcmp(magic, kMagic01, 8) == 0);
    ok = ok && std::fread(&seed, sizeof seed, 1, f) == 1;
    ok = ok && std::fread(&sweep, sizeof sweep, 1, f) == 1;
    ok = ok && std::fread(&ng, sizeof ng, 1, f) == 1 && ng == (int32_t)ctx->g.size();
    for (auto &g : ctx->g) {
        muca_group s{};
        ok = ok && std::fread(&s, sizeof s, 1, f) == 1 && s.L == g.spec.L && s.T == g.spec.T &&
             s.n_walkers == g.spec.n_walkers && s.e_min == g.spec.e_min &&
             s.e_max == g.spec.e_max;
    }
    std::vector<int32_t> recs(ctx->g.size(), MUCA_REC_PLAIN);
    if (v2)
        for (auto &r : recs)
            ok = ok && std::fread(&r, sizeof r, 1, f) == 1 &&
                 (r == MUCA_REC_PLAIN || r == MUCA_REC_ACCUMULATED);
    // the walkers of each group: written by format 03; earlier formats held
    // every walker of the group
    for (auto &g : ctx->g) {
        int32_t shard[2] = {0, g.spec.n_walkers};
        if (v3) ok = ok && std::fread(shard, sizeof shard, 1, f) == 1;
        ok = ok && shard[1] == g.W && (!v3 || (uint32_t)shard[0] == g.walker0);
    }
    // the active window and its growth rule: written by format 04; earlier
    // formats ran in the fixed window [e_min, e_max]
    struct Win {
        int32_t lo, hi, step;
        double flat;
    };
    std::vector<Win> wins;
    for (auto &g : ctx->g) {
        int32_t w3[3] = {g.e_min, g.e_max, 0};
        double flat = 0.0;
        if (v4)
            ok = ok && std::fread(w3, sizeof w3, 1, f) == 1 &&
                 std::fread(&flat, sizeof flat, 1, f) == 1;
        ok = ok && w3[0] >= g.e_min && w3[1] <= g.e_max && w3[0] <= w3[1] && flat >= 0.0 &&
             std::isfinite(flat) && (flat == 0.0 || w3[2] >= 1);
        wins.push_back({w3[0], w3[1], w3[2], flat});
    }
    // the couplings: written by format 05; earlier formats hold the clean model
    std::vector<int32_t> jms(ctx->g.size(), 0);
    std::vector<std::vector<int8_t>> Js(ctx->g.size());
    for (size_t gi = 0; gi < ctx->g.size() && ok; ++gi) {
        if (!v5) break;
        ok = std::fread(&jms[gi], sizeof(int32_t), 1, f) == 1 && jms[gi] >= 0 &&
             jms[gi] <= MUCA_MAX_JMAX;
        if (ok && jms[gi]) {
            Js[gi].resize((size_t)3 * ctx->g[gi].V);
            ok = std::fread(Js[gi].data(), 1, Js[gi].size(), f) == Js[gi].size();
            for (size_t k = 0; ok && k < Js[gi].size(); ++k)
                ok = Js[gi][k] >= -jms[gi] && Js[gi][k] <= jms[gi];
        }
    }
    if (!ok) {
        std::fclose(f);
        return fail(ctx, MUCA_ERR_INVALID_ARG, "restore: %s does not match this context", path);
    }
    for (size_t gi = 0; gi < ctx->g.size(); ++gi) {
        Group &g = ctx->g[gi];
        std::vector<double> lnW(g.nE), acc(g.acc.size(), 0.0);
        std::vector<unsigned long long> h(g.nE);
        std::vector<int32_t> t((size_t)3 * g.Wpad);
        std::vector<uint32_t> s((size_t)g.L * g.L * g.Lw * g.Wpad);
        ok = std::fread(lnW.data(), 8, g.nE, f) == (size_t)g.nE &&
             (!v2 || std::fread(acc.data(), 8, acc.size(), f) == acc.size()) &&
             std::fread(h.data(), 8, h.size(), f) == h.size() &&
             std::fread(t.data(), 4, t.size(), f) == t.size() &&
             std::fread(s.data(), 4, s.size(), f) == s.size();
        if (!ok) {
            std::fclose(f);
            return fail(ctx, MUCA_ERR_IO, "restore: %s is truncated", path);
        }
        g.lnW = lnW;
        g.acc = acc;
        g.recursion = recs[gi];
        g.win_lo = wins[gi].lo - g.e_min;
        g.win_hi = wins[gi].hi - g.e_min;
        g.grow_step = wins[gi].step;
        g.grow_flat = wins[gi].flat;
        g.flat[0] = g.flat[1] = g.flat[2] = 0.0;
        g.flat_full = false;
        g.injected.clear();
        g.in_window = true;
        if (cudaMemcpy(g.hist, h.data(), h.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(g.tal, t.data(), t.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(g.spins, s.data(), s.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            std::fclose(f);
            return fail(ctx, MUCA_ERR_CUDA, "restore: device write failed");
        }
        if (jms[gi] != g.jmax || (jms[gi] && Js[gi] != g.J)) {
            const int rb = apply_bonds(ctx, (int)gi, jms[gi] ? Js[gi].data() : nullptr, jms[gi],
                                       false);
            if (rb) {
                std::fclose(f);
                return rb;
            }
        }
        build_packed(g);
        int rc = upload_table(ctx, g);
        if (rc) {
            std::fclose(f);
            return rc;
        }
    }
    std::fclose(f);
    ctx->seed = seed;
    ctx->sweep = sweep;
    CK(cudaStreamSynchronize(ctx->stream));
    return MUCA_OK;
}

}  // extern "C"
