// shg_eval_2c_noalloc: the two-center evaluation of shg_eval_2c for callers
// that must not allocate device memory during the call.
//
// Who needs this: code that runs where cudaMalloc / cudaMallocAsync are not
// allowed or not wanted at call time - for example a framework whose memory
// is handed out only by its own pool, a real-time loop that has to avoid the
// implicit synchronisation and latency of allocation, or a host that has
// already reserved all device memory.  shg_eval_2c builds its plan in memory
// from cudaMallocAsync; this variant builds the same plan (pair bucketing and
// tile list) in a fixed device array that belongs to the library instead.
//
// The array is a file-scope __device__ variable, so every GPU that loads this
// library keeps it (kNoAllocBytes, about 10.5 MB) until the process exits.
// Host code cannot use its name as a device address; the address is taken
// with cudaGetSymbolAddress once per device, on the first call made on that
// device (so that first call should not be made while a stream is being
// captured), and kept for the life of the process: after cudaDeviceReset the
// cached address is stale, so the entry point must not be used across one.
//
// All calls share the one array and it keeps the contents of the previous
// call; every part that has to start at zero is cleared by the call itself.
// Two calls whose GPU work overlaps (different streams, or different host
// threads without ordering) race on the array and give wrong results: order
// them on one stream or synchronise between them.
#include "../../include/shg.h"
#include "shg_internal.h"

#include <mutex>

namespace shg {
namespace {

constexpr int64_t kNoAllocMaxPairs = int64_t(1) << 20;
// layout: tiles | perm | counter, err | key | hist | bin_start | cursor | tile_start
constexpr int64_t kNoAllocMaxTiles = kNoAllocMaxPairs / kTile + kNBins2c + 1;
constexpr size_t kTilesBytes = ((size_t)kNoAllocMaxTiles * sizeof(Tile) + 255) / 256 * 256;
constexpr size_t kPermBytes = ((size_t)kNoAllocMaxPairs * sizeof(int32_t) + 255) / 256 * 256;
constexpr size_t kFlagsBytes = 256;
constexpr size_t kWsBytes = (plan_ws_ints(kNoAllocMaxPairs, kNBins2c, kNClass) * sizeof(int) + 255) / 256 * 256;
constexpr size_t kNoAllocBytes = kTilesBytes + kPermBytes + kFlagsBytes + kWsBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {};

// Device address of g_noalloc_scratch on the current device (set-up on the
// first call per device).
int scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(SHG_ECUDA, "cudaGetDevice failed");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(SHG_ECUDA, "cudaGetSymbolAddress(scratch) failed on device %d: %s", dev, cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SHG_OK;
}

}  // namespace
}  // namespace shg

using namespace shg;

extern "C" int shg_eval_2c_noalloc(const shg_basis_t *basis, int64_t n_pairs, const int32_t *d_pair_a,
                                   const int32_t *d_pair_b, int op, double omega, int precision,
                                   const int64_t *d_out_offsets, double *d_out, void *stream)
{
    clear_error();
    if (!basis) return fail(SHG_EINVAL, "basis is NULL");
    if (precision != SHG_PREC_FP64)
        return fail(SHG_EINVAL, "shg_eval_2c_noalloc: precision %d not available (FP64 only)", precision);
    int r = check_op(op, omega, precision);
    if (r) return r;
    if (n_pairs < 0) return fail(SHG_EINVAL, "n_pairs < 0");
    if (n_pairs > kNoAllocMaxPairs)
        return fail(SHG_ERANGE, "shg_eval_2c_noalloc: %lld pairs exceed the fixed maximum of %lld", (long long)n_pairs,
                    (long long)kNoAllocMaxPairs);
    if (n_pairs == 0) return SHG_OK;
    if (!d_pair_a || !d_pair_b || !d_out_offsets || !d_out) return fail(SHG_EINVAL, "NULL device pointer");
    const BasisDev &b = basis->d;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return fail(SHG_ECUDA, "cudaGetDevice failed");
    if (cur != b.device) return fail(SHG_EINVAL, "current device %d differs from the basis device %d", cur, b.device);
    const int *ranks[2] = {nullptr, nullptr};
    const DeviceTables *t = device_tables_if_ready(ranks);
    if (!t) return fail(SHG_EINVAL, "library tables missing on this device: create a basis on it first");
    void *base = nullptr;
    r = scratch_address(&base);
    if (r) return r;

    cudaStream_t s = (cudaStream_t)stream;
    char *c = (char *)base;
    PlanDev plan;
    plan.basis = &b;
    plan.kind = 2;
    plan.n_pairs = n_pairs;
    plan.schedule = SHG_SCHED_PERSISTENT;
    plan.pair_a = d_pair_a;
    plan.pair_b = d_pair_b;
    plan.tiles = (Tile *)c;                c += kTilesBytes;
    plan.perm = (int32_t *)c;              c += kPermBytes;
    plan.counter = (int *)c;               c += kFlagsBytes;
    int *ws = (int *)c;

    cudaError_t e = launch_plan_build(plan, ws, kNBins2c, ranks[SHG_SCHED_PERSISTENT], s);
    // the end of the build summary: tile count and error flag
    int h_sum[2] = {0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_sum, plan_summary(ws, kNBins2c) + kNClass, sizeof(h_sum), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(SHG_ECUDA, "shg_eval_2c_noalloc planning: %s", cudaGetErrorString(e));
    if (h_sum[1]) return fail(SHG_EINVAL, "pair list holds a shell index outside 0..%d", b.n_shells - 1);
    const int n_tiles = h_sum[0];
    if (n_tiles <= 0) return SHG_OK;

    Args2c a;
    a.shells = b.shells;
    a.prims = b.prims;
    a.centers = b.centers;
    a.pair_a = d_pair_a;
    a.pair_b = d_pair_b;
    a.perm = plan.perm;
    a.tiles = plan.tiles;
    a.tile_begin = 0;
    a.tile_end = n_tiles;
    a.counter = plan.counter;
    a.out_off = reinterpret_cast<const long long *>(d_out_offsets);
    a.out = d_out;
    a.omega = omega;
    a.screen_thresh = 0.0;
    a.screen = b.screen;
    a.boys = t->boys;
    a.boys_e = t->boys_e;
    a.k = consts();
    e = cudaMemsetAsync(plan.counter, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_2c(a, op, precision, persistent_grid_2c(op, precision), true, s);
    if (e != cudaSuccess) return fail(SHG_ECUDA, "shg_eval_2c_noalloc launch: %s", cudaGetErrorString(e));
    return SHG_OK;
}
