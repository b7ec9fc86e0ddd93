// Molecular assembly kernels: blocks <-> dense AO matrix, and the per-center
// reduction of per-pair gradients.  A group of 8 lanes per pair (blocks hold
// 1 to 13 x 13 elements, a few on average), so a warp keeps four pairs'
// index loads in flight; HBM- or latency-bound.
#include "shg_internal.h"

namespace shg {
namespace {

constexpr int kWarpsPerCta = 8;
constexpr int kGroup = 8;                       // lanes per pair
constexpr int kGroupsPerCta = kWarpsPerCta * 32 / kGroup;

__global__ void __launch_bounds__(256) k_scatter_2c(const ShellRec *__restrict__ shells, int64_t n,
                                                    const int32_t *__restrict__ pa, const int32_t *__restrict__ pb,
                                                    const long long *__restrict__ boff,
                                                    const double *__restrict__ blocks,
                                                    const long long *__restrict__ ao, long long ld, int sym,
                                                    double *__restrict__ M)
{
    const int lane = threadIdx.x % kGroup;
    const int64_t groups = (int64_t)gridDim.x * kGroupsPerCta;
    for (int64_t p = (int64_t)blockIdx.x * kGroupsPerCta + threadIdx.x / kGroup; p < n; p += groups) {
        const int a = pa[p], b = pb[p];
        const int na = 2 * shells[a].l + 1, nb = 2 * shells[b].l + 1;
        const long long ra = ao[a], rb = ao[b];
        const double *blk = blocks + boff[p];
        const int ne = na * nb;
        // rows of the block: consecutive lanes write consecutive columns
        for (int e = lane; e < ne; e += kGroup) {
            const int i = e / nb, j = e - i * nb;
            M[(ra + i) * ld + rb + j] = blk[e];
        }
        if (sym && a != b) {
            // transposed block: consecutive lanes write consecutive columns of row rb + j
            for (int e = lane; e < ne; e += kGroup) {
                const int j = e / na, i = e - j * na;
                M[(rb + j) * ld + ra + i] = blk[i * nb + j];
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_gather_2c(const ShellRec *__restrict__ shells, int64_t n,
                                                   const int32_t *__restrict__ pa, const int32_t *__restrict__ pb,
                                                   const long long *__restrict__ boff,
                                                   const double *__restrict__ M, const long long *__restrict__ ao,
                                                   long long ld, int sym, double *__restrict__ blocks)
{
    const int lane = threadIdx.x % kGroup;
    const int64_t groups = (int64_t)gridDim.x * kGroupsPerCta;
    for (int64_t p = (int64_t)blockIdx.x * kGroupsPerCta + threadIdx.x / kGroup; p < n; p += groups) {
        const int a = pa[p], b = pb[p];
        const int na = 2 * shells[a].l + 1, nb = 2 * shells[b].l + 1;
        const long long ra = ao[a], rb = ao[b];
        double *blk = blocks + boff[p];
        const int ne = na * nb;
        const bool both = sym && a != b;
        for (int e = lane; e < ne; e += kGroup) {
            const int i = e / nb, j = e - i * nb;
            double v = M[(ra + i) * ld + rb + j];
            if (both) v += M[(rb + j) * ld + ra + i];
            blk[e] = v;
        }
    }
}

__global__ void k_reduce_centers(const ShellRec *__restrict__ shells, int64_t n, const int32_t *__restrict__ pa,
                                 const int32_t *__restrict__ pb, const double *__restrict__ ga,
                                 const double *__restrict__ gb, double *__restrict__ out)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 3 * n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / 3;
        const int d = (int)(t - 3 * p);
        atomicAdd(out + 3 * (int64_t)shells[pa[p]].center + d, ga[t]);
        atomicAdd(out + 3 * (int64_t)shells[pb[p]].center + d, gb[t]);
    }
}

int warp_grid(int64_t n)
{
    const int64_t ctas = (n + kGroupsPerCta - 1) / kGroupsPerCta;
    return (int)(ctas < 152 * 8 ? (ctas > 0 ? ctas : 1) : 152 * 8);
}

}  // namespace

cudaError_t launch_scatter_2c(const ShellRec *shells, int64_t n, const int32_t *pa, const int32_t *pb,
                              const int64_t *boff, const double *blocks, const int64_t *ao, int64_t ld, int sym,
                              double *M, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_scatter_2c<<<warp_grid(n), 32 * kWarpsPerCta, 0, s>>>(shells, n, pa, pb, reinterpret_cast<const long long *>(boff),
                                                           blocks, reinterpret_cast<const long long *>(ao), ld, sym, M);
    return cudaGetLastError();
}

cudaError_t launch_gather_2c(const ShellRec *shells, int64_t n, const int32_t *pa, const int32_t *pb,
                             const int64_t *boff, const double *M, const int64_t *ao, int64_t ld, int sym,
                             double *blocks, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_gather_2c<<<warp_grid(n), 32 * kWarpsPerCta, 0, s>>>(shells, n, pa, pb, reinterpret_cast<const long long *>(boff),
                                                          M, reinterpret_cast<const long long *>(ao), ld, sym, blocks);
    return cudaGetLastError();
}

cudaError_t launch_reduce_centers(const ShellRec *shells, int64_t n, const int32_t *pa, const int32_t *pb,
                                  const double *ga, const double *gb, double *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (3 * n + 255) / 256;
    k_reduce_centers<<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(shells, n, pa, pb, ga, gb, out);
    return cudaGetLastError();
}

}  // namespace shg
