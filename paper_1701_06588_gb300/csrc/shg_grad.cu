// Gradients of the two-center SHG integrals with respect to the centers
// (Sec. II C of arXiv:1701.06588, Eq. dev_ab), as a vector-Jacobian product
// with upstream weights W:
//
//   g_i = sum_{ma,mb} W[ma][mb] d(a|O|b)[ma][mb] / dR_{a,i}
//       = 2 (R_a - R_b)_i sum_j O^{(la+lb-j+1)} <W, Q~_j>
//         + sum_j O^{(la+lb-j)} <W, dQ~_j/dR_{a,i}>,
//
// and d/dR_b = -d/dR_a (translation invariance).  Q~_j = (-1)^lb A_a A_b
// 2^{la+lb-j} (2j-1)!! sum_kappa B_{j,kappa} W_a W_b^T; its derivative is
// built from (l-1) harmonics by the lowering rules of the regular scaled
// solid harmonics, applied to the entries of the translation matrices:
//   dR_{l,m}/dz = R_{l-1,m}
//   dR_{l,m}/dx = (R_{l-1,m+1} - R_{l-1,m-1}) / 2
//   dR_{l,m}/dy = -i (R_{l-1,m+1} + R_{l-1,m-1}) / 2      (R = R^c + i R^s)
// which is the construction of Eqs. cartesian_dev_x/y/z one level down.
// The radial terms are recomputed here up to order la+lb+1; nothing is kept
// from a forward evaluation.
#include "shg_device.cuh"
#include "shg_grad_angular.cuh"

namespace shg {
namespace {
using namespace dev;

template <int OP, int J>
__device__ void pair_grad_fp64(const Args2c &g, int p)
{
    const ShellRec sa = g.shells[g.pair_a[p]];
    const ShellRec sb = g.shells[g.pair_b[p]];
    const int la = sa.l, lb = sb.l;
    const Vec4 A = g.centers[sa.center];
    const Vec4 B = g.centers[sb.center];
    const double v[3] = {A.x - B.x, A.y - B.y, A.z - B.z};
    const double R2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const int kmax = la + lb;

    // Ox[j] = O^{(kmax+1-j)}, j = 0..J
    double Ox[J + 1], Ex[J + 1];
#pragma unroll
    for (int j = 0; j <= J; ++j) Ox[j] = Ex[j] = 0.0;
    const int Kb = sb.nprim, npp = sa.nprim * Kb;
    for (int q = 0; q < npp; ++q) {
        const int ia = q / Kb, ib = q - ia * Kb;
        radial_acc_fp64<OP, J + 1>(g.prims[sa.prim_off + ia], g.prims[sb.prim_off + ib], R2, kmax + 1, la, g, Ox, Ex);
    }
    radial_finish_fp64<OP, J + 1>(R2, kmax + 1, g.k, Ox, Ex);
    // f0[e]: factor of Q~_j with O^{(kmax-j)}, f1[e]: with O^{(kmax-j+1)}
    double f0[J * J], f1[J * J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const double p2 = g.k.pow2[kmax - j];
#pragma unroll
        for (int kp = 0; kp <= j; ++kp) {
            const double b = p2 * g.k.jB[j][kp];
            const int e0 = j * j + (kp == 0 ? 0 : 2 * kp - 1);
            f0[e0] = b * Ox[j + 1];
            f1[e0] = b * Ox[j];
            if (kp) {
                f0[e0 + 1] = f0[e0];
                f1[e0 + 1] = f1[e0];
            }
        }
    }

    gradang::grad_from_orders<J>(g, p, la, lb, v, f0, f1);
}

template <int OP>
__device__ __forceinline__ void grad_dispatch(const Args2c &g, int p, int J)
{
    switch (J) {
    case 1: pair_grad_fp64<OP, 1>(g, p); break;
    case 2: pair_grad_fp64<OP, 2>(g, p); break;
    case 3: pair_grad_fp64<OP, 3>(g, p); break;
    case 4: pair_grad_fp64<OP, 4>(g, p); break;
    case 5: pair_grad_fp64<OP, 5>(g, p); break;
    case 6: pair_grad_fp64<OP, 6>(g, p); break;
    default: pair_grad_fp64<OP, 7>(g, p); break;
    }
}

// With a tile counter every warp takes tiles from it until none are left; with
// none (g.counter == nullptr) warp w of block b takes tile tile_begin + b *
// warps_per_block + w once (a static launch over a short tile range).
template <int OP>
__global__ void __launch_bounds__(128) k_2c_grad_fp64_persistent(const Args2c g)
{
    const int lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    for (int it = 0;; ++it) {
        int t = 0;
        if (g.counter) {
            if (lane == 0) t = atomicAdd(g.counter, 1);
            t = __shfl_sync(0xffffffffu, t, 0) + g.tile_begin;
        } else {
            if (it) break;
            t = g.tile_begin + blockIdx.x * nw + (threadIdx.x >> 5);
        }
        if (t >= g.tile_end) break;
        const Tile tl = g.tiles[t];
        if (lane < tl.count) {
            const int la = tl.cls / (kLmax2c + 1), lb = tl.cls % (kLmax2c + 1);
            grad_dispatch<OP>(g, g.perm[tl.start + lane], (la < lb ? la : lb) + 1);
        }
        __syncwarp();
    }
}

template <int OP>
static int grid_for()
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_grad_fp64_persistent<OP>, 128, 0) != cudaSuccess ||
        per < 1)
        per = 1;
    return (sms > 0 ? sms : 1) * per;
}

}  // namespace

cudaError_t launch_2c_grad(const Args2c &a, int op, int precision, int grid, cudaStream_t s, int threads)
{
    (void)precision;
    if (threads < 32 || threads > 128 || threads % 32) return cudaErrorInvalidValue;
    if (!a.counter) {
        // static: one warp per tile of [tile_begin, tile_end)
        const int per = threads / 32;
        grid = (a.tile_end - a.tile_begin + per - 1) / per;
        if (grid <= 0) return cudaSuccess;
    }
    switch (op) {
    case OP_OVERLAP: k_2c_grad_fp64_persistent<OP_OVERLAP><<<grid, threads, 0, s>>>(a); break;
    case OP_COULOMB: k_2c_grad_fp64_persistent<OP_COULOMB><<<grid, threads, 0, s>>>(a); break;
    case OP_ERFC: k_2c_grad_fp64_persistent<OP_ERFC><<<grid, threads, 0, s>>>(a); break;
    case OP_ERF: k_2c_grad_fp64_persistent<OP_ERF><<<grid, threads, 0, s>>>(a); break;
    case OP_GAUSS: k_2c_grad_fp64_persistent<OP_GAUSS><<<grid, threads, 0, s>>>(a); break;
    case OP_GCOUL: k_2c_grad_fp64_persistent<OP_GCOUL><<<grid, threads, 0, s>>>(a); break;
    case OP_RA2N: k_2c_grad_fp64_persistent<OP_RA2N><<<grid, threads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int persistent_grid_2c_grad(int op, int precision)
{
    (void)precision;
    switch (op) {
    case OP_OVERLAP: return grid_for<OP_OVERLAP>();
    case OP_COULOMB: return grid_for<OP_COULOMB>();
    case OP_ERFC: return grid_for<OP_ERFC>();
    case OP_ERF: return grid_for<OP_ERF>();
    case OP_GAUSS: return grid_for<OP_GAUSS>();
    case OP_GCOUL: return grid_for<OP_GCOUL>();
    default: return grid_for<OP_RA2N>();
    }
}

}  // namespace shg
