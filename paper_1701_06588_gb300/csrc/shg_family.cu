// Family basis sets (all shells of an element share one exponent set, as in
// the MOLOPT bases the paper measures): the radial terms G^{(k)} of Table S1
// depend on the primitive pair and the separation only, so for a group of
// shell pairs whose a-shells share one family on one center (and likewise
// for b) they are computed once per primitive pair, for every order the
// group needs, and each shell pair contracts them with its own weights,
//   O^{(k)}_{ab} = sum_{i,j} w_a[i] w_b[j] G^{(k)}[i][j],
//   w = N c (2 alpha)^{-l}                               (Eq. O_rab2_deriv),
// instead of recomputing the radial terms per shell pair.  One warp per
// group: G in shared memory, lanes over primitive pairs, then over (shell
// pair, order) items.  The angular part follows in the class-tiled kernel
// (OP_PRE).
#include "shg_device.cuh"

namespace shg {
namespace {
using namespace dev;

constexpr int kFamWarps = 4;

// Unit-weight radial terms G[k] = (0_a|O|0_b)^{(k)}, k = 0..kmax, of one primitive pair.
template <int OP>
__device__ __forceinline__ void radial_all(double alpha, double beta, double inv_a, double inv_b, double R2, int kmax,
                                           const ArgsFam &g, double *G)
{
    const double c = alpha + beta;
    const double rc = rsqrt(c);
    const double ic = rc * rc;
    const double rho = alpha * beta * ic;
    const double T = rho * R2;
    if (OP == OP_OVERLAP) {
        double q = kPi32 * ic * rc * exp(-T);
        for (int k = 0; k <= kmax; ++k) {
            G[k] = q;
            q *= -rho;
        }
    } else if (OP == OP_GAUSS) {
        const double rd = rsqrt(rho + g.omega);
        const double id = rd * rd;
        const double f = -g.omega * rho * id;
        double q = kPi3 * ic * rc * id * rd * exp(-g.omega * T * id);
        for (int k = 0; k <= kmax; ++k) {
            G[k] = q;
            q *= f;
        }
    } else if (OP == OP_GCOUL) {
        const double id = 1.0 / (rho + g.omega);
        const double p = -g.omega * rho * id, q = -rho * rho * id;
        const double pre = kPi32 * ic * rc * (2.0 * kPi) * id * exp(-g.omega * T * id);
        double F[kBoysN];
        boys_all(T * rho * id, kmax, g.boys, g.boys_e, g.k, F);
        G[0] = pre * F[0];
        for (int m = 1; m <= kmax; ++m) {
            for (int i = 0; i <= kmax - m; ++i) F[i] = fma(p, F[i], q * F[i + 1]);
            G[m] = pre * F[0];
        }
    } else {
        const double pre = kTwoPi52 * inv_a * inv_b * rc;
        for (int k = 0; k <= kmax; ++k) G[k] = 0.0;
        double F[kBoysN];
        if (OP == OP_COULOMB || OP == OP_ERFC) {
            boys_all(T, kmax, g.boys, g.boys_e, g.k, F);
            double q = pre;
            for (int k = 0; k <= kmax; ++k) {
                G[k] = q * F[k];
                q *= -rho;
            }
        }
        if (OP == OP_ERF || OP == OP_ERFC) {
            const double w2 = g.omega * g.omega;
            const double rw = rsqrt(w2 + rho);
            const double s = w2 * rw * rw;
            const double f = -rho * s;
            boys_all(s * T, kmax, g.boys, g.boys_e, g.k, F);
            double q = pre * g.omega * rw;
            if (OP == OP_ERFC) q = -q;
            for (int k = 0; k <= kmax; ++k) {
                G[k] += q * F[k];
                q *= f;
            }
        }
    }
}

template <int OP>
__global__ void __launch_bounds__(32 * kFamWarps) k_family_radial(const ArgsFam g)
{
    __shared__ double Gs[kFamWarps][kFamOrd * kFamPP];
    __shared__ int Js[kFamWarps][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double *gs = Gs[w];
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(g.counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= g.n_groups) break;
        const FamGroup gr = g.groups[t];
        const Vec4 A = g.centers[gr.ca], B = g.centers[gr.cb];
        const double vx = A.x - B.x, vy = A.y - B.y, vz = A.z - B.z;
        const double R2 = vx * vx + vy * vy + vz * vz;
        const int npp = gr.fa_k * gr.fb_k;
        for (int ij = lane; ij < npp; ij += 32) {
            const int i = ij / gr.fb_k, j = ij - i * gr.fb_k;
            const PrimRec pa = g.prims[gr.fa_prim + i], pb = g.prims[gr.fb_prim + j];
            double G[kFamOrd];
            radial_all<OP>(pa.alpha, pb.alpha, pa.inv_alpha, pb.inv_alpha, R2, gr.kmax, g, G);
            for (int k = gr.kmin; k <= gr.kmax; ++k) gs[(k - gr.kmin) * kFamPP + ij] = G[k];
        }
        __syncwarp();
        // contraction: lanes over (shell pair, order) items, 32 shell pairs at a
        // time; item it belongs to the pair r with js[r] <= it < js[r + 1]
        int *js = Js[w];
        for (int q0 = 0; q0 < gr.count; q0 += 32) {
            int Jq = 0;
            if (q0 + lane < gr.count) {
                const int p = gr.start + q0 + lane;
                const int la = g.shells[g.pair_a[p]].l, lb = g.shells[g.pair_b[p]].l;
                Jq = (la < lb ? la : lb) + 1;
            }
            int inc = Jq;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            js[lane + 1] = inc;
            if (lane == 0) js[0] = 0;
            const int total = __shfl_sync(0xffffffffu, inc, 31);
            __syncwarp();
            for (int it = lane; it < total; it += 32) {
                int r = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1)
                    if (js[r + step] <= it) r += step;
                const int tj = it - js[r];
                const int p = gr.start + q0 + r;      // the subset is stored in group order
                const ShellRec sa = g.shells[g.pair_a[p]], sb = g.shells[g.pair_b[p]];
                const int kmax = sa.l + sb.l;
                const double *gk = gs + (kmax - tj - gr.kmin) * kFamPP;
                double s = 0.0;
                for (int i = 0; i < gr.fa_k; ++i) {
                    double si = 0.0;
                    for (int j = 0; j < gr.fb_k; ++j) si = fma(g.prims[sb.prim_off + j].w2c, gk[i * gr.fb_k + j], si);
                    s = fma(g.prims[sa.prim_off + i].w2c, si, s);
                }
                g.o_pre[(int64_t)p * kJmax + tj] = s;
            }
            __syncwarp();
        }
    }
}

__global__ void k_gather_i64(const int64_t *__restrict__ src, const int32_t *__restrict__ idx, int64_t n,
                             int64_t *__restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}

template <int OP>
cudaError_t launch_fam(const ArgsFam &a, cudaStream_t s)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_family_radial<OP>, 32 * kFamWarps, 0) != cudaSuccess ||
        per < 1)
        per = 1;
    k_family_radial<OP><<<sms * per, 32 * kFamWarps, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_family_radial(const ArgsFam &a, int op, cudaStream_t s)
{
    if (a.n_groups <= 0) return cudaSuccess;
    switch (op) {
    case OP_OVERLAP: return launch_fam<OP_OVERLAP>(a, s);
    case OP_COULOMB: return launch_fam<OP_COULOMB>(a, s);
    case OP_ERFC: return launch_fam<OP_ERFC>(a, s);
    case OP_ERF: return launch_fam<OP_ERF>(a, s);
    case OP_GAUSS: return launch_fam<OP_GAUSS>(a, s);
    case OP_GCOUL: return launch_fam<OP_GCOUL>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_gather_i64(const int64_t *src, const int32_t *idx, int64_t n, int64_t *dst, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    k_gather_i64<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(src, idx, n, dst);
    return cudaGetLastError();
}

}  // namespace shg
