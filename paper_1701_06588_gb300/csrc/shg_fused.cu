// Several operators of one pair list in one pass (FP64): the two-center
// formula of Sec. II B of arXiv:1701.06588 with the operators of Table S1,
// rearranged so that everything that depends on the geometry only is built
// once per shell pair and shared by the operators:
//
//   (a|O|b)[ma][mb] = (-1)^lb A_{la,ma} A_{lb,mb} sum_j 2^{la+lb-j} O^{(la+lb-j)} Q_j[ma][mb],
//   Q_j[ma][mb]     = (2j-1)!! sum_kappa B_{j,kappa} sum_z W_a[ma][j,kappa,z] W_b[mb][j,kappa,z],
//
// Q_j is the operator-independent part (Eq. Q_matrix with the B weights of
// Eq. B); per element it costs J^2 multiply-adds once, and each operator then
// needs only its J radial orders (J multiply-adds).  The radial sums share the
// primitive-pair setup (c, rho, T, the prefactors), erfc(wr)/r is formed as
// 1/r - erf(wr)/r from the Coulomb and attenuated Boys sums (Table S1), and
// when erf and erfc are both requested with the same omega the attenuated
// sum is computed once.
//
// Work mapping as the single-operator kernel: one thread per shell pair, a
// warp per class-pure tile of up to 32 pairs, tiles from the same plan.
#include "shg_device.cuh"

namespace shg {
namespace {
using namespace dev;

// Downward recursion after the contraction.  For one primitive pair the
// Coulomb-type radial term of order n, X_n = P q^n F_n(T') (1/r: P = pre,
// q = -rho, T' = T; attenuated: P = pre omega / sqrt(omega^2 + rho),
// q = -rho s, T' = s T with s = omega^2 / (omega^2 + rho)), obeys, by the
// Boys recursion F_n = (2T' F_{n+1} + exp(-T')) / (2n+1),
//   X_n = (-2R^2 X_{n+1} + P q^n exp(-T')) / (2n+1),
// since 2T'/q = -2R^2 for both.  -2R^2 is the same for every primitive pair
// of the shell pair, so the contracted orders follow the same recursion:
// per primitive pair only the top order (from the Taylor head) and the
// terms E_n = P q^n exp(-T') are summed.  The two terms of each step have
// the same sign for every primitive pair, so the contracted recursion
// loses nothing against the magnitude sum of the contraction.

// attenuated part (the erf(omega r)/r term of Table S1) of one primitive pair:
// pk = pre (-rho)^kmin, so P q^kmin = pk u s^kmin with u = omega / sqrt(omega^2 + rho)
template <int J>
__device__ __forceinline__ void att_head(double om, double w2, double rho, double T, int kmax, int kmin, double pk,
                                         const ArgsFused &g, double (&O)[J], double (&E)[J])
{
    const double u = om * rsqrt(w2 + rho);
    const double s = u * u;
    double F, e;
    boys_head(s * T, kmax, g.boys, g.boys_e, g.k, F, e);
    double w = pk * u * powi(s, kmin);
    const double q = -rho * s;
#pragma unroll
    for (int j = J - 1; j >= 1; --j) {
        E[j] = fma(w, e, E[j]);
        w *= q;
    }
    O[0] = fma(w, F, O[0]);
}

template <int J>
__device__ void pair_2c_fused(const ArgsFused &g, int p)
{
    const ShellRec sa = g.shells[g.pair_a[p]];
    const ShellRec sb = g.shells[g.pair_b[p]];
    const int la = sa.l, lb = sb.l;
    const Vec4 A = g.centers[sa.center];
    const Vec4 B = g.centers[sb.center];
    const double vx = A.x - B.x, vy = A.y - B.y, vz = A.z - B.z;
    const double R2 = vx * vx + vy * vy + vz * vz;
    const int kmax = la + lb, kmin = kmax - J + 1;

    // which sums the requested operators need (uniform over the launch)
    const bool f_ov = g.out[OP_OVERLAP] != nullptr;
    const bool f_ga = g.out[OP_GAUSS] != nullptr;
    const bool f_co = g.out[OP_COULOMB] != nullptr || g.out[OP_ERFC] != nullptr;
    const bool f_er = g.out[OP_ERF] != nullptr;
    const bool f_x = g.out[OP_ERFC] != nullptr && !(f_er && g.share_att);
    // exp(-T) from the Boys head: the downward recursion needs it for J > 1,
    // the overlap reuses it
    const bool need_e = J > 1 || f_ov;
    const double w2_erf = g.w_erf * g.w_erf, w2_erfc = g.w_erfc * g.w_erfc;

    // O*[j]: contracted order kmax - j of each operator; E*[j], j >= 1: the
    // exp(-T') terms of the contracted recursion (index 0 unused)
    double Oov[J], Oco[J], Oer[J], Ox[J], Oga[J], Eco[J], Eer[J], Ex[J];
#pragma unroll
    for (int j = 0; j < J; ++j) Oov[j] = Oco[j] = Oer[j] = Ox[j] = Oga[j] = Eco[j] = Eer[j] = Ex[j] = 0.0;
    // far-field part of the 1/r sum: sum of fw_a fw_b over the primitive pairs
    // with T >= kBoysTmax (see CoulPrim), multiplied by the per-pair order
    // factors after the loop
    double far = 0.0;

    const int Kb = sb.nprim, npp = sa.nprim * Kb;
    for (int q = 0; q < npp; ++q) {
        const int ia = q / Kb, ib = q - ia * Kb;
        const PrimRec pa = g.prims[sa.prim_off + ia], pb = g.prims[sb.prim_off + ib];
        const double c = pa.alpha + pb.alpha;
        const double rc = rsqrt(c);
        const double ic = rc * rc;
        const double rho = pa.alpha * pb.alpha * ic;
        const double T = rho * R2;
        const bool near = T < kBoysTmax;
        const double mrk = (f_ov || f_co || f_er || f_x) ? powi(-rho, kmin) : 0.0;
        // Boys head of the 1/r sum first: it also yields exp(-T) for the overlap
        // (0 for T >= kBoysTmax, where the overlap term is below e^-120 of its prefactor)
        double Fc = 0.0, eT = 0.0;
        if (f_co && near) {
            if (need_e) boys_head_near<true>(T, kmax, g.boys, g.boys_e, Fc, eT);
            else boys_head_near<false>(T, kmax, g.boys, g.boys_e, Fc, eT);
        }
        if (f_ov) {
            // (pi/c)^{3/2} exp(-T) (-rho)^k
            const double w = pa.w2c * pb.w2c;
            double t = w * kPi32 * ic * rc * (f_co ? eT : exp(-T)) * mrk;
#pragma unroll
            for (int j = J - 1; j >= 0; --j) {
                Oov[j] += t;
                t *= -rho;
            }
        }
        if (f_ga) {
            // (pi^2/(c (rho+w)))^{3/2} exp(-w T/(rho+w)) (-w rho/(rho+w))^k
            const double w = pa.w2c * pb.w2c;
            const double rd = rsqrt(rho + g.w_gauss);
            const double id = rd * rd;
            const double f = -g.w_gauss * rho * id;
            double t = w * kPi3 * ic * rc * id * rd * exp(-g.w_gauss * T * id) * powi(f, kmin);
#pragma unroll
            for (int j = J - 1; j >= 0; --j) {
                Oga[j] += t;
                t *= f;
            }
        }
        if (f_co || f_er || f_x) {
            // 2 pi^{5/2} w / (alpha beta sqrt(c)) (-rho)^kmin, times the Boys sums
            const CoulPrim ca = g.cprims[sa.prim_off + ia], cb = g.cprims[sb.prim_off + ib];
            const double pk = ca.cw * cb.cw * rc * mrk;
            if (f_co) {
                if (near) {
                    double w = pk;
#pragma unroll
                    for (int j = J - 1; j >= 1; --j) {
                        Eco[j] = fma(w, eT, Eco[j]);
                        w *= -rho;
                    }
                    Oco[0] = fma(w, Fc, Oco[0]);
                } else {
                    far = fma(ca.fw, cb.fw, far);
                }
            }
            if (f_er) att_head<J>(g.w_erf, w2_erf, rho, T, kmax, kmin, pk, g, Oer, Eer);
            if (f_x) att_head<J>(g.w_erfc, w2_erfc, rho, T, kmax, kmin, pk, g, Ox, Ex);
        }
    }
    // contracted downward recursion, orders kmax-1 .. kmin (the far field,
    // exact per order, is added afterwards)
    const double m2R2 = -2.0 * R2;
#pragma unroll
    for (int j = 1; j < J; ++j) {
        const double inv = g.k.inv_int[2 * (kmax - j) + 1];
        Oco[j] = fma(m2R2, Oco[j - 1], Eco[j]) * inv;
        Oer[j] = fma(m2R2, Oer[j - 1], Eer[j]) * inv;
        Ox[j] = fma(m2R2, Ox[j - 1], Ex[j]) * inv;
    }
    if (far != 0.0) {
        // pi^3 (-1)^n (2n-1)!! (2R^2)^{-n} / R for n = kmin .. kmax (R > 0: T >= kBoysTmax)
        const double ir2 = 1.0 / R2;
        double t = far * kPi3 * sqrt(ir2) * g.k.dfact[kmin] * powi(-0.5 * ir2, kmin);
#pragma unroll
        for (int j = J - 1; j >= 0; --j) {
            Oco[j] += t;
            t *= -0.5 * ir2 * g.k.dint[2 * (kmax - j) + 1];
        }
    }
    // erfc = coulomb - attenuated; then every operator's orders scaled by 2^{kmax-j}
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const double p2 = g.k.pow2[kmax - j];
        Ox[j] = (Oco[j] - (f_x ? Ox[j] : Oer[j])) * p2;
        Oov[j] *= p2;
        Oco[j] *= p2;
        Oer[j] *= p2;
        Oga[j] *= p2;
    }

    double Rc[(kLmax2c + 1) * (kLmax2c + 2) / 2], Rs[(kLmax2c + 1) * (kLmax2c + 2) / 2];
    scaled_harmonics(vx, vy, vz, la > lb ? la : lb, g.k, Rc, Rs);
    const int nb = 2 * lb + 1;
    double Wb[2 * kLmax2c + 1][J * J];
    for (int mb = -lb; mb <= lb; ++mb) {
        double w[J * J];
        w_row<J>(Rc, Rs, lb, mb, w);
#pragma unroll
        for (int e = 0; e < J * J; ++e) Wb[mb + lb][e] = w[e];
    }
    const double sgn_b = (lb & 1) ? -1.0 : 1.0;
    const long long o = g.out_off[p];
    for (int ma = -la; ma <= la; ++ma) {
        double ua[J * J];
        w_row<J>(Rc, Rs, la, ma, ua);
#pragma unroll
        for (int j = 0; j < J; ++j) {
#pragma unroll
            for (int kp = 0; kp <= j; ++kp) {
                const int e0 = j * j + (kp == 0 ? 0 : 2 * kp - 1);
                ua[e0] *= g.k.jB[j][kp];
                if (kp) ua[e0 + 1] *= g.k.jB[j][kp];
            }
        }
        const double Aa = g.k.A[la][ma < 0 ? -ma : ma] * sgn_b;
        for (int mb = -lb; mb <= lb; ++mb) {
            // Q_j[ma][mb] for j = 0..J-1 (block j holds the 2j+1 entries e = j^2 .. j^2+2j)
            double Q[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                double s = 0.0;
#pragma unroll
                for (int e = j * j; e < (j + 1) * (j + 1); ++e) s = fma(ua[e], Wb[mb + lb][e], s);
                Q[j] = s;
            }
            const double aa = Aa * g.k.A[lb][mb < 0 ? -mb : mb];
            const long long idx = o + (ma + la) * nb + (mb + lb);
#define SHG_FUSED_STORE(OPID, ARR)                                          \
    if (g.out[OPID]) {                                                      \
        double s = 0.0;                                                     \
        _Pragma("unroll") for (int j = 0; j < J; ++j) s = fma(ARR[j], Q[j], s); \
        g.out[OPID][idx] = aa * s;                                          \
    }
            SHG_FUSED_STORE(OP_OVERLAP, Oov)
            SHG_FUSED_STORE(OP_COULOMB, Oco)
            SHG_FUSED_STORE(OP_ERFC, Ox)
            SHG_FUSED_STORE(OP_ERF, Oer)
            SHG_FUSED_STORE(OP_GAUSS, Oga)
#undef SHG_FUSED_STORE
        }
    }
}

__device__ __forceinline__ void run_tile_fused(const ArgsFused &g, const Tile &t, int lane)
{
    if (lane >= t.count) return;
    const int p = g.perm[t.start + lane];
    const int la = t.cls / (kLmax2c + 1), lb = t.cls % (kLmax2c + 1);
    switch ((la < lb ? la : lb) + 1) {
    case 1: pair_2c_fused<1>(g, p); break;
    case 2: pair_2c_fused<2>(g, p); break;
    case 3: pair_2c_fused<3>(g, p); break;
    case 4: pair_2c_fused<4>(g, p); break;
    case 5: pair_2c_fused<5>(g, p); break;
    case 6: pair_2c_fused<6>(g, p); break;
    default: pair_2c_fused<7>(g, p); break;
    }
}

// MinB: CTAs of 128 threads that must fit on an SM (a register cap: 1 leaves the
// compiler's allocation, 3 caps at 170 registers, 4 at 128)
template <int MinB>
__global__ void __launch_bounds__(128, MinB) k_2c_fp64_fused_persistent(const ArgsFused g)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(g.counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0) + g.tile_begin;
        if (t >= g.tile_end) break;
        run_tile_fused(g, g.tiles[t], lane);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(128) k_2c_fp64_fused_static(const ArgsFused g)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int t = g.tile_begin + warp;
    if (t >= g.tile_end) return;
    run_tile_fused(g, g.tiles[t], lane);
}

}  // namespace

cudaError_t launch_2c_fused(const ArgsFused &a, int n_tiles_or_grid, bool persistent, cudaStream_t s, int threads,
                            int variant)
{
    if (persistent) {
        switch (variant) {
        case 1: k_2c_fp64_fused_persistent<3><<<n_tiles_or_grid, threads, 0, s>>>(a); break;
        case 2: k_2c_fp64_fused_persistent<4><<<n_tiles_or_grid, threads, 0, s>>>(a); break;
        default: k_2c_fp64_fused_persistent<1><<<n_tiles_or_grid, threads, 0, s>>>(a); break;
        }
    } else {
        const int tiles = a.tile_end - a.tile_begin;
        if (tiles <= 0) return cudaSuccess;
        const int wpb = threads / 32;
        k_2c_fp64_fused_static<<<(tiles + wpb - 1) / wpb, threads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

int persistent_grid_2c_fused(int threads, int ctas_per_sm, int variant)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e;
    switch (variant) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_fp64_fused_persistent<3>, threads, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_fp64_fused_persistent<4>, threads, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_fp64_fused_persistent<1>, threads, 0); break;
    }
    if (e != cudaSuccess || per < 1) per = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per) per = ctas_per_sm;
    return (sms > 0 ? sms : 1) * per;
}

}  // namespace shg
