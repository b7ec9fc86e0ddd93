// CUDA kernels of the SHG integral library (sm_103a), FP64 two-center path,
// planning kernels, Boys debug kernel and the ALU throughput probe.
//
// Two-center integrals follow Sec. II B of Golze et al. (arXiv:1701.06588):
//   (a|O|b) = (-1)^lb A_{la,ma} A_{lb,mb} sum_j 2^{la+lb-j} O^{(la+lb-j)}
//             (2j-1)!! sum_kappa B_{j,kappa} Q^{c/s,c/s}_{la,|ma|,lb,|mb|,j,kappa}
// with Q = W_a W_b^T (Eq. Q_matrix), W built from the regular scaled solid
// harmonics R^{c/s}_{l,m} of the vector R_a - R_b (Sec. II E), and
// O^{(k)} = sum_{alpha,beta} w_alpha w_beta (d/dR^2)^k (0_a|O|0_b)  (Eq. O_rab2_deriv,
// Table S1).
//
// Work mapping: one thread evaluates one shell pair (radial terms of every
// primitive pair in registers, then the (2la+1)(2lb+1) block); a warp owns a
// tile of up to 32 pairs of one (la, lb) class with similar Ka*Kb, so the
// lanes run the same loop trip counts.

#include "shg_device.cuh"

#include <cstdio>

namespace shg {

namespace {
using namespace dev;

// ------------------------------------------------------------------------- //
// One shell pair, FP64.                                                     //
// ------------------------------------------------------------------------- //
template <int OP, int J>
__device__ void pair_2c_fp64(const Args2c &g, int p)
{
    const ShellRec sa = g.shells[g.pair_a[p]];
    const ShellRec sb = g.shells[g.pair_b[p]];
    const int la = sa.l, lb = sb.l;
    const Vec4 A = g.centers[sa.center];
    const Vec4 B = g.centers[sb.center];
    const double vx = A.x - B.x, vy = A.y - B.y, vz = A.z - B.z;
    const double R2 = vx * vx + vy * vy + vz * vz;
    const int kmax = la + lb;
    if ((OP == OP_OVERLAP || OP == OP_GAUSS) && g.screen_thresh > 0.0 &&
        screen_bound(g.screen[g.pair_a[p]], g.screen[g.pair_b[p]], R2, OP, g.omega) < g.screen_thresh) {
        double *o = g.out + g.out_off[p];
        for (int i = 0; i < (2 * la + 1) * (2 * lb + 1); ++i) o[i] = 0.0;
        return;
    }

    double O[J], E[J];
#pragma unroll
    for (int j = 0; j < J; ++j) O[j] = E[j] = 0.0;
    if (OP == OP_PRE) {
#pragma unroll
        for (int j = 0; j < J; ++j) O[j] = g.o_pre[(int64_t)p * kJmax + j];
    } else {
        // one flat loop over the Ka*Kb primitive pairs: a tile holds one class's
        // pairs in descending Ka*Kb, so the lanes' trip counts differ only where
        // a tile straddles two Ka*Kb values
        const int Kb = sb.nprim, npp = sa.nprim * Kb;
        for (int q = 0; q < npp; ++q) {
            const int ia = q / Kb, ib = q - ia * Kb;
            radial_acc_fp64<OP, J>(g.prims[sa.prim_off + ia], g.prims[sb.prim_off + ib], R2, kmax, la, g, O, E);
        }
        radial_finish_fp64<OP, J>(R2, kmax, g.k, O, E);
    }

    // g_e = 2^{kmax-j} (2j-1)!! B_{j,kappa} O^{(kmax-j)}, shared by z = c, s
    double ge[J * J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const double oj = O[j] * g.k.pow2[kmax - j];
#pragma unroll
        for (int kp = 0; kp <= j; ++kp) {
            const double v = oj * g.k.jB[j][kp];
            const int e0 = j * j + (kp == 0 ? 0 : 2 * kp - 1);
            ge[e0] = v;
            if (kp) ge[e0 + 1] = v;
        }
    }

    double Rc[(kLmax2c + 1) * (kLmax2c + 2) / 2], Rs[(kLmax2c + 1) * (kLmax2c + 2) / 2];
    scaled_harmonics(vx, vy, vz, la > lb ? la : lb, g.k, Rc, Rs);

    const int nb = 2 * lb + 1;
    double Ub[2 * kLmax2c + 1][J * J];
    for (int mb = -lb; mb <= lb; ++mb) {
        double w[J * J];
        w_row<J>(Rc, Rs, lb, mb, w);
#pragma unroll
        for (int e = 0; e < J * J; ++e) Ub[mb + lb][e] = w[e];
    }
    const double sgn_b = (lb & 1) ? -1.0 : 1.0;
    double *out = g.out + g.out_off[p];
    for (int ma = -la; ma <= la; ++ma) {
        double ua[J * J];
        w_row<J>(Rc, Rs, la, ma, ua);
#pragma unroll
        for (int e = 0; e < J * J; ++e) ua[e] *= ge[e];
        const double Aa = g.k.A[la][ma < 0 ? -ma : ma] * sgn_b;
        for (int mb = -lb; mb <= lb; ++mb) {
            double s = 0.0;
#pragma unroll
            for (int e = 0; e < J * J; ++e) s = fma(ua[e], Ub[mb + lb][e], s);
            out[(ma + la) * nb + (mb + lb)] = Aa * (g.k.A[lb][mb < 0 ? -mb : mb] * s);
        }
    }
}

// ------------------------------------------------------------------------- //
// (a|r_a^{2n}|b) in double-double (Sec. II C, Eqs. ara2nb and T_rab2_deriv). //
// Its radial orders grow like (beta^2 R^2 / c)^n while the block does not:  //
// the sum over j of Eq. final_r12int_ab cancels by up to ~1e8 at n = 5 for a //
// diffuse a and a tight b, so every term of it must carry ~1e-20 relative   //
// precision: the contracted orders, the harmonics of the (exact) separation,//
// the W rows, the (2j-1)!! B weights and the block sums run in double-      //
// double.  Factors common to all orders of one primitive pair (weights,     //
// exp(-rho R^2)) and to a whole block (A_{l,m}) stay FP64: their rounding   //
// scales a term of the sum as a whole and does not survive the cancellation.//
// ------------------------------------------------------------------------- //
__device__ __forceinline__ ddv dd_const(double h, double l) { return ddv{h, l}; }

__device__ __forceinline__ ddv rcd_get(const ddv *Rc, int L, int m)
{
    const int am = m < 0 ? -m : m;
    if (L < 0 || am > L) return ddv{0.0, 0.0};
    const ddv v = Rc[L * (L + 1) / 2 + am];
    return (m < 0 && (am & 1)) ? dd_neg(v) : v;
}
__device__ __forceinline__ ddv rsd_get(const ddv *Rs, int L, int m)
{
    const int am = m < 0 ? -m : m;
    if (L < 0 || am > L) return ddv{0.0, 0.0};
    const ddv v = Rs[L * (L + 1) / 2 + am];
    return (m < 0 && !(am & 1)) ? dd_neg(v) : v;
}

// scaled_harmonics with double-double arithmetic and constants
__device__ void scaled_harmonics_dd(ddv x, ddv y, ddv z, int lmax, const Consts &k, ddv *Rc, ddv *Rs)
{
    const ddv r2 = dd_add(dd_add(dd_mul(x, x), dd_mul(y, y)), dd_mul(z, z));
    Rc[0] = ddv{1.0, 0.0};
    Rs[0] = ddv{0.0, 0.0};
    for (int l = 0; l < lmax; ++l) {
        const int d0 = l * (l + 1) / 2, d1 = (l + 1) * (l + 2) / 2, dm = (l - 1) * l / 2;
        const ddv cll = Rc[d0 + l], sll = Rs[d0 + l];
        const ddv inv = dd_const(k.inv_int[2 * l + 2], k.inv_int_lo[2 * l + 2]);
        Rc[d1 + l + 1] = dd_neg(dd_mul(dd_sub(dd_mul(x, cll), dd_mul(y, sll)), inv));
        Rs[d1 + l + 1] = dd_neg(dd_mul(dd_add(dd_mul(y, cll), dd_mul(x, sll)), inv));
        const ddv zl = dd_mul_d(z, k.dint[2 * l + 1]);
        for (int m = 0; m <= l; ++m) {
            const int q = (l + m + 1) * (l - m + 1);
            const ddv im = dd_const(k.inv_int[q], k.inv_int_lo[q]);
            ddv vc = dd_mul(zl, Rc[d0 + m]);
            if (m <= l - 1) vc = dd_sub(vc, dd_mul(r2, Rc[dm + m]));
            Rc[d1 + m] = dd_mul(vc, im);
            if (m == 0) {
                Rs[d1] = ddv{0.0, 0.0};
            } else {
                ddv vs = dd_mul(zl, Rs[d0 + m]);
                if (m <= l - 1) vs = dd_sub(vs, dd_mul(r2, Rs[dm + m]));
                Rs[d1 + m] = dd_mul(vs, im);
            }
        }
    }
}

template <int J>
__device__ __forceinline__ void w_row_dd(const ddv *Rc, const ddv *Rs, int l, int m, ddv (&w)[J * J])
{
    const int mu = m < 0 ? -m : m;
    const bool sine = m < 0;
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int L = l - j;
        w[j * j] = sine ? rsd_get(Rs, L, mu) : rcd_get(Rc, L, mu);
#pragma unroll
        for (int kp = 1; kp <= j; ++kp) {
            const int e0 = j * j + 2 * kp - 1;
            const ddv cm = rcd_get(Rc, L, mu - kp), cp = rcd_get(Rc, L, mu + kp);
            const ddv sm = rsd_get(Rs, L, mu - kp), sp = rsd_get(Rs, L, mu + kp);
            const bool odd = kp & 1;
            if (!sine) {
                w[e0] = odd ? dd_sub(cm, cp) : dd_add(cm, cp);
                w[e0 + 1] = odd ? dd_neg(dd_add(sm, sp)) : dd_sub(sp, sm);
            } else {
                w[e0] = odd ? dd_sub(sm, sp) : dd_add(sm, sp);
                w[e0 + 1] = odd ? dd_add(cm, cp) : dd_sub(cm, cp);
            }
        }
    }
}

// Radial orders of one primitive pair, accumulated in double-double into
// O[j] = O^{(kmax-j)} (the FP64 radial_acc_fp64<OP_RA2N> with the Horner
// variable R^2 and the accumulation kept in double-double).
template <int J>
__device__ __forceinline__ void radial_ra2n_dd(const PrimRec &pa, const PrimRec &pb, ddv R2d, int kmax, int la,
                                               const Args2c &g, ddv (&O)[J])
{
    const int kmin = kmax - J + 1;
    const double w = pa.w2c * pb.w2c;
    const double c = pa.alpha + pb.alpha;
    const double rc = rsqrt(c);
    const double ic = rc * rc;
    const double rho = pa.alpha * pb.alpha * ic;
    const double T = rho * R2d.h;
    const int n = __double2int_rn(g.omega);
    const ddv cc = dd_sum(pa.alpha, pb.alpha);
    const ddv icd = dd_inv(cc);
    const ddv rhod = dd_mul(dd_prod(pa.alpha, pb.alpha), icd);
    const ddv bcd = dd_mul(dd_prod(pb.alpha, pb.alpha), icd);
    const ddv iad = dd_inv(ddv{pa.alpha, 0.0});
    ddv tm[kRa2nMax + 1];
#pragma unroll
    for (int m = 0; m <= kRa2nMax; ++m) {
        tm[m] = ddv{0.0, 0.0};
        if (m <= n) {
            const int j = n - m;
            double rf = g.k.binom[n][j];                 // C(n, j) (la)_j: exact integer
            for (int i = 0; i < j; ++i) rf *= (double)(la + i);
            ddv t = ddv{rf, 0.0};
            for (int i = 0; i < j; ++i) t = dd_mul(t, iad);
            for (int i = 0; i < m; ++i) t = dd_mul(t, icd);
            tm[m] = t;
        }
    }
    ddv q[kRa2nMax + 2];
    ddv bd = ddv{1.0, 0.0};
#pragma unroll
    for (int d = 0; d <= kRa2nMax; ++d) {
        ddv sum = ddv{0.0, 0.0};
#pragma unroll
        for (int m = d; m <= kRa2nMax; ++m) sum = dd_add(sum, dd_mul_d(tm[m], g.k.ra2n_k[m][d]));
        q[d] = dd_mul(bd, sum);
        bd = dd_mul(bd, bcd);
    }
    q[kRa2nMax + 1] = ddv{0.0, 0.0};
    const ddv mrho = dd_neg(rhod);
    for (int k = 0; k < kmin; ++k) {
#pragma unroll
        for (int d = 0; d <= kRa2nMax; ++d) q[d] = dd_add(dd_mul_d(q[d + 1], (double)(d + 1)), dd_mul(mrho, q[d]));
    }
    // common factor of every order of this primitive pair (FP64: it scales each
    // pair's term of the final sum as a whole)
    const double we = w * kPi32 * ic * rc * exp(-T);
#pragma unroll
    for (int t = 0; t < J; ++t) {
        ddv val = q[kRa2nMax];
#pragma unroll
        for (int d = kRa2nMax - 1; d >= 0; --d) val = dd_add(dd_mul(val, R2d), q[d]);
        O[J - 1 - t] = dd_add(O[J - 1 - t], dd_mul_d(val, we));
        if (t + 1 < J) {
#pragma unroll
            for (int d = 0; d <= kRa2nMax; ++d)
                q[d] = dd_add(dd_mul_d(q[d + 1], (double)(d + 1)), dd_mul(mrho, q[d]));
        }
    }
}

template <int J>
__device__ void pair_2c_ra2n_dd(const Args2c &g, int p)
{
    const ShellRec sa = g.shells[g.pair_a[p]];
    const ShellRec sb = g.shells[g.pair_b[p]];
    const int la = sa.l, lb = sb.l;
    const Vec4 A = g.centers[sa.center];
    const Vec4 B = g.centers[sb.center];
    // the separation exactly (TwoSum) and R^2 in double-double
    const ddv vx = dd_sum(A.x, -B.x), vy = dd_sum(A.y, -B.y), vz = dd_sum(A.z, -B.z);
    const ddv R2d = dd_add(dd_add(dd_mul(vx, vx), dd_mul(vy, vy)), dd_mul(vz, vz));
    const int kmax = la + lb;
    ddv O[J];
#pragma unroll
    for (int j = 0; j < J; ++j) O[j] = ddv{0.0, 0.0};
    const int Kb = sb.nprim, npp = sa.nprim * Kb;
    for (int q = 0; q < npp; ++q) {
        const int ia = q / Kb, ib = q - ia * Kb;
        radial_ra2n_dd<J>(g.prims[sa.prim_off + ia], g.prims[sb.prim_off + ib], R2d, kmax, la, g, O);
    }
    // g_e = 2^{kmax-j} (2j-1)!! B_{j,kappa} O^{(kmax-j)}
    ddv ge[J * J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const ddv oj = ddv{O[j].h * g.k.pow2[kmax - j], O[j].l * g.k.pow2[kmax - j]};
#pragma unroll
        for (int kp = 0; kp <= j; ++kp) {
            const ddv v = dd_mul(oj, dd_const(g.k.jB[j][kp], g.k.jB_lo[j][kp]));
            const int e0 = j * j + (kp == 0 ? 0 : 2 * kp - 1);
            ge[e0] = v;
            if (kp) ge[e0 + 1] = v;
        }
    }
    ddv Rc[(kLmax2c + 1) * (kLmax2c + 2) / 2], Rs[(kLmax2c + 1) * (kLmax2c + 2) / 2];
    scaled_harmonics_dd(vx, vy, vz, la > lb ? la : lb, g.k, Rc, Rs);
    const int nb = 2 * lb + 1;
    ddv Ub[2 * kLmax2c + 1][J * J];
    for (int mb = -lb; mb <= lb; ++mb) {
        ddv w[J * J];
        w_row_dd<J>(Rc, Rs, lb, mb, w);
#pragma unroll
        for (int e = 0; e < J * J; ++e) Ub[mb + lb][e] = w[e];
    }
    const double sgn_b = (lb & 1) ? -1.0 : 1.0;
    double *out = g.out + g.out_off[p];
    for (int ma = -la; ma <= la; ++ma) {
        ddv ua[J * J];
        w_row_dd<J>(Rc, Rs, la, ma, ua);
#pragma unroll
        for (int e = 0; e < J * J; ++e) ua[e] = dd_mul(ua[e], ge[e]);
        const double Aa = g.k.A[la][ma < 0 ? -ma : ma] * sgn_b;
        for (int mb = -lb; mb <= lb; ++mb) {
            ddv s = ddv{0.0, 0.0};
#pragma unroll
            for (int e = 0; e < J * J; ++e) s = dd_fma(ua[e], Ub[mb + lb][e], s);
            out[(ma + la) * nb + (mb + lb)] = Aa * (g.k.A[lb][mb < 0 ? -mb : mb] * (s.h + s.l));
        }
    }
}

template <int OP>
__device__ __forceinline__ void pair_2c_fp64_dispatch(const Args2c &g, int p, int J)
{
    if (OP == OP_RA2N) {
        switch (J) {
        case 1: pair_2c_ra2n_dd<1>(g, p); return;
        case 2: pair_2c_ra2n_dd<2>(g, p); return;
        case 3: pair_2c_ra2n_dd<3>(g, p); return;
        case 4: pair_2c_ra2n_dd<4>(g, p); return;
        case 5: pair_2c_ra2n_dd<5>(g, p); return;
        case 6: pair_2c_ra2n_dd<6>(g, p); return;
        default: pair_2c_ra2n_dd<7>(g, p); return;
        }
    }
    switch (J) {
    case 1: pair_2c_fp64<OP, 1>(g, p); break;
    case 2: pair_2c_fp64<OP, 2>(g, p); break;
    case 3: pair_2c_fp64<OP, 3>(g, p); break;
    case 4: pair_2c_fp64<OP, 4>(g, p); break;
    case 5: pair_2c_fp64<OP, 5>(g, p); break;
    case 6: pair_2c_fp64<OP, 6>(g, p); break;
    default: pair_2c_fp64<OP, 7>(g, p); break;
    }
}

__device__ __forceinline__ void run_tile_fp64(const Args2c &g, int op, const Tile &t, int lane)
{
    if (lane >= t.count) return;
    const int p = g.perm[t.start + lane];
    const int la = t.cls / (kLmax2c + 1), lb = t.cls % (kLmax2c + 1);
    const int J = (la < lb ? la : lb) + 1;
    switch (op) {
    case OP_OVERLAP: pair_2c_fp64_dispatch<OP_OVERLAP>(g, p, J); break;
    case OP_COULOMB: pair_2c_fp64_dispatch<OP_COULOMB>(g, p, J); break;
    case OP_ERFC: pair_2c_fp64_dispatch<OP_ERFC>(g, p, J); break;
    case OP_ERF: pair_2c_fp64_dispatch<OP_ERF>(g, p, J); break;
    case OP_GAUSS: pair_2c_fp64_dispatch<OP_GAUSS>(g, p, J); break;
    case OP_GCOUL: pair_2c_fp64_dispatch<OP_GCOUL>(g, p, J); break;
    case OP_RA2N: pair_2c_fp64_dispatch<OP_RA2N>(g, p, J); break;
    default: pair_2c_fp64_dispatch<OP_PRE>(g, p, J); break;
    }
}

template <int OP>
__global__ void __launch_bounds__(128) k_2c_fp64_static(const Args2c g)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int t = g.tile_begin + warp;
    if (t >= g.tile_end) return;
    run_tile_fp64(g, OP, g.tiles[t], lane);
}

template <int OP>
__global__ void __launch_bounds__(128) k_2c_fp64_persistent(const Args2c g)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(g.counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0) + g.tile_begin;
        if (t >= g.tile_end) break;
        run_tile_fp64(g, OP, g.tiles[t], lane);
        __syncwarp();
    }
}

// ------------------------------------------------------------------------- //
// Planning: counting sort of pairs into (class, Ka*Kb) bins, bins visited in //
// a schedule-specific rank order, then class-pure tiles of <= 32 pairs.     //
// ------------------------------------------------------------------------- //
__global__ void k_classify(int64_t n, const int32_t *__restrict__ pa, const int32_t *__restrict__ pb,
                           const ShellRec *__restrict__ shells, int n_shells, const int *__restrict__ bin_rank,
                           int *__restrict__ key, int *__restrict__ hist, int *__restrict__ err)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int a = pa[p], b = pb[p];
        int r = 0;
        if (a < 0 || a >= n_shells || b < 0 || b >= n_shells) {
            atomicOr(err, 1);
        } else {
            const ShellRec sa = shells[a], sb = shells[b];
            const int cls = sa.l * (kLmax2c + 1) + sb.l;
            const int kk = sa.nprim * sb.nprim;
            r = bin_rank[cls * kKbins2c + (kk - 1)];
        }
        key[p] = r;
        atomicAdd(hist + r, 1);
    }
}

__global__ void k_classify_3c(int64_t n, const int32_t *__restrict__ ta, const int32_t *__restrict__ tt,
                              const int32_t *__restrict__ tb, const ShellRec *__restrict__ orb, int n_orb,
                              const ShellRec *__restrict__ aux, int n_aux, const int *__restrict__ bin_rank,
                              int *__restrict__ key, int *__restrict__ hist, int *__restrict__ err)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int a = ta[p], t = tt[p], b = tb[p];
        int r = 0;
        if (a < 0 || a >= n_orb || t < 0 || t >= n_orb || b < 0 || b >= n_aux) {
            atomicOr(err, 1);
        } else {
            const ShellRec sa = orb[a], st = orb[t], sb = aux[b];
            if (sa.center != st.center) atomicOr(err, 2);
            if (sa.l + st.l > kLmaxAabA) atomicOr(err, 4);
            const int cls = (sa.l * 7 + st.l) * 7 + sb.l;
            int kk = sa.nprim * st.nprim * sb.nprim;
            kk = kk < kKbins3c ? kk : kKbins3c;
            r = bin_rank[cls * kKbins3c + (kk - 1)];
        }
        key[p] = r;
        atomicAdd(hist + r, 1);
    }
}

// Exclusive prefix sums over the bins in rank order, one block per chunk of
// `chunk` consecutive ranks (blockDim.x == chunk <= 1024).  Both planners'
// rank orders are class-major, and a chunk is the bins of one class: tiles
// are cut per chunk, so each class ends in one partial tile.
//   cursor[r]            offset of bin r inside its chunk (the scatter cursor)
//   bin_start[c*chunk]   first pair of chunk c
//   tile_start[c*chunk]  first tile of chunk c; tile_start[n_bins] = all tiles
// Every block scans its own chunk and posts the chunk's count; the last block
// to finish (an atomic ticket, *ticket zero on entry) scans the counts.  No
// block waits for another.
__device__ __forceinline__ int block_incl_scan(int x, int *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const int r = x + (warp ? s_warp[warp - 1] : 0);
    __syncthreads();   // s_warp free for the next scan
    return r;
}

__global__ void __launch_bounds__(1024) k_scan_chunks(int n_bins, int chunk, const int *__restrict__ hist,
                                                      int *__restrict__ bin_start, int *__restrict__ cursor,
                                                      int *__restrict__ tile_start, int *ticket,
                                                      int *__restrict__ summary, const int *err)
{
    __shared__ int s_warp[32];
    __shared__ int s_last;
    const int c = blockIdx.x;
    const int r = c * chunk + threadIdx.x;
    const int v = hist[r];
    const int incl = block_incl_scan(v, s_warp);
    cursor[r] = incl - v;
    if (threadIdx.x == blockDim.x - 1) {
        bin_start[c * chunk] = incl;                  // the chunk's count for now
        __threadfence();
        s_last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last block: offsets of the chunks (gridDim.x <= blockDim.x chunks, one per thread)
    const int k = threadIdx.x;
    const int cnt = k < (int)gridDim.x ? __ldcg(bin_start + k * chunk) : 0;
    const int til = (cnt + kTile - 1) / kTile;
    const int ic = block_incl_scan(cnt, s_warp);
    const int it = block_incl_scan(til, s_warp);
    if (k < (int)gridDim.x) {
        bin_start[k * chunk] = ic - cnt;
        tile_start[k * chunk] = it - til;
        summary[k] = it - til;
    }
    if (k == (int)gridDim.x - 1) {
        tile_start[n_bins] = it;
        summary[k + 1] = it;
        summary[k + 2] = __ldcg(err);
        *ticket = 0;
    }
}

__global__ void k_scatter(int64_t n, int chunk, const int *__restrict__ key, const int *__restrict__ bin_start,
                          int *__restrict__ cursor, int32_t *__restrict__ perm)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int r = key[p];
        const int pos = bin_start[r - r % chunk] + atomicAdd(cursor + r, 1);
        perm[pos] = (int32_t)p;
    }
}

// One thread per tile: the tile's chunk by bisection over the chunks' first tiles.
__global__ void k_make_tiles(int n_chunks, int chunk, int bins_per_class, int n_pairs, const int *__restrict__ bin_start,
                             const int *__restrict__ tile_start, const int *__restrict__ rank_to_bin,
                             Tile *__restrict__ tiles)
{
    const int total = tile_start[n_chunks * chunk];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int lo = 0, hi = n_chunks;                    // tile_start[lo*chunk] <= t < tile_start[hi*chunk]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tile_start[mid * chunk] <= t) lo = mid;
            else hi = mid;
        }
        const int first = bin_start[lo * chunk] + (t - tile_start[lo * chunk]) * kTile;
        const int end = lo + 1 < n_chunks ? bin_start[(lo + 1) * chunk] : n_pairs;
        Tile tl;
        tl.start = first;
        tl.count = end - first < kTile ? end - first : kTile;
        tl.cls = rank_to_bin[lo * chunk] / bins_per_class;
        tl.pad = 0;
        tiles[t] = tl;
    }
}

// ------------------------------------------------------------------------- //
// Debug: Boys values through the device code path.                          //
// ------------------------------------------------------------------------- //
__global__ void k_debug_boys(int64_t n, const double *__restrict__ T, int nmax, double *__restrict__ F,
                             const double *tab, const double *etab, const Consts k)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double f[kBoysN];
        boys_top<kBoysN>(T[i], kBoysN - 1, tab, etab, k, f);
        for (int m = 0; m <= nmax; ++m) F[i * (nmax + 1) + m] = f[kBoysN - 1 - m];
    }
}

// ------------------------------------------------------------------------- //
// Center packing for shg_basis_set_centers: FP64 Vec4 and the double-float   //
// split (hi = nearest float, lo = nearest float of the exact remainder).     //
// ------------------------------------------------------------------------- //
__device__ __forceinline__ float2 split_df(double v)
{
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}

__global__ void k_pack_centers(const double *__restrict__ raw, int n, Vec4 *__restrict__ ctr,
                               MixCenter *__restrict__ mctr, int *bad)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const double x = raw[3 * c], y = raw[3 * c + 1], z = raw[3 * c + 2];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicMin(bad, c);
        ctr[c] = Vec4{x, y, z, 0.0};
        mctr[c] = MixCenter{split_df(x), split_df(y), split_df(z), make_float2(0.f, 0.f)};
    }
}

// ------------------------------------------------------------------------- //
// ALU throughput probe: 8 independent FMA chains per thread.                //
// ------------------------------------------------------------------------- //
template <typename T>
__global__ void __launch_bounds__(256) k_alu_probe(int iters, T *sink)
{
    T a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
    const T b = (T)0.999999, c = (T)1e-6;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == (T)-12345.0) sink[0] = s;
}

// FP64 tensor-core probe: 8 independent chains of mma.sync m8n8k4 (FP64 in,
// FP64 accumulate) per warp; 2*8*8*4 = 512 flops per warp instruction.
__global__ void __launch_bounds__(256) k_dmma_probe(int iters, double *sink)
{
    const double a = 1e-3 * (double)((threadIdx.x & 31) + 1), b = 0.999;
    double c0[8], c1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) c0[i] = c1[i] = 1e-3 * (double)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c0[i]), "+d"(c1[i])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += c0[i] + c1[i];
    if (s == -12345.0) sink[0] = s;
}

}  // namespace

// ------------------------------------------------------------------------- //
// Launchers                                                                 //
// ------------------------------------------------------------------------- //
cudaError_t launch_plan_build(PlanDev &plan, int *d_ws, int n_bins, const int *d_bin_rank, cudaStream_t s)
{
    // d_ws layout (plan_ws_ints): err | ticket | 2 spare | hist[n_bins] | bin_start[n_bins] | cursor[n_bins] |
    // tile_start[n_bins+1] | summary[n_chunks+2] | key[n]; one memset clears err, ticket and hist.
    // d_bin_rank: bin_rank[n_bins] followed by rank_to_bin[n_bins]
    const int64_t n = plan.n_pairs;
    int *d_err = d_ws;
    int *ticket = d_ws + 1;
    int *hist = d_ws + 4;
    int *bin_start = hist + n_bins;
    int *cursor = bin_start + n_bins;
    int *tile_start = cursor + n_bins;
    const int bpc = plan.kind == 2 ? kKbins2c : kKbins3c;
    const int n_chunks = n_bins / bpc;
    int *summary = tile_start + n_bins + 1;
    int *key = summary + n_chunks + 2;
    cudaError_t e = cudaMemsetAsync(d_ws, 0, sizeof(int) * (4 + (size_t)n_bins), s);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const int blocks = (int)((n + threads - 1) / threads < 4096 ? (n + threads - 1) / threads : 4096);
    if (n > 0 && plan.kind == 2) {
        k_classify<<<blocks, threads, 0, s>>>(n, plan.pair_a, plan.pair_b, plan.basis->shells, plan.basis->n_shells,
                                              d_bin_rank, key, hist, d_err);
    } else if (n > 0) {
        k_classify_3c<<<blocks, threads, 0, s>>>(n, plan.pair_a, plan.trip_t, plan.pair_b, plan.basis->shells,
                                                 plan.basis->n_shells, plan.aux->shells, plan.aux->n_shells,
                                                 d_bin_rank, key, hist, d_err);
    }
    // both rank orders are class-major (each class a chunk of bins_per_class ranks): one tiling per class
    k_scan_chunks<<<n_chunks, bpc, 0, s>>>(n_bins, bpc, hist, bin_start, cursor, tile_start, ticket, summary, d_err);
    if (n > 0) k_scatter<<<blocks, threads, 0, s>>>(n, bpc, key, bin_start, cursor, plan.perm);
    const int64_t max_tiles = n / kTile + n_chunks + 1;
    const int tb = (int)((max_tiles + 255) / 256 < 1024 ? (max_tiles + 255) / 256 : 1024);
    k_make_tiles<<<tb, 256, 0, s>>>(n_chunks, bpc, bpc, (int)n, bin_start, tile_start, d_bin_rank + n_bins,
                                    plan.tiles);
    return cudaGetLastError();
}

template <int OP>
static cudaError_t launch_2c_op(const Args2c &a, int n, int threads, bool persistent, cudaStream_t s)
{
    if (persistent) {
        k_2c_fp64_persistent<OP><<<n, threads, 0, s>>>(a);
    } else {
        const int tiles = a.tile_end - a.tile_begin;
        if (tiles <= 0) return cudaSuccess;
        const int wpb = threads / 32;
        k_2c_fp64_static<OP><<<(tiles + wpb - 1) / wpb, threads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_2c(const Args2c &a, int op, int precision, int n, bool persistent, cudaStream_t s, int threads)
{
    (void)precision;
    switch (op) {
    case OP_OVERLAP: return launch_2c_op<OP_OVERLAP>(a, n, threads, persistent, s);
    case OP_COULOMB: return launch_2c_op<OP_COULOMB>(a, n, threads, persistent, s);
    case OP_ERFC: return launch_2c_op<OP_ERFC>(a, n, threads, persistent, s);
    case OP_ERF: return launch_2c_op<OP_ERF>(a, n, threads, persistent, s);
    case OP_GAUSS: return launch_2c_op<OP_GAUSS>(a, n, threads, persistent, s);
    case OP_GCOUL: return launch_2c_op<OP_GCOUL>(a, n, threads, persistent, s);
    case OP_RA2N: return launch_2c_op<OP_RA2N>(a, n, threads, persistent, s);
    case OP_PRE: return launch_2c_op<OP_PRE>(a, n, threads, persistent, s);
    default: return cudaErrorInvalidValue;
    }
}

int persistent_grid_2c(int op, int precision, int threads, int ctas_per_sm)
{
    (void)precision;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaSuccess;
    switch (op) {
    case OP_OVERLAP: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_fp64_persistent<OP_OVERLAP>, threads, 0); break;
    case OP_COULOMB: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_fp64_persistent<OP_COULOMB>, threads, 0); break;
    case OP_ERFC: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_fp64_persistent<OP_ERFC>, threads, 0); break;
    case OP_ERF: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_fp64_persistent<OP_ERF>, threads, 0); break;
    case OP_GAUSS: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_fp64_persistent<OP_GAUSS>, threads, 0); break;
    case OP_GCOUL: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_fp64_persistent<OP_GCOUL>, threads, 0); break;
    case OP_RA2N: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_fp64_persistent<OP_RA2N>, threads, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_2c_fp64_persistent<OP_PRE>, threads, 0); break;
    }
    if (e != cudaSuccess || per < 1) per = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per) per = ctas_per_sm;
    if (sms < 1) sms = 1;
    return sms * per;
}

cudaError_t launch_pack_centers(const double *raw, int n, Vec4 *ctr, MixCenter *mctr, int *bad, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int blocks = (n + 255) / 256 < 1216 ? (n + 255) / 256 : 1216;
    k_pack_centers<<<blocks, 256, 0, s>>>(raw, n, ctr, mctr, bad);
    return cudaGetLastError();
}

cudaError_t launch_debug_boys(int64_t n, const double *T, int nmax, double *F, const DeviceTables &t, cudaStream_t s)
{
    Consts k;
    fill_consts(k);
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)((n + 127) / 128 < 4096 ? (n + 127) / 128 : 4096);
    k_debug_boys<<<blocks, 128, 0, s>>>(n, T, nmax, F, t.boys, t.boys_e, k);
    return cudaGetLastError();
}

cudaError_t launch_alu_probe(int kind, int iters, int blocks, int threads, double *sink, cudaStream_t s)
{
    if (kind == 0)
        k_alu_probe<double><<<blocks, threads, 0, s>>>(iters, sink);
    else if (kind == 1)
        k_alu_probe<float><<<blocks, threads, 0, s>>>(iters, reinterpret_cast<float *>(sink));
    else
        k_dmma_probe<<<blocks, threads, 0, s>>>(iters, sink);
    return cudaGetLastError();
}

}  // namespace shg
