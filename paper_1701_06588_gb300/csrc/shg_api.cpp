// Host side of the SHG integral library: C ABI, input validation, shell
// normalisation, device tables, planning and kernel dispatch.
#include "../../include/shg.h"
#include "shg_internal.h"

#include <algorithm>
#include <string>
#include <unordered_map>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

namespace shg {

// NVTX range around one phase of a call (plan, exec, copies), visible to
// profilers that trace NVTX (ncu --nvtx, nsys); no cost without a tool.
struct Phase {
    explicit Phase(const char *name) { nvtxRangePushA(name); }
    ~Phase() { nvtxRangePop(); }
    Phase(const Phase &) = delete;
    Phase &operator=(const Phase &) = delete;
};

static thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

void clear_error() { g_err.clear(); }

#define SHG_CUDA(call)                                                                                    \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return fail(SHG_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                                           __FILE__, __LINE__);                                          \
    } while (0)

// ------------------------------------------------------------------------- //
// Constant tables                                                           //
// ------------------------------------------------------------------------- //
static long double lfact(int n)
{
    long double f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// Double-double arithmetic for the host precomputation (shell normalisation
// and per-primitive weights): as accurate as 80-bit long double and much
// faster than the software binary128 long double of aarch64 hosts.
struct dd {
    double hi, lo;
};
static inline dd dd_two_sum(double a, double b)
{
    const double s = a + b, bb = s - a;
    return dd{s, (a - (s - bb)) + (b - bb)};
}
static inline dd dd_norm(double h, double l) { const double s = h + l; return dd{s, l - (s - h)}; }
static inline dd dd_add(dd a, dd b)
{
    dd s = dd_two_sum(a.hi, b.hi), t = dd_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = dd_norm(s.hi, s.lo);
    s.lo += t.lo;
    return dd_norm(s.hi, s.lo);
}
static inline dd dd_mul(dd a, dd b)
{
    const double p = a.hi * b.hi;
    double e = std::fma(a.hi, b.hi, -p);
    e += a.hi * b.lo + a.lo * b.hi;
    return dd_norm(p, e);
}
static inline dd dd_div(dd a, dd b)
{
    const double q1 = a.hi / b.hi;
    const dd r = dd_add(a, dd_mul(b, dd{-q1, 0.0}));
    const double q2 = r.hi / b.hi;
    const dd r2 = dd_add(r, dd_mul(b, dd{-q2, 0.0}));
    const double q3 = r2.hi / b.hi;
    return dd_add(dd_norm(q1, q2), dd{q3, 0.0});
}
static inline dd dd_sqrt(dd a)
{
    if (!(a.hi > 0)) return dd{0.0, 0.0};
    const double x = std::sqrt(a.hi);
    const dd x2 = dd_mul(dd{x, 0.0}, dd{x, 0.0});
    const dd d = dd_add(a, dd{-x2.hi, -x2.lo});
    return dd_norm(x, d.hi / (2 * x));
}
static inline dd dd_from(long double v)
{
    const double h = (double)v;
    return dd{h, (double)(v - (long double)h)};
}

void fill_consts(Consts &k)
{
    std::memset(&k, 0, sizeof k);
    // A_{l,mu} = (-1)^mu sqrt((2 - delta_{mu,0}) (l+mu)! (l-mu)!)      Eq. (A)
    for (int l = 0; l <= kLmaxR; ++l)
        for (int mu = 0; mu <= l; ++mu) {
            long double v = std::sqrt((long double)(mu == 0 ? 1 : 2) * lfact(l + mu) * lfact(l - mu));
            k.A[l][mu] = (double)((mu & 1) ? -v : v);
        }
    // (2j-1)!! B_{j,kappa},  B_{j,kappa} = 1 / ((2 - delta_{kappa,0}) (j+kappa)! (j-kappa)!)   Eq. (B)
    for (int j = 0; j < kJmax; ++j) {
        long double df = 1;
        for (int i = 2 * j - 1; i > 1; i -= 2) df *= i;
        for (int kp = 0; kp <= j; ++kp) {
            const long double v = df / ((kp == 0 ? 1 : 2) * lfact(j + kp) * lfact(j - kp));
            k.jB[j][kp] = (double)v;
            k.jB_lo[j][kp] = (double)(v - (long double)k.jB[j][kp]);
        }
    }
    for (int i = 0; i < 32; ++i) k.pow2[i] = std::ldexp(1.0, i);
    for (int i = 0; i < 64; ++i) k.dint[i] = (double)i;
    for (int i = 1; i < 192; ++i) k.inv_int[i] = (double)(1.0L / (long double)i);
    k.inv_int_lo[0] = 0.0;
    for (int i = 1; i < 64; ++i) k.inv_int_lo[i] = (double)(1.0L / (long double)i - (long double)k.inv_int[i]);
    long double df = 1;
    for (int n = 0; n < 32; ++n) {
        k.dfact[n] = (double)df;                 // (2n-1)!!
        df *= (2 * n + 1);
    }
    // (a|r_a^{2n}|b): C(n, j) and the coefficients 2^{d-m} (2m+1)!! C(m,d) / (2d+1)!!
    // of Eqs. sra2ms and I_jab
    auto odd_fact = [](int n) { long double f = 1; for (int i = n; i > 1; i -= 2) f *= i; return f; };
    for (int n = 0; n <= kRa2nMax; ++n)
        for (int j = 0; j <= n; ++j) {
            k.binom[n][j] = (double)(lfact(n) / (lfact(j) * lfact(n - j)));
            k.ra2n_k[n][j] = (double)(std::ldexp(1.0L, j - n) * odd_fact(2 * n + 1) * (lfact(n) / (lfact(j) * lfact(n - j))) /
                                      odd_fact(2 * j + 1));
        }
}

// Boys tables, computed in long double: F_N(T) from its power series
//   F_N(T) = exp(-T) sum_k (2T)^k / ((2N+1)(2N+3)...(2N+2k+1))
// at N = 48, then the stable downward recursion
//   F_{n-1}(T) = (2T F_n(T) + exp(-T)) / (2n-1);
// at T_i = i / per_unit, i = 0..ngrid-1: tab[(i kBoysN + n) nterms + t] =
// F_{n+t}(T_i) / t!, etab[i] = exp(-T_i).
void make_boys_table(int per_unit, int ngrid, int nterms, double *tab, double *etab)
{
    const int ntop = 48;
    for (int i = 0; i < ngrid; ++i) {
        const long double T = (long double)i / (long double)per_unit;
        const long double e = std::exp(-T);
        long double term = 1.0L / (2 * ntop + 1), sum = term;
        for (int k = 1; k < 20000; ++k) {
            term *= 2 * T / (long double)(2 * ntop + 2 * k + 1);
            sum += term;
            if (term < sum * 1e-24L) break;
        }
        long double F[ntop + 1];
        F[ntop] = e * sum;
        for (int n = ntop; n > 0; --n) F[n - 1] = (2 * T * F[n] + e) / (long double)(2 * n - 1);
        for (int n = 0; n < kBoysN; ++n) {
            long double tf = 1;
            for (int t = 0; t < nterms; ++t) {
                if (t > 0) tf *= t;
                tab[((size_t)i * kBoysN + n) * nterms + t] = (double)(F[n + t] / tf);
            }
        }
        etab[i] = (double)e;
    }
}

static float2 split2(long double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (long double)hi));
}

// same for a double: v - hi is exact in double (hi holds v's leading 24 bits)
static inline float2 split2d(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

void fill_consts_mix(ConstsMix &k)
{
    std::memset(&k, 0, sizeof k);
    for (int l = 0; l <= kLmaxR; ++l)
        for (int mu = 0; mu <= l; ++mu) {
            long double v = std::sqrt((long double)(mu == 0 ? 1 : 2) * lfact(l + mu) * lfact(l - mu));
            k.A[l][mu] = split2((mu & 1) ? -v : v);
        }
    for (int j = 0; j < kJmax; ++j) {
        long double df = 1;
        for (int i = 2 * j - 1; i > 1; i -= 2) df *= i;
        for (int kp = 0; kp <= j; ++kp) k.jB[j][kp] = split2(df / ((kp == 0 ? 1 : 2) * lfact(j + kp) * lfact(j - kp)));
    }
    for (int i = 1; i < 128; ++i) k.inv_int[i] = split2(1.0L / i);
    for (int t = 0; t < 14; ++t) {
        k.inv_fact[t] = split2(1.0L / lfact(t));
        k.inv_fact_f[t] = (float)(1.0L / lfact(t));
    }
    const long double pi = 3.14159265358979323846264338327950288L;
    k.pi32 = split2(std::pow(pi, 1.5L));
    k.pi3 = split2(pi * pi * pi);
    k.two_pi52 = split2(2 * std::pow(pi, 2.5L));
    k.sqrt_pi_half = split2(std::sqrt(pi) / 2);
    k.two_pi = split2(2 * pi);
    long double dfc = 1;
    for (int n = 0; n < kBoysN; ++n) {
        k.dfact[n] = split2(dfc);
        dfc *= (2 * n + 1);
    }
}

void fill_consts3(Consts3 &k)
{
    std::memset(&k, 0, sizeof k);
    for (int n = 0; n < 18; ++n)
        for (int i = 0; i <= n; ++i) k.binom[n][i] = (double)(lfact(n) / (lfact(i) * lfact(n - i)));
    // d_{m,j} = 2^j (2m+1)!! binom(m,j) / (2j+1)!!   (Eq. I_jab); dd[m][i][j] = d_{m,j} j!/(j-i)!
    auto dfact = [](int n) { long double f = 1; for (int i = n; i > 1; i -= 2) f *= i; return f; };
    for (int m = 0; m < 6; ++m)
        for (int j = 0; j <= m; ++j) {
            const long double d = std::ldexp(1.0L, j) * dfact(2 * m + 1) * (lfact(m) / (lfact(j) * lfact(m - j))) /
                                  dfact(2 * j + 1);
            for (int i = 0; i <= j; ++i) k.dd[m][i][j] = (double)(d * lfact(j) / lfact(j - i));
        }
    // binom(p, j) (L)_j with the rising factorial (L)_j = L (L+1) ... (L+j-1), (0)_0 = 1, (0)_j = 0
    for (int L = 0; L < 11; ++L)
        for (int p = 0; p < 6; ++p)
            for (int j = 0; j <= p; ++j) {
                long double r = 1;
                for (int i = 0; i < j; ++i) r *= (L + i);
                k.bj[L][p][j] = (double)((lfact(p) / (lfact(j) * lfact(p - j))) * r);
            }
    for (int n = 0; n < 32; ++n) k.sqrt_int[n] = (double)std::sqrt((long double)n);
}

// Real orthonormal spherical harmonics Y_{l,m} = A_{l,|m|} R^{c/s}_{l,|m|} / sqrt(4pi/(2l+1))
// at a unit vector (Sec. II E recursions), l <= lmax, stored at l*l + l + m.
static void real_ylm(long double x, long double y, long double z, int lmax, long double *Y)
{
    long double Rc[16][16] = {}, Rs[16][16] = {};
    const long double r2 = x * x + y * y + z * z;
    Rc[0][0] = 1;
    for (int l = 0; l < lmax; ++l) {
        Rc[l + 1][l + 1] = -(x * Rc[l][l] - y * Rs[l][l]) / (2 * l + 2);
        Rs[l + 1][l + 1] = -(y * Rc[l][l] + x * Rs[l][l]) / (2 * l + 2);
        for (int m = 0; m <= l; ++m) {
            const long double pc = (l >= 1 && m <= l - 1) ? Rc[l - 1][m] : 0, ps = (l >= 1 && m <= l - 1) ? Rs[l - 1][m] : 0;
            Rc[l + 1][m] = ((2 * l + 1) * z * Rc[l][m] - r2 * pc) / ((l + m + 1) * (l - m + 1));
            Rs[l + 1][m] = ((2 * l + 1) * z * Rs[l][m] - r2 * ps) / ((l + m + 1) * (l - m + 1));
        }
    }
    const long double pi = 3.14159265358979323846264338327950288L;
    for (int l = 0; l <= lmax; ++l) {
        const long double nrm = std::sqrt((2 * l + 1) / (4 * pi));
        for (int m = -l; m <= l; ++m) {
            const int mu = m < 0 ? -m : m;
            long double A = std::sqrt((long double)(mu == 0 ? 1 : 2) * lfact(l + mu) * lfact(l - mu));
            if (mu & 1) A = -A;
            Y[l * l + l + m] = nrm * A * (m >= 0 ? Rc[l][mu] : Rs[l][mu]);
        }
    }
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n).
static void gauss_legendre(int n, std::vector<long double> &x, std::vector<long double> &w)
{
    const long double pi = 3.14159265358979323846264338327950288L;
    x.assign(n, 0);
    w.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        long double t = std::cos(pi * (i + 0.75L) / (n + 0.5L)), dp = 0;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const long double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1);
            const long double dt = p1 / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-19L) break;
        }
        x[i] = t;
        w[i] = 2 / ((1 - t * t) * dp * dp);
    }
}

// Real Gaunt coefficients G = int Y_{L,M} Y_{l,m} Y_{l~,m~} dOmega for
// l, l~ <= 6, l + l~ <= kLmaxAabA, L = |l-l~|..l+l~ step 2 (the expansion of
// Eq. CG_expansion written for real harmonics), by product quadrature that is
// exact for these degrees: 16-point Gauss-Legendre in cos(theta) (polynomial
// degree <= 20) times the 32-point trapezoid rule in phi (|frequency| <= 20).
static void make_gaunt(std::vector<int> &base, std::vector<int> &row, std::vector<GauntEnt> &ent)
{
    const int nt = 16, np = 32, LY = 16;
    const long double pi = 3.14159265358979323846264338327950288L;
    std::vector<long double> gx, gw;
    gauss_legendre(nt, gx, gw);
    std::vector<double> Y((size_t)nt * np * LY * LY), W((size_t)nt * np);
    long double Yl[LY * LY];
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < np; ++j) {
            const long double ct = gx[i], st = std::sqrt(1 - ct * ct), ph = 2 * pi * j / np;
            real_ylm(st * std::cos(ph), st * std::sin(ph), ct, 12, Yl);
            for (int q = 0; q < LY * LY; ++q) Y[((size_t)i * np + j) * LY * LY + q] = (double)Yl[q];
            W[(size_t)i * np + j] = (double)(gw[i] * 2 * pi / np);
        }
    base.assign(49, -1);
    row.clear();
    ent.clear();
    row.push_back(0);
    for (int l = 0; l <= 6; ++l)
        for (int lt = 0; lt <= 6; ++lt) {
            if (l + lt > kLmaxAabA) continue;
            base[l * 7 + lt] = (int)row.size() - 1;
            for (int m = -l; m <= l; ++m)
                for (int mt = -lt; mt <= lt; ++mt) {
                    for (int L = std::abs(l - lt); L <= l + lt; L += 2)
                        for (int M = -L; M <= L; ++M) {
                            double g = 0;
                            for (size_t q = 0; q < W.size(); ++q) {
                                const double *Yq = &Y[q * LY * LY];
                                g += W[q] * Yq[L * L + L + M] * Yq[l * l + l + m] * Yq[lt * lt + lt + mt];
                            }
                            if (std::fabs(g) > 1e-13) ent.push_back(GauntEnt{g, L, M});
                        }
                    row.push_back((int)ent.size());
                }
        }
}

// ------------------------------------------------------------------------- //
// Per-device tables                                                          //
// ------------------------------------------------------------------------- //
constexpr int kNBins = kNClass * kKbins2c;

constexpr int kNBins3 = kNClass3 * kKbins3c;

struct DevState {
    DeviceTables t{};
    int *bin_rank[2] = {nullptr, nullptr};   // [2 * kNBins]: rank of bin, then bin of rank
    int *bin_rank3 = nullptr;                // [2 * kNBins3], three-index bins by cost
    bool ready = false;
};

static double class_cost3(int la, int lt, int lb, int kk)
{
    const int Lmin = std::abs(la - lt), Lmax = la + lt, nL = (Lmax - Lmin) / 2 + 1;
    double rad = 30.0, ang = 0;
    for (int L = Lmin; L <= Lmax; L += 2) {
        const int J = std::min(L, lb) + 1;
        rad += 4.0 * J * ((Lmax - L) / 2 + 1);
        ang += (2.0 * L + 1) * (2 * lb + 1) * (J * J + 2) + (2.0 * L + 1) * J * J;
    }
    return kk * rad + ang + (2.0 * la + 1) * (2 * lt + 1) * (2 * lb + 1) * nL * 2;
}

static std::mutex g_mu;
static DevState g_dev[64];

static double class_cost(int la, int lb, int kk)
{
    const int J = std::min(la, lb) + 1;
    const double radial = kk * (40.0 + 4.0 * J);
    const double na = 2 * la + 1, nb = 2 * lb + 1;
    const double angular = na * nb * (J * J + 2) + (2 * na + nb) * J * J + 10.0 * (std::max(la, lb) + 1) * (std::max(la, lb) + 1);
    return radial + angular;
}

static void make_ranks(int schedule, std::vector<int> &rank, std::vector<int> &inv)
{
    rank.assign(kNBins, 0);
    inv.assign(kNBins, 0);
    std::vector<int> order(kNBins);
    for (int b = 0; b < kNBins; ++b) order[b] = b;
    if (schedule == SHG_SCHED_PER_CLASS) {
        // class-major, Ka*Kb descending inside a class
        std::sort(order.begin(), order.end(), [](int x, int y) {
            const int cx = x / kKbins2c, cy = y / kKbins2c;
            if (cx != cy) return cx < cy;
            return (x % kKbins2c) > (y % kKbins2c);
        });
    } else {
        // class-major; classes grouped by J = min(la, lb) + 1 (descending), then by
        // decreasing estimated cost of their heaviest pairs; Ka*Kb descending
        // inside a class.  Longest tiles come first (J-major is close to cost
        // order), and the warps resident on one SM mostly run one J
        // instantiation at a time (instruction-cache locality)
        std::vector<double> ccost(kNClass);
        std::vector<int> cJ(kNClass);
        for (int cls = 0; cls < kNClass; ++cls) {
            const int la = cls / (kLmax2c + 1), lb = cls % (kLmax2c + 1);
            ccost[cls] = class_cost(la, lb, 64);
            cJ[cls] = std::min(la, lb) + 1;
        }
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            const int cx = x / kKbins2c, cy = y / kKbins2c;
            if (cx != cy) {
                if (cJ[cx] != cJ[cy]) return cJ[cx] > cJ[cy];
                return ccost[cx] > ccost[cy] || (ccost[cx] == ccost[cy] && cx < cy);
            }
            return (x % kKbins2c) > (y % kKbins2c);
        });
    }
    for (int r = 0; r < kNBins; ++r) {
        rank[order[r]] = r;
        inv[r] = order[r];
    }
}

const DeviceTables *device_tables_impl(int **ranks, int **rank3 = nullptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        fail(SHG_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &st = g_dev[dev];
    if (!st.ready) {
        // FP64 table (step 1/32): c0..c3 as doubles, c4..c6 as floats
        std::vector<double> raw((size_t)kBoysGrid * kBoysN * 7), etab(kBoysGrid);
        make_boys_table(32, kBoysGrid, 7, raw.data(), etab.data());
        std::vector<double> tab((size_t)kBoysGrid * kBoysN * kBoysStride, 0.0);
        for (size_t q = 0; q < (size_t)kBoysGrid * kBoysN; ++q) {
            double *d = &tab[q * kBoysStride];
            const double *r = &raw[q * 7];
            for (int t = 0; t < 4; ++t) d[t] = r[t];
            const float f[4] = {(float)r[4], (float)r[5], (float)r[6], 0.0f};
            std::memcpy(d + 4, f, sizeof f);
        }
        // double-float table (the same grid): c0..c2 as hi/lo float pairs, c3..c6 as floats
        std::vector<float4> mtab((size_t)kBoysGrid * kBoysN * 3);
        std::vector<float2> metab(kBoysGrid);
        for (int i = 0; i < kBoysGrid; ++i) {
            for (int n = 0; n < kBoysN; ++n) {
                const double *cf = &raw[((size_t)i * kBoysN + n) * 7];
                float4 *q = &mtab[((size_t)i * kBoysN + n) * 3];
                const float2 c0 = split2(cf[0]), c1 = split2(cf[1]), c2 = split2(cf[2]);
                q[0] = make_float4(c0.x, c0.y, c1.x, c1.y);
                q[1] = make_float4(c2.x, c2.y, (float)cf[3], (float)cf[4]);
                q[2] = make_float4((float)cf[5], (float)cf[6], 0.0f, 0.0f);
            }
            metab[i] = split2(etab[i]);
        }
        double *d_tab = nullptr, *d_e = nullptr;
        float4 *d_mtab = nullptr;
        float2 *d_metab = nullptr;
        int *d_r[2] = {nullptr, nullptr};
        if (cudaMalloc(&d_tab, tab.size() * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&d_e, etab.size() * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&d_r[0], 2 * kNBins * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&d_r[1], 2 * kNBins * sizeof(int)) != cudaSuccess) {
            cudaFree(d_tab); cudaFree(d_e); cudaFree(d_r[0]); cudaFree(d_r[1]);
            fail(SHG_ENOMEM, "device tables: cudaMalloc failed");
            return nullptr;
        }
        bool ok = cudaMemcpy(d_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(d_e, etab.data(), etab.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMalloc(&d_mtab, mtab.size() * sizeof(float4)) == cudaSuccess &&
                  cudaMalloc(&d_metab, metab.size() * sizeof(float2)) == cudaSuccess &&
                  cudaMemcpy(d_mtab, mtab.data(), mtab.size() * sizeof(float4), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(d_metab, metab.data(), metab.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess;
        for (int s = 0; s < 2 && ok; ++s) {
            std::vector<int> rank, inv;
            make_ranks(s, rank, inv);
            rank.insert(rank.end(), inv.begin(), inv.end());
            ok = cudaMemcpy(d_r[s], rank.data(), rank.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
        }
        // three-index bins ordered by estimated cost
        int *d_r3 = nullptr;
        if (ok) {
            // class-major like the two-center ranks (each class one contiguous chunk
            // of kKbins3c ranks, tiled as a whole): classes by decreasing cost of
            // their heaviest bin, Ka*Ka~*Kb descending inside a class
            std::vector<int> order(kNBins3), rank3(2 * kNBins3);
            std::vector<double> ccost(kNClass3);
            for (int cls = 0; cls < kNClass3; ++cls)
                ccost[cls] = class_cost3(cls / 49, (cls / 7) % 7, cls % 7, kKbins3c);
            for (int b = 0; b < kNBins3; ++b) order[b] = b;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
                const int cx = x / kKbins3c, cy = y / kKbins3c;
                if (cx != cy) return ccost[cx] > ccost[cy] || (ccost[cx] == ccost[cy] && cx < cy);
                return (x % kKbins3c) > (y % kKbins3c);
            });
            for (int r = 0; r < kNBins3; ++r) {
                rank3[order[r]] = r;
                rank3[kNBins3 + r] = order[r];
            }
            ok = cudaMalloc(&d_r3, rank3.size() * sizeof(int)) == cudaSuccess &&
                 cudaMemcpy(d_r3, rank3.data(), rank3.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
        }
        // real Gaunt coefficients
        int *d_gb = nullptr, *d_gr = nullptr;
        GauntEnt *d_ge = nullptr;
        if (ok) {
            std::vector<int> gb, gr;
            std::vector<GauntEnt> ge;
            make_gaunt(gb, gr, ge);
            ok = cudaMalloc(&d_gb, gb.size() * sizeof(int)) == cudaSuccess &&
                 cudaMalloc(&d_gr, gr.size() * sizeof(int)) == cudaSuccess &&
                 cudaMalloc(&d_ge, ge.size() * sizeof(GauntEnt)) == cudaSuccess &&
                 cudaMemcpy(d_gb, gb.data(), gb.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
                 cudaMemcpy(d_gr, gr.data(), gr.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
                 cudaMemcpy(d_ge, ge.data(), ge.size() * sizeof(GauntEnt), cudaMemcpyHostToDevice) == cudaSuccess;
        }
        if (!ok) {
            fail(SHG_ECUDA, "device tables: upload failed");
            return nullptr;
        }
        st.bin_rank3 = d_r3;
        st.t.gaunt_base = d_gb;
        st.t.gaunt_row = d_gr;
        st.t.gaunt = d_ge;
        st.t.boys_mix = d_mtab;
        st.t.boys_e_mix = d_metab;
        st.t.boys = d_tab;
        st.t.boys_e = d_e;
        st.bin_rank[0] = d_r[0];
        st.bin_rank[1] = d_r[1];
        st.ready = true;
    }
    if (ranks) {
        ranks[0] = st.bin_rank[0];
        ranks[1] = st.bin_rank[1];
    }
    if (rank3) *rank3 = st.bin_rank3;
    return &st.t;
}

const DeviceTables *device_tables() { return device_tables_impl(nullptr); }

const DeviceTables *device_tables_if_ready(const int **ranks)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &st = g_dev[dev];
    if (!st.ready) return nullptr;
    if (ranks) {
        ranks[0] = st.bin_rank[0];
        ranks[1] = st.bin_rank[1];
    }
    return &st.t;
}

const ConstsMix &consts_mix()
{
    static ConstsMix k;
    static std::once_flag once;
    std::call_once(once, [] { fill_consts_mix(k); });
    return k;
}

const Consts3 &consts3()
{
    static Consts3 k;
    static std::once_flag once;
    std::call_once(once, [] { fill_consts3(k); });
    return k;
}

const Consts &consts()
{
    static Consts k;
    static std::once_flag once;
    std::call_once(once, [] { fill_consts(k); });
    return k;
}

static bool is_finite_d(double x) { return std::isfinite(x); }

static int current_device_matches(int dev)
{
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return fail(SHG_ECUDA, "cudaGetDevice failed");
    if (cur != dev) return fail(SHG_EINVAL, "current device %d differs from the basis device %d", cur, dev);
    return SHG_OK;
}

int check_op(int op, double omega, int precision)
{
    if (op < SHG_OP_OVERLAP || op > SHG_OP_RA2N) return fail(SHG_EINVAL, "bad operator %d", op);
    if (op == SHG_OP_RA2N) {
        if (!(omega >= 0 && omega <= kRa2nMax && omega == std::floor(omega)))
            return fail(SHG_EINVAL, "SHG_OP_RA2N takes n = 0..%d in omega (got %g)", kRa2nMax, omega);
        if (precision != SHG_PREC_FP64) return fail(SHG_EINVAL, "SHG_OP_RA2N is available in FP64 only");
    } else if (op != SHG_OP_OVERLAP && op != SHG_OP_COULOMB && !(omega > 0 && std::isfinite(omega))) {
        return fail(SHG_EINVAL, "operator %d needs omega > 0 (got %g)", op, omega);
    }
    if (precision != SHG_PREC_FP64 && precision != SHG_PREC_MIXED)
        return fail(SHG_EINVAL, "precision %d not available", precision);
    return SHG_OK;
}

}  // namespace shg

using namespace shg;

// ------------------------------------------------------------------------- //
// C ABI                                                                      //
// ------------------------------------------------------------------------- //
extern "C" {

const char *shg_last_error(void) { return g_err.c_str(); }

const char *shg_version(void) { return "shg-gb300 0.1 (sm_103a)"; }

int shg_basis_create(int n_shells, const int32_t *l, const int32_t *nprim, const double *exps, const double *coefs,
                     int n_centers, const double *centers, const int32_t *center_of_shell, int normalize,
                     shg_basis_t **out)
{
    Phase phase_("shg:basis_create");
    g_err.clear();
    if (!out) return fail(SHG_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_shells < 1 || n_centers < 1) return fail(SHG_EINVAL, "n_shells and n_centers must be >= 1");
    if (!l || !nprim || !exps || !coefs || !centers || !center_of_shell) return fail(SHG_EINVAL, "NULL input array");
    int64_t n_prims = 0;
    for (int s = 0; s < n_shells; ++s) {
        if (l[s] < 0 || l[s] > kLmax2c) return fail(SHG_EINVAL, "shell %d: l = %d outside 0..%d", s, l[s], kLmax2c);
        if (nprim[s] < 1 || nprim[s] > kKmax) return fail(SHG_EINVAL, "shell %d: K = %d outside 1..%d", s, nprim[s], kKmax);
        if (center_of_shell[s] < 0 || center_of_shell[s] >= n_centers)
            return fail(SHG_EINVAL, "shell %d: center index %d out of range", s, center_of_shell[s]);
        n_prims += nprim[s];
    }
    if (n_prims > (int64_t)INT32_MAX) return fail(SHG_ERANGE, "too many primitives");
    for (int64_t i = 0; i < n_prims; ++i) {
        if (!is_finite_d(exps[i]) || exps[i] <= 0) return fail(SHG_EINVAL, "primitive %lld: exponent %g not > 0", (long long)i, exps[i]);
        if (!is_finite_d(coefs[i])) return fail(SHG_EINVAL, "primitive %lld: coefficient not finite", (long long)i);
    }
    for (int64_t i = 0; i < 3 * (int64_t)n_centers; ++i)
        if (!is_finite_d(centers[i])) return fail(SHG_EINVAL, "center coordinate %lld not finite", (long long)i);

    std::vector<ShellRec> sh(n_shells);
    std::vector<PrimRec> pr(n_prims);
    std::vector<CoulPrim> cpr(n_prims);
    std::vector<int64_t> first(n_shells + 1, 0);
    for (int s = 0; s < n_shells; ++s) first[s + 1] = first[s] + nprim[s];
    // per-l constants: sqrt(pi) (2l+2)! / (2^{2l+3} (l+1)!) and K_l = sqrt((2l+1)/(4 pi))
    dd pref_l[kLmax2c + 1], K_l[kLmax2c + 1];
    for (int L = 0; L <= kLmax2c; ++L) {
        const long double pi = 3.14159265358979323846264338327950288L;
        pref_l[L] = dd_from(std::sqrt(pi) * lfact(2 * L + 2) / (std::ldexp(1.0L, 2 * L + 3) * lfact(L + 1)));
        K_l[L] = dd_from(std::sqrt((2 * L + 1) / (4 * pi)));
    }
    int bad_shell = -1;
#pragma omp parallel for schedule(dynamic, 256)
    for (int s = 0; s < n_shells; ++s) {
        const int L = l[s], K = nprim[s];
        const int64_t off = first[s];
        dd N = {1.0, 0.0};
        if (normalize) {
            // N_l = K_l [sum_ij sqrt(pi) (2l+2)! c_i c_j / (2^{2l+3} (l+1)! (a_i+a_j)^{l+3/2})]^{-1/2}
            dd sum = {0.0, 0.0};
            for (int i = 0; i < K; ++i)
                for (int j = i; j < K; ++j) {
                    const dd sij = dd_two_sum(exps[off + i], exps[off + j]);
                    const dd r = dd_div(dd{1.0, 0.0}, sij);
                    dd pw = r;
                    for (int t = 0; t < L; ++t) pw = dd_mul(pw, r);      // s^-(L+1)
                    dd term = dd_mul(pw, dd_sqrt(r));                    // s^-(L+3/2)
                    term = dd_mul(term, dd_mul(dd{coefs[off + i], 0.0}, dd{coefs[off + j], 0.0}));
                    if (j != i) term = dd{2 * term.hi, 2 * term.lo};
                    sum = dd_add(sum, term);
                }
            sum = dd_mul(sum, pref_l[L]);
            if (!(sum.hi > 0)) {
#pragma omp critical
                bad_shell = s;
                continue;
            }
            N = dd_div(K_l[L], dd_sqrt(sum));
        }
        for (int i = 0; i < K; ++i) {
            const double a = exps[off + i];
            const dd c = dd_mul(N, dd{coefs[off + i], 0.0});
            dd p2 = {1.0, 0.0};
            for (int t = 0; t < L; ++t) p2 = dd_mul(p2, dd{2 * a, 0.0});  // (2a)^l
            PrimRec p;
            const dd ia = dd_div(dd{1.0, 0.0}, dd{a, 0.0});
            const dd w2c = dd_div(c, p2);
            p.alpha = a;
            p.inv_alpha = ia.hi;
            p.w2c = w2c.hi;
            p.wN = c.hi;
            pr[off + i] = p;
            const dd cw = dd_mul(w2c, ia);
            // sqrt(2 pi^{5/2}) folded into cw: pre = cw_a cw_b / sqrt(c)
            const dd s2p52 = dd_sqrt(dd_from(2.0L * 17.493418327624862846262821679871554L));   // 2 pi^{5/2}
            cpr[off + i] = CoulPrim{dd_mul(cw, s2p52).hi, dd_mul(cw, dd_sqrt(ia)).hi};
        }
        sh[s] = ShellRec{L, K, (int)off, center_of_shell[s]};
    }
    if (bad_shell >= 0) return fail(SHG_EINVAL, "shell %d: contracted function has zero norm", bad_shell);
    // families: shells on one center whose exponent lists are bitwise identical
    std::vector<int32_t> fam(n_shells), fam_prim, fam_k;
    {
        std::unordered_map<std::string, int> ids;
        std::string key;
        for (int s = 0; s < n_shells; ++s) {
            key.assign(reinterpret_cast<const char *>(&center_of_shell[s]), sizeof(int32_t));
            key.append(reinterpret_cast<const char *>(exps + first[s]), sizeof(double) * (size_t)nprim[s]);
            auto it = ids.find(key);
            if (it == ids.end()) {
                it = ids.emplace(key, (int)fam_prim.size()).first;
                fam_prim.push_back((int32_t)first[s]);
                fam_k.push_back(nprim[s]);
            }
            fam[s] = it->second;
        }
    }
    std::vector<ScreenRec> scr(n_shells);
    for (int s = 0; s < n_shells; ++s) {
        double amin = exps[first[s]], sabs = 0;
        for (int64_t i = first[s]; i < first[s + 1]; ++i) {
            amin = std::min(amin, exps[i]);
            sabs += std::fabs(pr[i].wN);
        }
        const int L = l[s];
        const double lfac = L == 0 ? 1.0 : std::pow(L / (amin * 2.718281828459045), 0.5 * L);
        scr[s] = ScreenRec{amin, sabs, lfac, 0.0};
    }
    std::vector<Vec4> ctr(n_centers);
    std::vector<MixCenter> mctr(n_centers);
    for (int c = 0; c < n_centers; ++c) {
        ctr[c] = Vec4{centers[3 * c], centers[3 * c + 1], centers[3 * c + 2], 0.0};
        mctr[c] = MixCenter{split2d(centers[3 * c]), split2d(centers[3 * c + 1]), split2d(centers[3 * c + 2]),
                            make_float2(0, 0)};
    }
    std::vector<MixPrim> mpr(n_prims);
#pragma omp parallel for schedule(static)
    for (int64_t o = 0; o < n_prims; ++o) {
        const double a = exps[o];
        const dd ia = dd_div(dd{1.0, 0.0}, dd{a, 0.0});
        const float ih = (float)ia.hi;
        mpr[o] = MixPrim{split2d(a), make_float2(ih, (float)((ia.hi - (double)ih) + ia.lo)), split2d(pr[o].wN),
                         cpr[o].fw};
    }

    shg_basis_t *b = new (std::nothrow) shg_basis_t;
    if (!b) return fail(SHG_ENOMEM, "host allocation failed");
    BasisDev &d = b->d;
    d.n_shells = n_shells;
    d.n_centers = n_centers;
    d.n_prims = n_prims;
    cudaGetDevice(&d.device);
    d.h_l = new int32_t[n_shells];
    d.h_nprim = new int32_t[n_shells];
    d.h_center = new int32_t[n_shells];
    std::memcpy(d.h_l, l, sizeof(int32_t) * n_shells);
    std::memcpy(d.h_nprim, nprim, sizeof(int32_t) * n_shells);
    std::memcpy(d.h_center, center_of_shell, sizeof(int32_t) * n_shells);
    d.n_fams = (int)fam_prim.size();
    d.h_fam = new int32_t[n_shells];
    d.h_fam_prim = new int32_t[d.n_fams];
    d.h_fam_k = new int32_t[d.n_fams];
    std::memcpy(d.h_fam, fam.data(), sizeof(int32_t) * n_shells);
    std::memcpy(d.h_fam_prim, fam_prim.data(), sizeof(int32_t) * d.n_fams);
    std::memcpy(d.h_fam_k, fam_k.data(), sizeof(int32_t) * d.n_fams);
    if (cudaMalloc(&d.shells, sizeof(ShellRec) * n_shells) != cudaSuccess ||
        cudaMalloc(&d.prims, sizeof(PrimRec) * n_prims) != cudaSuccess ||
        cudaMalloc(&d.centers, sizeof(Vec4) * n_centers) != cudaSuccess ||
        cudaMalloc(&d.mprims, sizeof(MixPrim) * n_prims) != cudaSuccess ||
        cudaMalloc(&d.cprims, sizeof(CoulPrim) * n_prims) != cudaSuccess ||
        cudaMalloc(&d.screen, sizeof(ScreenRec) * n_shells) != cudaSuccess ||
        cudaMalloc(&d.mcenters, sizeof(MixCenter) * n_centers) != cudaSuccess) {
        shg_basis_destroy(b);
        return fail(SHG_ENOMEM, "basis: cudaMalloc failed");
    }
    if (cudaMemcpy(d.shells, sh.data(), sizeof(ShellRec) * n_shells, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.prims, pr.data(), sizeof(PrimRec) * n_prims, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.centers, ctr.data(), sizeof(Vec4) * n_centers, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.mprims, mpr.data(), sizeof(MixPrim) * n_prims, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.cprims, cpr.data(), sizeof(CoulPrim) * n_prims, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.screen, scr.data(), sizeof(ScreenRec) * n_shells, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d.mcenters, mctr.data(), sizeof(MixCenter) * n_centers, cudaMemcpyHostToDevice) != cudaSuccess) {
        shg_basis_destroy(b);
        return fail(SHG_ECUDA, "basis: upload failed");
    }
    if (!device_tables()) {
        shg_basis_destroy(b);
        return SHG_ECUDA;
    }
    *out = b;
    return SHG_OK;
}

int shg_basis_set_centers(shg_basis_t *b, const double *centers)
{
    Phase phase_("shg:set_centers");
    g_err.clear();
    if (!b || !centers) return fail(SHG_EINVAL, "NULL argument");
    BasisDev &d = b->d;
    const int n = d.n_centers;
    if (n == 0) return SHG_OK;
    if (!d.stage_raw) {
        if (cudaMalloc(&d.stage_raw, sizeof(double) * 3 * n) != cudaSuccess ||
            cudaMalloc(&d.stage_ctr, sizeof(Vec4) * n) != cudaSuccess ||
            cudaMalloc(&d.stage_mctr, sizeof(MixCenter) * n) != cudaSuccess ||
            cudaMalloc(&d.stage_bad, sizeof(int)) != cudaSuccess) {
            cudaFree(d.stage_raw);
            cudaFree(d.stage_ctr);
            cudaFree(d.stage_mctr);
            cudaFree(d.stage_bad);
            d.stage_raw = nullptr;
            d.stage_ctr = nullptr;
            d.stage_mctr = nullptr;
            d.stage_bad = nullptr;
            return fail(SHG_ENOMEM, "set_centers: cudaMalloc failed");
        }
    }
    // the legacy default stream orders this against work on blocking streams
    const cudaStream_t s = 0;
    SHG_CUDA(cudaMemcpyAsync(d.stage_raw, centers, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    SHG_CUDA(cudaMemsetAsync(d.stage_bad, 0x7f, sizeof(int), s));
    SHG_CUDA(launch_pack_centers(d.stage_raw, n, d.stage_ctr, d.stage_mctr, d.stage_bad, s));
    int bad = 0;
    SHG_CUDA(cudaMemcpyAsync(&bad, d.stage_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    SHG_CUDA(cudaStreamSynchronize(s));
    if (bad < n) return fail(SHG_EINVAL, "center %d has a non-finite coordinate", bad);
    SHG_CUDA(cudaMemcpyAsync(d.centers, d.stage_ctr, sizeof(Vec4) * n, cudaMemcpyDeviceToDevice, s));
    SHG_CUDA(cudaMemcpyAsync(d.mcenters, d.stage_mctr, sizeof(MixCenter) * n, cudaMemcpyDeviceToDevice, s));
    SHG_CUDA(cudaStreamSynchronize(s));
    return SHG_OK;
}

void shg_basis_destroy(shg_basis_t *b)
{
    if (!b) return;
    cudaFree(b->d.shells);
    cudaFree(b->d.prims);
    cudaFree(b->d.centers);
    cudaFree(b->d.mprims);
    cudaFree(b->d.cprims);
    cudaFree(b->d.mcenters);
    cudaFree(b->d.screen);
    cudaFree(b->d.stage_raw);
    cudaFree(b->d.stage_ctr);
    cudaFree(b->d.stage_mctr);
    cudaFree(b->d.stage_bad);
    delete[] b->d.h_l;
    delete[] b->d.h_nprim;
    delete[] b->d.h_center;
    delete[] b->d.h_fam;
    delete[] b->d.h_fam_prim;
    delete[] b->d.h_fam_k;
    delete b;
}

int64_t shg_basis_nshells(const shg_basis_t *b) { return b ? b->d.n_shells : 0; }
int64_t shg_basis_nprims(const shg_basis_t *b) { return b ? b->d.n_prims : 0; }

int64_t shg_pair_offsets(const shg_basis_t *b, int64_t n, const int32_t *pa, const int32_t *pb, int64_t *offsets)
{
    g_err.clear();
    if (!b || n < 0 || (n > 0 && (!pa || !pb || !offsets))) return fail(SHG_EINVAL, "bad argument");
    int64_t tot = 0;
    for (int64_t p = 0; p < n; ++p) {
        if (pa[p] < 0 || pa[p] >= b->d.n_shells || pb[p] < 0 || pb[p] >= b->d.n_shells)
            return fail(SHG_EINVAL, "pair %lld: shell index out of range", (long long)p);
        offsets[p] = tot;
        tot += (int64_t)(2 * b->d.h_l[pa[p]] + 1) * (2 * b->d.h_l[pb[p]] + 1);
    }
    return tot;
}

int64_t shg_triple_offsets(const shg_basis_t *orb, const shg_basis_t *aux, int64_t n, const int32_t *ta,
                           const int32_t *tt, const int32_t *tb, int64_t *offsets)
{
    g_err.clear();
    if (!orb || !aux || n < 0 || (n > 0 && (!ta || !tt || !tb || !offsets))) return fail(SHG_EINVAL, "bad argument");
    int64_t tot = 0;
    for (int64_t p = 0; p < n; ++p) {
        if (ta[p] < 0 || ta[p] >= orb->d.n_shells || tt[p] < 0 || tt[p] >= orb->d.n_shells || tb[p] < 0 ||
            tb[p] >= aux->d.n_shells)
            return fail(SHG_EINVAL, "triple %lld: shell index out of range", (long long)p);
        offsets[p] = tot;
        tot += (int64_t)(2 * orb->d.h_l[ta[p]] + 1) * (2 * orb->d.h_l[tt[p]] + 1) * (2 * aux->d.h_l[tb[p]] + 1);
    }
    return tot;
}

int shg_plan_2c_create(const shg_basis_t *basis, int64_t n, const int32_t *pa, const int32_t *pb, int schedule,
                       void *stream, shg_plan_t **out)
{
    Phase phase_("shg:plan_2c_create");
    g_err.clear();
    if (!out) return fail(SHG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!basis) return fail(SHG_EINVAL, "basis is NULL");
    if (n < 0 || n > (int64_t)INT32_MAX / 2) return fail(SHG_ERANGE, "n_pairs %lld out of range", (long long)n);
    if (n > 0 && (!pa || !pb)) return fail(SHG_EINVAL, "NULL pair list");
    if (schedule != SHG_SCHED_PER_CLASS && schedule != SHG_SCHED_PERSISTENT)
        return fail(SHG_EINVAL, "bad schedule %d", schedule);
    int r = current_device_matches(basis->d.device);
    if (r) return r;
    int *ranks[2];
    if (!device_tables_impl(ranks)) return SHG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;

    const int64_t max_tiles = n / kTile + std::min<int64_t>(n, kNBins) + 1;
    const size_t bytes_perm = sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1);
    const size_t bytes_tiles = sizeof(Tile) * (size_t)max_tiles;
    const size_t bytes_ws = sizeof(int) * plan_ws_ints(n, kNBins, kNClass);
    const size_t bytes = bytes_perm + bytes_tiles + bytes_ws + 256;
    void *blk = nullptr;
    SHG_CUDA(cudaMallocAsync(&blk, bytes, s));

    shg_plan_t *p = new (std::nothrow) shg_plan_t;
    if (!p) {
        cudaFreeAsync(blk, s);
        return fail(SHG_ENOMEM, "host allocation failed");
    }
    PlanDev &d = p->d;
    d.basis = &basis->d;
    d.n_pairs = n;
    d.schedule = schedule;
    d.pair_a = pa;
    d.pair_b = pb;
    d.owner_block = blk;
    d.stream = s;
    char *c = (char *)blk;
    d.tiles = (Tile *)c;                 c += (bytes_tiles + 15) / 16 * 16;
    d.perm = (int32_t *)c;               c += (bytes_perm + 15) / 16 * 16;
    d.counter = (int *)c;                c += 16;
    int *ws = (int *)c;

    auto cleanup = [&](int code) {
        cudaFreeAsync(blk, s);
        delete p;
        return code;
    };
    cudaError_t e = launch_plan_build(d, ws, kNBins, ranks[schedule], s);
    if (e != cudaSuccess) return cleanup(fail(SHG_ECUDA, "plan build: %s", cudaGetErrorString(e)));
    // first tile of every class chunk, the tile count and the error flag, in one read-back
    int chunk_tile[kNClass + 2];
    if (cudaMemcpyAsync(chunk_tile, plan_summary(ws, kNBins), sizeof(chunk_tile), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cleanup(fail(SHG_ECUDA, "plan build: %s", cudaGetErrorString(cudaGetLastError())));
    if (chunk_tile[kNClass + 1])
        return cleanup(fail(SHG_EINVAL, "pair list holds a shell index outside 0..%d", basis->d.n_shells - 1));
    d.n_tiles = chunk_tile[kNClass];
    for (int cls = 0; cls <= kNClass; ++cls) d.class_tile_begin[cls] = chunk_tile[cls];
    if (schedule == SHG_SCHED_PERSISTENT) {
        // the persistent rank order is J-major (J descending), so the classes with
        // both l >= kMixedFp64MinL are its first chunks
        int n_hi = 0;
        for (int cls = 0; cls < kNClass; ++cls) n_hi += mixed_runs_fp64(cls);
        d.mixed_fp64_tiles = chunk_tile[n_hi];
    }
    if (schedule == SHG_SCHED_PERSISTENT) {
        p->launches = d.n_tiles > 0 ? 1 : 0;
    } else {
        p->launches = 0;
        for (int cls = 0; cls < kNClass; ++cls) p->launches += d.class_tile_begin[cls + 1] > d.class_tile_begin[cls];
    }
    *out = p;
    return SHG_OK;
}

int shg_plan_launches(const shg_plan_t *p) { return p ? p->launches : 0; }

int shg_plan_launches_prec(const shg_plan_t *p, int precision)
{
    if (!p || (precision != SHG_PREC_FP64 && precision != SHG_PREC_MIXED)) return -1;
    if (precision == SHG_PREC_FP64 || p->d.schedule != SHG_SCHED_PERSISTENT) return p->launches;
    return (p->d.mixed_fp64_tiles > 0) + (p->d.n_tiles > p->d.mixed_fp64_tiles);
}

int shg_plan_2c_set_variant(shg_plan_t *p, int variant)
{
    g_err.clear();
    if (!p) return fail(SHG_EINVAL, "plan is NULL");
    if (variant < 0 || variant > 2) return fail(SHG_EINVAL, "kernel variant must be 0, 1 or 2");
    p->d.variant = variant;
    return SHG_OK;
}

int shg_plan_2c_set_launch(shg_plan_t *p, int threads, int ctas_per_sm)
{
    g_err.clear();
    if (!p) return fail(SHG_EINVAL, "plan is NULL");
    if (threads != 32 && threads != 64 && threads != 128) return fail(SHG_EINVAL, "threads per CTA must be 32, 64 or 128");
    if (ctas_per_sm < 0 || ctas_per_sm > 64) return fail(SHG_EINVAL, "ctas_per_sm must be 0..64");
    p->d.threads = threads;
    p->d.ctas_per_sm = ctas_per_sm;
    return SHG_OK;
}

struct shg_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// Capture the launches `issue` makes on a private stream into an instantiated graph.
extern "C++" {
template <class F>
static int capture_graph(F issue, shg_graph_t **out)
{
    cudaStream_t s = nullptr;
    SHG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s);
        return fail(SHG_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    }
    const int rc = issue(s);
    std::string msg = g_err;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    cudaStreamDestroy(s);
    if (rc != SHG_OK) {
        if (graph) cudaGraphDestroy(graph);
        return fail(rc, "capture: %s", msg.c_str());
    }
    if (e != cudaSuccess) return fail(SHG_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(SHG_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    shg_graph_t *g = new (std::nothrow) shg_graph_t;
    if (!g) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return fail(SHG_ENOMEM, "host allocation failed");
    }
    g->graph = graph;
    g->exec = exec;
    *out = g;
    return SHG_OK;
}
}  // extern "C++"

int shg_graph_2c_create(shg_plan_t *p, int n_ops, const int *ops, const double *omegas, int precision,
                        const int64_t *off, double *const *outs, shg_graph_t **out)
{
    g_err.clear();
    if (!out) return fail(SHG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!p || n_ops < 1 || !ops || !omegas || !outs) return fail(SHG_EINVAL, "bad argument");
    for (int i = 0; i < n_ops; ++i) {
        int r = check_op(ops[i], omegas[i], precision);
        if (r) return r;
    }
    return capture_graph(
        [&](cudaStream_t s) {
            int rc = SHG_OK;
            for (int i = 0; i < n_ops && rc == SHG_OK; ++i)
                rc = shg_plan_2c_exec(p, ops[i], omegas[i], 0.0, precision, off, outs[i], s);
            return rc;
        },
        out);
}

int shg_graph_launch(shg_graph_t *g, void *stream)
{
    Phase phase_("shg:graph_launch");
    g_err.clear();
    if (!g) return fail(SHG_EINVAL, "graph is NULL");
    SHG_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return SHG_OK;
}

void shg_graph_destroy(shg_graph_t *g)
{
    if (!g) return;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
}

void shg_plan_destroy(shg_plan_t *p)
{
    if (!p) return;
    cudaFreeAsync(p->d.owner_block, p->d.stream);
    if (p->d.ev_fork) cudaEventDestroy(p->d.ev_fork);
    if (p->d.ev_join) cudaEventDestroy(p->d.ev_join);
    if (p->d.ev_join2) cudaEventDestroy(p->d.ev_join2);
    if (p->d.side) cudaStreamDestroy(p->d.side);
    if (p->d.side2) cudaStreamDestroy(p->d.side2);
    delete p;
}


// Streams and events of a forked mixed-precision pass, created on the first
// execution that needs them: the FP64 launch of the classes with both l >=
// kMixedFp64MinL (a few hundred heavy tiles, one warp each) runs on `side`,
// the double-float persistent launch on `side2`, so that the FP64 pipes work
// on those tiles while the FP32 pipes of the rest of the GPU run the others.
// Neither launch goes to the caller's stream, which only forks and joins (on
// the legacy default stream a launch beside another stream's does not overlap
// it).  `side` has the highest stream priority: its CTAs are dispatched first
// and are resident before the persistent launch fills the SMs.
static int plan_side_streams(shg_plan_t *p)
{
    if (p->d.side) return SHG_OK;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&p->d.side, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&p->d.side2, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->d.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->d.ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->d.ev_join2, cudaEventDisableTiming) != cudaSuccess)
        return fail(SHG_ECUDA, "side streams: %s", cudaGetErrorString(cudaGetLastError()));
    return SHG_OK;
}

// fork: both side streams wait for the work already on s
static int fork_sides(shg_plan_t *p, cudaStream_t s)
{
    int r = plan_side_streams(p);
    if (r) return r;
    SHG_CUDA(cudaEventRecord(p->d.ev_fork, s));
    SHG_CUDA(cudaStreamWaitEvent(p->d.side, p->d.ev_fork, 0));
    SHG_CUDA(cudaStreamWaitEvent(p->d.side2, p->d.ev_fork, 0));
    return SHG_OK;
}

// join: s waits for both side streams
static int join_sides(shg_plan_t *p, cudaStream_t s)
{
    SHG_CUDA(cudaEventRecord(p->d.ev_join, p->d.side));
    SHG_CUDA(cudaEventRecord(p->d.ev_join2, p->d.side2));
    SHG_CUDA(cudaStreamWaitEvent(s, p->d.ev_join, 0));
    SHG_CUDA(cudaStreamWaitEvent(s, p->d.ev_join2, 0));
    return SHG_OK;
}

// which classes an FP64 execution covers: all of them, or only those the
// mixed-precision passes run in FP64
enum { kAllClasses = 0, kMixedFp64Classes = 1 };
static int exec_fp64(shg_plan_t *p, int op, double omega, double screen, const int64_t *off, double *out,
                     const double *o_pre, cudaStream_t s, int sel = kAllClasses);
static int exec_fp64_static_range(shg_plan_t *p, int op, double omega, double screen, const int64_t *off,
                                  double *out, int tile_begin, int tile_end, cudaStream_t s);

int shg_plan_2c_exec(shg_plan_t *p, int op, double omega, double screen, int precision, const int64_t *off,
                     double *out, void *stream)
{
    Phase phase_("shg:plan_2c_exec");
    g_err.clear();
    if (!p) return fail(SHG_EINVAL, "plan is NULL");
    int r = check_op(op, omega, precision);
    if (r) return r;
    if (!(screen >= 0.0) || !std::isfinite(screen)) return fail(SHG_EINVAL, "screening threshold must be >= 0");
    if (p->d.n_pairs == 0 || p->d.n_tiles == 0) return SHG_OK;
    if (!off || !out) return fail(SHG_EINVAL, "NULL output");
    r = current_device_matches(p->d.basis->device);
    if (r) return r;
    const DeviceTables *t = device_tables();
    if (!t) return SHG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == SHG_PREC_MIXED) {
        ArgsMix m;
        m.shells = p->d.basis->shells;
        m.prims = p->d.basis->mprims;
        m.centers = p->d.basis->mcenters;
        m.pair_a = p->d.pair_a;
        m.pair_b = p->d.pair_b;
        m.perm = p->d.perm;
        m.tiles = p->d.tiles;
        m.out_off = reinterpret_cast<const long long *>(off);
        m.out = out;
        m.omega = split2(omega);
        m.omega2 = split2((long double)omega * omega);
        m.omega_d = omega;
        m.screen_thresh = screen;
        m.screen = p->d.basis->screen;
        m.boys = t->boys_mix;
        m.boys_e = t->boys_e_mix;
        m.km = consts_mix();
        // classes with both l >= kMixedFp64MinL in FP64: beside the double-float
        // launch on the side streams (persistent plans holding both kinds), else first
        const bool fork = p->d.schedule == SHG_SCHED_PERSISTENT && p->d.mixed_fp64_tiles > 0 &&
                          p->d.n_tiles > p->d.mixed_fp64_tiles;
        if (fork) {
            r = fork_sides(p, s);
            if (r) return r;
            r = exec_fp64_static_range(p, op, omega, screen, off, out, 0, p->d.mixed_fp64_tiles, p->d.side);
            if (r) return r;
        } else {
            r = exec_fp64(p, op, omega, screen, off, out, nullptr, s, kMixedFp64Classes);
            if (r) return r;
        }
        if (p->d.schedule == SHG_SCHED_PERSISTENT) {
            m.tile_begin = p->d.mixed_fp64_tiles;
            m.tile_end = p->d.n_tiles;
            if (m.tile_end <= m.tile_begin) return SHG_OK;
            const cudaStream_t sm = fork ? p->d.side2 : s;
            SHG_CUDA(cudaMemsetAsync(p->d.counter, 0, sizeof(int), sm));
            m.counter = p->d.counter;
            SHG_CUDA(launch_2c_mixed(m, op, persistent_grid_2c_mixed(op, p->d.threads, p->d.ctas_per_sm), true, sm,
                                     p->d.threads));
            if (fork) return join_sides(p, s);
        } else {
            m.counter = nullptr;
            for (int cls = 0; cls < kNClass; ++cls) {
                if (mixed_runs_fp64(cls)) continue;
                m.tile_begin = p->d.class_tile_begin[cls];
                m.tile_end = p->d.class_tile_begin[cls + 1];
                if (m.tile_end <= m.tile_begin) continue;
                SHG_CUDA(launch_2c_mixed(m, op, 0, false, s, p->d.threads));
            }
        }
        return SHG_OK;
    }
    return exec_fp64(p, op, omega, screen, off, out, nullptr, s);
}

// FP64 execution of a plan; o_pre != null runs the angular part on
// precomputed contracted radial terms (op = OP_PRE, family path).
static int exec_fp64(shg_plan_t *p, int op, double omega, double screen, const int64_t *off, double *out,
                     const double *o_pre, cudaStream_t s, int sel)
{
    const DeviceTables *t = device_tables();
    if (!t) return SHG_ECUDA;
    const int precision = SHG_PREC_FP64;
    Args2c a;
    a.shells = p->d.basis->shells;
    a.prims = p->d.basis->prims;
    a.centers = p->d.basis->centers;
    a.pair_a = p->d.pair_a;
    a.pair_b = p->d.pair_b;
    a.perm = p->d.perm;
    a.tiles = p->d.tiles;
    a.out_off = reinterpret_cast<const long long *>(off);
    a.out = out;
    a.omega = omega;
    a.screen_thresh = screen;
    a.screen = p->d.basis->screen;
    a.boys = t->boys;
    a.boys_e = t->boys_e;
    a.o_pre = o_pre;
    a.k = consts();
    if (p->d.schedule == SHG_SCHED_PERSISTENT) {
        a.tile_begin = 0;
        a.tile_end = sel == kAllClasses ? p->d.n_tiles : p->d.mixed_fp64_tiles;
        if (a.tile_end <= 0) return SHG_OK;
        SHG_CUDA(cudaMemsetAsync(p->d.counter, 0, sizeof(int), s));
        a.counter = p->d.counter;
        SHG_CUDA(launch_2c(a, op, precision, persistent_grid_2c(op, precision, p->d.threads, p->d.ctas_per_sm), true, s,
                           p->d.threads));
    } else {
        a.counter = nullptr;
        for (int cls = 0; cls < kNClass; ++cls) {
            if (sel == kMixedFp64Classes && !mixed_runs_fp64(cls)) continue;
            a.tile_begin = p->d.class_tile_begin[cls];
            a.tile_end = p->d.class_tile_begin[cls + 1];
            if (a.tile_end <= a.tile_begin) continue;
            SHG_CUDA(launch_2c(a, op, precision, 0, false, s, p->d.threads));
        }
    }
    return SHG_OK;
}

// FP64 single-operator pass over the tiles [tile_begin, tile_end) of a plan,
// one warp per tile (no work counter: it may run beside a persistent launch
// of the same plan)
static int exec_fp64_static_range(shg_plan_t *p, int op, double omega, double screen, const int64_t *off,
                                  double *out, int tile_begin, int tile_end, cudaStream_t s)
{
    const DeviceTables *t = device_tables();
    if (!t) return SHG_ECUDA;
    Args2c a;
    a.shells = p->d.basis->shells;
    a.prims = p->d.basis->prims;
    a.centers = p->d.basis->centers;
    a.pair_a = p->d.pair_a;
    a.pair_b = p->d.pair_b;
    a.perm = p->d.perm;
    a.tiles = p->d.tiles;
    a.out_off = reinterpret_cast<const long long *>(off);
    a.out = out;
    a.omega = omega;
    a.screen_thresh = screen;
    a.screen = p->d.basis->screen;
    a.boys = t->boys;
    a.boys_e = t->boys_e;
    a.o_pre = nullptr;
    a.k = consts();
    a.tile_begin = tile_begin;
    a.tile_end = tile_end;
    a.counter = nullptr;
    SHG_CUDA(launch_2c(a, op, SHG_PREC_FP64, 0, false, s, 32));
    return SHG_OK;
}

// Arguments of a fused pass: the operators are checked (each of overlap,
// 1/r, erfc, erf and the Gaussian at most once, in the given precision),
// outputs placed by operator id.
static int fused_args(shg_plan_t *p, int n_ops, const int *ops, const double *omegas, int precision,
                      const int64_t *off, double *const *outs, ArgsFused &a)
{
    if (!p) return fail(SHG_EINVAL, "plan is NULL");
    if (n_ops < 1 || n_ops > 5) return fail(SHG_EINVAL, "n_ops must be 1..5 (got %d)", n_ops);
    if (!ops || !omegas || !outs) return fail(SHG_EINVAL, "NULL operator, omega or output array");
    for (int i = 0; i < 5; ++i) a.out[i] = nullptr;
    a.w_erf = a.w_erfc = a.w_gauss = 0.0;
    for (int i = 0; i < n_ops; ++i) {
        const int op = ops[i];
        if (op < SHG_OP_OVERLAP || op > SHG_OP_GAUSS)
            return fail(SHG_EINVAL, "the fused pass takes overlap, 1/r, erfc, erf and the Gaussian only (got %d)", op);
        int r = check_op(op, omegas[i], precision);
        if (r) return r;
        if (a.out[op]) return fail(SHG_EINVAL, "operator %d listed twice", op);
        if (!outs[i]) return fail(SHG_EINVAL, "NULL output for operator %d", op);
        a.out[op] = outs[i];
        if (op == SHG_OP_ERF) a.w_erf = omegas[i];
        if (op == SHG_OP_ERFC) a.w_erfc = omegas[i];
        if (op == SHG_OP_GAUSS) a.w_gauss = omegas[i];
    }
    if (!off) return fail(SHG_EINVAL, "NULL output offsets");
    a.share_att = (a.out[SHG_OP_ERF] && a.out[SHG_OP_ERFC] && a.w_erf == a.w_erfc) ? 1 : 0;
    return SHG_OK;
}

int shg_plan_2c_exec_fused(shg_plan_t *p, int n_ops, const int *ops, const double *omegas, int precision,
                           const int64_t *off, double *const *outs, void *stream)
{
    Phase phase_("shg:plan_2c_exec_fused");
    g_err.clear();
    ArgsFused a;
    int r = fused_args(p, n_ops, ops, omegas, precision, off, outs, a);
    if (r) return r;
    if (p->d.n_pairs == 0 || p->d.n_tiles == 0) return SHG_OK;
    r = current_device_matches(p->d.basis->device);
    if (r) return r;
    const DeviceTables *t = device_tables();
    if (!t) return SHG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    a.shells = p->d.basis->shells;
    a.prims = p->d.basis->prims;
    a.centers = p->d.basis->centers;
    a.pair_a = p->d.pair_a;
    a.pair_b = p->d.pair_b;
    a.perm = p->d.perm;
    a.tiles = p->d.tiles;
    a.out_off = reinterpret_cast<const long long *>(off);
    a.boys = t->boys;
    a.boys_e = t->boys_e;
    a.cprims = p->d.basis->cprims;
    a.k = consts();
    const bool mixed = precision == SHG_PREC_MIXED;
    const bool persistent = p->d.schedule == SHG_SCHED_PERSISTENT;
    // mixed precision on a persistent plan with both kinds of classes: the FP64
    // tiles (one warp each) and the double-float launch side by side on the plan's
    // side streams
    const bool fork = mixed && persistent && p->d.mixed_fp64_tiles > 0 && p->d.n_tiles > p->d.mixed_fp64_tiles;
    if (fork) {
        r = fork_sides(p, s);
        if (r) return r;
        a.tile_begin = 0;
        a.tile_end = p->d.mixed_fp64_tiles;
        a.counter = nullptr;
        SHG_CUDA(launch_2c_fused(a, 0, false, p->d.side, 32));
    } else if (persistent) {
        // FP64 pass: every tile, or under mixed precision the classes with both
        // l >= kMixedFp64MinL (a prefix of the persistent tile order)
        a.tile_begin = 0;
        a.tile_end = mixed ? p->d.mixed_fp64_tiles : p->d.n_tiles;
        if (a.tile_end > 0) {
            SHG_CUDA(cudaMemsetAsync(p->d.counter, 0, sizeof(int), s));
            a.counter = p->d.counter;
            // the variant applies to the FP64 pass of FP64 executions only
            const int v = mixed ? 0 : p->d.variant;
            SHG_CUDA(launch_2c_fused(a, persistent_grid_2c_fused(p->d.threads, p->d.ctas_per_sm, v), true, s,
                                     p->d.threads, v));
        }
    } else {
        a.counter = nullptr;
        for (int cls = 0; cls < kNClass; ++cls) {
            if (mixed && !mixed_runs_fp64(cls)) continue;
            a.tile_begin = p->d.class_tile_begin[cls];
            a.tile_end = p->d.class_tile_begin[cls + 1];
            if (a.tile_end <= a.tile_begin) continue;
            SHG_CUDA(launch_2c_fused(a, 0, false, s, p->d.threads));
        }
    }
    if (!mixed) return SHG_OK;
    ArgsMixFused m;
    m.shells = p->d.basis->shells;
    m.prims = p->d.basis->mprims;
    m.centers = p->d.basis->mcenters;
    m.pair_a = p->d.pair_a;
    m.pair_b = p->d.pair_b;
    m.perm = p->d.perm;
    m.tiles = p->d.tiles;
    m.out_off = reinterpret_cast<const long long *>(off);
    for (int i = 0; i < 5; ++i) m.out[i] = a.out[i];
    m.w_erf = split2(a.w_erf);
    m.w_erf2 = split2((long double)a.w_erf * a.w_erf);
    m.w_erfc = split2(a.w_erfc);
    m.w_erfc2 = split2((long double)a.w_erfc * a.w_erfc);
    m.w_gauss = split2(a.w_gauss);
    m.share_att = a.share_att;
    m.boys = t->boys_mix;
    m.boys_e = t->boys_e_mix;
    m.km = consts_mix();
    if (persistent) {
        m.tile_begin = p->d.mixed_fp64_tiles;
        m.tile_end = p->d.n_tiles;
        if (m.tile_end <= m.tile_begin) return SHG_OK;
        const cudaStream_t sm = fork ? p->d.side2 : s;
        SHG_CUDA(cudaMemsetAsync(p->d.counter, 0, sizeof(int), sm));
        m.counter = p->d.counter;
        SHG_CUDA(launch_2c_mixed_fused(m, persistent_grid_2c_mixed_fused(p->d.threads, p->d.ctas_per_sm, p->d.variant),
                                       true, sm, p->d.threads, p->d.variant));
        if (fork) return join_sides(p, s);
    } else {
        m.counter = nullptr;
        for (int cls = 0; cls < kNClass; ++cls) {
            if (mixed_runs_fp64(cls)) continue;
            m.tile_begin = p->d.class_tile_begin[cls];
            m.tile_end = p->d.class_tile_begin[cls + 1];
            if (m.tile_end <= m.tile_begin) continue;
            SHG_CUDA(launch_2c_mixed_fused(m, 0, false, s, p->d.threads, p->d.variant));
        }
    }
    return SHG_OK;
}

int shg_graph_2c_create_fused(shg_plan_t *p, int n_ops, const int *ops, const double *omegas, int precision,
                              const int64_t *off, double *const *outs, shg_graph_t **out)
{
    g_err.clear();
    if (!out) return fail(SHG_EINVAL, "out is NULL");
    *out = nullptr;
    ArgsFused chk;
    int r = fused_args(p, n_ops, ops, omegas, precision, off, outs, chk);
    if (r) return r;
    return capture_graph(
        [&](cudaStream_t s) { return shg_plan_2c_exec_fused(p, n_ops, ops, omegas, precision, off, outs, s); }, out);
}

int shg_eval_2c(const shg_basis_t *basis, int64_t n, const int32_t *pa, const int32_t *pb, int op, double omega,
                double screen, int precision, const int64_t *off, double *out, void *stream)
{
    g_err.clear();
    int r = check_op(op, omega, precision);
    if (r) return r;
    if (n == 0) return SHG_OK;
    shg_plan_t *p = nullptr;
    r = shg_plan_2c_create(basis, n, pa, pb, SHG_SCHED_PERSISTENT, stream, &p);
    if (r) return r;
    r = shg_plan_2c_exec(p, op, omega, screen, precision, off, out, stream);
    shg_plan_destroy(p);
    return r;
}

static int eval_3c_common(const shg_basis_t *orb, const shg_basis_t *aux, int64_t n, const int32_t *ta,
                          const int32_t *tt, const int32_t *tb, int precision, const int64_t *off, double *out,
                          const double *w, double *grad_a, double *grad_b, void *stream, double screen = 0.0)
{
    Phase phase_("shg:eval_3c");
    if (!orb || !aux) return fail(SHG_EINVAL, "basis is NULL");
    if (precision != SHG_PREC_FP64 && (precision != SHG_PREC_MIXED || grad_a))
        return fail(SHG_EINVAL, "precision %d not available for the (aab) %s", precision,
                    grad_a ? "gradient" : "integrals");
    if (n < 0 || n > (int64_t)INT32_MAX / 2) return fail(SHG_ERANGE, "n_triples %lld out of range", (long long)n);
    if (n == 0) return SHG_OK;
    if (!ta || !tt || !tb || !off || (!out && !grad_a)) return fail(SHG_EINVAL, "NULL device pointer");
    int r = current_device_matches(orb->d.device);
    if (r) return r;
    if (aux->d.device != orb->d.device) return fail(SHG_EINVAL, "orb and aux bases live on different devices");
    int *ranks[2], *rank3 = nullptr;
    const DeviceTables *t = device_tables_impl(ranks, &rank3);
    if (!t) return SHG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;

    const int64_t max_tiles = n / kTile + std::min<int64_t>(n, kNBins3) + 1;
    const size_t bytes_perm = sizeof(int32_t) * (size_t)n;
    const size_t bytes_tiles = sizeof(Tile) * (size_t)max_tiles;
    const size_t bytes_ws = sizeof(int) * plan_ws_ints(n, kNBins3, kNClass3);
    const size_t bytes = bytes_perm + bytes_tiles + bytes_ws + 512;
    void *blk = nullptr;
    SHG_CUDA(cudaMallocAsync(&blk, bytes, s));
    PlanDev d;
    d.basis = &orb->d;
    d.aux = &aux->d;
    d.kind = 3;
    d.n_pairs = n;
    d.schedule = SHG_SCHED_PERSISTENT;
    d.pair_a = ta;
    d.trip_t = tt;
    d.pair_b = tb;
    char *c = (char *)blk;
    d.tiles = (Tile *)c;                 c += (bytes_tiles + 15) / 16 * 16;
    d.perm = (int32_t *)c;               c += (bytes_perm + 15) / 16 * 16;
    d.counter = (int *)c;                c += 16;
    int *ws = (int *)c;
    // the end of the build summary: sm[0] = tile count, sm[1] = error flags
    int sm[2] = {0, 0};
    cudaError_t e = launch_plan_build(d, ws, kNBins3, rank3, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sm, plan_summary(ws, kNBins3) + kNClass3, sizeof(sm), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const int h[2] = {sm[1], sm[0]};              // error flags, tile count
    if (e != cudaSuccess) {
        cudaFreeAsync(blk, s);
        return fail(SHG_ECUDA, "(aab) planning: %s", cudaGetErrorString(e));
    }
    if (h[0]) {
        cudaFreeAsync(blk, s);
        if (h[0] & 1) return fail(SHG_EINVAL, "triple list holds a shell index out of range");
        if (h[0] & 2) return fail(SHG_EINVAL, "a and a~ of a triple are not on the same center");
        return fail(SHG_EINVAL, "la + la~ exceeds %d", kLmaxAabA);
    }
    Args3c a;
    a.orb_shells = orb->d.shells;
    a.aux_shells = aux->d.shells;
    a.orb_prims = orb->d.prims;
    a.aux_prims = aux->d.prims;
    a.orb_centers = orb->d.centers;
    a.aux_centers = aux->d.centers;
    a.t_a = ta;
    a.t_t = tt;
    a.t_b = tb;
    a.perm = d.perm;
    a.tiles = d.tiles;
    a.tile_begin = 0;
    a.tile_end = h[1];
    a.counter = d.counter;
    a.out_off = reinterpret_cast<const long long *>(off);
    a.out = out;
    a.gaunt_base = t->gaunt_base;
    a.gaunt_row = t->gaunt_row;
    a.gaunt = t->gaunt;
    a.w_off = grad_a ? reinterpret_cast<const long long *>(off) : nullptr;
    a.w = w;
    a.grad_a = grad_a;
    a.grad_b = grad_b;
    a.screen_thresh = grad_a ? 0.0 : screen;
    a.orb_screen = orb->d.screen;
    a.aux_screen = aux->d.screen;
    a.k = consts();
    a.k3 = consts3();
    a.km = consts_mix();
    e = cudaMemsetAsync(d.counter, 0, sizeof(int), s);
    if (e == cudaSuccess && h[1] > 0) e = launch_3c(a, precision, persistent_grid_3c(precision), s);
    cudaFreeAsync(blk, s);
    if (e != cudaSuccess) return fail(SHG_ECUDA, "(aab) launch: %s", cudaGetErrorString(e));
    return SHG_OK;
}

int shg_eval_3c_aab(const shg_basis_t *orb, const shg_basis_t *aux, int64_t n, const int32_t *ta, const int32_t *tt,
                    const int32_t *tb, int precision, double screen, const int64_t *off, double *out, void *stream)
{
    g_err.clear();
    if (!(screen >= 0.0) || !std::isfinite(screen)) return fail(SHG_EINVAL, "screening threshold must be >= 0");
    if (n > 0 && !out) return fail(SHG_EINVAL, "NULL output");
    return eval_3c_common(orb, aux, n, ta, tt, tb, precision, off, out, nullptr, nullptr, nullptr, stream, screen);
}

int shg_eval_2c_grad(const shg_basis_t *basis, int64_t n, const int32_t *pa, const int32_t *pb, int op, double omega,
                     int precision, const int64_t *w_off, const double *w, double *grad_a, double *grad_b,
                     void *stream)
{
    Phase phase_("shg:eval_2c_grad");
    g_err.clear();
    int r = check_op(op, omega, precision);
    if (r) return r;
    if (n == 0) return SHG_OK;
    if (!w_off || !w || !grad_a) return fail(SHG_EINVAL, "NULL device pointer");
    shg_plan_t *p = nullptr;
    r = shg_plan_2c_create(basis, n, pa, pb, SHG_SCHED_PERSISTENT, stream, &p);
    if (r) return r;
    const DeviceTables *t = device_tables();
    cudaStream_t s = (cudaStream_t)stream;
    Args2c a{};
    a.shells = basis->d.shells;
    a.prims = basis->d.prims;
    a.centers = basis->d.centers;
    a.pair_a = pa;
    a.pair_b = pb;
    a.perm = p->d.perm;
    a.tiles = p->d.tiles;
    a.tile_begin = 0;
    a.tile_end = p->d.n_tiles;
    a.counter = p->d.counter;
    a.omega = omega;
    a.boys = t->boys;
    a.boys_e = t->boys_e;
    a.w_off = reinterpret_cast<const long long *>(w_off);
    a.w = w;
    a.grad_a = grad_a;
    a.grad_b = grad_b;
    a.k = consts();
    // mixed precision: the classes with both l >= kMixedFp64MinL (the leading
    // tiles of the persistent order) in FP64, the others with double-float
    // radial orders and the FP64 angular part.  With both kinds present the
    // two launches run side by side on the plan's side streams (as in
    // shg_plan_2c_exec_fused): the FP64 tiles one warp each, statically.
    const bool mixed = precision == SHG_PREC_MIXED;
    const bool fork = mixed && p->d.mixed_fp64_tiles > 0 && p->d.n_tiles > p->d.mixed_fp64_tiles;
    a.tile_end = mixed ? p->d.mixed_fp64_tiles : p->d.n_tiles;
    cudaError_t e = cudaSuccess;
    if (fork) {
        r = fork_sides(p, s);
        if (r) {
            shg_plan_destroy(p);
            return r;
        }
        a.counter = nullptr;
        e = launch_2c_grad(a, op, SHG_PREC_FP64, 0, p->d.side, 32);
    } else if (a.tile_end > 0) {
        e = cudaMemsetAsync(p->d.counter, 0, sizeof(int), s);
        if (e == cudaSuccess) e = launch_2c_grad(a, op, SHG_PREC_FP64, persistent_grid_2c_grad(op, SHG_PREC_FP64), s);
    }
    if (e == cudaSuccess && mixed && p->d.n_tiles > p->d.mixed_fp64_tiles) {
        ArgsGradMix gm;
        gm.g = a;
        ArgsMix &m = gm.m;
        m.shells = basis->d.shells;
        m.prims = basis->d.mprims;
        m.centers = basis->d.mcenters;
        m.pair_a = pa;
        m.pair_b = pb;
        m.perm = p->d.perm;
        m.tiles = p->d.tiles;
        m.tile_begin = p->d.mixed_fp64_tiles;
        m.tile_end = p->d.n_tiles;
        m.counter = p->d.counter;
        m.out_off = nullptr;
        m.out = nullptr;
        m.omega = split2(omega);
        m.omega2 = split2((long double)omega * omega);
        m.omega_d = omega;
        m.screen_thresh = 0.0;
        m.screen = basis->d.screen;
        m.boys = t->boys_mix;
        m.boys_e = t->boys_e_mix;
        m.km = consts_mix();
        const cudaStream_t sm = fork ? p->d.side2 : s;
        e = cudaMemsetAsync(p->d.counter, 0, sizeof(int), sm);
        if (e == cudaSuccess) e = launch_2c_grad_mixed(gm, op, sm);
    }
    // the plan's memory is released in the order of s: join first, also after
    // a failed launch (the other side stream may hold a running kernel)
    if (fork) r = join_sides(p, s);
    shg_plan_destroy(p);
    if (r) return r;
    if (e != cudaSuccess) return fail(SHG_ECUDA, "gradient launch: %s", cudaGetErrorString(e));
    return SHG_OK;
}

int shg_eval_3c_aab_grad(const shg_basis_t *orb, const shg_basis_t *aux, int64_t n, const int32_t *ta,
                         const int32_t *tt, const int32_t *tb, int precision, const int64_t *w_off, const double *w,
                         double *grad_a, double *grad_b, void *stream)
{
    g_err.clear();
    if (n > 0 && (!w || !w_off || !grad_a)) return fail(SHG_EINVAL, "NULL device pointer");
    return eval_3c_common(orb, aux, n, ta, tt, tb, precision, w_off, nullptr, w, grad_a, grad_b, stream);
}

// ------------------------------------------------------------------------- //
// Family plans                                                               //
// ------------------------------------------------------------------------- //
void shg_family_plan_destroy(shg_family_plan_t *fp)
{
    if (!fp) return;
    if (fp->plan_fam) shg_plan_destroy(fp->plan_fam);
    if (fp->plan_rest) shg_plan_destroy(fp->plan_rest);
    cudaFree(fp->block);
    delete fp;
}

int shg_family_plan_create(const shg_basis_t *basis, int64_t n, const int32_t *d_pa, const int32_t *d_pb, void *stream,
                           shg_family_plan_t **out)
{
    Phase phase_("shg:family_plan_create");
    g_err.clear();
    if (!basis || !out || n < 0 || (n > 0 && (!d_pa || !d_pb))) return fail(SHG_EINVAL, "bad argument");
    if (n > (int64_t)INT32_MAX / 2) return fail(SHG_ERANGE, "n_pairs %lld out of range", (long long)n);
    *out = nullptr;
    int r = current_device_matches(basis->d.device);
    if (r) return r;
    const BasisDev &bd = basis->d;
    std::vector<int32_t> pa(n), pb(n);
    if (n > 0) {
        SHG_CUDA(cudaMemcpy(pa.data(), d_pa, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        SHG_CUDA(cudaMemcpy(pb.data(), d_pb, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    }
    for (int64_t i = 0; i < n; ++i)
        if (pa[i] < 0 || pa[i] >= bd.n_shells || pb[i] < 0 || pb[i] >= bd.n_shells)
            return fail(SHG_EINVAL, "pair list holds a shell index outside 0..%d", bd.n_shells - 1);
    // family subset, grouped by (family of a, family of b)
    std::vector<std::pair<int64_t, int32_t>> keyed;
    std::vector<int32_t> rest;
    keyed.reserve(n);
    for (int64_t i = 0; i < n; ++i) {
        const int fa = bd.h_fam[pa[i]], fb = bd.h_fam[pb[i]];
        if ((int64_t)bd.h_fam_k[fa] * bd.h_fam_k[fb] <= kFamPP)
            keyed.emplace_back((int64_t)fa * bd.n_fams + fb, (int32_t)i);
        else
            rest.push_back((int32_t)i);
    }
    std::stable_sort(keyed.begin(), keyed.end(), [](const std::pair<int64_t, int32_t> &x,
                                                    const std::pair<int64_t, int32_t> &y) { return x.first < y.first; });
    const int64_t nf = (int64_t)keyed.size(), nr = (int64_t)rest.size();
    std::vector<int32_t> idx_f(nf), pa_f(nf), pb_f(nf), pa_r(nr), pb_r(nr);
    std::vector<FamGroup> groups;
    for (int64_t i = 0; i < nf; ++i) {
        const int32_t o = keyed[i].second;
        idx_f[i] = o;
        pa_f[i] = pa[o];
        pb_f[i] = pb[o];
        const int la = bd.h_l[pa[o]], lb = bd.h_l[pb[o]];
        if (i == 0 || keyed[i].first != keyed[i - 1].first) {
            const int fa = bd.h_fam[pa[o]], fb = bd.h_fam[pb[o]];
            groups.push_back(FamGroup{bd.h_fam_prim[fa], bd.h_fam_k[fa], bd.h_fam_prim[fb], bd.h_fam_k[fb], (int)i, 0,
                                      std::max(la, lb), la + lb, bd.h_center[pa[o]], bd.h_center[pb[o]], 0, 0});
        }
        FamGroup &g = groups.back();
        g.count += 1;
        g.kmin = std::min(g.kmin, std::max(la, lb));
        g.kmax = std::max(g.kmax, la + lb);
    }
    for (int64_t i = 0; i < nr; ++i) {
        pa_r[i] = pa[rest[i]];
        pb_r[i] = pb[rest[i]];
    }
    shg_family_plan_t *fp = new (std::nothrow) shg_family_plan_t;
    if (!fp) return fail(SHG_ENOMEM, "host allocation failed");
    fp->basis = &bd;
    fp->n = n;
    fp->n_fam = nf;
    fp->n_rest = nr;
    fp->n_groups = (int)groups.size();
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_i32f = al(sizeof(int32_t) * (size_t)std::max<int64_t>(nf, 1));
    const size_t b_i32r = al(sizeof(int32_t) * (size_t)std::max<int64_t>(nr, 1));
    const size_t b_grp = al(sizeof(FamGroup) * (size_t)std::max(fp->n_groups, 1));
    const size_t b_o = al(sizeof(double) * kJmax * (size_t)std::max<int64_t>(nf, 1));
    const size_t b_offf = al(sizeof(int64_t) * (size_t)std::max<int64_t>(nf, 1));
    const size_t b_offr = al(sizeof(int64_t) * (size_t)std::max<int64_t>(nr, 1));
    const size_t total = 3 * b_i32f + 3 * b_i32r + b_grp + 256 + b_o + b_offf + b_offr;
    if (cudaMalloc(&fp->block, total) != cudaSuccess) {
        delete fp;
        return fail(SHG_ENOMEM, "family plan: cudaMalloc of %zu bytes failed", total);
    }
    char *c = (char *)fp->block;
    fp->d_idx_fam = (int32_t *)c; c += b_i32f;
    fp->d_pa_fam = (int32_t *)c; c += b_i32f;
    fp->d_pb_fam = (int32_t *)c; c += b_i32f;
    fp->d_idx_rest = (int32_t *)c; c += b_i32r;
    fp->d_pa_rest = (int32_t *)c; c += b_i32r;
    fp->d_pb_rest = (int32_t *)c; c += b_i32r;
    fp->d_groups = (FamGroup *)c; c += b_grp;
    fp->d_counter = (int *)c; c += 256;
    fp->d_o = (double *)c; c += b_o;
    fp->d_off_fam = (int64_t *)c; c += b_offf;
    fp->d_off_rest = (int64_t *)c;
    bool ok = true;
    if (nf > 0)
        ok = cudaMemcpy(fp->d_idx_fam, idx_f.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(fp->d_pa_fam, pa_f.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(fp->d_pb_fam, pb_f.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(fp->d_groups, groups.data(), sizeof(FamGroup) * groups.size(), cudaMemcpyHostToDevice) ==
                 cudaSuccess;
    if (ok && nr > 0)
        ok = cudaMemcpy(fp->d_idx_rest, rest.data(), sizeof(int32_t) * nr, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(fp->d_pa_rest, pa_r.data(), sizeof(int32_t) * nr, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(fp->d_pb_rest, pb_r.data(), sizeof(int32_t) * nr, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        shg_family_plan_destroy(fp);
        return fail(SHG_ECUDA, "family plan: upload failed");
    }
    if (nf > 0 && (r = shg_plan_2c_create(basis, nf, fp->d_pa_fam, fp->d_pb_fam, SHG_SCHED_PERSISTENT, stream,
                                          &fp->plan_fam)) != SHG_OK) {
        shg_family_plan_destroy(fp);
        return r;
    }
    if (nr > 0 && (r = shg_plan_2c_create(basis, nr, fp->d_pa_rest, fp->d_pb_rest, SHG_SCHED_PERSISTENT, stream,
                                          &fp->plan_rest)) != SHG_OK) {
        shg_family_plan_destroy(fp);
        return r;
    }
    *out = fp;
    return SHG_OK;
}

int64_t shg_family_plan_counts(const shg_family_plan_t *fp, int64_t *n_family_pairs, int64_t *n_groups)
{
    if (!fp) return -1;
    if (n_family_pairs) *n_family_pairs = fp->n_fam;
    if (n_groups) *n_groups = fp->n_groups;
    return fp->n;
}

int shg_family_plan_exec(shg_family_plan_t *fp, int op, double omega, const int64_t *off, double *out, void *stream)
{
    Phase phase_("shg:family_plan_exec");
    g_err.clear();
    if (!fp) return fail(SHG_EINVAL, "plan is NULL");
    int r = check_op(op, omega, SHG_PREC_FP64);
    if (r) return r;
    if (op == SHG_OP_RA2N) return fail(SHG_EINVAL, "SHG_OP_RA2N has no family path (its radial term depends on la)");
    if (fp->n == 0) return SHG_OK;
    if (!off || !out) return fail(SHG_EINVAL, "NULL output");
    r = current_device_matches(fp->basis->device);
    if (r) return r;
    const DeviceTables *t = device_tables();
    if (!t) return SHG_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (fp->n_fam > 0) {
        SHG_CUDA(launch_gather_i64(off, fp->d_idx_fam, fp->n_fam, fp->d_off_fam, s));
        ArgsFam a;
        a.shells = fp->basis->shells;
        a.prims = fp->basis->prims;
        a.centers = fp->basis->centers;
        a.pair_a = fp->d_pa_fam;
        a.pair_b = fp->d_pb_fam;
        a.groups = fp->d_groups;
        a.n_groups = fp->n_groups;
        a.counter = fp->d_counter;
        a.o_pre = fp->d_o;
        a.omega = omega;
        a.boys = t->boys;
        a.boys_e = t->boys_e;
        a.k = consts();
        SHG_CUDA(cudaMemsetAsync(fp->d_counter, 0, sizeof(int), s));
        SHG_CUDA(launch_family_radial(a, op, s));
        r = exec_fp64(fp->plan_fam, 7 /* OP_PRE */, omega, 0.0, fp->d_off_fam, out, fp->d_o, s);
        if (r) return r;
    }
    if (fp->n_rest > 0) {
        SHG_CUDA(launch_gather_i64(off, fp->d_idx_rest, fp->n_rest, fp->d_off_rest, s));
        r = shg_plan_2c_exec(fp->plan_rest, op, omega, 0.0, SHG_PREC_FP64, fp->d_off_rest, out, stream);
        if (r) return r;
    }
    return SHG_OK;
}

int shg_scatter_2c(const shg_basis_t *b, int64_t n, const int32_t *pa, const int32_t *pb, const int64_t *boff,
                   const double *blocks, const int64_t *ao, int64_t ld, int symmetric, double *M, void *stream)
{
    g_err.clear();
    if (!b || n < 0 || ld < 1) return fail(SHG_EINVAL, "bad argument");
    if (n == 0) return SHG_OK;
    if (!pa || !pb || !boff || !blocks || !ao || !M) return fail(SHG_EINVAL, "NULL device pointer");
    int r = current_device_matches(b->d.device);
    if (r) return r;
    SHG_CUDA(launch_scatter_2c(b->d.shells, n, pa, pb, boff, blocks, ao, ld, symmetric, M, (cudaStream_t)stream));
    return SHG_OK;
}

int shg_gather_2c(const shg_basis_t *b, int64_t n, const int32_t *pa, const int32_t *pb, const int64_t *boff,
                  const double *M, const int64_t *ao, int64_t ld, int symmetric, double *blocks, void *stream)
{
    g_err.clear();
    if (!b || n < 0 || ld < 1) return fail(SHG_EINVAL, "bad argument");
    if (n == 0) return SHG_OK;
    if (!pa || !pb || !boff || !blocks || !ao || !M) return fail(SHG_EINVAL, "NULL device pointer");
    int r = current_device_matches(b->d.device);
    if (r) return r;
    SHG_CUDA(launch_gather_2c(b->d.shells, n, pa, pb, boff, M, ao, ld, symmetric, blocks, (cudaStream_t)stream));
    return SHG_OK;
}

int shg_reduce_centers(const shg_basis_t *b, int64_t n, const int32_t *pa, const int32_t *pb, const double *ga,
                       const double *gb, double *out, void *stream)
{
    g_err.clear();
    if (!b || n < 0) return fail(SHG_EINVAL, "bad argument");
    if (n == 0) return SHG_OK;
    if (!pa || !pb || !ga || !gb || !out) return fail(SHG_EINVAL, "NULL device pointer");
    int r = current_device_matches(b->d.device);
    if (r) return r;
    SHG_CUDA(launch_reduce_centers(b->d.shells, n, pa, pb, ga, gb, out, (cudaStream_t)stream));
    return SHG_OK;
}

int shg_debug_boys(int64_t n, const double *T, int nmax, double *F, void *stream)
{
    g_err.clear();
    if (n < 0 || nmax < 0 || nmax >= kBoysN) return fail(SHG_EINVAL, "bad n or nmax (nmax <= %d)", kBoysN - 1);
    if (n == 0) return SHG_OK;
    if (!T || !F) return fail(SHG_EINVAL, "NULL pointer");
    const DeviceTables *t = device_tables();
    if (!t) return SHG_ECUDA;
    SHG_CUDA(launch_debug_boys(n, T, nmax, F, *t, (cudaStream_t)stream));
    return SHG_OK;
}

int shg_measure_alu_peak(int kind, int iters, double *flops, void *stream)
{
    g_err.clear();
    if (kind < 0 || kind > 2 || iters < 1 || !flops) return fail(SHG_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    SHG_CUDA(cudaGetDevice(&dev));
    SHG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = sms * 8;
    double *sink = nullptr;
    SHG_CUDA(cudaMalloc(&sink, 16));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch_alu_probe(kind, iters, blocks, threads, sink, s);   // warm-up
    cudaEventRecord(e0, s);
    cudaError_t le = launch_alu_probe(kind, iters, blocks, threads, sink, s);
    cudaEventRecord(e1, s);
    cudaError_t se = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (le != cudaSuccess || se != cudaSuccess) return fail(SHG_ECUDA, "probe failed");
    // flops per thread per chain step: one FMA (2) for kinds 0 and 1; kind 2 a
    // warp-wide m8n8k4 MMA (512 flops) shared by the warp's 32 threads (16)
    const double per = kind == 2 ? 16.0 : 2.0;
    *flops = per * 8.0 * (double)iters * threads * (double)blocks / (ms * 1e-3);
    return SHG_OK;
}

}  // extern "C"
