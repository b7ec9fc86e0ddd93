// Internal declarations shared by the host API (shg_api.cpp) and the CUDA
// kernels (shg_*.cu).  Plain C++: no device code, no torch types.
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>

namespace shg {

constexpr int kLmax2c = 6;        // largest l of a two-center shell
constexpr int kLmaxAabA = 10;     // largest la + la~ of an (aab) triple
constexpr int kLmaxR = 10;        // largest l of the scaled solid harmonics table
constexpr int kKmax = 32;         // largest contraction length
constexpr int kJmax = 7;          // min(la, lb) + 1 <= 7
constexpr int kRa2nMax = 5;                // largest n of the (a|r_a^{2n}|b) operator
constexpr int kNClass = (kLmax2c + 1) * (kLmax2c + 1);
constexpr int kTile = 32;         // pairs per warp tile
// Two-center classes that the mixed-precision passes evaluate in FP64: both
// la and lb >= kMixedFp64MinL (J = min(la, lb) + 1 >= 5).  There the sum over
// j of Eq. final_r12int_ab cancels by up to ~1e4 (l = 6, exponents to 5000),
// beyond what double-float (2^-44 of the largest term) carries to 1e-10.
constexpr int kMixedFp64MinL = 4;
inline bool mixed_runs_fp64(int cls) { return cls / 7 >= kMixedFp64MinL && cls % 7 >= kMixedFp64MinL; }

// Boys tables: Taylor coefficients c_t = F_{n+t}(T_i)/t!, t = 0..6, about the
// grid points T_i = i/32, i = 0..kBoysGrid-1 (|delta| <= 1/64), n < kBoysN;
// Taylor expansion about the nearest grid point.
//   FP64 table: per (i, n) kBoysStride doubles: c0..c3 as doubles, c4..c6 as
//     floats (and one float of padding), 48 bytes.
//   double-float table: per (i, n) three float4: c0..c2 as hi/lo float pairs,
//     c3..c6 as floats (and two floats of padding), 48 bytes.
// Above kBoysTmax, F_n(T) = (2n-1)!! / (2T)^n sqrt(pi/(4T)) to better than
// 1e-30 relative for n <= 16 (the neglected terms carry exp(-T)).
constexpr int kBoysGrid = 3841;     // covers T < 120 at step 1/32
constexpr int kBoysStride = 6;
constexpr double kBoysTmax = 120.0;
constexpr int kBoysN = 16;          // orders n = 0..15 from the tables

// Per-shell screening data (host-computed): smallest exponent, sum |N c| over
// the primitives, and (l / (alpha_min e))^{l/2} (1 for l = 0).
struct alignas(32) ScreenRec {
    double amin, sabs, lfac, pad;
};

// Per-shell record on the device (16 bytes): l, K, first primitive, center.
struct ShellRec {
    int l, nprim, prim_off, center;
};

// Center coordinates on the device (x, y, z, padding), 32-byte aligned.
struct alignas(32) Vec4 {
    double x, y, z, w;
};

// Per-primitive record on the device (32 bytes).
//   alpha, 1/alpha, w2c = N_l c / (2 alpha)^l (the two-center weight of
//   Eq. O_rab2_deriv), wN = N_l c (normalised coefficient, used by (aab)).
struct alignas(32) PrimRec {
    double alpha, inv_alpha, w2c, wN;
};

// Real Gaunt coefficient entry G = int Y_{L,M} Y_{l,m} Y_{l~,m~} dOmega.
struct GauntEnt {
    double g;
    int L, M;
};

// Per-primitive weights of the Coulomb-type radial terms (Table S1), 16 bytes:
//   cw = sqrt(2 pi^{5/2}) w2c / alpha   so that 2 pi^{5/2} w / (alpha beta sqrt(c)) = cw_a cw_b / sqrt(c)
//   fw = w2c alpha^{-3/2}       the far-field weight: for T >= kBoysTmax every order of
//                               w 2 pi^{5/2} / (alpha beta sqrt(c)) (-rho)^n F_n(T) equals
//                               fw_a fw_b pi^3 (-1)^n (2n-1)!! (2R^2)^{-n} / R
struct alignas(16) CoulPrim {
    double cw, fw;
};

// Mixed-precision (double-float) copies: each value v as float2 (hi, lo),
// hi = fl32(v), lo = fl32(v - hi); fw is the FP64 far-field weight of CoulPrim.
struct alignas(32) MixPrim {
    float2 alpha, inv_alpha, wN;
    double fw;
};
struct alignas(32) MixCenter {
    float2 x, y, z, pad;
};

// Small constant tables, passed by value in kernel parameters.
struct Consts {
    double A[kLmaxR + 1][kLmaxR + 1];      // A_{l,mu} of Eq. (A)
    double jB[kJmax][kJmax];               // (2j-1)!! B_{j,kappa}, Eq. (B)
    double pow2[32];                       // 2^k
    double dint[64];                       // (double) n
    double inv_int[192];                   // 1/n (0 for n = 0)
    double dfact[32];                      // (2n-1)!!, (-1)!! = 1
    double binom[kRa2nMax + 1][kRa2nMax + 1];  // C(n, j)
    double ra2n_k[kRa2nMax + 1][kRa2nMax + 1]; // 2^{d-m} (2m+1)!! C(m,d) / (2d+1)!!, [m][d], d <= m
    // low parts of jB and inv_int (value - double(value), from long double) for
    // the double-double (a|r_a^{2n}|b) path
    double jB_lo[kJmax][kJmax];
    double inv_int_lo[64];
};

void fill_consts(Consts &k);

// Double-float constants of the mixed-precision kernels.
struct ConstsMix {
    float2 A[kLmaxR + 1][kLmaxR + 1];      // A_{l,mu} (l <= 10: two-center and (aab) L_a)
    float2 jB[kJmax][kJmax];               // (2j-1)!! B_{j,kappa}
    float2 inv_int[128];                   // 1/n
    float2 inv_fact[14];                   // 1/t!
    float inv_fact_f[14];
    float2 pi32, pi3, two_pi52, sqrt_pi_half, two_pi;
    float2 dfact[kBoysN];                  // (2n-1)!!
};

void fill_consts_mix(ConstsMix &k);

// Device-resident tables owned by the library, one set per device.
struct DeviceTables {
    const double *boys;   // [kBoysGrid][kBoysN][kBoysStride] (layout above)
    const double *boys_e; // [kBoysGrid] exp(-T_i), T_i = i/32
    // real Gaunt coefficients for l, l~ <= 6 with l + l~ <= kLmaxAabA:
    // rows (l, l~, m, m~) -> entries [gaunt_row[r], gaunt_row[r+1]) of gaunt
    const int *gaunt_base;     // [7*7] first row of the (l, l~) block
    const int *gaunt_row;      // row pointers
    const GauntEnt *gaunt;     // entries
    const float4 *boys_mix;    // [kBoysGrid][kBoysN][3] (layout above)
    const float2 *boys_e_mix;  // [kBoysGrid] exp(-T_i) as hi/lo
};

// Extra constants of the three-index kernels (by value).
struct Consts3 {
    double binom[18][18];       // binom(k, i)
    double dd[6][6][6];         // d_{m,j} j!/(j-i)!: D_m^{(i)}(x) = sum_j dd[m][i][j] x^{j-i}
    double bj[11][6][6];        // binom(p, j) (L)_j (rising factorial, (0)_0 = 1)
    double sqrt_int[32];        // sqrt(n)
};

void fill_consts3(Consts3 &k);

// Returns the tables of the current device (created on first use), or null
// and sets the error message.
const DeviceTables *device_tables();

// Tables of the current device if a basis was already created on it (never
// allocates); ranks[0..1] receive the bin rank tables of both schedules.
const DeviceTables *device_tables_if_ready(const int **ranks);

// Host helpers of shg_api.cpp.
int fail(int code, const char *fmt, ...);          // sets shg_last_error(), returns code
void clear_error();                                // empties shg_last_error() (start of a call)
const Consts &consts();                            // constant tables (host copy)
int check_op(int op, double omega, int precision);  // operator / omega / precision check

// Host generation of the Boys table (long double arithmetic).
void make_boys_table(int per_unit, int ngrid, int nterms, double *tab, double *etab);

struct BasisDev {
    int n_shells = 0, n_centers = 0;
    int64_t n_prims = 0;
    int device = 0;
    ShellRec *shells = nullptr;   // device
    PrimRec *prims = nullptr;     // device
    Vec4 *centers = nullptr;      // device
    MixPrim *mprims = nullptr;    // device, double-float copies for the mixed path
    CoulPrim *cprims = nullptr;   // device, Coulomb-type weights (fused passes)
    ScreenRec *screen = nullptr;  // device, per-shell screening data
    MixCenter *mcenters = nullptr;
    // shg_basis_set_centers staging (allocated on its first call): raw
    // coordinates, packed copies checked before they replace the live ones,
    // and the smallest non-finite center index
    double *stage_raw = nullptr;
    Vec4 *stage_ctr = nullptr;
    MixCenter *stage_mctr = nullptr;
    int *stage_bad = nullptr;
    // host copies used for validation and offsets
    int32_t *h_l = nullptr, *h_nprim = nullptr, *h_center = nullptr;
    // families: shells on one center with bitwise-identical exponent lists
    int32_t *h_fam = nullptr;                           // family of each shell
    int32_t *h_fam_prim = nullptr, *h_fam_k = nullptr;  // per family: first primitive record, K
    int n_fams = 0;
};

// A warp's unit of work: up to kTile consecutive entries of the sorted list,
// all of one class.  cls = la*7 + lb (two-center) or (la*7 + la~)*7 + lb.
struct Tile {
    int start, count, cls, pad;
};

constexpr int kKbins2c = kKmax * kKmax;      // two-center bins per class: Ka*Kb - 1
constexpr int kNBins2c = kNClass * kKbins2c;
constexpr int kNClass3 = 7 * 7 * 7;          // (la, la~, lb) classes
constexpr int kKbins3c = 512;                // three-index bins per class: min(Ka*Ka~*Kb, 512) - 1


struct PlanDev {
    const BasisDev *basis = nullptr;
    const BasisDev *aux = nullptr;  // three-index plans: basis of b
    int kind = 2;                   // 2: pairs, 3: (aab) triples
    int64_t n_pairs = 0;
    int schedule = 0;
    const int32_t *pair_a = nullptr, *pair_b = nullptr;   // device, caller-owned
    const int32_t *trip_t = nullptr;                      // a~ of triples (kind 3)
    int32_t *perm = nullptr;       // device [n_pairs], pairs sorted by bin
    Tile *tiles = nullptr;         // device [n_tiles]
    int *counter = nullptr;        // device, persistent work counter
    int n_tiles = 0;
    int class_tile_begin[kNClass + 1] = {};   // host, per-class tile ranges (class-major)
    int mixed_fp64_tiles = 0;      // persistent order: leading tiles of the classes that the
                                   // mixed-precision passes run in FP64 (both l >= kMixedFp64MinL)
    int threads = 128;             // launch shape (autotuned): threads per CTA (32, 64 or 128)
    int ctas_per_sm = 0;           // persistent CTAs per SM, 0 = occupancy limit
    int variant = 1;               // compiled variant of the fused kernels (shg_plan_2c_set_variant)
                                   // (0: free register count, 1: <= 96 registers, 5 CTAs per SM)
    // streams of a mixed-precision pass that runs the FP64 high-l tiles beside the
    // double-float launch (created on first use): side (highest priority) takes the
    // FP64 launch, side2 the double-float one; the caller's stream forks and joins
    cudaStream_t side = nullptr, side2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    void *owner_block = nullptr;   // device allocation holding all of the above
    cudaStream_t stream = nullptr;
};

// Arguments of the two-center kernels (by value).
struct Args2c {
    const ShellRec *shells;
    const PrimRec *prims;
    const Vec4 *centers;
    const int32_t *pair_a, *pair_b;
    const int32_t *perm;
    const Tile *tiles;
    int tile_begin, tile_end;
    int *counter;                 // persistent schedule (null: static)
    const long long *out_off;
    double *out;
    double omega;
    double screen_thresh;         // > 0: overlap / Gaussian-operator pairs bounded below it write zeros
    const ScreenRec *screen;
    const double *boys, *boys_e;
    // gradient kernels only: upstream weights W (blocks at w + w_off[p]) and
    // the per-pair outputs dI/dR_a . W and dI/dR_b . W
    const long long *w_off;
    const double *w;
    double *grad_a, *grad_b;
    // family path: contracted radial terms O[j] of pair p precomputed at
    // o_pre[p * kJmax + j] (read by the OP_PRE instantiation only)
    const double *o_pre = nullptr;
    Consts k;
};

// Fused multi-operator FP64 pass (overlap, 1/r, erfc, erf, Gaussian): one
// output per requested operator (null = not requested), all with the block
// offsets out_off.
struct ArgsFused {
    const ShellRec *shells;
    const PrimRec *prims;
    const Vec4 *centers;
    const int32_t *pair_a, *pair_b;
    const int32_t *perm;
    const Tile *tiles;
    int tile_begin, tile_end;
    int *counter;                 // persistent schedule (null: static)
    const long long *out_off;
    double *out[5];               // indexed by OP_OVERLAP .. OP_GAUSS
    double w_erf, w_erfc, w_gauss;
    int share_att;                // erf and erfc requested with the same omega
    const double *boys, *boys_e;
    const CoulPrim *cprims;       // Coulomb-type weights per primitive
    Consts k;
};

// Family basis sets: a group of shell pairs whose shells a share one
// exponent set (family) on one center, and likewise for b.
constexpr int kFamPP = 100;                // largest K_a * K_b of the family path
constexpr int kFamOrd = 2 * kLmax2c + 1;   // derivative orders 0..la+lb
struct FamGroup {
    int fa_prim, fa_k, fb_prim, fb_k;   // first primitive record and K of each family
    int start, count;                   // range of the group in the grouped pair order
    int kmin, kmax;                     // derivative orders the group's pairs need
    int ca, cb, pad0, pad1;             // centers
};
struct ArgsFam {
    const ShellRec *shells;
    const PrimRec *prims;
    const Vec4 *centers;
    const int32_t *pair_a, *pair_b;     // the family subset of the pair list, in group order
    const FamGroup *groups;
    int n_groups;
    int *counter;
    double *o_pre;                      // [n_subset][kJmax]
    double omega;
    const double *boys, *boys_e;
    Consts k;
};

// Arguments of the mixed-precision two-center kernels (by value).
struct ArgsMix {
    const ShellRec *shells;
    const MixPrim *prims;
    const MixCenter *centers;
    const int32_t *pair_a, *pair_b;
    const int32_t *perm;
    const Tile *tiles;
    int tile_begin, tile_end;
    int *counter;
    const long long *out_off;
    double *out;
    float2 omega, omega2;
    double omega_d, screen_thresh;
    const ScreenRec *screen;
    const float4 *boys;
    const float2 *boys_e;
    ConstsMix km;
};

// Mixed-precision gradient: double-float radial orders (m) and the FP64 angular
// vector-Jacobian product (g: centers, constants, upstream weights, outputs).
struct ArgsGradMix;

// Fused multi-operator pass in double-float (outputs as ArgsFused).
struct ArgsMixFused {
    const ShellRec *shells;
    const MixPrim *prims;
    const MixCenter *centers;
    const int32_t *pair_a, *pair_b;
    const int32_t *perm;
    const Tile *tiles;
    int tile_begin, tile_end;
    int *counter;
    const long long *out_off;
    double *out[5];                     // indexed by OP_OVERLAP .. OP_GAUSS
    float2 w_erf, w_erf2, w_erfc, w_erfc2, w_gauss;   // omega (and omega^2) as double-float
    int share_att;
    const float4 *boys;
    const float2 *boys_e;
    ConstsMix km;
};

struct ArgsGradMix {
    Args2c g;
    ArgsMix m;
};

// Arguments of the three-index kernels (by value).
struct Args3c {
    const ShellRec *orb_shells, *aux_shells;
    const PrimRec *orb_prims, *aux_prims;
    const Vec4 *orb_centers, *aux_centers;
    const int32_t *t_a, *t_t, *t_b;
    const int32_t *perm;
    const Tile *tiles;
    int tile_begin, tile_end;
    int *counter;
    const long long *out_off;
    double *out;
    const int *gaunt_base, *gaunt_row;
    const GauntEnt *gaunt;
    // gradient kernels only (grad_a != null selects the VJP kernel)
    const long long *w_off;
    const double *w;
    double *grad_a, *grad_b;
    // screening: > 0 writes zeros for a triple whose bound on every element is below it
    double screen_thresh;
    const ScreenRec *orb_screen, *aux_screen;
    Consts k;
    Consts3 k3;
    ConstsMix km;                 // mixed-precision angular part
};

// Kernel launchers (shg_kernels.cu, shg_3c.cu).
// Planning workspace (ints): err, ticket, 2 spare, hist, bin_start, cursor
// (n_bins each), tile_start (n_bins + 1), summary (n_chunks + 2), key (n).
// After the build, summary[c] is the first tile of class chunk c
// (c = 0..n_chunks-1), summary[n_chunks] the number of tiles and
// summary[n_chunks + 1] the error flag of the classification.
constexpr size_t plan_ws_ints(int64_t n, int n_bins, int n_chunks)
{
    return 4 + 4 * (size_t)n_bins + 1 + (size_t)n_chunks + 2 + (size_t)n;
}
inline int *plan_summary(int *ws, int n_bins) { return ws + 4 + 4 * (size_t)n_bins + 1; }
cudaError_t launch_plan_build(PlanDev &plan, int *d_ws, int n_bins, const int *d_bin_rank, cudaStream_t s);
cudaError_t launch_3c(const Args3c &args, int precision, int grid, cudaStream_t s);
// grid is ignored when args.counter is null (static launch, one warp per tile)
cudaError_t launch_2c_grad(const Args2c &args, int op, int precision, int grid, cudaStream_t s, int threads = 128);
cudaError_t launch_2c_grad_mixed(const ArgsGradMix &args, int op, cudaStream_t s);
cudaError_t launch_2c_mixed(const ArgsMix &args, int op, int grid, bool persistent, cudaStream_t s,
                            int threads = 128);
int persistent_grid_2c_mixed(int op, int threads = 128, int ctas_per_sm = 0);
cudaError_t launch_2c_mixed_fused(const ArgsMixFused &args, int grid, bool persistent, cudaStream_t s,
                                  int threads, int variant = 0);
int persistent_grid_2c_mixed_fused(int threads = 128, int ctas_per_sm = 0, int variant = 0);
int persistent_grid_2c_grad(int op, int precision);
int persistent_grid_3c(int precision);
cudaError_t launch_2c(const Args2c &args, int op, int precision, int n_tiles_or_grid, bool persistent,
                      cudaStream_t s, int threads = 128);
int persistent_grid_2c(int op, int precision, int threads = 128, int ctas_per_sm = 0);
// variant (persistent launches): 0 = the compiler's register allocation, 1 = at
// most 170 registers (three 128-thread CTAs per SM), 2 = at most 128 (four)
cudaError_t launch_2c_fused(const ArgsFused &args, int n_tiles_or_grid, bool persistent, cudaStream_t s,
                            int threads, int variant = 0);
int persistent_grid_2c_fused(int threads = 128, int ctas_per_sm = 0, int variant = 0);
cudaError_t launch_pack_centers(const double *raw, int n, Vec4 *ctr, MixCenter *mctr, int *bad, cudaStream_t s);
cudaError_t launch_family_radial(const ArgsFam &a, int op, cudaStream_t s);
cudaError_t launch_gather_i64(const int64_t *src, const int32_t *idx, int64_t n, int64_t *dst, cudaStream_t s);
cudaError_t launch_scatter_2c(const ShellRec *shells, int64_t n, const int32_t *pa, const int32_t *pb,
                              const int64_t *boff, const double *blocks, const int64_t *ao, int64_t ld, int sym,
                              double *M, cudaStream_t s);
cudaError_t launch_gather_2c(const ShellRec *shells, int64_t n, const int32_t *pa, const int32_t *pb,
                             const int64_t *boff, const double *M, const int64_t *ao, int64_t ld, int sym,
                             double *blocks, cudaStream_t s);
cudaError_t launch_reduce_centers(const ShellRec *shells, int64_t n, const int32_t *pa, const int32_t *pb,
                                  const double *ga, const double *gb, double *out, cudaStream_t s);
cudaError_t launch_debug_boys(int64_t n, const double *T, int nmax, double *F, const DeviceTables &t,
                              cudaStream_t s);
cudaError_t launch_alu_probe(int kind, int iters, int blocks, int threads, double *sink, cudaStream_t s);

}  // namespace shg

// Opaque handles of the C ABI.
struct shg_basis {
    shg::BasisDev d;
};

struct shg_plan {
    shg::PlanDev d;
    int launches = 0;
};

// Family plan: the pairs whose shells both belong to families with
// K_a * K_b <= kFamPP, grouped by family pair, plus the rest (regular path).
struct shg_family_plan {
    const shg::BasisDev *basis = nullptr;
    int64_t n = 0, n_fam = 0, n_rest = 0;
    int n_groups = 0;
    int32_t *d_idx_fam = nullptr, *d_idx_rest = nullptr;   // original pair indices
    int32_t *d_pa_fam = nullptr, *d_pb_fam = nullptr, *d_pa_rest = nullptr, *d_pb_rest = nullptr;
    shg::FamGroup *d_groups = nullptr;
    int *d_counter = nullptr;
    double *d_o = nullptr;                                  // [n_fam][kJmax]
    int64_t *d_off_fam = nullptr, *d_off_rest = nullptr;    // offsets gathered at execution
    shg_plan *plan_fam = nullptr, *plan_rest = nullptr;
    void *block = nullptr;
};

