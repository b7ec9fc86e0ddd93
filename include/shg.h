/*
 * shg.h - C ABI of the GB300 (sm_103a) solid-harmonic Gaussian integral library.
 *
 * The library evaluates, on the GPU, batched integrals over contracted real
 * solid-harmonic Gaussian shells by the SHG scheme of Golze, Benedikter,
 * Iannuzzi, Wilhelm and Hutter (arXiv:1701.06588):
 *   - two-center integrals (a|O|b) for O = delta (overlap), 1/r, erfc(w r)/r,
 *     erf(w r)/r, exp(-w r^2) and exp(-w r^2)/r (Sec. II B, Eq.
 *     final_r12int_ab; Table S1, whose s-type rows define all six), and
 *     (a|r_a^{2n}|b) (Sec. II C, Eq. ara2nb),
 *   - three-index overlaps (a b a~) with a and a~ on one center (Sec. II D),
 *   - gradients of both with respect to the centers (Sec. II E, Eq. dev_ab).
 *
 * Conventions (all entry points):
 *   * A shell is (l, K primitives with exponents alpha_i > 0 and contraction
 *     coefficients c_i, a center).  Its functions are
 *         phi_{l,m}(r) = N_l sum_i c_i S_{l,m}(r - R) exp(-alpha_i |r - R|^2),
 *     S_{l,m} the unit-normalised real solid harmonics (S_{1,1} = x,
 *     S_{1,-1} = y, S_{1,0} = z; S_{l,m} = A_{l,|m|} R^{c/s}_{l,|m|} of
 *     Sec. II E), m = -l..l.  N_l is the closed form of Sec. II A (unit
 *     self-overlap) when `normalize` != 0, else 1.
 *   * A two-center block is stored row-major [m_a = -la..la][m_b = -lb..lb],
 *     (2la+1)(2lb+1) doubles, at d_out + d_out_offsets[p].
 *   * A three-index block is row-major [m_a][m_a~][m_b].
 *   * Arguments named d_* are DEVICE pointers on the current CUDA device and
 *     are owned by the caller (for example PyTorch tensors).  Arguments named
 *     h_* or without prefix are host pointers, read during the call only.
 *   * `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Evaluation calls are asynchronous with respect to the host
 *     unless stated otherwise.
 *   * Every int-returning call returns SHG_OK (0) or a negative SHG_E* code;
 *     shg_last_error() then gives a message (thread-local).
 */
#ifndef SHG_H
#define SHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SHG_LMAX_2C 6      /* largest l of a shell in two-center calls            */
#define SHG_LMAX_AAB_A 10  /* largest la + la~ in (aab) calls                     */
#define SHG_KMAX 32        /* largest number of primitives of one shell           */

enum shg_status {
    SHG_OK = 0,
    SHG_EINVAL = -1,   /* invalid argument (l, K, exponent, index, operator, ...) */
    SHG_ENOMEM = -2,   /* host or device allocation failed                        */
    SHG_ECUDA = -3,    /* a CUDA runtime call failed                              */
    SHG_ETIMEOUT = -4, /* a bounded device-side wait gave up                      */
    SHG_ERANGE = -5    /* size beyond a documented maximum                        */
};

enum shg_operator {
    SHG_OP_OVERLAP = 0, /* delta(r12):       (a|b)                                */
    SHG_OP_COULOMB = 1, /* 1/r12                                                  */
    SHG_OP_ERFC = 2,    /* erfc(w r12)/r12, short range, w > 0                    */
    SHG_OP_ERF = 3,     /* erf(w r12)/r12, long range, w > 0                      */
    SHG_OP_GAUSS = 4,   /* exp(-w r12^2), w > 0                                   */
    SHG_OP_GAUSS_COULOMB = 5, /* exp(-w r12^2)/r12, Gaussian-damped Coulomb, w > 0 */
    SHG_OP_RA2N = 6     /* r_a^{2n} = |r - R_a|^{2n}: (a|r_a^{2n}|b) of Sec. II C;
                           n = 0..5 is passed in omega as an exact integer; FP64
                           only (SHG_EINVAL for SHG_PREC_MIXED)                 */
};

enum shg_precision {
    SHG_PREC_FP64 = 0,  /* every step in FP64                                     */
    SHG_PREC_MIXED = 1  /* FP32-based compensated arithmetic, FP64 where needed:
                           two-center passes evaluate the classes with both la
                           and lb >= 4 in FP64 (their sum over j of Eq.
                           final_r12int_ab cancels beyond double-float reach),
                           every other class in double-float; the FP64 far
                           field of 1/r (T >= 120) is summed on the FP64 pipe */
};

enum shg_schedule {
    SHG_SCHED_PER_CLASS = 0,  /* one launch per (la, lb) class                    */
    SHG_SCHED_PERSISTENT = 1  /* one launch, warps pull class-pure tiles          */
};

typedef struct shg_basis shg_basis_t;
typedef struct shg_plan shg_plan_t;
typedef struct shg_family_plan shg_family_plan_t;

/*
 * shg_basis_create - upload a shell set to the current device.
 * Definition: contracted shells phi_{l,m} of Sec. II A, Eq. contracted_phi,
 * with N_l of the equation after it (includes K_l = sqrt((2l+1)/4pi)).
 *   n_shells          number of shells (>= 1)
 *   l[n_shells]       angular momentum, 0 <= l <= SHG_LMAX_2C
 *   nprim[n_shells]   primitives per shell, 1 <= K <= SHG_KMAX
 *   exps, coefs       sum(nprim) values each, concatenated shell by shell
 *   n_centers         number of centers
 *   centers           n_centers x 3 doubles (bohr)
 *   center_of_shell   center index of each shell, 0 <= c < n_centers
 *   normalize         non-zero: multiply coefficients by N_l
 * All input pointers are host pointers, copied; the caller keeps them.
 * Returns SHG_EINVAL for l or K out of range, a non-positive or non-finite
 * exponent, a non-finite coefficient or center, or a bad center index;
 * SHG_ENOMEM / SHG_ECUDA on allocation or copy failure.  On success *out
 * owns device memory until shg_basis_destroy.  Synchronous.
 */
int shg_basis_create(int n_shells, const int32_t *l, const int32_t *nprim, const double *exps,
                     const double *coefs, int n_centers, const double *centers,
                     const int32_t *center_of_shell, int normalize, shg_basis_t **out);

/*
 * shg_basis_set_centers - replace all center coordinates (host array of
 * n_centers x 3 doubles, same count as at creation; pinned memory is copied
 * by DMA, pageable memory through the driver's staging).  The coordinates are
 * packed and checked on the device, in buffers of ~88 B per center that the
 * first call allocates and the basis keeps.  Returns SHG_EINVAL, naming the
 * first center with a non-finite coordinate, and then keeps the previous
 * centers.  Plans made on the basis stay valid: they depend only on l and K.
 * Runs on the legacy default stream and returns when the new centers are in
 * place (synchronous).
 */
int shg_basis_set_centers(shg_basis_t *basis, const double *centers);

/* shg_basis_destroy - free the device copy.  NULL is ignored. */
void shg_basis_destroy(shg_basis_t *basis);

/* Number of shells and primitives of a basis (0 for NULL). */
int64_t shg_basis_nshells(const shg_basis_t *basis);
int64_t shg_basis_nprims(const shg_basis_t *basis);

/*
 * shg_pair_offsets - host helper: offsets[p] = sum_{q<p} (2la_q+1)(2lb_q+1)
 * for host pair lists; returns the total number of doubles, or a negative
 * SHG_E* code for an out-of-range shell index.
 */
int64_t shg_pair_offsets(const shg_basis_t *basis, int64_t n_pairs, const int32_t *pair_a,
                         const int32_t *pair_b, int64_t *offsets);

/* As shg_pair_offsets for (aab) triples: blocks (2la+1)(2la~+1)(2lb+1). */
int64_t shg_triple_offsets(const shg_basis_t *orb, const shg_basis_t *aux, int64_t n_triples,
                           const int32_t *t_a, const int32_t *t_atilde, const int32_t *t_b, int64_t *offsets);

/*
 * shg_eval_2c - two-center integrals (a|O|b) of Sec. II B:
 *   (a|O|b) = (-1)^lb A_{la,ma} A_{lb,mb} sum_j 2^{la+lb-j} O^{(la+lb-j)}(R^2)
 *             (2j-1)!! sum_kappa B_{j,kappa} Q_{la,|ma|,lb,|mb|,j,kappa}
 * with O^{(k)} the contracted R_ab^2-derivatives of Eq. O_rab2_deriv and the
 * s-type integrals of Table S1.
 *   basis          shells for both sides
 *   n_pairs        number of pairs (0 is allowed and does nothing)
 *   d_pair_a/b     device int32[n_pairs] shell indices
 *   op, omega      operator (enum shg_operator); omega > 0 for ERF, ERFC, GAUSS,
 *                  GAUSS_COULOMB; omega = n (0..5) for RA2N, whose radial
 *                  term is T^{(k)} of Eq. T_rab2_deriv in place of O^{(k)}
 *   screen_thresh  0 disables screening; > 0: a pair whose bound on every
 *                  element magnitude is below it writes zeros (overlap and
 *                  Gaussian operator only; Coulomb-type pairs are never
 *                  screened).  The bound uses |S_{l,m}(r)| <= sqrt(2) r^l,
 *                  r^l exp(-a r^2) <= (l/(a e))^{l/2} exp(-a r^2/2), the
 *                  s-type integral at half the smallest exponents of each
 *                  shell and sum |N c|; so every element of a screened
 *                  block is below the threshold in magnitude.
 *   precision      enum shg_precision
 *   d_out_offsets  device int64[n_pairs] start of each block in d_out
 *   d_out          device doubles, large enough for every block
 * One-shot convenience: builds a plan (device memory, one host sync to read
 * class counts), executes it on `stream` and frees it.  Returns SHG_EINVAL
 * for a bad operator, omega, precision or shell index.
 */
int shg_eval_2c(const shg_basis_t *basis, int64_t n_pairs, const int32_t *d_pair_a, const int32_t *d_pair_b,
                int op, double omega, double screen_thresh, int precision, const int64_t *d_out_offsets,
                double *d_out, void *stream);

/*
 * shg_plan_2c_create - bucket a pair list by (la, lb, Ka*Kb) class on the
 * device and build the tile list of a schedule (enum shg_schedule).  The plan
 * owns device memory (about 12 bytes per pair) and depends only on the pair
 * list and the l and K of the shells, not on centers, exponents or operator.
 * Validates the shell indices on the device and synchronises `stream` once.
 * d_pair_a/b must stay valid and unchanged for the plan's lifetime.
 */
int shg_plan_2c_create(const shg_basis_t *basis, int64_t n_pairs, const int32_t *d_pair_a,
                       const int32_t *d_pair_b, int schedule, void *stream, shg_plan_t **out);

/*
 * shg_plan_2c_exec - evaluate the integrals of a plan (see shg_eval_2c for the
 * arguments).  Asynchronous; issues only kernel launches and a memset on
 * `stream`, so it can be captured in a CUDA graph.
 */
int shg_plan_2c_exec(shg_plan_t *plan, int op, double omega, double screen_thresh, int precision,
                     const int64_t *d_out_offsets, double *d_out, void *stream);

/*
 * shg_plan_2c_set_variant - compiled variant of the persistent fused kernel
 * used by later fused executions of the plan (an autotuner knob).
 *   FP64:  0 = registers as the compiler allocates them (253 per thread),
 *          1 = at most 170 (three 128-thread CTAs per SM), 2 = at most 128
 *          (four); the capped variants spill some values to local memory.
 *   mixed: 0 = registers as the compiler allocates them (about 124),
 *          1 = at most 96 (five 128-thread CTAs per SM), 2 = at most 85 (six).
 * A new plan uses variant 1 (the fastest of the three on GB300 for both
 * precisions on the 2M-pair workload).  The variants run the same operations
 * in the same order, so the results are bitwise equal.  SHG_EINVAL for a
 * value outside 0..2.
 */
int shg_plan_2c_set_variant(shg_plan_t *plan, int variant);

/* Number of kernel launches one FP64 shg_plan_2c_exec (or fused pass) issues
 * (for accounting). */
int shg_plan_launches(const shg_plan_t *plan);

/* Number of kernel launches one execution of the plan issues in `precision`
 * (SHG_PREC_MIXED adds the FP64 launch of the classes with both l >= 4 to a
 * persistent plan that holds any); -1 for a NULL plan or bad precision. */
int shg_plan_launches_prec(const shg_plan_t *plan, int precision);

/*
 * shg_plan_2c_set_launch - launch shape of later executions of a plan (the
 * autotuner's knobs): threads per CTA (32, 64 or 128; each warp owns one
 * tile of up to 32 pairs) and, for the persistent schedule, CTAs per SM
 * (0 = as many as occupancy allows).  Returns SHG_EINVAL for other values.
 */
int shg_plan_2c_set_launch(shg_plan_t *plan, int threads_per_cta, int ctas_per_sm);

/*
 * CUDA-graph form of a plan: shg_graph_2c_create captures shg_plan_2c_exec of
 * n_ops operators (ops[i], omegas[i], all with `precision`, block offsets
 * d_out_offsets, outputs d_outs[i]) on a private stream and instantiates the
 * graph; shg_graph_launch replays it on `stream`.  The graph keeps the
 * pointers it was captured with; geometry changes made with
 * shg_basis_set_centers are seen by later replays.  The plan must outlive
 * the graph.
 */
typedef struct shg_graph shg_graph_t;
int shg_graph_2c_create(shg_plan_t *plan, int n_ops, const int *ops, const double *omegas, int precision,
                        const int64_t *d_out_offsets, double *const *d_outs, shg_graph_t **out);
int shg_graph_launch(shg_graph_t *graph, void *stream);
void shg_graph_destroy(shg_graph_t *graph);

/*
 * shg_plan_2c_exec_fused - several operators of one plan in a single pass.  The two-center formula of Sec. II B factors as
 *   (a|O|b)[ma][mb] = (-1)^lb A_{la,ma} A_{lb,mb} sum_j 2^{la+lb-j} O^{(la+lb-j)} Q_j[ma][mb],
 * where Q_j (Eq. Q_matrix contracted with the weights (2j-1)!! B_{j,kappa} of
 * Eq. B) depends on the geometry only; the pass builds Q_j once per shell
 * pair and contracts it with the radial orders of every requested operator
 * (Table S1).  The radial sums share their primitive-pair setup, erfc(wr)/r
 * is formed as 1/r - erf(wr)/r, and erf and erfc with the same omega share
 * one attenuated sum.  Results agree with shg_plan_2c_exec of each operator
 * up to the order of the floating-point sums.  SHG_PREC_MIXED runs the same
 * scheme in double-float (each block sum of Q_j a compensated dot product);
 * its accuracy bar is that of the mixed single-operator pass.
 *   ops[n_ops], omegas[n_ops]  host arrays, 1 <= n_ops <= 5; each of
 *                  SHG_OP_OVERLAP, SHG_OP_COULOMB, SHG_OP_ERFC, SHG_OP_ERF,
 *                  SHG_OP_GAUSS at most once; omega rules of shg_eval_2c
 *   precision      SHG_PREC_FP64 or SHG_PREC_MIXED
 *   d_out_offsets  device int64[n_pairs], block offsets shared by all outputs
 *   d_outs[n_ops]  host array of device output pointers (operator i writes
 *                  d_outs[i], layout of shg_eval_2c); owned by the caller
 * No screening threshold (every block is evaluated).  Asynchronous on
 * `stream`; issues a memset and kernel launches only (graph-capturable).
 * SHG_EINVAL for other operators, a repeated operator, n_ops outside 1..5,
 * a bad omega or precision, or a NULL array or output.
 * shg_graph_2c_create_fused - the CUDA-graph form of one fused pass (same
 * arguments; see shg_graph_2c_create for the graph's lifetime rules).
 */
int shg_plan_2c_exec_fused(shg_plan_t *plan, int n_ops, const int *ops, const double *omegas, int precision,
                           const int64_t *d_out_offsets, double *const *d_outs, void *stream);
int shg_graph_2c_create_fused(shg_plan_t *plan, int n_ops, const int *ops, const double *omegas, int precision,
                              const int64_t *d_out_offsets, double *const *d_outs, shg_graph_t **out);

/*
 * shg_plan_destroy - free a plan.  NULL ok.  The plan's device memory is
 * released in the order of the stream the plan was created on
 * (cudaFreeAsync), without a host synchronisation: executions queued on that
 * stream finish first, and executions on another stream must be ordered
 * before it by the caller (an event that stream waits for).  The side streams
 * and events of mixed-precision executions are destroyed with the plan; the
 * executions have already joined them into the caller's stream.
 */
void shg_plan_destroy(shg_plan_t *plan);

/*
 * shg_eval_3c_aab - three-index overlaps (a b a~) = int phi_a phi_a~ phi_b of
 * Sec. II D: the product phi_a phi_a~ is expanded with real Gaunt
 * coefficients into shells L_a = |la-la~|..la+la~ (step 2) with exponent
 * alpha + alpha~ (Eq. product_SHG_STGO), the radial part is P^{(k)} of
 * Eq. Pa_aba built from (0_a'|r_a^{2m}|0_b)^{(k)} (Eqs. sra2ms, devsra2ms),
 * and the angular part reuses Q of Sec. II E.
 *   orb            basis of a and a~ (both on one center, checked)
 *   aux            basis of b (may be the same handle as orb)
 *   d_a, d_atilde  device int32[n_triples] indices into orb
 *   d_b            device int32[n_triples] indices into aux
 *   precision      enum shg_precision (FP64, or MIXED: radial sums FP64,
 *                  angular part and Gaunt sum double-float)
 *   screen_thresh  0 disables screening; > 0: a triple whose bound on every
 *                  element magnitude is below it writes zeros.  The bound
 *                  multiplies the single-shell bounds of a and a~ used by
 *                  shg_eval_2c (one Gaussian of exponent (amin_a+amin_a~)/2
 *                  on A) and takes the two-center overlap bound with b
 *   d_out_offsets  device int64[n_triples]; d_out device doubles
 * Limits: la + la~ <= SHG_LMAX_AAB_A, lb <= SHG_LMAX_2C.  Returns SHG_EINVAL
 * when a and a~ of a triple are not on the same center.
 */
int shg_eval_3c_aab(const shg_basis_t *orb, const shg_basis_t *aux, int64_t n_triples, const int32_t *d_a,
                    const int32_t *d_atilde, const int32_t *d_b, int precision, double screen_thresh,
                    const int64_t *d_out_offsets, double *d_out, void *stream);

/*
 * shg_eval_2c_grad - vector-Jacobian product of the two-center integrals with
 * respect to the centers (Sec. II E, Eq. dev_ab):
 *   d_grad_a[p][i] = sum_{ma,mb} W_p[ma][mb] d(a|O|b)[ma][mb] / dR_{a,i}
 *   d_grad_b[p][i] = -d_grad_a[p][i]   (translation invariance)
 * using O^{(k+1)} with Q~ and O^{(k)} with dQ~/dR_a (Eqs. cartesian_dev_x/y/z);
 * radial terms are recomputed, nothing is stored from a forward call.
 *   d_w_offsets, d_upstream_w   device int64[n_pairs] / doubles: W_p blocks,
 *                               same layout as shg_eval_2c output
 *   d_grad_a, d_grad_b          device double[n_pairs][3]; d_grad_b may be NULL
 *   precision                   SHG_PREC_FP64, or SHG_PREC_MIXED: radial orders
 *                               in double-float on the FP32 pipes, the angular
 *                               part (harmonics, their gradients, W and the
 *                               contractions with W_p) in FP64; the classes with
 *                               both la and lb >= 4 wholly in FP64.  Not for
 *                               SHG_OP_RA2N (SHG_EINVAL)
 * No atomics: per-atom sums are left to the caller.
 */
int shg_eval_2c_grad(const shg_basis_t *basis, int64_t n_pairs, const int32_t *d_pair_a, const int32_t *d_pair_b,
                     int op, double omega, int precision, const int64_t *d_w_offsets, const double *d_upstream_w,
                     double *d_grad_a, double *d_grad_b, void *stream);

/*
 * shg_eval_3c_aab_grad - as shg_eval_2c_grad for (a b a~):
 *   d_grad_a[t][i] = sum W_t[ma][ma~][mb] d(a b a~)/dR_{a,i}, with R_a the
 *   common center of a and a~; d_grad_b = -d_grad_a.
 */
int shg_eval_3c_aab_grad(const shg_basis_t *orb, const shg_basis_t *aux, int64_t n_triples, const int32_t *d_a,
                         const int32_t *d_atilde, const int32_t *d_b, int precision, const int64_t *d_w_offsets,
                         const double *d_upstream_w, double *d_grad_a, double *d_grad_b, void *stream);

/*
 * shg_eval_2c_noalloc - shg_eval_2c for callers that cannot allocate device
 * memory during the call.  The paper has no counterpart: this is a property
 * of the library, not of the integral scheme.
 *
 * shg_eval_2c allocates its plan (the bucketed pair list and tile list) with
 * cudaMallocAsync.  Some callers cannot allow that at call time: a framework
 * that hands out device memory only from its own pool, a real-time loop that
 * must not pay allocation latency or its implicit synchronisation, a process
 * that has reserved all device memory up front.  This entry point builds the
 * same plan in a fixed array inside the library (a file-scope __device__
 * array of about 10.5 MB that every GPU loading the library keeps until the
 * process exits) and calls no cudaMalloc, cudaFree or other allocating
 * routine.  Results equal those of shg_eval_2c with the persistent schedule.
 *   arguments      as shg_eval_2c (no screening threshold); FP64 and the
 *                  basis must have been created on the current device, which
 *                  also set up the library's tables there
 *   limit          n_pairs <= 1,048,576; larger lists return SHG_ERANGE
 *                  with a message, before any device work
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call outside stream capture;
 * the address is kept for the life of the process, so do not use this entry
 * point across a cudaDeviceReset.  Any precision other than SHG_PREC_FP64
 * returns SHG_EINVAL.
 * The call synchronises `stream` once, after planning, to read the pair-index
 * check and the tile count.  All calls share the one array and each clears
 * what must start at zero; calls whose GPU work overlaps (other streams or
 * unordered host threads) race on it, so order them on one stream.
 */
int shg_eval_2c_noalloc(const shg_basis_t *basis, int64_t n_pairs, const int32_t *d_pair_a,
                        const int32_t *d_pair_b, int op, double omega, int precision,
                        const int64_t *d_out_offsets, double *d_out, void *stream);

/*
 * Family path (the structure of the bases the paper measures, Sec. III):
 * when the shells of an element share one exponent set, the radial terms
 * (0_a|O|0_b)^{(k)} of Table S1 depend only on the primitive pair and R_ab,
 * so for all shell pairs of one pair of families they are computed once per
 * primitive pair and contracted per shell pair with its weights
 * N c (2 alpha)^{-l} (Eq. O_rab2_deriv); the angular part is the same
 * class-tiled kernel as shg_eval_2c.  Families are found at
 * shg_basis_create: shells on one center whose exponent lists are bitwise
 * identical.
 *
 * shg_family_plan_create - group a device pair list (as shg_plan_2c_create;
 *   copied to the host once, synchronously) by family pair.  Pairs whose two
 *   families have K_a * K_b > 100 go to the regular path inside the plan.
 * shg_family_plan_exec - blocks of every pair at d_out + d_out_offsets[p],
 *   FP64, for op = OVERLAP, COULOMB, ERFC, ERF, GAUSS, GAUSS_COULOMB (not
 *   RA2N: its radial term depends on la); equal to shg_eval_2c up to the
 *   order of the contraction sums.  Asynchronous on `stream`.
 * shg_family_plan_counts - total pairs (return value), pairs on the family
 *   path and number of family-pair groups.
 * Errors as shg_plan_2c_create / shg_plan_2c_exec.
 */
int shg_family_plan_create(const shg_basis_t *basis, int64_t n_pairs, const int32_t *d_pair_a,
                           const int32_t *d_pair_b, void *stream, shg_family_plan_t **out);
int shg_family_plan_exec(shg_family_plan_t *plan, int op, double omega, const int64_t *d_out_offsets,
                         double *d_out, void *stream);
int64_t shg_family_plan_counts(const shg_family_plan_t *plan, int64_t *n_family_pairs, int64_t *n_groups);
void shg_family_plan_destroy(shg_family_plan_t *plan);

/*
 * Molecular assembly (the caller-side use of the blocks; no paper formula).
 * A basis whose shells carry AO offsets ao_off[s] (device int64[n_shells],
 * the first row/column of shell s in an n_ao x n_ao matrix, functions of a
 * shell consecutive in m = -l..l) maps a pair list onto a dense matrix.
 *
 * shg_scatter_2c - write every block (layout of shg_eval_2c) into the dense
 *   row-major matrix d_matrix (leading dimension ld >= n_ao): rows
 *   ao_off[a].., columns ao_off[b]..; with symmetric != 0 and a != b also
 *   the transposed block at rows ao_off[b].., columns ao_off[a]...  Entries
 *   no pair touches are left unchanged; the caller lists each unordered pair
 *   once (pairs that write the same entries race).  HBM-bound.
 * shg_gather_2c - the adjoint: d_blocks[p] = M[a rows, b columns], plus the
 *   transpose of M[b rows, a columns] when symmetric != 0 and a != b.  With a
 *   symmetric weight matrix W this gives the upstream weights of the
 *   gradient call for sum_{mu,nu} W_{mu nu} M_{mu nu}.
 * shg_reduce_centers - d_center_grad[c][i] += sum of d_grad_a[p][i] over the
 *   pairs whose shell a sits on center c, and the same for d_grad_b with the
 *   center of b (FP64 atomics: the order of the additions, hence the last
 *   bits, may differ between runs).
 * All pointers are device pointers owned by the caller; asynchronous on
 * `stream`.  SHG_EINVAL for NULL pointers, n_pairs < 0 or ld < 1.  Shell
 * indices are not checked (they come from a pair list already checked by the
 * evaluation call).
 */
int shg_scatter_2c(const shg_basis_t *basis, int64_t n_pairs, const int32_t *d_pair_a, const int32_t *d_pair_b,
                   const int64_t *d_block_off, const double *d_blocks, const int64_t *d_ao_off, int64_t ld,
                   int symmetric, double *d_matrix, void *stream);
int shg_gather_2c(const shg_basis_t *basis, int64_t n_pairs, const int32_t *d_pair_a, const int32_t *d_pair_b,
                  const int64_t *d_block_off, const double *d_matrix, const int64_t *d_ao_off, int64_t ld,
                  int symmetric, double *d_blocks, void *stream);
int shg_reduce_centers(const shg_basis_t *basis, int64_t n_pairs, const int32_t *d_pair_a, const int32_t *d_pair_b,
                       const double *d_grad_a, const double *d_grad_b, double *d_center_grad, void *stream);

/*
 * shg_debug_boys - device Boys function F_n(T) = int_0^1 exp(-T t^2) t^{2n} dt
 * (SI Eq. 3) as used by the Coulomb-type radial terms: for every T in
 * d_T[n_T] writes F_n for n = 0..nmax (nmax <= 24) to d_F[i*(nmax+1) + n].
 */
int shg_debug_boys(int64_t n_T, const double *d_T, int nmax, double *d_F, void *stream);

/*
 * shg_measure_alu_peak - ALU throughput probe: a grid of independent FMA
 * chains in FP64 (kind 0) or FP32 (kind 1), `iters` FMAs per thread per
 * chain, or of FP64 tensor-core MMA chains (kind 2: mma.sync m8n8k4 with FP64
 * operands and accumulator, 512 flops per warp instruction), timed with CUDA
 * events on `stream`.  Writes FLOP/s (2 per FMA) to *flops.  Synchronous.
 */
int shg_measure_alu_peak(int kind, int iters, double *flops, void *stream);

/* Message describing the last failure on this host thread ("" if none). */
const char *shg_last_error(void);

/* Library version string. */
const char *shg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SHG_H */
