/*
 * discloop.h -- C ABI of the GB300 (sm_103a) disconnected-quark-loop library.
 *
 * The calls follow the paper's statement of the workflow (Alexandrou et al.,
 * "Evaluation of disconnected quark loops for hadron structure using GPUs",
 * App. A "Interfaces and workflow"): load a gauge field, set kappa and a*mu,
 * generate Z4 noise, invert the even-odd preconditioned twisted-mass operator,
 * contract the solutions into local and one-derivative loops per time slice and
 * momentum, and combine low- and high-precision solves with the Truncated
 * Solver Method.
 *
 * Conventions shared by every call
 *   - Lattice dims[4] = {X, Y, Z, T}; every extent even, X*Y*Z*T/2 < 2^31.
 *   - Site order lex = x + X*(y + Y*(z + Z*t)); parity (x+y+z+t)&1, even = 0.
 *   - Gauge field: complex128 [T][Z][Y][X][mu][3][3], mu = 0:x 1:y 2:z 3:t,
 *     U_mu(x) row-major.  The time-boundary factor is applied by the kernels.
 *   - "Natural" spinor fields: complex [n][T][Z][Y][X][4][3] (spin-major,
 *     colour-minor), complex128 (DL_C128) or complex64 (DL_C64), in DEVICE
 *     memory unless a call says otherwise.
 *   - Chiral Euclidean gammas: gamma_k = [[0,-i s_k],[i s_k,0]] (k = x,y,z),
 *     gamma_t = [[0,1],[1,0]], gamma_5 = diag(1,1,-1,-1).  Gamma_b for
 *     b = 0..15 is g_x^b0 g_y^b1 g_z^b2 g_t^b3.
 *   - Operator (kappa normalisation, App. A Eq. A.1):
 *       M_f psi = (1 + 2 i kappa amu f gamma_5) psi
 *                 - kappa sum_mu [(1-gamma_mu) U_mu(x) psi(x+mu) + (1+gamma_mu) U_mu(x-mu)^+ psi(x-mu)]
 *     f = +1 (u) or -1 (d).  Physical units: M_phys = M / (2 kappa).
 *   - All device work is ordered on the context's stream; the stream passed
 *     to dl_create (or the legacy default stream if NULL) waits for it before
 *     a call returns.  Calls on one context are not thread-safe.
 *   - Negative status = error (message in dl_last_error); positive status =
 *     a non-fatal outcome (outputs and stats are filled).  No exceptions cross
 *     this boundary.
 *   - Ownership: the caller owns every pointer it passes; the context owns the
 *     gauge field copies and all workspaces and frees them in dl_destroy.
 */
#ifndef DISCLOOP_H
#define DISCLOOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dl_ctx dl_ctx;
typedef struct dl_nn dl_nn;   /* learned preconditioner (see the section at the end) */

typedef enum {
  DL_OK = 0,
  DL_ERR_ARG = -1,    /* invalid argument (sizes, enum values, NULL) */
  DL_ERR_CUDA = -2,   /* a CUDA call failed; the message names it */
  DL_ERR_OOM = -3,    /* device allocation failed */
  DL_ERR_STATE = -4,  /* call out of order (e.g. no gauge field loaded) */
  DL_ERR_IO = -5,     /* a file could not be read or written, or failed its checks */
  DL_NOT_CONVERGED = 1, /* a solve reached max_iter; last iterate returned */
  DL_BREAKDOWN = 3      /* a CG scalar became zero, negative or non-finite */
} dl_status;

/* Storage precision.  DL_F16 is the 16-bit format: signed 16-bit fixed point
 * with one float scale per site and right-hand side (value = q * scale / 32767,
 * scale = the site's largest |re|,|im|), i.e. the paper's "half" precision
 * (App. A, Table A.1); arithmetic on it is FP32. */
typedef enum { DL_F64 = 0, DL_F32 = 1, DL_F16 = 2, DL_F64_IEEE = 5 } dl_prec;
/* DL_F64 runs as double-float arithmetic (two floats per value, ~48 significant bits,
 * relative rounding ~1e-14) because GB300 executes IEEE binary64 at a small fraction of
 * its FP32 rate; DL_F64_IEEE requests IEEE binary64 kernels (dl_apply, dl_solve), e.g. for
 * a plain FP64 baseline. */
typedef enum { DL_C128 = 0, DL_C64 = 1 } dl_dtype;              /* natural field element type */

/* Operators applied by dl_apply (natural full-lattice fields in and out). */
typedef enum {
  DL_OP_M = 0,       /* out = M_f in                                       (Eq. A.1) */
  DL_OP_MDAG = 1,    /* out = M_f^dagger in                                          */
  DL_OP_HOP = 2,     /* out = D in (hopping sum, no kappa)                           */
  DL_OP_MHAT = 3,    /* out_e = Mhat in_e, out_o = 0                        (Eq. A.2) */
  DL_OP_MHAT_DAG = 4,/* out_e = Mhat^dagger in_e                                     */
  DL_OP_PREP = 5,    /* out_e = in_e + kappa D_eo R_oo^-1 in_o (bhat of Eq. A.2)     */
  DL_OP_RECON = 6,   /* out = in_e + R_oo^-1 (aux_o + kappa D_oe in_e)      (Eq. A.4) */
  DL_OP_BH = 7       /* out = B H in, B = R_f^-1, H = -kappa D              (Eq. HPE) */
} dl_op;

/* Loop estimators (Sec. 2.3, 2.5). Output = factor * sum xi^dagger_a phi_b. */
typedef enum {
  DL_EST_STANDARD = 0, /* (eta, s)                 factor 1       -> Tr[M_u^-1 X]            (Eq. loopSt)  */
  DL_EST_ONE_END = 1,  /* (g5 s, s)                factor -4i k amu -> Tr[(M_u^-1 - M_d^-1) X] (Eq. loopVv)  */
  DL_EST_GEN = 2,      /* (g5 s, g5 (eta - 2i k amu g5 s)) factor 2 -> Tr[(M_u^-1 + M_d^-1) X] (Eq. loopStD) */
  DL_EST_HPE = 3       /* (eta, (BH)^4 s)          factor 1       -> Tr[X (BH)^4 M_u^-1]     (Eq. loopHPE1) */
} dl_estimator;

#define DL_MAX_RHS 32   /* right-hand sides per block */

/* ---- context ------------------------------------------------------------ */

/* Create a context for one lattice on CUDA device `device`.  `cuda_stream`
 * (a cudaStream_t, may be NULL) is the caller's stream that every call orders
 * itself after and before returning.  Allocates nothing large. */
dl_status dl_create(dl_ctx** ctx, const int dims[4], int device, void* cuda_stream);
void dl_destroy(dl_ctx* ctx);
const char* dl_last_error(const dl_ctx* ctx);
dl_status dl_set_stream(dl_ctx* ctx, void* cuda_stream);

/* Load the gauge field (App. A, "Twisted mass fermion operator": links stored
 * with 18, 12 or 8 reals; the 16-bit copy uses int16 fixed point).  `links` is complex128 [T][Z][Y][X][4][3][3] in host
 * memory (links_on_device = 0) or device memory (1).  t_boundary = -1
 * (antiperiodic in time, the default reading) or +1.  recon_f32 in {18,12,8}
 * and recon_f16 in {12,8} choose the compressed copies the FP32 and FP16
 * operators read; the FP64 operator always reads all 18 reals.  The links must
 * be SU(3) for recon 12/8. */
dl_status dl_load_gauge(dl_ctx* ctx, const double* links, int links_on_device,
                        double t_boundary, int recon_f32, int recon_f16);

/* Set kappa and the twisted mass a*mu (App. A Eq. A.1). */
dl_status dl_set_params(dl_ctx* ctx, double kappa, double amu);

/* ---- noise (Sec. 2.1, Eqs. eq1/eq2) ------------------------------------- */

/* Z2 x iZ2 noise (entries (+-1 +- i)/sqrt(2)), or {1,i,-1,-i} if quadrant != 0,
 * for noise indices first_index .. first_index+n-1, written as a natural field
 * `out` of type dtype.  Entry (r, lex, spin a, colour c) is bits 0 and 1 of
 * splitmix64(seed, (r*V + lex)*12 + 3a + c), splitmix64 as published by Steele,
 * Lea & Flood (2014): state = seed + (counter+1)*0x9E3779B97F4A7C15. */
dl_status dl_noise_z4(dl_ctx* ctx, uint64_t seed, uint64_t first_index, int n,
                      void* out, int dtype, int quadrant);
/* Time-diluted noise (Sec. 2.3, time dilution and coherent sources): the fields
 * of dl_noise_z4 with every time slice t != t0 (mod dt) set to zero, so that a
 * source fills the slices t0, t0 + dt, ... only (dt = T: one slice; smaller dt:
 * coherent sources on several slices dt apart).  The dt sources t0 = 0 .. dt-1
 * of one noise index sum to its dl_noise_z4 field.  Solving for such a source
 * and contracting it with dl_contract (DL_EST_STANDARD, or DL_EST_HPE plus
 * dl_hpe_exact times X*Y*Z at zero momentum on each kept slice) gives loops that
 * vanish off the kept slices.  Needs 1 <= dt <= T and 0 <= t0 < dt. */
dl_status dl_noise_z4_tdil(dl_ctx* ctx, uint64_t seed, uint64_t first_index, int n,
                           void* out, int dtype, int quadrant, int t0, int dt);

/* ---- operators (App. A) -------------------------------------------------- */

/* Apply `op` (dl_op) with flavour f (+1/-1) in storage precision `prec` to n
 * natural fields `in` (and `aux` for DL_OP_RECON; else NULL), writing `out`.
 * in/aux/out are device pointers of type dtype; out must not alias in. */
dl_status dl_apply(dl_ctx* ctx, int op, int prec, int flavour, int n,
                   const void* in, const void* aux, void* out, int dtype);

/* ---- solver (Sec. 2.2) ---------------------------------------------------- */

typedef struct {
  double tol;       /* stop when |r| / |Mhat^dag bhat| < tol, r the CG residual (Sec. 2.2) */
  int max_iter;     /* per right-hand side */
  int prec_hi;      /* DL_F64 or DL_F32: solution accumulator, reliable-update residual */
  int prec_lo;      /* DL_F64, DL_F32 or DL_F16: Krylov vectors and operator in the loop */
  double delta;     /* reliable update when |r| < delta * max|r| since the last one; 0 = never */
  int flavour;      /* +1 (u) or -1 (d) */
  int chunk;        /* iterations per CUDA-graph launch between host checks (>= 1) */
} dl_solve_params;

typedef struct {
  int iters[DL_MAX_RHS];          /* CG iterations per right-hand side */
  double resid[DL_MAX_RHS];       /* final |r|/|Mhat^dag bhat| from the recomputed residual */
  double true_resid[DL_MAX_RHS];  /* |b - M psi| / |b| on the full lattice, in FP64 */
  int reliable_updates;           /* total over right-hand sides */
  int max_iters;
  double seconds;
} dl_solve_stats;

/* Solve M_f psi = b for n <= DL_MAX_RHS natural fields b (src) into sol, by CG
 * on the normal equations of the even-odd system (App. A Eq. A.2) with
 * per-right-hand-side convergence masks, then Eq. A.4 for the odd sites.
 * stats may be NULL.  Returns DL_NOT_CONVERGED if any column hit max_iter. */
dl_status dl_solve(dl_ctx* ctx, const void* src, void* sol, int n, int dtype,
                   const dl_solve_params* params, dl_solve_stats* stats);

/* ---- contractions (App. A, "Contraction kernels") ------------------------- */

/* Number of momenta n with |n|^2 <= p2max, and (if list != NULL) the list as
 * int[3*count] (nx, ny, nz), ordered nz, ny, nx outer to inner, ascending. */
dl_status dl_momenta(int p2max, int* count, int* list);

/* Loops of estimator `est` for n pairs (eta[i], sol[i]) (natural fields of
 * type dtype, device), with momenta |n|^2 <= p2max and phases exp(-i p.x).
 * out (device, complex128) is [n][T][Np][nd][4][4], nd = 1 (local) or 5 with
 * with_deriv (local, then the symmetric covariant derivative in x, y, z, t):
 *   out[..][a][b] = factor * sum_x exp(-i p.x) xi^dagger_a(x) phi_b(x)
 * so that the loop of insertion X is sum_ab X_ab out[..][a][b] (colour traced).
 * accumulate != 0 adds into out instead of overwriting it. */
dl_status dl_contract(dl_ctx* ctx, int est, const void* eta, const void* sol, int n,
                      int dtype, int with_deriv, int p2max, double* out, int accumulate);

/* dl_contract for time-diluted sources (Sec. 2.3, dl_noise_z4_tdil): the local loops
 * (no derivative) on the time slices t = t0 (mod dt) only, 1 <= dt <= T, 0 <= t0 < dt.
 * out has dl_contract's layout [n][T][Np][1][4][4]; the other slices are written as zero
 * (or left unchanged with accumulate), where a source that vanishes off its slices has
 * loops that vanish too.  The contraction work is proportional to the slices kept.
 * Needs X <= 256. */
dl_status dl_contract_slices(dl_ctx* ctx, int est, const void* eta, const void* sol, int n,
                             int dtype, int p2max, int t0, int dt, double* out, int accumulate);

/* Exact part of the hopping-parameter expansion for local insertions (Eq. HPE:
 * orders 0 and 2; orders 1 and 3 vanish on the diagonal): the per-site 4x4
 * matrix C_ab (colour traced) with Tr_x[X (B - BHB + (BH)^2 B - (BH)^3 B)] =
 * sum_ab X_ab C_ab, written to out16 (host, complex128 [4][4]).  The second order
 * is the gauge-independent sum over back-and-forth hops, exact when every extent
 * is at least 4; DL_ERR_ARG otherwise (on an extent of 2, two forward hops also
 * return to the site).  dl_tsm_run with hpe = 1 has the same requirement. */
dl_status dl_hpe_exact(dl_ctx* ctx, int flavour, double* out16);

/* ---- truncated solver method (Sec. 2.2, Eq. estiTSM) --------------------- */

typedef struct {
  int n_hp, n_lp;        /* HP-LP pairs and fresh LP solves */
  double tol_hp, tol_lp; /* CG residual bounds */
  int prec_hp_lo;        /* Krylov storage of HP solves (FP64 accumulation, reliable updates) */
  int prec_lp_lo;        /* Krylov storage of LP solves (FP32 accumulation) */
  double delta_hp;       /* reliable-update trigger for HP solves */
  int block;             /* right-hand sides per batched solve, 1..DL_MAX_RHS; 0: chosen by
                            the autotuner: the first call on a context for a given LP
                            precision, p2max, with_deriv, hpe and time dilution runs one LP
                            block (noise, truncated solve, contractions) of 8, 16 and 32
                            right-hand sides on extra noise indices (from 2^32), each once
                            untimed and once timed, and keeps the block with the least time
                            per right-hand side for that call and later ones (info->block) */
  uint64_t seed;         /* noise seed; HP pairs use indices 0..n_hp-1, LP n_hp.. */
  int p2max;             /* momentum cut */
  int with_deriv;        /* add the one-derivative loops */
  int hpe;               /* add the HPE standard-estimator loops */
  int max_iter;
  int chunk;
  dl_nn* lp_net;         /* NULL: LP solutions by truncated CG.  Otherwise the learned
                            map's output N(eta) stands in for every LP solution (on the
                            context's first-flavour operator); the HP correction of
                            Eq. estiTSM keeps the estimate unbiased for any map. */
  int hp_guess;          /* 1: every HP solve starts from the LP solution of its noise
                            vector (the HP tolerance is unchanged, so the HP solution is
                            the same to that tolerance); 0: from zero */
  int hpe_diff;          /* 1: the HPE estimator's HP-LP correction (Eq. estiTSM) is
                            computed from s_HP - s_LP, which the estimator is linear in:
                            eta^+ X (BH)^4 (s_HP - s_LP) with (BH)^4 applied in FP32 to the
                            difference taken in high precision (relative error ~1e-7 of the
                            correction, not of the loop); 0: both terms in high precision */
  int tdil_dt, tdil_t0;  /* time dilution (Sec. 2.3): tdil_dt = 0 uses full noise vectors;
                            otherwise every source is the noise vector restricted to the time
                            slices t = tdil_t0 (mod tdil_dt) (1 <= tdil_dt <= T, 0 <= tdil_t0 <
                            tdil_dt; tdil_dt = T: one slice, smaller: coherent sources), as
                            dl_noise_z4_tdil makes them, and its loops are contracted on those
                            slices only (zero elsewhere, contraction work in proportion to
                            the slices kept); local loops only (with_deriv = 0).  The
                            estimators are then the standard one (Eq. loopSt) and, with hpe,
                            the HPE one: the one-end trick sums over every sink time of a
                            source and does not restrict to its slices */
} dl_tsm_params;

typedef struct {
  int np, nd, n_est;     /* momenta, derivative slots, estimators (ONE_END, GEN, [HPE]) */
  double seconds_total, seconds_hp, seconds_lp, seconds_contract;
  long long iters_hp, iters_lp; /* summed over right-hand sides */
  int not_converged;     /* 1 when a right-hand side hit max_iter (status DL_NOT_CONVERGED) or
                            an HP solve broke down (status DL_BREAKDOWN: the loops are not
                            valid); an LP solve that breaks down keeps its last iterate, which
                            Eq. estiTSM accepts as the LP map of that noise vector */
  int block;             /* right-hand sides per batched solve used (params->block or the tuned one) */
  double seconds_tune;   /* spent by the autotuner in this call (0 when cached or not asked) */
} dl_tsm_info;

/* Run the TSM for one gauge field: n_hp HP/LP pairs and n_lp fresh LP solves,
 * each followed by its contractions (one-end, generalised one-end, and the HPE
 * standard estimator with its exact part added), noise generated on the
 * device and never stored beyond a block.  Outputs (host memory, may be NULL):
 *   loops  complex128 [n_est][T][Np][nd][4][4]: Eq. estiTSM per element;
 *   obs_hp, obs_lp_pair  double [n_hp][4], obs_lp double [n_lp][4]: per-noise
 *          scalar observables (sigma loop Re, Im; isoscalar axial loop Re, Im;
 *          zero momentum, summed over t) for error estimates.
 * With time dilution (tdil_dt > 0) the estimators are the standard one and, with
 * hpe, the HPE one (n_est = 1 + hpe), and the observables are the standard
 * estimator's i g5 and g_z g5 loops on the kept slices. */
dl_status dl_tsm_run(dl_ctx* ctx, const dl_tsm_params* params, double* loops,
                     double* obs_hp, double* obs_lp_pair, double* obs_lp, dl_tsm_info* info);

/* ---- several lattices in one batch ------------------------------------------ */

/* A context over nlat independent lattices (dims: int[nlat][4]), e.g. several
 * gauge configurations or ensembles, whose solves share every kernel launch.
 * Only dl_load_gauge_lat, dl_set_params_lat, dl_set_params (all lattices) and
 * dl_batch_loops accept a multi-lattice context; nlat <= 16. */
dl_status dl_create_multi(dl_ctx** ctx, int nlat, const int* dims, int device, void* cuda_stream);
/* dl_load_gauge for lattice `lat` (every lattice must use the same recon choice). */
dl_status dl_load_gauge_lat(dl_ctx* ctx, int lat, const double* links, int links_on_device,
                            double t_boundary, int recon_f32, int recon_f16);
/* kappa and a*mu of lattice `lat` (Eq. A.1). */
dl_status dl_set_params_lat(dl_ctx* ctx, int lat, double kappa, double amu);

typedef struct {
  int n;            /* noise vectors per lattice; n * nlat <= 256 */
  double tol;       /* CG residual bound (Sec. 2.2), as in dl_solve_params */
  int prec_hi;      /* DL_F64 or DL_F32 */
  int prec_lo;      /* Krylov storage, DL_F64 / DL_F32 / DL_F16 */
  double delta;     /* reliable-update trigger, 0 = never */
  uint64_t seed;    /* noise r of lattice l is index l * n + r of the dl_noise_z4 stream */
  int max_iter;
  int tile;         /* right-hand sides per instance: 4, 8, 16 or 32; 0 = fastest of 8/16/32
                       from a short timed run (autotuning) */
} dl_batch_params;

typedef struct {
  int tile, instances;
  double seconds_tune, seconds_solve, seconds_contract;
  int iters_max[16];     /* per lattice */
  double resid_max[16];  /* per lattice, CG residual |r|/|Mhat^dag bhat| */
  int not_converged;
} dl_batch_info;

/* Z4 noise, even-odd solve (flavour u) and local loops at zero momentum for n
 * noise vectors on every lattice of a multi-lattice context.  Every lattice's
 * n right-hand sides are split into instances of `tile` columns that share its
 * gauge field; one CUDA-graph loop (conditional WHILE node) iterates CG over all
 * instances of all lattices at once, each column masked out when it converges.
 * loops (host, complex128, may be NULL): per lattice in order,
 *   [2][n][T_l][4][4]: one-end (Eq. loopVv, factor -4i kappa amu) then
 *   generalised one-end (Eq. loopStD, factor 2), summed over space per t.
 * sol (device, complex128, may be NULL): per lattice in order, natural fields
 *   [n][T_l][Z_l][Y_l][X_l][4][3]. */
dl_status dl_batch_loops(dl_ctx* ctx, const dl_batch_params* params, double* loops, void* sol,
                         dl_batch_info* info);

/* ---- instrumentation ------------------------------------------------------ */

/* Live timing of the stencil kernels inside the solver's CUDA graphs.  With
 * profiling on, every captured chunk of CG iterations records CUDA events
 * around the four operator launches of its first iteration (on the context's
 * stream); durations are summed per stage and Krylov precision.  out (host,
 * may be NULL) receives double[4 stages][3 precisions][3] = (launches sampled,
 * milliseconds, site-column items processed) accumulated since the last reset.
 * Stages: 0 = R^-1 D_oe, 1 = R - kappa^2 D_eo (+|q|^2), 2 = daggered stage 0,
 * 3 = daggered stage 1 fused with the CG update.  enable = 1/0 switches
 * profiling on/off and resets the sums; enable = -1 only reads them. */
dl_status dl_profile(dl_ctx* ctx, int enable, double* out);

/* Number of kernels this library has launched in the process so far (direct
 * launches plus the kernel nodes of every CUDA-graph launch).  Thread-safe. */
long long dl_kernel_launches(void);

/* Stencil launch statistics of the process since profiling was last switched on
 * (dl_profile with enable = 1 on any context): out (host) receives
 * double[4 storages][4 epilogues][2][4] = (launches executed, launches timed, summed
 * milliseconds of the timed ones, summed site-column items of the timed ones) per
 * class.  Storages: 0 double-float (DL_F64), 1 FP32, 2 16-bit, 3 IEEE FP64.
 * Epilogues: 0 plain (R^-1 D, B H), 1 with an auxiliary field (R aux - kappa^2 D,
 * source preparation, reconstruction, M), 2 the same with |.|^2 sums, 3 fused with
 * the CG update.  The last index is 1 for the daggered hop.  Launches inside the
 * solver's CUDA graphs are counted per replay and timed through the samples that
 * dl_profile describes; every other stencil launch is timed with CUDA events on its
 * stream.  Waits for those events.  Not thread-safe against concurrent profiling. */
dl_status dl_profile_stencils(double* out);

/* ---- allocation-free variant ----------------------------------------------- */

/* dl_apply without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at the
 * moment they apply an operator, for example a host framework whose caching
 * allocator already owns the device memory, or a latency-critical loop that
 * must not wait on cudaMalloc's implicit synchronisation.  It computes exactly
 * what dl_apply computes (same kernels, same arguments and layouts; the
 * context's gauge field must be loaded), but its seven working fields come
 * from one fixed device array of 64 MiB that the library holds on every GPU
 * that loads it, until the process exits.  Sizes whose working fields exceed
 * that array are rejected with DL_ERR_ARG and a message (the limit is
 * 7 x ceil256(V/2 x npad x site bytes [+ 4-byte scales for DL_F16]) <= 64 MiB,
 * npad = n rounded up to a power of two, site bytes 192 / 96 / 48 for
 * DL_F64 / DL_F32 / DL_F16; e.g. 16^3 x 8 with n = 2 in FP64 needs ~44 MB and
 * fits, with n = 4 it needs ~88 MB and is rejected).
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  The address
 * is kept for the life of the process: after a cudaDeviceReset (or anything else
 * that destroys the device's primary context) it is stale, so do not call this
 * entry point on that device again in the same process.  The array
 * is shared by every call and keeps the previous call's contents (each call
 * overwrites all of it that it reads), so calls that may overlap on the GPU,
 * from any context or stream, race and must be serialised by the caller. */
dl_status dl_apply_noalloc(dl_ctx* ctx, int op, int prec, int flavour, int n,
                           const void* in, const void* aux, void* out, int dtype);

/* ---- learned preconditioner (no counterpart in the paper) ------------------- */

/* A gauge-covariant network N of parallel-transport convolution layers on the
 * context's lattice and gauge field.  Layer l maps C_in channel fields x_i to
 * C_out fields
 *   y_o(x) = sum_i [ sum_b W[0][b][o][i] L_b x_i(x)
 *                  + sum_mu sum_b W[1+2mu][b][o][i] H_b(mu) U_mu(x) x_i(x+mu)
 *                  + sum_mu sum_b W[2+2mu][b][o][i] H_b(mu) U_mu(x-mu)^+ x_i(x-mu) ]
 * with L_b in {1, g5} (b < 2; W[0][2..3] unused, keep them zero) and
 * H_b(mu) in {1, g_mu, g5, g5 g_mu}; hops across t = T-1 <-> 0 carry the
 * context's time-boundary factor.  Weights act on channels and spin only, so
 * N commutes with gauge transformations.  Channels run 1 -> C -> ... -> C -> 1.
 * Weights are complex64, per layer [9][4][C_out][C_in], layers concatenated;
 * activations are stored in FP32 (act_prec = DL_F32) or bfloat16 (act_prec =
 * 3), arithmetic is FP32.  The network uses the FP32 gauge copy (its recon). */
#define DL_BF16 3
dl_status dl_nn_create(dl_ctx* ctx, int n_layers, int channels, int act_prec, dl_nn** out);
void dl_nn_destroy(dl_nn* nn);
/* Complex weights over all layers (the length of the set/get arrays / 2 floats). */
long long dl_nn_weight_count(const dl_nn* nn);
/* Layers of bfloat16 networks: 1 (the default for DL_BF16 activations) runs the channel
 * mixing of the forward pass, of the adjoint (N^+, the input gradients of training) and of
 * the weight gradients as tcgen05 matrix products (bf16 operands from shared memory, FP32
 * accumulators in tensor memory; the adjoint as a layer of the same form with
 * conjugate-transposed weights and the two hops of each direction swapped; the weight
 * gradients with the lattice sites as the reduction dimension), 0 on the CUDA cores (FP32
 * FMA).  DL_ERR_ARG for FP32 activations. */
dl_status dl_nn_set_tensor_cores(dl_nn* nn, int enable);
dl_status dl_nn_set_weights(dl_nn* nn, const float* host_w);   /* host complex64 */
dl_status dl_nn_get_weights(dl_nn* nn, float* host_w);
/* out_k = N(in_k) for n natural full-lattice fields (device, dtype). */
dl_status dl_nn_apply(dl_nn* nn, int n, const void* in, void* out, int dtype);
/* out_k = N^+(in_k), the adjoint map (conjugate weights, adjoint spin factors and
 * transports, layers in reverse order). */
dl_status dl_nn_apply_adjoint(dl_nn* nn, int n, const void* in, void* out, int dtype);
/* Loss sum_k |N(eta_k) - s_k|^2 / |s_k|^2 over n pairs (device natural fields)
 * and its gradient with respect to conj(W) times 2 (host complex64, weight
 * layout); either output may be NULL. */
dl_status dl_nn_loss_grad(dl_nn* nn, int n, const void* eta, const void* s, int dtype, double* loss,
                          float* grad);

/* The residual loss sum_k |M_u N(eta_k) - eta_k|^2 / |eta_k|^2 over n sources (device
 * natural fields) and its gradient (as dl_nn_loss_grad: 2 dL/d conj(W), host complex64);
 * the operator is applied in FP32 with the context's kappa, a*mu and FP32 links. */
dl_status dl_nn_loss_grad_residual(dl_nn* nn, int n, const void* eta, int dtype, double* loss, float* grad);

typedef struct {
  int steps;            /* Adam steps */
  int batch;            /* pairs per step (mean loss) */
  double lr, beta1, beta2, eps;
  uint64_t seed;        /* order of the pairs: a seeded shuffle per pass */
  int loss;             /* 0: |N eta - s|^2 / |s|^2 over (eta, s) pairs; 1: the residual
                           |M_u N eta - eta|^2 / |eta|^2 (s may be NULL), which weighs the
                           error of N by M itself rather than by M^-1 */
} dl_nn_train_params;

/* Adam on the mean loss over minibatches of the n_pairs (eta, s) pairs (device
 * natural fields, dtype).  loss_hist (host, may be NULL) receives the mean
 * minibatch loss of every step. */
dl_status dl_nn_train(dl_nn* nn, const dl_nn_train_params* params, int n_pairs, const void* eta,
                      const void* s, int dtype, double* loss_hist);

/* Flexible GCR (Eisenstat, Elman & Schultz 1983; flexible preconditioning as
 * in Saad 1993) on the full operator M_f (or its normal operator), preconditioned
 * by the network (or by the identity when nn is NULL): FP32 inner cycles of at
 * most `restart` directions, each started from the FP64 true residual b - M x and
 * stopped at inner_tol relative to its start; the FP64 solution is updated after
 * every cycle until ||b - M x|| <= tol ||b||.  The full operator's spectrum can
 * surround the origin near the critical hopping parameter, where restarted GCR on
 * M stagnates; the normal mode cannot stagnate. */
typedef struct {
  double tol;        /* true relative residual bound */
  int max_iter;      /* inner iterations per right-hand side */
  int restart;       /* directions per inner cycle, 1..256 (two FP32 full-lattice fields each) */
  double inner_tol;  /* relative residual reduction per inner cycle */
  int flavour;       /* +1 (u) or -1 (d) */
  int normal;        /* 0: GCR on M, right-preconditioned by N.  1: GCR on the normal
                        operator M^+ M (Hermitian positive definite), preconditioned by
                        N N^+ (N^+ by the network's adjoint kernels), the inner right-hand
                        side M^+ r; the outer FP64 residual is b - M x in both modes */
} dl_fgcr_params;

typedef struct {
  int iters[DL_MAX_RHS];        /* inner iterations */
  int cycles[DL_MAX_RHS];       /* inner cycles (FP64 residual recomputations) */
  double true_resid[DL_MAX_RHS];
  long long op_applications;    /* M applications, FP32 and FP64 */
  long long nn_applications;
  double seconds;
} dl_fgcr_stats;

dl_status dl_fgcr_solve(dl_ctx* ctx, dl_nn* precond, const dl_fgcr_params* params, int n,
                        const void* src, void* sol, int dtype, dl_fgcr_stats* stats);

/* ---- base-2 storage of per-noise loops (App. A, "Binary storage system") ----
 *
 * Loops are averaged over noise vectors ("sources"), so it is enough to keep
 * sums over groups of sources whose sizes are powers of two (Fig. St): the file
 * of weight w = 2^k holds the elementwise sum of the loop arrays of sources
 * w-1 .. 2w-2, counted from 0 in the order they were added (weight 1: source 0,
 * weight 2: sources 1 and 2, weight 4: sources 3-6, ...).  The sum over a set of
 * any n sources with n < 2^K, K the number of complete files, is the sum of the
 * files whose weights are the set bits of n (n = 13: weights 1, 4 and 8), so N
 * sources take O(log2 N) files.  A source is any array of n_values doubles, for
 * example one noise vector's dl_contract output ([T][Np][nd][4][4] complex128 =
 * 32*T*Np*nd doubles) copied to host memory.  These calls are host-only and need
 * no GPU.
 *
 * Files: "<prefix>.<w>" for each complete group and "<prefix>.partial" for the
 * group being filled when the writer is closed.  Format, integers little-endian:
 * char[8] "DLLOOPB2", u32 version 1, u32 0, u64 weight, u64 sources summed (the
 * weight, or fewer for .partial), u64 first source (weight - 1), u64 n_values,
 * u64 FNV-1a-64 of the payload bytes, then n_values IEEE binary64 little-endian.
 * Each file is written beside its name and renamed into place. */
typedef struct dl_store dl_store;

/* Message of the last failed dl_store_* call on this thread. */
const char* dl_store_last_error(void);
/* Open a writer of n_values-double sources under `prefix` (a path without
 * suffix; its directory must exist).  resume = 0: a new store; DL_ERR_STATE if a
 * file of a store already exists under the prefix.  resume = 1: continue the
 * store found there (complete files 1, 2, 4, ... without a gap, then .partial),
 * DL_ERR_IO if its files are inconsistent or n_values differs.  *st is NULL on
 * failure; a writer is freed by dl_store_close. */
dl_status dl_store_open(dl_store** st, const char* prefix, int64_t n_values, int resume);
/* Add n_sources sources (host double[n_sources][n_values]) in order; every group
 * that completes is written at once.  On DL_ERR_IO the sources before the
 * failing write are kept and the write is retried by the next add or close. */
dl_status dl_store_add(dl_store* st, const double* values, int64_t n_sources);
/* Sources added so far, including those of a resumed store. */
dl_status dl_store_count(const dl_store* st, int64_t* total);
/* Write the incomplete group (if any) as .partial, remove a stale .partial
 * otherwise, and free the writer (also when the write fails). */
dl_status dl_store_close(dl_store* st);
/* out (host double[n_values]) = sum over the set of n sources, read from the
 * files of the set bits of n and checked (header, size, checksum); n = 0 gives
 * zeros; DL_ERR_IO if a file is missing or fails a check. */
dl_status dl_store_load(const char* prefix, int64_t n_values, int64_t n, double* out);
/* The source indices of the set of n (if list != NULL, int64[n], ascending). */
dl_status dl_store_sources(int64_t n, int64_t* list);

#ifdef __cplusplus
}
#endif
#endif /* DISCLOOP_H */
