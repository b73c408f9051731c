/*
 * agis.h -- C ABI of the GB300 (sm_103a) library for the data-parallel hot path of the
 * Astrometric Global Iterative Solution (Lindegren et al. 2012, arXiv:1112.4139).
 *
 * The library owns its device memory.  Every pointer argument may be host or device
 * memory (unified addressing); sizes are element counts.  No call throws; every call
 * returns AGIS_OK (0) or a negative code, and agis_last_error() gives a message.
 * One context per host thread.  Rank deficiency is reported in the statistics, never as
 * an error (App. C.3).
 *
 * Units: radians, radians per Julian year (365.25 d), int64 nanoseconds of TCB since a
 * fixed origin.  Astrometric parameters are (alpha, delta, parallax, mu_alpha*, mu_delta)
 * with mu_r = 0 (Sect. 3.2); attitude coefficients are quaternions {x, y, z, w} of the
 * cubic B-spline of Eq. qspline; calibration parameters are the r = 0 offsets of
 * Eq. etazeta, indexed as described at agis_init.
 */
#ifndef AGIS_H
#define AGIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AGIS_ABI_VERSION 8

#define AGIS_OK 0
#define AGIS_E_INVALID (-1)    /* bad argument or call order                            */
#define AGIS_E_CUDA (-2)       /* CUDA runtime error                                    */
#define AGIS_E_OOM (-3)        /* device allocation failed                              */
#define AGIS_E_TIMEOUT (-4)    /* a bounded device-side wait gave up                    */
#define AGIS_E_NONFINITE (-5)  /* a non-finite value appeared in a reduction            */

#define AGIS_N_CCD 62          /* astrometric-field CCDs (Sect. 3.4)                    */
#define AGIS_N_ROW 7           /* across-scan CCD rows                                  */
#define AGIS_N_COL 1966        /* AC pixel columns of a CCD (Eq. etazeta, small-scale terms) */
#define AGIS_MAX_GATE 16       /* gates of the full calibration model (g = 0 .. n_gate-1) */

/* Instrument, ephemeris, epochs and knots (Sects. 3.2-3.4). */
typedef struct agis_geometry {
    double gamma_c;              /* conventional basic angle Gamma_c, Eq. srspropeta     */
    double focal_length;         /* F (m), Eq. etazeta0                                  */
    double p_ac;                 /* AC pixel size (m)                                    */
    double mu_c;                 /* AC pixel coordinate of the CCD centre                */
    double eta0[AGIS_N_CCD];     /* nominal AL observation line -Y_FPA/F per CCD (rad)   */
    double x_fpa[AGIS_N_CCD];    /* X_FPA of the CCD centre (m)                          */
    double x_centre[2];          /* X_FPA^centre[f]: index 0 for f = +1, 1 for f = -1    */
    int32_t ccd_row[AGIS_N_CCD]; /* AC row of each CCD (0..6)                            */
    double orb_L0;               /* ecliptic longitude of the observer at t = 0 (rad)   */
    double obliquity;            /* ecliptic -> ICRS rotation angle (rad)                */
    double au_light_s;           /* A_u / c (s)                                          */
    double year_s;               /* length of the year for proper motions and the orbit  */
    int64_t t_ep_ns;             /* reference epoch of the astrometric parameters        */
    int64_t t_fr_ns;             /* frame rotator epoch (Eq. fr1)                        */
    int64_t knot0_ns;            /* t_beg = tau_{M-1}: first regular knot (App. B.3)     */
    int64_t knot_dt_ns;          /* uniform knot interval; 4-fold knots at both ends     */
    int64_t cal_t0_ns;           /* start of the first calibration interval              */
    int64_t cal_dt_ns;           /* length of the calibration intervals                  */
    int32_t n_coef;              /* N: number of B-spline coefficients                   */
    int32_t n_cal_days;          /* number of calibration intervals                      */
} agis_geometry;

/* Algorithm switches.  agis_default_config() fills the paper's values. */
typedef struct agis_config {
    int32_t robust;              /* 1: inner iteration with downweighting and excess noise (Sect. 5.1.2) */
    int32_t n_rounds;            /* weight rounds of the inner iteration (4)             */
    int32_t n_eps;               /* excess-noise steps per round (3)                     */
    int32_t weight_fn;           /* 0: Eq. dw, 1: Huber Eq. dwH with c = 2               */
    double lambda_att;           /* lambda of Eq. JfuncMod (1e-3)                        */
    int32_t rhs_norm_term;       /* 1: lambda^2 dD D W also on the right-hand side       */
    int32_t seg_len;             /* attitude segment length in knot intervals (Sect. 5.2.2) */
    int32_t seg_overlap;         /* L (12): 2L overlapping knot intervals                */
    int32_t frame_each_iter;     /* agis_iterate runs the frame rotator after each iteration */
    int32_t block_mask;          /* bit 0: S, bit 1: A, bit 2: C (agis_iterate)          */
    int32_t use_graph;           /* agis_iterate replays one captured CUDA graph per iteration */
    double pivot_tol;            /* robust Cholesky: pivots <= pivot_tol * N_jj count as zero (1e-12) */
    int32_t max_obs_per_source;  /* largest n_i accepted (bounds the S-pass scratch), 0: derived */
    int32_t precision;           /* 0: FP64 throughout; 1: mixed (see below)                 */
    int32_t refresh_every;       /* mixed: full FP64 residual refresh every n source updates */
    int32_t block_order;         /* 0: S[AC], 1: Gauss-Seidel SAC, 2: Jacobi [SAC] (below) */
    int32_t cal_model;           /* 0: r = 0 offsets per interval; 1: full geometric model (below) */
    int32_t n_gate;              /* cal_model 1: gates g = 0 .. n_gate-1 (1..AGIS_MAX_GATE)   */
    int32_t cal_j_per_k;         /* cal_model 1: short calibration intervals per long one      */
    int32_t cal_col_bin;         /* cal_model 1: AC pixel columns per small-scale parameter    */
} agis_config;

/* Full geometric calibration (cal_model = 1; Sect. 3.4, Eq. etazeta; Sect. 5.3).  The
 * observation lines of field f, CCD n, gate g, at AC pixel coordinate mu and time t in short
 * interval j (the calibration intervals of the geometry) and long interval k = j / j_per_k:
 *   AL  eta0_n + sum_r Deta_{r f n g j} L*_r(x) + deta_{n g k b}
 *   AC  zeta0_fn(mu) + sum_r Dzeta_{r f n g k} L*_r(x)
 * r = 0, 1, 2, x = (mu - 13.5) / AGIS_N_COL, L*_r the shifted Legendre polynomials, b the bin
 * (of cal_col_bin columns) of the nearest column m = floor(mu + 1/2) - 14 (clamped to
 * 0 .. AGIS_N_COL-1).  AL observations carry mu too (the AC pixel coordinate of the image).
 * Parameter layout: groups (n, g, k) in the order n, g, k; AL group of 6 j_per_k + n_bin values
 * (Deta[j within k][f][r], then deta[b]), then all AC groups of 6 values (Dzeta[f][r]);
 * n_bin = ceil(AGIS_N_COL / cal_col_bin), n_k = ceil(n_cal_days / j_per_k),
 * n_cal = 62 n_gate n_k (6 j_per_k + n_bin + 6).
 * The C block solves each AL group's normals (Eq. normC) as the least-squares solution under
 * Eq. cc2 (every gate), by eliminating each short interval's 6x6 block of large-scale terms
 * onto the small-scale terms, imposing cc2 on that reduced system (null-space method) and
 * back-substituting; each AC group's 6x6 normals by Algorithms C.1-C.3; then Eqs. cc1 and cc3
 * by the projection of Eq. calCon.  Parameters without observations are held and counted as
 * rank defects.  FP64 form only (precision 0). */

/* Block order within an iteration (Sect. 4.6).  0, S[AC] (Eq. precondS(CAG)): A and C both
 * from the residuals after the source update, R = h - A d.  1, SAC (block Gauss-Seidel, Eq.
 * precond): C from those residuals with the attitude update added to first order,
 * R + (dR/da) (a^(k+1) - a^(k)) (the N_ca block).  2, [SAC] (block Jacobi, Eq.
 * precond(SCAG)): A and C from the residuals before the source update, R = h.  All three
 * use the weights of the source update.  The learned proposal and ASI extrapolate the
 * source update for A and C to read and need orders 0 or 1. */

/* Mixed precision (precision = 1).  The residuals stay FP64; partials and normal-equation
 * accumulation run in FP32, and the outer block iteration acts as iterative refinement.
 * Every refresh_every-th source update evaluates the full FP64 observation model
 * (Eqs. resAL, resAC) and stores R (FP64) with the FP32 partials.  The source updates in
 * between take the residuals from the linear identity of Eq. precond2:
 * R <- R + (dR/da) d_a + (dR/dc) d_c after each A and C update, and R <- R - A d after the
 * source solve.  The 5x5 and banded Cholesky factorisations and the frame rotator stay
 * FP64.  The first source update after agis_init or an agis_set_* call always refreshes.
 * Device memory per observation: 64 bytes of records (128 in the FP64 form) besides the
 * inputs.  Converged solutions agree with the FP64 form to well below 1 uas; between
 * refreshes the residuals carry second-order terms of the updates since the last refresh. */

/* Observations in structure-of-arrays form, sorted by source index (ascending; any order
 * within a source).  AL and AC components are separate observations (Sect. 3.6). */
typedef struct agis_obs {
    const int64_t* t_ns;         /* observation time                                     */
    const int32_t* src;          /* source index 0..n_src-1                              */
    const uint8_t* ccd;          /* AF CCD index 0..61                                   */
    const uint8_t* fov;          /* 0: preceding field (f = +1), 1: following (f = -1)   */
    const uint8_t* kind;         /* 0: AL (observed t), 1: AC (observed mu)              */
    const float* sigma;          /* formal standard uncertainty (rad)                    */
    const double* mu;            /* AC pixel coordinate (AC; AL too with cal_model 1)    */
    const uint8_t* gate;         /* gate 0..n_gate-1 (cal_model 1), or NULL: all 0       */
} agis_obs;

/* Statistics of one block call. */
typedef struct agis_block_stats {
    double chi2;                 /* sum_l W_l R_l^2 after the block                      */
    double q_sum;                /* S: sum_i Q_i (Eq. Qi)                                */
    int64_t nu_sum;              /* S: sum_i nu_i                                        */
    int64_t n_out;               /* S: observations with w_l < 0.2                       */
    int64_t rank_defect;         /* robust Cholesky rank-defect count (App. C)           */
    double d_rms[5];             /* S: RMS of the 5 parameter updates                    */
    double elapsed_ms;           /* device time of the block (CUDA events)               */
    double pass_ms;              /* S: device time of the observation pass within it     */
    int32_t full_eval;           /* S: 1 if the pass evaluated the full FP64 model       */
    int32_t reserved_;
} agis_block_stats;

typedef struct agis_iter_stats {
    agis_block_stats s, a, c;
    double frame[6];             /* (eps, omega) applied by the frame rotator            */
    double elapsed_ms;           /* device time, including work redone after a rollback  */
    int32_t proposal;            /* learned proposal: 0 none, 1 applied after this S,     */
                                 /* 2 the previous proposal was rolled back and its      */
                                 /* iteration redone without it before this one          */
    int32_t asi_n;               /* ASI: sample ratios the estimate used (0: not applied) */
    double asi_lambda;           /* ASI: median ratio of successive parallax updates     */
    double asi_factor;           /* ASI: factor 1/(1 - lambda) applied (1: none)         */
} agis_iter_stats;

typedef struct agis_ctx agis_ctx;

/* Fill cfg with the paper's defaults (4 rounds, 3 excess-noise steps, Eq. dw, lambda = 1e-3,
 * L = 12, S[ACG] with the frame rotator each iteration). */
void agis_default_config(agis_config* cfg);

/* Create a context: validate and upload the observations (sorted by source), the starting
 * values and the optional frame-rotator reference; build the time-ordered and
 * calibration-ordered permutations.  Eq. synth, Sect. 3.6.
 *   obs        n_obs observations (host or device pointers)
 *   src0       n_src x 5 starting astrometric parameters
 *   src_ref    n_src x 4 reference (alpha, delta, mu_a*, mu_d) at t_ep in the ICRS for the
 *              frame rotator (subset S_PM of Sect. 6.1.4), or NULL (frame rotator disabled)
 *   att0       n_coef x 4 starting spline coefficients
 *   cal0       n_cal starting calibration parameters; with cal_model 1 the layout above,
 *              otherwise n_cal = n_cal_days * 2 * (62 + 7):
 *              AL offset of (interval d, field f, CCD n) at (d*2 + f)*62 + n,
 *              AC offset of (d, f, row r) at n_cal_days*124 + (d*2 + f)*7 + r
 *   stream     cudaStream_t to run on (NULL: the legacy default stream)
 * Errors: AGIS_E_INVALID (unsorted sources, index out of range, non-finite input,
 * n_coef < 4, inconsistent sizes), AGIS_E_OOM, AGIS_E_CUDA.  On error *out is NULL. */
int agis_init(const agis_geometry* geo, const agis_config* cfg, const agis_obs* obs, int64_t n_obs,
              const double* src0, const double* src_ref, int32_t n_src, const double* att0, int32_t n_coef,
              const double* cal0, int32_t n_cal, void* stream, agis_ctx** out);

/* S block (Sect. 5.1): evaluate residuals and partials of every observation at the current
 * (s, a, c) (Eqs. resAL, resAC, srsprop1diffsol, dfadq), solve the per-source 5x5 normal
 * equations (Eq. normS) with the inner iteration, update s, and keep the residuals
 * R_l = h_l - A_l d and weights W_l for the A and C blocks (Eq. precond2). */
int agis_source_update(agis_ctx* ctx, agis_block_stats* out);

/* A block (Sect. 5.2): banded attitude normals (Eq. normAmod) from the residuals and weights
 * of the latest S block, segmented robust banded Cholesky (Sect. 5.2.2, App. C), update a.
 * Error AGIS_E_INVALID if no S block ran since the context was created or restored. */
int agis_attitude_update(agis_ctx* ctx, agis_block_stats* out);

/* C block (Sect. 5.3): block-diagonal calibration normals (Eq. normC), robust solves and the
 * constraint projection of Eq. calCon for Eqs. cc1 and cc3; update c.  Same call-order rule. */
int agis_calibration_update(agis_ctx* ctx, agis_block_stats* out);

/* Frame rotator (Sect. 6.1): least-squares (eps, omega) from Eq. cond-mu3 over all sources
 * (or the n_subset listed in subset) with unit weights, then the rigorous transformation of
 * the sources (Sect. 6.1.2) and a_n <- f(t_n)^-1 a_n (Eq. fr-q4).  eps_omega_out (6 doubles,
 * host) receives the applied parameters.  AGIS_E_INVALID without a reference. */
int agis_frame_rotate(agis_ctx* ctx, const int32_t* subset, int32_t n_subset, double eps_omega_out[6]);

/* n_iter iterations of the S[ACG] simple iteration (Sects. 4.5-4.6) with the blocks of
 * cfg->block_mask and, if cfg->frame_each_iter, the frame rotator.  per_iter (host, may be
 * NULL) receives n_iter records; *n_done the number completed. */
int agis_iterate(agis_ctx* ctx, int32_t n_iter, agis_iter_stats* per_iter, int32_t* n_done);

/* Residuals R_l of all observations at the current (s, a, c) without updating anything
 * (Eqs. resAL, resAC); out has n_obs doubles in the caller's observation order. */
int agis_evaluate(agis_ctx* ctx, double* R_out);

/* State export and checkpoint restore; buffers are caller-owned, sized as at agis_init. */
int agis_get_sources(agis_ctx* ctx, double* src_out);           /* n_src x 5 */
int agis_get_attitude(agis_ctx* ctx, double* att_out);          /* n_coef x 4 */
int agis_get_calibration(agis_ctx* ctx, double* cal_out);       /* n_cal */
int agis_set_sources(agis_ctx* ctx, const double* src);
int agis_set_attitude(agis_ctx* ctx, const double* att);
int agis_set_calibration(agis_ctx* ctx, const double* cal);
/* Residuals and weights handed from the latest S block to A and C (caller order): available
 * after any source update until a state is set (a frame rotation leaves them as they are; in
 * block order 1 they include the first-order attitude correction that the C block read).
 * AGIS_E_INVALID before the first source update or after an agis_set_* call. */
int agis_get_residuals(agis_ctx* ctx, double* R_out, double* W_out);
/* Per-source results of the latest S block: eps_i^2, Q_i, nu_i, n_out_i, D_i (5 x n_src doubles,
 * row-major by quantity) and the 5x5 inverse normal matrices (n_src x 25 doubles, or NULL). */
int agis_get_source_stats(agis_ctx* ctx, double* stats_out, double* cov_out);

/* Sizes of the context (n_obs, n_src, n_coef, n_cal). */
int agis_get_sizes(const agis_ctx* ctx, int64_t* n_obs, int32_t* n_src, int32_t* n_coef, int32_t* n_cal);
/* Device time in ms of the kernels of the latest call, per kernel class (S pass, A
 * accumulation, A solve, C, frame): 5 doubles. */
int agis_get_kernel_times(const agis_ctx* ctx, double* ms_out);

void agis_destroy(agis_ctx* ctx);
const char* agis_last_error(const agis_ctx* ctx);
int agis_abi_version(void);

/* Largest max_obs_per_source accepted by agis_source_update_static. */
#define AGIS_STATIC_MAX_OBS 16384

/* Source update that allocates no device memory.  The paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory themselves or through this
 * library, e.g. code running inside a host framework that owns the allocator, or a process
 * that reserved all device memory up front.  It runs the S block of agis_source_update()
 * (observation pass, inner iteration, 5x5 solves, parameter update) on caller-owned device
 * arrays, and keeps its scratch in a 32 MiB file-scope device array that every GPU loading
 * this library holds until the process exits.
 *   obs        n_obs observations, DEVICE pointers, sorted by source (as for agis_init)
 *   src        n_src x 5 parameters, device, updated in place
 *   att, cal   device arrays of n_coef x 4 and n_cal (geo->n_cal_days * 138) values
 *   R_out, W_out  device, n_obs each (residuals h - A d and weights), or NULL
 *   stats_out  device, 5 x n_src (eps^2, Q, nu, n_out, D by rows), or NULL
 *   max_obs_per_source  upper bound on the observations of any source, 1..AGIS_STATIC_MAX_OBS
 * The first call on a device looks up the array's device address with that device current;
 * make it before any stream capture.  All calls share the array and it keeps the last
 * call's contents: calls that overlap on the GPU race and must be serialised.  Errors:
 * AGIS_E_INVALID for bad arguments, and for inputs that a check kernel finds before anything
 * is written (source index out of range, sources not sorted, ccd, fov or kind out of range,
 * sigma not positive and finite, non-finite mu of an AC observation, non-finite src, att or
 * cal, a source with more than max_obs_per_source observations): src and the outputs are
 * then unchanged; the message is in agis_last_error(NULL).  AGIS_E_CUDA.  Synchronises the
 * stream before returning (twice: after the check and after the update). */
int agis_source_update_static(const agis_geometry* geo, const agis_config* cfg, const agis_obs* obs, int64_t n_obs,
                              double* src, int32_t n_src, const double* att, const double* cal, double* R_out,
                              double* W_out, double* stats_out, int32_t max_obs_per_source, void* stream);

/* ---- Learned iteration proposal ---------------------------------------------------------
 * Not part of the paper; its analogue there is the accelerated simple iteration (Sect. 4.7),
 * which extrapolates the source updates with a factor estimated from successive updates.
 * A network maps the last four updates of each source (and its observation count and
 * ecliptic latitude) to a correction towards the converged solution:
 *   features  22 per source: the last four updates d (oldest first; alpha* and delta as arcs,
 *             rad and rad/yr) divided by their RMS sigma, log10(n_obs) - 2.5, sin(ecliptic
 *             latitude)
 *   network   22 -> 64 -> 64 -> 5, ReLU hidden layers; parameters as one FP32 vector in the
 *             order W1[64][22], b1[64], W2[64][64], b2[64], W3[5][64], b3[5]
 *   output    the correction sigma * y in the tangent units of d, added to the sources
 * The forward runs on tensor cores with BF16 inputs, weights and hidden activations and
 * FP32 accumulation; the training gradient is that of the same rounded forward. */
#define AGIS_MLP_N_IN 22
#define AGIS_MLP_N_HIDDEN 64
#define AGIS_MLP_N_OUT 5
#define AGIS_MLP_N_PARAMS 5957
/* bytes of the packed (BF16, padded) weights that agis_mlp_pack writes */
#define AGIS_MLP_PACKED_BYTES 16032

/* Device-pointer kernels on `stream` (NULL: the legacy default stream); asynchronous.
 * agis_mlp_pack        params (FP32, AGIS_MLP_N_PARAMS) -> packed weights for the forward
 * agis_mlp_forward     X (n x 22 FP32, row-major) -> Y (n x 5 FP32)
 * agis_mlp_loss_grad   loss = mean over the n rows of sum_j (y_j - t_j)^2 and its gradient
 *                      with respect to params (grad: AGIS_MLP_N_PARAMS FP32, overwritten;
 *                      loss: 1 FP32, overwritten); T: rows of 5; row r of the batch is row
 *                      idx[r] of X and T (idx: n int32, device), or row r when idx is NULL
 * agis_mlp_adam        one Adam step (Kingma & Ba 2015) with bias correction at step t >= 1;
 *                      m, v: moment vectors (AGIS_MLP_N_PARAMS FP32, zero before step 1)
 * agis_proposal_targets  T = (x_ref - x_k) / sigma in the tangent units of d, n x 5 FP32,
 *                      from x_k, x_ref (n x 5 FP64) and sigma (n FP64)
 * Errors: AGIS_E_INVALID (null pointer, n < 0, t < 1), AGIS_E_CUDA (launch failure). */
int agis_mlp_pack(const float* params, void* packed, void* stream);
int agis_mlp_forward(const void* packed, const float* X, int32_t n, float* Y, void* stream);
int agis_mlp_loss_grad(const float* params, const float* X, const float* T, const int32_t* idx, int32_t n,
                       float* grad, float* loss, void* stream);
int agis_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t t, float lr, float beta1, float beta2,
                  float eps, void* stream);
int agis_proposal_targets(const double* src_k, const double* src_ref, const double* sigma, int32_t n, float* T,
                          void* stream);

/* Enable the proposal in agis_iterate: params (host or device, AGIS_MLP_N_PARAMS FP32) are
 * copied; every >= 5 is the number of iterations between proposals (the four updates the
 * network sees are then plain ones).  After the S block of an iteration that qualifies, the
 * proposal is added to the sources (and, to first order, to the residuals the A and C blocks
 * read); the robust chi^2 of the next S block decides: if it is larger than before the
 * proposal, the state before that iteration is restored and the iteration is redone without
 * it.  params = NULL disables.  Errors: AGIS_E_INVALID, AGIS_E_OOM, AGIS_E_CUDA. */
int agis_set_proposal(agis_ctx* ctx, const float* params, int32_t every);
/* Features of the context's last four source updates and the current sources (device
 * pointers: X n_src x 22 FP32, sigma n_src FP64), as the proposal uses them; a source with
 * fewer than four updates since agis_init has zero history entries.  For training data. */
int agis_get_proposal_features(agis_ctx* ctx, float* X, double* sigma);
/* The current source parameters into a device array (n_src x 5 FP64, no host copy). */
int agis_copy_sources_device(agis_ctx* ctx, double* src_dev);

/* ---------------------------------------------------------------------------------------
 * Accelerated simple iteration (ASI, Sect. 4.7)
 *
 * Once the updates of successive iterations are nearly proportional, d^(k+1) ~ lambda d^(k),
 * the updates still to come sum to d^(k+1) / (1 - lambda) (a geometric series), and ASI
 * applies that factor to the update of the iteration.  In agis_iterate, after the S block
 * of every iteration that has the source updates of two S blocks behind it:
 *   r_i     = d_varpi,i^(k+1) / d_varpi,i^(k) for the sample sources i = 0, m, 2m, ...
 *             (m = stride; parallax updates, which a change of the frame orientation
 *             leaves alone); sources with a zero or non-finite ratio are skipped
 *   lambda  = the lower median of the r_i, clamped to [0, lambda_max]
 *   sources += (1/(1 - lambda) - 1) d^(k+1), alpha* turned into alpha with cos(delta),
 *             and the residuals the A and C blocks read -= A times that correction
 *             (first order), so that A and C solve against the extrapolated sources.
 * The factor multiplies the source update only: for two coupled blocks iterated in
 * Gauss-Seidel order the error component along the slowest eigenvector vanishes when the
 * update of one block is extrapolated with its exact lambda, and overshoots when both are.
 * The ratios are those of the plain S-block updates, before extrapolation.  An iteration
 * that carries a learned proposal is not also extrapolated.
 * stride <= 0 disables; lambda_max in [0, 1).  Errors: AGIS_E_INVALID, AGIS_E_OOM,
 * AGIS_E_CUDA. */
int agis_set_asi(agis_ctx* ctx, int32_t stride, double lambda_max);
/* The ASI estimate on its own, from two source updates in device memory (d_prev, d_cur:
 * n_src x 5 FP64, parallax at column 2): est[0] the lower median of the ratios
 * d_cur/d_prev over the sources i = 0, stride, 2 stride, ... with d_prev != 0 and a finite
 * ratio, est[1] that median clamped to [0, lambda_max], est[2] = 1/(1 - est[1]), est[3] the
 * number of ratios (all zero but est[2] = 1 when there are none).  est: 4 FP64 on the device;
 * scratch: ceil(n_src / stride) x 8 bytes on the device.  Asynchronous on `stream`.
 * Errors: AGIS_E_INVALID (null pointer, n_src < 1, stride < 1, lambda_max outside [0, 1)),
 * AGIS_E_CUDA. */
int agis_asi_estimate(const double* d_prev, const double* d_cur, int32_t n_src, int32_t stride, double lambda_max,
                      void* scratch, double* est, void* stream);

/* ---------------------------------------------------------------------------------------
 * Excess attitude noise (Sect. 5.2.5, Eqs. excess, W, wl, e09)
 *
 * The excess noise of an observation is modelled as eps_i^2 (its source, estimated by the
 * source update) plus eps_a^2(t), one function of time per component: AL, AC in the
 * preceding field of view (fov 0) and AC in the following one (fov 1).  Each is constant on
 * buckets [knot0_ns + j bucket_ns, knot0_ns + (j+1) bucket_ns), j = 0 .. n_buckets - 1,
 * n_buckets reaching the last observation.  With the noise on, every source update (in
 * agis_iterate and agis_source_update):
 *   uses sigma~^2 = sigma^2 + eps_a^2(t) in place of sigma^2 (robust scale, weights and
 *             normals; Eq. W), eps_a^2 being the estimate of the previous source update
 *             (0 after this call);
 *   estimates eps_a^2(j) = max(0, F_0.68{R_l^2 - sigma_l^2 - eps_i^2}) over the observations
 *             l of bucket j and the component (Eq. e09; R the residual after the update,
 *             sigma the formal one, F_0.68 the 68% quantile with linear interpolation between
 *             order statistics, 0 for an empty bucket);
 *   and the next attitude update weighs observation l with w(R_l / sqrt(v)) / v,
 *             v = sigma_l^2 + eps_a^2(t_l) + eps_i^2 (Eqs. W, wl) in place of the weights of
 *             the source update; the calibration update keeps the latter.
 * bucket_ns > 0 switches the noise on (eps_a^2 = 0), 0 switches it off.  Both forms: the mixed
 * form (precision 1) forms x_l and the attitude weights from its float-pair residuals in FP64,
 * hands the attitude update the pairs (W_l, W_l R_l) in FP32, and keeps sigma~_l as the FP32
 * sigma of its observation records (its next source update after this call starts with a full
 * FP64 evaluation).  Block orders S[AC] and SAC, not together with ASI or the learned proposal.
 * Errors: AGIS_E_INVALID (bucket_ns < 0, one of those combinations, an observation before
 * knot0_ns, more than 2^30 / 3 buckets), AGIS_E_OOM, AGIS_E_CUDA.  Device memory: 20 bytes
 * per observation and 48 bytes per bucket, owned by the context (and 12 bytes per
 * observation during this call, for the sort of the (component, bucket) order). */
int agis_set_attnoise(agis_ctx* ctx, int64_t bucket_ns);
/* *n_buckets = the number of buckets (0 when the noise is off); if eps2_a is not NULL and
 * the noise is on, eps2_a[c * n_buckets + j] = eps_a^2 of component c (0 AL, 1 AC preceding
 * field, 2 AC following field) in bucket j, rad^2, from the last source update (host or
 * device memory, 3 x n_buckets FP64, caller-owned).  Synchronous.  Errors: AGIS_E_INVALID
 * (null ctx or n_buckets), AGIS_E_CUDA. */
int agis_get_attnoise(agis_ctx* ctx, double* eps2_a, int32_t* n_buckets);

/* ---------------------------------------------------------------------------------------
 * Source partitions (Sects. 4.6, 7.1): several contexts, each holding the observations of one
 * part of the sources (sorted, indices 0 .. n_src-1 of its own) and the whole attitude and
 * calibration, iterate one problem.  The source update is local.  The attitude and
 * calibration normals are sums over observations (Eqs. normAmod, normC), and the frame
 * rotator's over sources (Eq. cond-mu3): each context accumulates its part, the caller adds
 * the parts over the contexts (an all-reduce: the paper's accumulation of the DataTrain's
 * normals on the servers, Sect. 7.1) and gives the sums back, and every context solves the
 * same sums, so that all hold the same attitude and calibration.  One iteration:
 *   agis_source_update;
 *   for X in (AGIS_X_ATTITUDE, AGIS_X_CALIBRATION): agis_accumulate(X), agis_get_exchange(X),
 *       sum over the contexts, agis_set_exchange(X), agis_solve_exchange(X);
 *   the same with AGIS_X_FRAME (its sums are over the context's sources and need no source
 *       update; it applies the rotation to the local sources and to the attitude).
 * With one context this is agis_iterate's S[AC] iteration (the sums of one part are the sums).
 *   AGIS_X_ATTITUDE     per knot interval, the 136 upper entries of the 16x16 normals of its four
 *                       coefficients and the 16 right-hand sides (n_coef - 3) x 152 doubles
 *   AGIS_X_CALIBRATION  per calibration parameter, sum W and -sum W R (n_cal x 2)
 *   AGIS_X_FRAME        the 21 upper entries of the 6x6 normals and the 6 right-hand sides (27)
 * Buffers are caller-owned (host or device).  FP64 form; the calibration exchange needs the
 * offsets model (cal_model 0).  agis_accumulate synchronises; agis_solve_exchange returns the
 * rank defects in out (and the applied (eps, omega) for the frame, if eps_omega_out is not
 * NULL).  Errors: AGIS_E_INVALID (unknown buffer, call order, the restrictions above),
 * AGIS_E_OOM, AGIS_E_CUDA. */
#define AGIS_X_ATTITUDE 0
#define AGIS_X_CALIBRATION 1
#define AGIS_X_FRAME 2
int agis_exchange_size(const agis_ctx* ctx, int32_t which, int64_t* n_doubles);
int agis_accumulate(agis_ctx* ctx, int32_t which);
int agis_get_exchange(agis_ctx* ctx, int32_t which, double* out);
int agis_set_exchange(agis_ctx* ctx, int32_t which, const double* in);
int agis_solve_exchange(agis_ctx* ctx, int32_t which, agis_block_stats* out, double eps_omega_out[6]);

/* ---------------------------------------------------------------------------------------
 * Launch-shape autotuner (iteration control)
 *
 * Knobs and their parameters (a, b):
 *   AGIS_KNOB_OBS_PASS    observation pass (FP64 model in the FP64 form, the linearized
 *                         correction in the mixed form): a threads per block (128, 256),
 *                         b blocks per SM of the grid-stride grid (1..64)
 *   AGIS_KNOB_SRC_BATCH   FP64 form, per-source solves: a sources per work fetch of the
 *                         persistent kernel (1..32; 0: n_src / 2432 within 1..32); b unused
 *   AGIS_KNOB_MIX_SUMS    mixed form, S-block sums and final pass: a warps per block
 *                         (2, 4, 8), b blocks per SM (1..64)
 *   AGIS_KNOB_MIX_SOLVE5  mixed form, 5x5 solves (a thread per source): a threads per block
 *                         (64, 128, 256); b unused
 *   AGIS_KNOB_ATT_ACCUM   A-block accumulation (a warp per knot interval): b blocks per SM
 *                         (1..64; 0: 32 in the FP64 form, 64 in the mixed form); a unused
 *   AGIS_KNOB_CAL_ACCUM   C-block accumulation (a warp per parameter): a threads per block
 *                         (128, 256), b blocks per SM (1..64)
 * Every kernel a knob shapes gives each observation, source, knot interval or calibration
 * parameter to one thread or one warp with the same arithmetic whatever the shape, so the
 * solution does not depend on the knobs (bit for bit).
 *
 * agis_autotune runs up to max_iter S[ACG] iterations, exactly as agis_iterate would (they
 * advance the solution; the learned proposal and ASI pause meanwhile, and the blocks run
 * without graph capture).  Each iteration gives each timed block (S observation pass, S
 * solves, A, C) one candidate shape of one of its knobs; the device time of the block (CUDA
 * events) rates it.  The mixed form rates its observation pass only in iterations that use
 * the linearized correction.  When every candidate of a knob has been rated, the fastest is
 * kept; the candidates include the default.  out (may be NULL): AGIS_N_KNOBS entries in knob
 * order; *n_done: iterations run.  Errors: AGIS_E_INVALID, AGIS_E_CUDA, AGIS_E_NONFINITE.
 *
 * agis_get_tuning / agis_set_tuning read and set the shapes (for instance to reuse a tuning
 * on another context of the same workload); set validates every value against the ranges
 * above and changes nothing on AGIS_E_INVALID. */
#define AGIS_KNOB_OBS_PASS 0
#define AGIS_KNOB_SRC_BATCH 1
#define AGIS_KNOB_MIX_SUMS 2
#define AGIS_KNOB_MIX_SOLVE5 3
#define AGIS_KNOB_ATT_ACCUM 4
#define AGIS_KNOB_CAL_ACCUM 5
#define AGIS_N_KNOBS 6
typedef struct agis_tune_entry {
    int32_t knob;                /* AGIS_KNOB_*                                          */
    int32_t a, b;                /* the shape (meaning per knob, above)                  */
    int32_t n_tried;             /* candidates rated (0: the knob does not apply)        */
    double best_ms;              /* device time of the block with the kept shape         */
    double default_ms;           /* ... with the default shape (-1: not rated)           */
} agis_tune_entry;
int agis_autotune(agis_ctx* ctx, int32_t max_iter, int32_t* n_done, agis_tune_entry* out);
int agis_get_tuning(const agis_ctx* ctx, agis_tune_entry* out);
int agis_set_tuning(agis_ctx* ctx, const agis_tune_entry* in, int32_t n);

#ifdef __cplusplus
}
#endif
#endif /* AGIS_H */
