// agis_internal.cuh -- device-side data layout and the per-observation model of the AGIS
// hot path (Lindegren et al. 2012).  Shared by the kernels of this library only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>

#include "agis.h"

namespace agis {

constexpr int kWarp = 32;
constexpr int kNccd = AGIS_N_CCD;
constexpr int kRecDoubles = 8;   // A/C hand-over record: 64 bytes per observation
constexpr int kBlkVals = 152;    // per knot interval: 136 upper entries of the 16x16 + 16 rhs
constexpr int kScr = 8;          // S-pass scratch per observation: h, A[5], w, sigma^2

// Packed per-observation descriptor: bits 0-5 CCD, 6 field (0: f=+1), 7 kind (0: AL),
// 8-31 calibration parameter index.
__host__ __device__ inline uint32_t meta_ccd(uint32_t m) { return m & 63u; }
__host__ __device__ inline uint32_t meta_fov(uint32_t m) { return (m >> 6) & 1u; }
__host__ __device__ inline uint32_t meta_kind(uint32_t m) { return (m >> 7) & 1u; }
__host__ __device__ inline uint32_t meta_cal(uint32_t m) { return m >> 8; }

// Full geometric calibration (Eq. etazeta; agis_config.cal_model = 1): sizes of the parameter
// layout described in agis.h.  on = 0: the r = 0 offsets of the packed index.
struct CalGen {
    int32_t on;
    int32_t n_gate, j_per_k, col_bin, n_bin, n_k, n_j, al_size;
    int64_t n_al;                // AL parameters (62 n_gate n_k al_size); the AC groups follow
    int64_t t0, dt;              // calibration intervals (the short intervals j)
    double inv_ncol;
};
// generic model: gate in bits 8-15 of the packed descriptor (no packed parameter index)
__host__ __device__ inline uint32_t meta_gate(uint32_t m) { return (m >> 8) & 255u; }

// Geometry passed by value to the kernels.
struct DevGeo {
    double gamma_half;
    double cos_gh, sin_gh;       // cos and sin of gamma_half
    double F, p_ac, mu_c;
    double eta0[kNccd];
    double x_fpa[kNccd];
    double x_centre[2];
    double orb_L0, cos_obl, sin_obl, au_light_s, year_s, orb_rate;
    double orb_L0_pi, inv_year_s, vk;   // L0 / pi, 1 / year, orbital speed / c
    int64_t t_ep_ns, t_fr_ns, knot0_ns, knot_dt_ns;
    double inv_knot_dt;
    int32_t n_coef;
    CalGen cg;
    // orbital longitude tabulated every 2^kOrbShift ns from orb_t0: (sin L, cos L) pairs, and
    // the longitude rate per ns (null table: sincospi of the linear longitude)
    const double* orb_tab;
    int64_t orb_t0;
    int32_t orb_n;
    double orb_rad_per_ns;
};
constexpr int kOrbShift = 42;   // 4398 s: 8.8e-4 rad of orbital longitude per table step

inline void fill_devgeo(const agis_geometry* geo, int32_t n_coef, DevGeo& G) {
    const double pi = 3.141592653589793;
    std::memset(&G, 0, sizeof(G));
    G.gamma_half = 0.5 * geo->gamma_c;
    G.cos_gh = std::cos(G.gamma_half);
    G.sin_gh = std::sin(G.gamma_half);
    G.F = geo->focal_length;
    G.p_ac = geo->p_ac;
    G.mu_c = geo->mu_c;
    for (int i = 0; i < kNccd; i++) {
        G.eta0[i] = geo->eta0[i];
        G.x_fpa[i] = geo->x_fpa[i];
    }
    G.x_centre[0] = geo->x_centre[0];
    G.x_centre[1] = geo->x_centre[1];
    G.orb_L0 = geo->orb_L0;
    G.cos_obl = std::cos(geo->obliquity);
    G.sin_obl = std::sin(geo->obliquity);
    G.au_light_s = geo->au_light_s;
    G.year_s = geo->year_s;
    G.orb_rate = 2.0 * pi / geo->year_s;
    G.orb_L0_pi = geo->orb_L0 / pi;
    G.inv_year_s = 1.0 / geo->year_s;
    G.vk = G.orb_rate * geo->au_light_s;
    G.t_ep_ns = geo->t_ep_ns;
    G.t_fr_ns = geo->t_fr_ns;
    G.knot0_ns = geo->knot0_ns;
    G.knot_dt_ns = geo->knot_dt_ns;
    G.inv_knot_dt = 1.0 / (double)geo->knot_dt_ns;
    G.n_coef = n_coef;
    G.orb_rad_per_ns = G.orb_rate * 1e-9;
}

// (sin L, cos L) of the tabulated longitude L(t_j) = L0 + 2 pi (t_j / 1e9) / year at
// t_j = t0 + j 2^kOrbShift, j = 0 .. n-1 (host, at set-up)
inline void fill_orbit_table(const DevGeo& G, int64_t t0, int32_t n, double* tab) {
    const double pi = 3.141592653589793;
    for (int32_t j = 0; j < n; j++) {
        const int64_t t = t0 + ((int64_t)j << kOrbShift);
        const double x = G.orb_L0_pi + 2.0 * ((double)t * 1e-9) * G.inv_year_s;
        tab[2 * j] = std::sin(pi * x);
        tab[2 * j + 1] = std::cos(pi * x);
    }
}

// Hand-over record written by the S pass and read (gathered) by the A and C passes.
struct __align__(16) ObsRec {
    int64_t t_ns;
    double R;       // residual after the source update, h - A d
    double W;       // statistical weight w / (sigma^2 + eps^2)
    uint32_t meta;
    int32_t pad;
    double g[4];    // dR/dq / ||s||  (so that dR/da_n = g B_n)
};
static_assert(sizeof(ObsRec) == 64, "record must be 64 bytes");

// Mixed-precision per-observation arrays (source order).  Every per-observation operation
// of the mixed form runs on the FP32 pipe; the residual is kept as an unevaluated float pair
// R = Rh + Rl (about 48 significant bits).
//   s   what the source solve reads besides R: the FP32 design row A = (Ap, Aq, Aw, Ap tau,
//       Aq tau) (Eq. ubardiff) and sigma (negative for AC)                     20 B
//   r   the residual pair (Rh, Rl), in its own array so that the linearized observation
//       pass reads and writes 8 B of it per observation                        8 B
//   ac  what the A and C blocks read besides the partials: (W, W Rh) after the source
//       update; the per-observation path of the S block keeps its round weights in .x    8 B
//   t   the attitude partial g, the descriptor, and the time as knot interval l with the
//       offset u = (t - tau_l) / dt                                            32 B
struct MixS {
    float Ap, Aq, Aw, tau;
    float sig;      // +sigma for AL, -sigma for AC
};
struct __align__(16) MixT {
    float g[4];     // dR/dq / ||s||
    uint32_t meta;
    int32_t l;      // left knot index of the observation time
    float u;        // (t - tau_l) / knot interval
    uint32_t pad;
};
static_assert(sizeof(MixS) == 20 && sizeof(MixT) == 32, "mixed record sizes");
struct MixObs {
    MixS* s;
    float2* r;
    float2* ac;
    MixT* t;
};

// Per-source state of the mixed S block between its kernels.
struct __align__(16) SrcScale {
    double s2c[2];  // sigma^2 of the AL and AC observations (one value per class)
    double s2min;
    float vs;       // robust scale of x = R / sigma
    int32_t flags;  // bit 0: one sigma per class (class-sum path); bit 1: no observations
};
// FP32 inputs of one weight round's per-observation pass (written by the per-source solve of
// the previous round, so that the passes need no FP64 arithmetic)
struct __align__(16) SrcRound {
    float dp[5];    // previous solution: the shift of the sums
    float isd[2];   // 1 / sqrt(sigma_c^2 + eps^2_prev)
    float sigc[2];
    float vs;
    int32_t mode;   // 0 first robust round, 1 later robust rounds, 2 plain weights
    int32_t pad;
};
struct __align__(16) SrcFinal {  // the final update as float pairs and 1 / (sigma_c^2 + eps^2)
    float dh[5], dl[5];
    float iw[2];
};
struct RoundSums {  // FP32 class sums of one weight round, shifted to the previous solution
    float AA[2][15];
    float Ah[2][5];
    float hh[2];
    int32_t nout;
    int32_t pad;
};
struct MixSrcWork {
    SrcScale* scale;
    SrcRound* round;
    SrcFinal* fin;
    RoundSums* sums;
};

// Per-source outputs of the S block (device arrays).
struct SrcOutPtrs {
    double* src;      // n_src x 5, updated in place
    double* d;        // n_src x 5 updates
    double* eps2;     // excess source variance
    double* q;        // Q_i
    double* dsig;     // significance D
    double* chi2;     // sum over the source of W R^2
    double* cov;      // n_src x 25 inverse normal matrix
    int* nu;
    int* nout;
    int* rankdef;
};

struct Settings {
    int robust, n_rounds, n_eps, weight_fn;
    double lambda2;
    int rhs_norm_term;
    double pivot_tol;
    int handover_h;   // block Jacobi: A and C read h (the residual before the source update)
};

// Launch shapes chosen by the autotuner.  Every kernel they shape gives each observation,
// source, knot interval or calibration parameter to one thread or one warp with the same
// arithmetic whatever the shape, so the results do not depend on them.
struct Shapes {
    int obs_threads = 256, obs_bps = 64;  // observation pass: threads per block, blocks per SM (grid cap)
    int src_batch = 0;                    // FP64 S solves: sources per work fetch (0: n_src / 2432 in 1..32)
    int sums_warps = 4, sums_bps = 16;    // mixed S sums and final pass: warps per block, blocks per SM
    int solve5_threads = 128;             // mixed 5x5 solves: threads per block
    int att_bps = 0;                      // A accumulation: blocks per SM (0: 32 FP64 form, 64 mixed form)
    int cal_threads = 256, cal_bps = 16;  // C accumulation: threads per block, blocks per SM
};

// ---------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Downweighting factor, Eq. dw (weight_fn 0) or Huber Eq. dwH with c = 2 (weight_fn 1).
__device__ __forceinline__ double wfun(double z, int fn) {
    double a = fabs(z);
    if (fn == 0) {
        if (a <= 2.0) return 1.0;
        if (a < 3.0) {
            double t = a - 2.0;
            return 1.0 - 1.773735 * t * t + 1.141615 * t * t * t;
        }
        return exp(-a / 3.0);
    }
    if (a <= 2.0) return 1.0;
    return 2.0 * (2.0 * a - 2.0) / (a * a);
}

// knot tau_k (ns) of the uniform sequence with 4-fold end knots
// order-preserving map of an FP64 value to an unsigned key (and back), for radix selection
__device__ __forceinline__ uint64_t dkey(double x) {
    long long b = __double_as_longlong(x);
    return b < 0 ? ~(uint64_t)b : ((uint64_t)b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(uint64_t k) {
    long long b = (k & 0x8000000000000000ull) ? (long long)(k & 0x7fffffffffffffffull) : (long long)(~k);
    return __longlong_as_double(b);
}

// Excess attitude noise (Sect. 5.2.5): eps_a^2 of the three components (AL, AC in the
// preceding field, AC in the following field) per time bucket [t0 + j dt, t0 + (j+1) dt),
// stored eps2[comp * n_b + j].  eps2 null: off.
// 1/d for d > 0 by Newton's iteration for the reciprocal, y <- y + y (1 - d y), two steps
// from an FP32 seed (rcp.approx of d rounded to FP32).  The seed's relative error e0 (below
// 2^-22: the FP32 rounding of d plus the approximate reciprocal) becomes e0^2 after one step
// and e0^4 < 2^-88 after two, so the result differs from 1/d by the rounding of the last
// FMA: at most one FP64 ulp (the GPU unit test measures the largest difference from the
// correctly rounded 1.0 / d over random and edge values).  d outside [2^-100, 2^101)
// (exponent bits) takes the plain division.
__device__ __forceinline__ double rcp_pos(double d) {
    const int ex = (__double2hiint(d) >> 20) & 0x7ff;
    if (ex < 1023 - 100 || ex > 1023 + 100) return 1.0 / d;
    float y0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(__double2float_rn(d)));
    double y = (double)y0;
    y = fma(y, fma(-d, y, 1.0), y);
    y = fma(y, fma(-d, y, 1.0), y);
    return y;
}

struct AttNoise {
    const double* eps2 = nullptr;
    int64_t t0 = 0, dt = 1;
    int32_t n_b = 0;
};
__device__ __forceinline__ int an_comp(uint32_t m) { return meta_kind(m) == 0 ? 0 : 1 + (int)meta_fov(m); }
__device__ __forceinline__ int64_t an_index(const AttNoise& a, int64_t t, uint32_t m) {
    return (int64_t)an_comp(m) * a.n_b + (t - a.t0) / a.dt;   // t >= t0 (checked when switched on)
}

__device__ __forceinline__ int64_t knot_at(const DevGeo& G, int64_t k) {
    int64_t K = (int64_t)G.n_coef - 3;
    int64_t j = k - 3;
    j = j < 0 ? 0 : (j > K ? K : j);
    return G.knot0_ns + j * G.knot_dt_ns;
}

__device__ __forceinline__ int left_index(const DevGeo& G, int64_t t) {
    int64_t rel = t - G.knot0_ns;
    if (rel < 0) return 3;
    int64_t l = 3 + rel / G.knot_dt_ns;
    if (l > G.n_coef - 1) l = G.n_coef - 1;
    return (int)l;
}

// The four non-zero cubic B-splines B_{l-3..l}(t) (App. B): closed form where the six
// knots around the interval are regular, Algorithm B.1 near the multiple end knots.
__device__ __forceinline__ void bspline4(const DevGeo& G, int64_t t, int l, double b[4]) {
    if (l >= 5 && l <= G.n_coef - 3) {
        double u = (double)(t - knot_at(G, l)) * G.inv_knot_dt;
        double v = 1.0 - u;
        double u2 = u * u, u3 = u2 * u;
        b[0] = v * v * v * (1.0 / 6.0);
        b[1] = (3.0 * u3 - 6.0 * u2 + 4.0) * (1.0 / 6.0);
        b[2] = (-3.0 * u3 + 3.0 * u2 + 3.0 * u + 1.0) * (1.0 / 6.0);
        b[3] = u3 * (1.0 / 6.0);
        return;
    }
    double R[3], L[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        R[i] = (double)(knot_at(G, l + i + 1) - t);
        L[i] = (double)(t - knot_at(G, l - i));
    }
    b[0] = 1.0; b[1] = b[2] = b[3] = 0.0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j <= i; j++) {
            double u = b[j] / (R[j] + L[i - j]);
            b[j] = s + R[j] * u;
            s = L[i - j] * u;
        }
        b[i + 1] = s;
    }
}

// quaternion product ab, Eq. quatmult
__device__ __forceinline__ void qmul(const double* a, const double* b, double* c) {
    c[0] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    c[1] = -a[0] * b[2] + a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    c[2] = a[0] * b[1] - a[1] * b[0] + a[2] * b[3] + a[3] * b[2];
    c[3] = -a[0] * b[0] - a[1] * b[1] - a[2] * b[2] + a[3] * b[3];
}

// |s|^2 times the attitude matrix of the quaternion s / |s| (Eq. quat2mat in homogeneous
// form; rows: SRS axes in the ICRS).  The field angles are invariant to the scale.
__device__ __forceinline__ void quat2mat_h(const double* q, double m[9]) {
    const double x = q[0], y = q[1], z = q[2], w = q[3];
    const double xx = x * x, yy = y * y, zz = z * z, ww = w * w;
    m[0] = ww + xx - yy - zz; m[1] = 2.0 * (x * y + z * w); m[2] = 2.0 * (x * z - y * w);
    m[3] = 2.0 * (x * y - z * w); m[4] = ww - xx + yy - zz; m[5] = 2.0 * (y * z + x * w);
    m[6] = 2.0 * (x * z + y * w); m[7] = 2.0 * (y * z - x * w); m[8] = ww - xx - yy + zz;
}

// atan2(y, x) for a direction within 0.02 rad of the x axis by the Taylor series of arctan
// (the remainder after the t^9 term is below 2e-20 rad; t = y / x by the Newton reciprocal
// of x > 0, within an ulp of the quotient); atan2 elsewhere.
__device__ __forceinline__ double atan2_small(double y, double x) {
    if (x > 0.0 && fabs(y) <= 0.02 * x) {
        const double t = y * rcp_pos(x), t2 = t * t;
        return t * (1.0 + t2 * (-1.0 / 3.0 + t2 * (1.0 / 5.0 + t2 * (-1.0 / 7.0 + t2 * (1.0 / 9.0)))));
    }
    return atan2(y, x);
}

// sin and cos of the orbital longitude L(t) = L0 + 2 pi (t / 1e9) / year: from the table point
// at or before t by the angle-addition formulas, with sin and cos of the offset d < 8.8e-4 rad
// by their Taylor series to d^5 and d^6 (remainders below 1e-25); sincospi of L / pi where
// there is no table or t lies outside it.
__device__ __forceinline__ void orbit_sincos(const DevGeo& G, int64_t t, double& sL, double& cL) {
    if (G.orb_tab) {
        const int64_t rel = t - G.orb_t0;
        const int64_t j = rel >> kOrbShift;
        if (rel >= 0 && j < G.orb_n) {
            const double d = (double)(rel - (j << kOrbShift)) * G.orb_rad_per_ns;
            const double d2 = d * d;
            const double sd = d * (1.0 + d2 * (-1.0 / 6.0 + d2 * (1.0 / 120.0)));
            const double cd = 1.0 + d2 * (-0.5 + d2 * (1.0 / 24.0 + d2 * (-1.0 / 720.0)));
            const double s0 = G.orb_tab[2 * j], c0 = G.orb_tab[2 * j + 1];
            sL = fma(s0, cd, c0 * sd);
            cL = fma(c0, cd, -(s0 * sd));
            return;
        }
    }
    sincospi(G.orb_L0_pi + 2.0 * ((double)t * 1e-9) * G.inv_year_s, &sL, &cL);
}

// Per-source geometry: normal triad (Eq. normal-triad) and the parameters.
struct SrcGeo {
    double p[3], q[3], r[3];
    double par, pma, pmd, cosd;
    float pf[3], qf[3];   // p, q rounded to FP32 (the mixed form's FP32 partials)
};

__device__ __forceinline__ void source_geo(const double* s5, SrcGeo& S) {
    double sa, ca, sd, cd;
    sincos(s5[0], &sa, &ca);
    sincos(s5[1], &sd, &cd);
    S.p[0] = -sa; S.p[1] = ca; S.p[2] = 0.0;
    S.q[0] = -sd * ca; S.q[1] = -sd * sa; S.q[2] = cd;
    S.r[0] = cd * ca; S.r[1] = cd * sa; S.r[2] = sd;
    S.par = s5[2]; S.pma = s5[3]; S.pmd = s5[4];
    S.cosd = cd;
}

struct ObsOut {
    double R;       // residual
    double A[5];    // -dR/ds'
    double g[4];    // dR/dq / ||s||
    double tau;     // proper-motion time (years), A[3] = A[0] tau, A[4] = A[1] tau
    float Af[3];    // FP32 partials (kPartials == 2): A[0..2], g, tau
    float gf[4];
    float tauf;
};

__device__ __forceinline__ float dot3f(const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ __forceinline__ void qmulf(const float* a, const float* b, float* c) {
    c[0] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    c[1] = -a[0] * b[2] + a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    c[2] = a[0] * b[1] - a[1] * b[0] + a[2] * b[3] + a[3] * b[2];
    c[3] = -a[0] * b[0] - a[1] * b[1] - a[2] * b[2] + a[3] * b[3];
}

// Device arrays of the full calibration model's C block (k_calgen.cu).
struct CalGenWork {
    const uint32_t* perm;      // observations by (AL cell, bin), then by AC group
    const int64_t* off;        // n_cells + n_groups + 1 offsets into perm
    double* V;                 // AL cell: 6 x n_bin, V_j = U_j'^-1 B_j
    double* E;                 // AL cell: n_bin, sum W per bin
    double* bs;                // AL cell: n_bin, -sum W R per bin
    double* cw;                // AL cell: 18 = w_j (6) and the two upper 3x3 factors (6 + 6)
    double* S;                 // AL group: n_bin x n_bin reduced normals
    double* r;                 // AL group: n_bin reduced right-hand side
    double* Et;                // AL group: n_bin, sum of E over the group's cells
    double* H;                 // AL group: 3 x n_bin Householder vectors of the cc2 columns
    double* v;                 // AL group: n_bin small-scale update
    int* idx;                  // AL group: n_bin observed bins (compacted)
    const double* cc2w;        // 3 x n_bin: sum of L*_r over the columns of each bin
    double* d;                 // n_cal update
    int* rd;                   // n_cells + 2 n_groups rank defects (cells, AL groups, AC groups)
};

// Short interval j and long interval k of an observation time, the AL/AC group (n, g, k) and
// the shifted Legendre factors L*_1, L*_2 of x = (mu - 13.5) / n_col (Eq. etazeta).
struct CalPos {
    int64_t grp;
    int jj;        // j within its long interval
    int bin;       // small-scale bin of the nearest column (AL)
    double L1, L2;
};
__device__ __forceinline__ CalPos cal_position(const CalGen& C, int64_t t, uint32_t meta, double mu) {
    CalPos p;
    const int64_t rel = t - C.t0;
    int64_t j = rel < 0 ? 0 : rel / C.dt;
    if (j > C.n_j - 1) j = C.n_j - 1;
    const int k = (int)(j / C.j_per_k);
    p.jj = (int)(j - (int64_t)k * C.j_per_k);
    p.grp = ((int64_t)meta_ccd(meta) * C.n_gate + meta_gate(meta)) * C.n_k + k;
    const double x = (mu - 13.5) * C.inv_ncol;
    p.L1 = 2.0 * x - 1.0;
    p.L2 = 6.0 * x * x - 6.0 * x + 1.0;
    int m = (int)floor(mu + 0.5) - 14;
    m = m < 0 ? 0 : (m > AGIS_N_COL - 1 ? AGIS_N_COL - 1 : m);
    p.bin = m / C.col_bin;
    return p;
}

// The calibration term of an observation line: the r = 0 offset of its packed index, or the
// full model's sum of Legendre-weighted large-scale terms and the small-scale term.
__device__ __forceinline__ double cal_term(const DevGeo& G, int64_t t, uint32_t meta, double mu,
                                           const double* __restrict__ cal) {
    if (!G.cg.on) return cal[meta_cal(meta)];
    const CalGen& C = G.cg;
    const CalPos p = cal_position(C, t, meta, mu);
    const int f = (int)meta_fov(meta);
    if (meta_kind(meta) == 0) {
        const double* c = cal + p.grp * C.al_size + p.jj * 6 + f * 3;
        return c[0] + p.L1 * c[1] + p.L2 * c[2] + cal[p.grp * C.al_size + 6 * C.j_per_k + p.bin];
    }
    const double* c = cal + C.n_al + p.grp * 6 + f * 3;
    return c[0] + p.L1 * c[1] + p.L2 * c[2];
}

// Residual and partial derivatives of one observation (FP64).
//   proper direction: Eqs. astro-standard, roemer, classAberr
//   field angles: Eqs. srsprop, srsprop1, srspropeta; lines: Eqs. etazeta0, etazeta (r = 0)
//   source partials: Eqs. srspqr, srsprop1diffsol, ubardiff, duds (evaluated in the ICRS by
//   turning m and n back with the attitude matrix)
//   attitude partials: Eq. dfadq divided by ||s|| (normalisation of Eq. qspline)
// The field angles depend on the direction only, so neither the aberrated direction nor the
// attitude quaternion is normalised: the rotation uses |s|^2 R(s/|s|), and the along-scan
// angle is measured from the field centre after turning by -f Gamma / 2.
// kPartials: 0 residual only, 1 FP64 partials, 2 FP32 partials (Af, gf, tauf)
template <int kPartials>
__device__ __forceinline__ void observe(const DevGeo& G, const SrcGeo& S, int64_t t, uint32_t meta, double mu,
                                        const double* __restrict__ att, const double* __restrict__ cal,
                                        ObsOut& o) {
    // ephemeris: circular orbit, ICRS components (AU, AU/s in units of c)
    double sL, cL;
    orbit_sincos(G, t, sL, cL);
    const double b[3] = {cL, G.cos_obl * sL, G.sin_obl * sL};
    const double vc[3] = {-G.vk * sL, G.vk * G.cos_obl * cL, G.vk * G.sin_obl * cL};
    // Roemer delay and proper-motion time
    const double rb = dot3(S.r, b);
    const double tau = ((double)(t - G.t_ep_ns) * 1e-9 + rb * G.au_light_s) * G.inv_year_s;
    double ub[3];
#pragma unroll
    for (int i = 0; i < 3; i++) ub[i] = S.r[i] + tau * (S.p[i] * S.pma + S.q[i] * S.pmd) - S.par * b[i];
    const double inb = rsqrt(dot3(ub, ub));
    ub[0] *= inb; ub[1] *= inb; ub[2] *= inb;
    const double u[3] = {ub[0] + vc[0], ub[1] + vc[1], ub[2] + vc[2]};
    // attitude
    const int l = left_index(G, t);
    double B[4];
    bspline4(G, t, l, B);
    const double* a = att + 4 * (int64_t)(l - 3);
    double s[4];
#pragma unroll
    for (int c = 0; c < 4; c++) s[c] = B[0] * a[c] + B[1] * a[4 + c] + B[2] * a[8 + c] + B[3] * a[12 + c];
    double Am[9];
    quat2mat_h(s, Am);
    const double us[3] = {dot3(Am, u), dot3(Am + 3, u), dot3(Am + 6, u)};
    const uint32_t fov = meta_fov(meta), kind = meta_kind(meta), ccd = meta_ccd(meta);
    const double f = fov == 0 ? 1.0 : -1.0;
    const double c_k = cal_term(G, t, meta, mu, cal);
    const double rho2 = us[0] * us[0] + us[1] * us[1];
    const double irho = rsqrt(rho2);
    const double zeta = atan2_small(us[2], rho2 * irho);
    if (kind == 0) {
        // eta = phi - f Gamma/2 from the direction turned by -f Gamma/2 about the z axis
        const double c0 = G.cos_gh * us[0] + f * G.sin_gh * us[1];
        const double c1 = G.cos_gh * us[1] - f * G.sin_gh * us[0];
        o.R = (G.eta0[ccd] + c_k) - atan2_small(c1, c0);
    } else {
        const double zeta0 = -(G.x_fpa[ccd] - (mu - G.mu_c) * G.p_ac - G.x_centre[fov]) / G.F;
        o.R = (zeta0 + c_k) - zeta;
    }
    if (kPartials == 0) return;
    if (kPartials == 2) {
        // FP32 partials from the FP64 intermediates rounded once (the mixed form keeps its
        // partials in FP32; their rounding changes the rate of the iteration, not its fixed
        // point).  Same equations as the FP64 branch below; r = p x q for the normal triad.
        const float usf[3] = {(float)us[0], (float)us[1], (float)us[2]};
        const float sf[4] = {(float)s[0], (float)s[1], (float)s[2], (float)s[3]};
        const float r2 = usf[0] * usf[0] + usf[1] * usf[1];
        const float ir = rsqrtf(r2);
        const float cphi = usf[0] * ir, sphi = usf[1] * ir;
        const float in = rsqrtf(r2 + usf[2] * usf[2]);
        const float czeta = r2 * ir * in, szeta = usf[2] * in;
        const bool al = kind == 0;
        // e = m (AL) or n (AC), and w = the other one (selects, not pointers: registers)
        const float e[3] = {al ? -sphi : -szeta * cphi, al ? cphi : -szeta * sphi, al ? 0.0f : czeta};
        const float w3[3] = {al ? -szeta * cphi : -sphi, al ? -szeta * sphi : cphi, al ? czeta : 0.0f};
        const float x = sf[0], y = sf[1], z = sf[2], w = sf[3];
        const float xx = x * x, yy = y * y, zz = z * z, ww = w * w;
        const float Af[9] = {ww + xx - yy - zz,      2.0f * (x * y + z * w), 2.0f * (x * z - y * w),
                             2.0f * (x * y - z * w), ww - xx + yy - zz,      2.0f * (y * z + x * w),
                             2.0f * (x * z + y * w), 2.0f * (y * z - x * w), ww - xx - yy + zz};
        const float ins2 = 1.0f / (xx + yy + zz + ww);
        const float ec[3] = {(Af[0] * e[0] + Af[3] * e[1] + Af[6] * e[2]) * ins2,
                             (Af[1] * e[0] + Af[4] * e[1] + Af[7] * e[2]) * ins2,
                             (Af[2] * e[0] + Af[5] * e[1] + Af[8] * e[2]) * ins2};
        const float sLf = (float)sL, cLf = (float)cL;
        const float co = (float)G.cos_obl, so = (float)G.sin_obl, vk = (float)G.vk;
        const float bf[3] = {cLf, co * sLf, so * sLf};
        const float vcf[3] = {-vk * sLf, vk * co * cLf, vk * so * cLf};
        const float ubf[3] = {(float)ub[0], (float)ub[1], (float)ub[2]};
        const float* pf = S.pf;
        const float* qf = S.qf;
        const float rf[3] = {pf[1] * qf[2] - pf[2] * qf[1], pf[2] * qf[0] - pf[0] * qf[2],
                             pf[0] * qf[1] - pf[1] * qf[0]};
        const float rbf = dot3f(rf, bf);
        const float ubv = dot3f(ubf, vcf);
        const float eub = dot3f(ec, ubf);
        const float dpar[3] = {-(bf[0] - rf[0] * rbf), -(bf[1] - rf[1] * rbf), -(bf[2] - rf[2] * rbf)};
        const float secz = 1.0f / czeta;
        const float sc = (kind == 0) ? secz : 1.0f;
        o.Af[0] = ((1.0f - ubv) * dot3f(ec, pf) - eub * dot3f(vcf, pf)) * sc;
        o.Af[1] = ((1.0f - ubv) * dot3f(ec, qf) - eub * dot3f(vcf, qf)) * sc;
        o.Af[2] = ((1.0f - ubv) * dot3f(ec, dpar) - eub * dot3f(vcf, dpar)) * sc;
        o.tauf = (float)tau;
        const float v4[4] = {w3[0], w3[1], w3[2], 0.0f};
        float gq[4];
        qmulf(sf, v4, gq);
        const float k2 = ((kind == 0) ? 2.0f * secz : -2.0f) * ins2;
        o.gf[0] = gq[0] * k2; o.gf[1] = gq[1] * k2; o.gf[2] = gq[2] * k2; o.gf[3] = gq[3] * k2;
        return;
    }
    // m, n in the SRS (Eq. srspqr)
    const double cphi = us[0] * irho, sphi = us[1] * irho;
    double czeta, szeta;
    if (fabs(zeta) <= 0.02) {
        const double z2 = zeta * zeta;
        czeta = 1.0 + z2 * (-0.5 + z2 * (1.0 / 24.0 + z2 * (-1.0 / 720.0)));
        szeta = zeta * (1.0 + z2 * (-1.0 / 6.0 + z2 * (1.0 / 120.0 + z2 * (-1.0 / 5040.0))));
    } else {
        const double in = rsqrt(rho2 + us[2] * us[2]);
        czeta = rho2 * irho * in;
        szeta = us[2] * in;
    }
    const double ms[3] = {-sphi, cphi, 0.0};
    const double nsv[3] = {-szeta * cphi, -szeta * sphi, czeta};
    // back to the ICRS: x_C = R' x_S with R = Am / |s|^2
    const double ins2 = rcp_pos(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3]);
    const double* e = (kind == 0) ? ms : nsv;
    const double ec[3] = {(Am[0] * e[0] + Am[3] * e[1] + Am[6] * e[2]) * ins2,
                          (Am[1] * e[0] + Am[4] * e[1] + Am[7] * e[2]) * ins2,
                          (Am[2] * e[0] + Am[5] * e[1] + Am[8] * e[2]) * ins2};
    // du/ds' = [(1 - ub'v/c) I - ub v'/c] dub/ds'  (Eq. duds); e'du = (1-ubv) e'x - (e'ub)(v'x)
    const double ubv = dot3(ub, vc);
    const double eub = dot3(ec, ub);
    const double dpar[3] = {-(b[0] - S.r[0] * rb), -(b[1] - S.r[1] * rb), -(b[2] - S.r[2] * rb)};
    const double secz = rcp_pos(czeta);
    const double sc = (kind == 0) ? secz : 1.0;
    const double Ap = ((1.0 - ubv) * dot3(ec, S.p) - eub * dot3(vc, S.p)) * sc;
    const double Aq = ((1.0 - ubv) * dot3(ec, S.q) - eub * dot3(vc, S.q)) * sc;
    const double Aw = ((1.0 - ubv) * dot3(ec, dpar) - eub * dot3(vc, dpar)) * sc;
    o.A[0] = Ap; o.A[1] = Aq; o.A[2] = Aw; o.A[3] = Ap * tau; o.A[4] = Aq * tau;
    o.tau = tau;
    // attitude: dR_AL/dq = 2 sec(zeta) q {n,0};  dR_AC/dq = -2 q {m,0}; divided by ||s||, with
    // q = s / ||s||: g = k qmul(s, {e,0}) / ||s||^2
    double v4[4], gq[4];
    const double* w3 = (kind == 0) ? nsv : ms;
    v4[0] = w3[0]; v4[1] = w3[1]; v4[2] = w3[2]; v4[3] = 0.0;
    qmul(s, v4, gq);
    const double k2 = ((kind == 0) ? 2.0 * secz : -2.0) * ins2;
    o.g[0] = gq[0] * k2; o.g[1] = gq[1] * k2; o.g[2] = gq[2] * k2; o.g[3] = gq[3] * k2;
}

// ---------------------------------------------------------------------------------------
// 5x5 robust Cholesky (Algorithms C.1-C.3) in registers; N upper-packed row-major:
// (0,0) (0,1) .. (0,4) (1,1) .. (1,4) (2,2) .. (4,4)
// ---------------------------------------------------------------------------------------
__host__ __device__ constexpr int up5(int i, int j) { return i * 5 - i * (i - 1) / 2 + (j - i); }

// U holds the 15 upper-packed entries of the factor, then the reciprocals of its 5 diagonal
// entries (0 where the pivot test failed): each pivot takes one reciprocal square root, and the
// off-diagonal entries and both substitutions multiply by the stored reciprocals instead of
// dividing (equal to the divisions up to rounding).
constexpr int kU5 = 20;

__device__ __forceinline__ int chol5(const double* N, double* U, double tol) {
    int d = 0;
#pragma unroll
    for (int j = 0; j < 5; j++) {
#pragma unroll
        for (int i = 0; i <= j; i++) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < i; k++) s += U[up5(k, i)] * U[up5(k, j)];
            if (i < j) {
                const double ri = U[15 + i];
                U[up5(i, j)] = ri > 0.0 ? (N[up5(i, j)] - s) * ri : 0.0;
            } else {
                double v = N[up5(j, j)] - s;
                if (v > tol * N[up5(j, j)]) {
                    const double r = rsqrt(v);
                    U[up5(j, j)] = v * r;
                    U[15 + j] = r;
                } else {
                    U[up5(j, j)] = 0.0;
                    U[15 + j] = 0.0;
                    d++;
                }
            }
        }
    }
    return d;
}

__device__ __forceinline__ void chol5_solve(const double* U, const double* b, double* x) {
    double y[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        double s = b[i];
#pragma unroll
        for (int k = 0; k < i; k++) s -= U[up5(k, i)] * y[k];
        y[i] = U[15 + i] > 0.0 ? s * U[15 + i] : 0.0;
    }
#pragma unroll
    for (int i = 4; i >= 0; i--) {
        double s = y[i];
#pragma unroll
        for (int k = i + 1; k < 5; k++) s -= U[up5(i, k)] * x[k];
        x[i] = U[15 + i] > 0.0 ? s * U[15 + i] : 0.0;
    }
}

// ---- per-class sums: when every AL observation of a source has one sigma and every AC
// observation another, N(y) = sum_c AA_c / (s2_c + y), b(y) = sum_c Ah_c / (s2_c + y) and
// Q(y) = sum_c [hh_c - 2 d'Ah_c + d'AA_c d] / (s2_c + y): one pass over the observations per
// weight round serves every excess-noise step (exact algebra; only the rounding differs).
struct ClassSums {
    double AA[2][15];
    double Ah[2][5];
    double hh[2];
};

// solve at excess variance y from the class sums; returns Q(y) and S2 = sum num_c/(s2_c+y)^2
static __device__ __noinline__ void class_solve(const ClassSums& S, const double* s2c, double y, double tol_piv,
                                            double* U, double* d, int& rd, double& Q, double& S2) {
    const double i0 = 1.0 / (s2c[0] + y), i1 = 1.0 / (s2c[1] + y);
    double N[15], b[5];
#pragma unroll
    for (int i = 0; i < 15; i++) N[i] = S.AA[0][i] * i0 + S.AA[1][i] * i1;
#pragma unroll
    for (int i = 0; i < 5; i++) b[i] = S.Ah[0][i] * i0 + S.Ah[1][i] * i1;
    rd = chol5(N, U, tol_piv);
    chol5_solve(U, b, d);
    double num[2];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        double dMd = 0.0, db = 0.0;
#pragma unroll
        for (int a = 0; a < 5; a++) {
            db += d[a] * S.Ah[c][a];
            dMd += S.AA[c][up5(a, a)] * d[a] * d[a];
#pragma unroll
            for (int k = a + 1; k < 5; k++) dMd += 2.0 * S.AA[c][up5(a, k)] * d[a] * d[k];
        }
        num[c] = S.hh[c] - 2.0 * db + dMd;
    }
    Q = num[0] * i0 + num[1] * i1;
    S2 = num[0] * i0 * i0 + num[1] * i1 * i1;
}

}  // namespace agis
