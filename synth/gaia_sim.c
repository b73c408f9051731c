/*
 * gaia_sim.c -- seeded synthetic Gaia-like sky, scanning law and observation
 * generator.  This is the "truth world" that both the FP64 oracle and the GPU
 * library consume: it plays the role that the Gaia System Simulator plays for
 * the demonstration solution of Lindegren et al. (2012), Sect. 7.2.
 *
 * It simulates the instrument; it does not contain the astrometric solution
 * (no residual weighting, partial derivatives, normal equations or solvers).
 * Its geometry is written with rotation matrices and the Cox-de Boor
 * recursion, independently of the oracle and of the CUDA kernels.
 *
 * Conventions (all stated in the accompanying Python wrapper as well):
 *   time      int64 nanoseconds since mission start (TCB); year = 365.25 d
 *   angles    radians; proper motions rad/yr; parallax rad
 *   ephemeris circular 1-AU orbit in the ecliptic, rotated to ICRS by the
 *             J2000 obliquity (auxiliary data h of Sect. 3.2)
 *   attitude  quaternion {x,y,z,w} of the frame rotation ICRS -> SRS
 *             (Eq. att-q), represented by a cubic B-spline (Eq. qspline)
 *             with 4-fold end knots (App. B.3)
 *   focal plane 7 AC rows x 9 AL strips minus (row 3, strip 8) = 62 AF CCDs
 *
 * Build: cc -O2 -fopenmp -shared -fPIC gaia_sim.c -o libgaia_sim.so -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SIM_PI 3.14159265358979323846
#define SIM_ARCSEC (SIM_PI / 648000.0)
#define SIM_MAS (SIM_ARCSEC * 1e-3)
#define SIM_UAS (SIM_ARCSEC * 1e-6)
#define SIM_DAY_S 86400.0
#define SIM_YEAR_S (365.25 * 86400.0)
#define SIM_NROW 7
#define SIM_NSTRIP 9
#define SIM_NCCD 62
#define SIM_MISSING_ROW 3
#define SIM_MISSING_STRIP 8

/* ------------------------------------------------------------------------ */
/* configuration and geometry                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n_src;
    int64_t span_ns;          /* mission span */
    int64_t knot_dt_ns;       /* attitude knot interval */
    int64_t cal_dt_ns;        /* calibration interval (1 day) */
    uint64_t seed;
    double sigma_al;          /* rad, used when mag_dependent == 0 */
    double sigma_ac;          /* rad */
    int32_t mag_dependent;    /* 1: G ~ U(12,18), sigma_AL = 50 uas 10^((G-12)/6) */
    int32_t noise_free;       /* 1: no Gaussian noise and no outliers */
    double outlier_frac;      /* fraction of components with an outlier */
    double outlier_nsigma;    /* outlier offset in units of sigma */
    double att_pert_rms;      /* rad, total RMS of the smooth attitude perturbation */
    double cal_al_rms;        /* rad, per (f, ccd, day) AL offset */
    double cal_ac_rms;        /* rad, per (f, row, day) AC offset */
    double start_src_err;     /* rad, starting error of alpha*, delta */
    double start_att_err;     /* rad, starting error per attitude coefficient and axis */
    int32_t min_transits;     /* keep sources with at least this many field transits (0: all) */
    int32_t max_transits;     /* and at most this many (0: no limit) */
    double dec_min, dec_max;  /* declination range for sources (rad) */
    double ra_min, ra_max;    /* right ascension range (rad) */
    double parallax_mean;     /* rad */
    double pm_sigma;          /* rad/yr */
    int32_t n_threads;        /* 0: default */
    /* full geometric calibration of Eq. etazeta (cal_generic = 1); otherwise the per-day
     * offsets above */
    int32_t cal_generic;
    int32_t n_gate;           /* gates 0 .. n_gate - 1 */
    int32_t cal_j_per_k;      /* days (short intervals) per long interval */
    int32_t cal_col_bin;      /* pixel columns per small-scale parameter */
    double gate_g0;           /* observations of sources brighter than this magnitude are gated */
    double gate_step;         /* magnitudes per gate */
    double gate_fuzz;         /* rms of the per-observation jitter of the gate threshold (mag) */
    double cal_l12_rms;       /* rad, the r = 1, 2 large-scale AL and AC terms */
    double cal_small_rms;     /* rad, the small-scale AL terms */
} sim_config;

typedef struct {
    /* instrument */
    double gamma_c;           /* basic angle */
    double focal_length;      /* m */
    double p_ac;              /* m */
    double mu_c;              /* AC pixel coordinate of CCD centre */
    double eta0[SIM_NCCD];    /* nominal AL line per AF CCD, Eq. etazeta0 */
    double x_fpa[SIM_NCCD];   /* X_FPA of the CCD centre (m) */
    double x_centre[2];       /* X_FPA^centre[f] for fov index 0 (f=+1) and 1 (f=-1) */
    int32_t ccd_row[SIM_NCCD];
    int32_t ccd_strip[SIM_NCCD];
    /* scanning law */
    double xi;                /* solar aspect angle */
    double spin_rate;         /* rad/s */
    double prec_rate;         /* rad/s */
    double spin0, prec0;      /* phases at t=0 */
    /* ephemeris */
    double orb_L0;            /* ecliptic longitude of the barycentre of Earth+Gaia at t=0 */
    double obliquity;
    double cos_obl, sin_obl;
    double au_light_s;        /* A_u / c in seconds */
    /* epochs */
    int64_t t_ep_ns;
    int64_t t_fr_ns;
    /* knots */
    int64_t knot0_ns;         /* tau_{M-1} = t_beg */
    int64_t n_coef;           /* N */
    int64_t n_cal_days;
} sim_geometry;

/* ------------------------------------------------------------------------ */
/* random numbers: splitmix64-seeded xoshiro256** per stream                 */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static void rng_seed(rng_t *r, uint64_t seed, uint64_t stream, uint64_t sub) {
    uint64_t x = seed * 0x2545F4914F6CDD1DULL ^ (stream + 0x632BE59BD9B4E019ULL) * 0x9E3779B97F4A7C15ULL
                 ^ (sub + 1) * 0xD1B54A32D192ED03ULL;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}
static inline uint64_t rotl(const uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t rng_next(rng_t *r) {
    const uint64_t result = rotl(r->s[1] * 5, 7) * 9;
    const uint64_t t = r->s[1] << 17;
    r->s[2] ^= r->s[0]; r->s[3] ^= r->s[1]; r->s[1] ^= r->s[2]; r->s[0] ^= r->s[3];
    r->s[2] ^= t; r->s[3] = rotl(r->s[3], 45);
    return result;
}
static double rng_uniform(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static double rng_gauss(rng_t *r) {
    double u1 = rng_uniform(r), u2 = rng_uniform(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * SIM_PI * u2);
}

/* ------------------------------------------------------------------------ */
/* small vector / matrix helpers                                             */
/* ------------------------------------------------------------------------ */
static inline void v_cross(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double v_dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void v_unit(double a[3]) {
    double n = sqrt(v_dot(a, a));
    a[0] /= n; a[1] /= n; a[2] /= n;
}
/* ecliptic -> equatorial (ICRS) by the obliquity */
static inline void ecl2eq(double ce, double se, const double e[3], double q[3]) {
    q[0] = e[0];
    q[1] = ce * e[1] - se * e[2];
    q[2] = se * e[1] + ce * e[2];
}

/* rows of the matrix are the SRS axes expressed in ICRS -> quaternion of the
 * frame rotation ICRS -> SRS (Shepperd's largest-component method). */
static void mat2quat(const double m[3][3], double q[4]) {
    double tr = m[0][0] + m[1][1] + m[2][2];
    double c[4] = {1.0 + 2.0 * m[0][0] - tr, 1.0 + 2.0 * m[1][1] - tr, 1.0 + 2.0 * m[2][2] - tr, 1.0 + tr};
    int k = 0;
    for (int i = 1; i < 4; i++) if (c[i] > c[k]) k = i;
    double s = 0.5 * sqrt(c[k]);
    double f = 0.25 / s;
    /* m = [[1-2(y2+z2), 2(xy+zw), 2(xz-yw)], [2(xy-zw), 1-2(x2+z2), 2(yz+xw)], [2(xz+yw), 2(yz-xw), 1-2(x2+y2)]] */
    double x, y, z, w;
    if (k == 0) { x = s; y = (m[0][1] + m[1][0]) * f; z = (m[0][2] + m[2][0]) * f; w = (m[1][2] - m[2][1]) * f; }
    else if (k == 1) { y = s; x = (m[0][1] + m[1][0]) * f; z = (m[1][2] + m[2][1]) * f; w = (m[2][0] - m[0][2]) * f; }
    else if (k == 2) { z = s; x = (m[0][2] + m[2][0]) * f; y = (m[1][2] + m[2][1]) * f; w = (m[0][1] - m[1][0]) * f; }
    else { w = s; x = (m[1][2] - m[2][1]) * f; y = (m[2][0] - m[0][2]) * f; z = (m[0][1] - m[1][0]) * f; }
    q[0] = x; q[1] = y; q[2] = z; q[3] = w;
}
/* quaternion -> matrix with rows = SRS axes in ICRS */
static void quat2mat(const double q[4], double m[3][3]) {
    double x = q[0], y = q[1], z = q[2], w = q[3];
    m[0][0] = 1 - 2 * (y * y + z * z); m[0][1] = 2 * (x * y + z * w); m[0][2] = 2 * (x * z - y * w);
    m[1][0] = 2 * (x * y - z * w); m[1][1] = 1 - 2 * (x * x + z * z); m[1][2] = 2 * (y * z + x * w);
    m[2][0] = 2 * (x * z + y * w); m[2][1] = 2 * (y * z - x * w); m[2][2] = 1 - 2 * (x * x + y * y);
}
static void m_mul(const double a[3][3], const double b[3][3], double c[3][3]) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) c[i][j] = a[i][0] * b[0][j] + a[i][1] * b[1][j] + a[i][2] * b[2][j];
}
/* rotation matrix of a small rotation vector phi (frame rotation by the angle |phi| about phi) */
static void rotvec_mat(const double phi[3], double m[3][3]) {
    double th = sqrt(v_dot(phi, phi));
    double k[3] = {0, 0, 1};
    if (th > 0) { k[0] = phi[0] / th; k[1] = phi[1] / th; k[2] = phi[2] / th; }
    double c = cos(th), s = sin(th), C = 1 - c;
    /* frame rotation: coordinates in the new frame = R' * old, i.e. rows = new axes in old frame */
    double R[3][3] = {{c + k[0] * k[0] * C, k[0] * k[1] * C - k[2] * s, k[0] * k[2] * C + k[1] * s},
                      {k[1] * k[0] * C + k[2] * s, c + k[1] * k[1] * C, k[1] * k[2] * C - k[0] * s},
                      {k[2] * k[0] * C - k[1] * s, k[2] * k[1] * C + k[0] * s, c + k[2] * k[2] * C}};
    /* rows of the frame-rotation matrix = new axes = R applied to old axes -> transpose */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) m[i][j] = R[j][i];
}

/* ------------------------------------------------------------------------ */
/* geometry set-up                                                           */
/* ------------------------------------------------------------------------ */
static void setup_geometry(const sim_config *c, sim_geometry *g) {
    memset(g, 0, sizeof(*g));
    g->gamma_c = 106.5 * SIM_PI / 180.0;
    g->focal_length = 35.0;
    g->p_ac = 30e-6;
    g->mu_c = 996.5;
    const double strip_pitch = 49.4e-3; /* m, ~291 arcsec at F = 35 m */
    const double row_pitch = 60.2e-3;   /* m, ~0.0986 deg */
    int n = 0;
    for (int r = 0; r < SIM_NROW; r++)
        for (int s = 0; s < SIM_NSTRIP; s++) {
            if (r == SIM_MISSING_ROW && s == SIM_MISSING_STRIP) continue;
            double y_fpa = (s - 4) * strip_pitch;
            g->eta0[n] = -y_fpa / g->focal_length;
            g->x_fpa[n] = (r - 3) * row_pitch;
            g->ccd_row[n] = r;
            g->ccd_strip[n] = s;
            n++;
        }
    g->x_centre[0] = -37.5e-3 * (+1.0);
    g->x_centre[1] = -37.5e-3 * (-1.0);
    g->xi = 45.0 * SIM_PI / 180.0;
    g->spin_rate = 60.0 * SIM_ARCSEC;
    g->prec_rate = 2.0 * SIM_PI * 5.8 / SIM_YEAR_S;
    rng_t r;
    rng_seed(&r, c->seed, 0xA77ULL, 0);
    g->spin0 = 2.0 * SIM_PI * rng_uniform(&r);
    g->prec0 = 2.0 * SIM_PI * rng_uniform(&r);
    g->orb_L0 = 2.0 * SIM_PI * rng_uniform(&r);
    g->obliquity = 23.4392911 * SIM_PI / 180.0;
    g->cos_obl = cos(g->obliquity);
    g->sin_obl = sin(g->obliquity);
    g->au_light_s = 499.004783836;
    g->t_ep_ns = c->span_ns / 2;
    g->t_fr_ns = g->t_ep_ns;
    g->knot0_ns = 0;
    g->n_coef = c->span_ns / c->knot_dt_ns + 3;
    g->n_cal_days = (c->span_ns + c->cal_dt_ns - 1) / c->cal_dt_ns;
}

/* barycentric position (AU) and velocity (AU/s) of Gaia, ICRS components */
static void ephemeris(const sim_geometry *g, double t_s, double b[3], double v[3]) {
    double L = g->orb_L0 + 2.0 * SIM_PI * (t_s / SIM_YEAR_S);
    double n = 2.0 * SIM_PI / SIM_YEAR_S;
    double be[3] = {cos(L), sin(L), 0.0};
    double ve[3] = {-n * sin(L), n * cos(L), 0.0};
    ecl2eq(g->cos_obl, g->sin_obl, be, b);
    ecl2eq(g->cos_obl, g->sin_obl, ve, v);
}

/* nominal scanning law: rows of the returned matrix are the SRS axes in ICRS */
static void nominal_axes(const sim_geometry *g, double t_s, double m[3][3]) {
    double b[3], v[3];
    double L = g->orb_L0 + 2.0 * SIM_PI * (t_s / SIM_YEAR_S);
    (void)b; (void)v;
    double lam = L + SIM_PI; /* Sun as seen from Gaia */
    double s[3] = {cos(lam), sin(lam), 0.0};
    double np[3] = {0.0, 0.0, 1.0};
    double e2[3];
    v_cross(np, s, e2);
    double nu = g->prec0 + g->prec_rate * t_s;
    double cx = cos(g->xi), sx = sin(g->xi), cn = cos(nu), sn = sin(nu);
    double z[3], a[3], bb[3], x[3], y[3];
    for (int i = 0; i < 3; i++) z[i] = cx * s[i] + sx * (cn * np[i] + sn * e2[i]);
    v_unit(z);
    v_cross(np, z, a);
    v_unit(a);
    v_cross(z, a, bb);
    double om = g->spin0 + g->spin_rate * t_s;
    double co = cos(om), so = sin(om);
    for (int i = 0; i < 3; i++) x[i] = co * a[i] + so * bb[i];
    v_cross(z, x, y);
    double xq[3], yq[3], zq[3];
    ecl2eq(g->cos_obl, g->sin_obl, x, xq);
    ecl2eq(g->cos_obl, g->sin_obl, y, yq);
    ecl2eq(g->cos_obl, g->sin_obl, z, zq);
    for (int i = 0; i < 3; i++) { m[0][i] = xq[i]; m[1][i] = yq[i]; m[2][i] = zq[i]; }
}

/* smooth attitude perturbation: per SRS axis a sum of 8 sinusoids */
#define SIM_NPERT 8
typedef struct { double amp[3][SIM_NPERT], per[3][SIM_NPERT], ph[3][SIM_NPERT]; } pert_t;

static void setup_pert(const sim_config *c, pert_t *p) {
    rng_t r;
    rng_seed(&r, c->seed, 0xBEEFULL, 0);
    double dt = (double)c->knot_dt_ns * 1e-9;
    for (int a = 0; a < 3; a++) {
        double sum2 = 0;
        for (int k = 0; k < SIM_NPERT; k++) {
            p->per[a][k] = dt * (4.0 + 44.0 * rng_uniform(&r));
            p->ph[a][k] = 2.0 * SIM_PI * rng_uniform(&r);
            p->amp[a][k] = 0.5 + rng_uniform(&r);
            sum2 += 0.5 * p->amp[a][k] * p->amp[a][k];
        }
        /* total RMS over the three axes = att_pert_rms */
        double scale = c->att_pert_rms / sqrt(3.0 * sum2);
        for (int k = 0; k < SIM_NPERT; k++) p->amp[a][k] *= scale;
    }
}

/* target attitude (nominal law followed by the perturbation as a frame rotation) */
static void target_quat(const sim_geometry *g, const pert_t *p, double t_s, double q[4]) {
    double m0[3][3], mp[3][3], m[3][3], phi[3];
    nominal_axes(g, t_s, m0);
    for (int a = 0; a < 3; a++) {
        double s = 0;
        for (int k = 0; k < SIM_NPERT; k++) s += p->amp[a][k] * sin(2.0 * SIM_PI * t_s / p->per[a][k] + p->ph[a][k]);
        phi[a] = s;
    }
    rotvec_mat(phi, mp);
    /* successive frame rotation: first nominal (ICRS -> S0), then S0 -> S1 */
    m_mul(mp, m0, m);
    mat2quat(m, q);
}

/* knot value tau_k in ns (4-fold end knots) */
static inline int64_t knot_ns(const sim_geometry *g, int64_t k, int64_t dt) {
    int64_t K = g->n_coef - 3; /* number of intervals */
    int64_t j = k - 3;
    if (j < 0) j = 0;
    if (j > K) j = K;
    return g->knot0_ns + j * dt;
}

/* Cox-de Boor recursion for the 4 non-zero cubic B-splines at t = base_ns + off_ns.
 * Returns the left index l (3 <= l <= N-1), b[0..3] = B_{l-3..l}(t). */
static int64_t bspline4(const sim_geometry *g, int64_t dt, int64_t base_ns, double off_ns, double b[4]) {
    int64_t K = g->n_coef - 3;
    /* left index from the (rounded) time */
    int64_t tr = base_ns + (int64_t)llround(off_ns);
    int64_t rel = tr - g->knot0_ns;
    int64_t l;
    if (rel < 0) l = 3;
    else {
        l = 3 + rel / dt;
        if (l > g->n_coef - 1) l = g->n_coef - 1;
    }
    (void)K;
    if (l >= 5 && l <= g->n_coef - 3) {
        /* uniform knots around the interval: closed-form cubic B-splines */
        double u = ((double)(base_ns - knot_ns(g, l, dt)) + off_ns) / (double)dt;
        double v = 1.0 - u;
        b[0] = v * v * v / 6.0;
        b[1] = (3.0 * u * u * u - 6.0 * u * u + 4.0) / 6.0;
        b[2] = (-3.0 * u * u * u + 3.0 * u * u + 3.0 * u + 1.0) / 6.0;
        b[3] = u * u * u / 6.0;
        return l;
    }
    /* x_j = t - tau_j in ns, computed from integer differences */
    double xt[8];
    for (int j = 0; j < 8; j++) {
        int64_t kk = l - 3 + j;
        xt[j] = (double)(base_ns - knot_ns(g, kk, dt)) + off_ns;
    }
    /* order-1 */
    double B[8] = {0};
    B[3] = 1.0; /* B_{l,1} = 1 on [tau_l, tau_{l+1}) */
    for (int k = 2; k <= 4; k++) {
        double nb[8] = {0};
        for (int j = 4 - k; j <= 3; j++) {
            int64_t jj = l - 3 + j;
            double v = 0;
            double d1 = (double)(knot_ns(g, jj + k - 1, dt) - knot_ns(g, jj, dt));
            double d2 = (double)(knot_ns(g, jj + k, dt) - knot_ns(g, jj + 1, dt));
            if (d1 > 0) v += xt[j] / d1 * B[j];
            if (d2 > 0) v += (-xt[j + k] / d2) * B[j + 1];
            nb[j] = v;
        }
        memcpy(B, nb, sizeof(B));
    }
    for (int j = 0; j < 4; j++) b[j] = B[j];
    return l;
}

/* ------------------------------------------------------------------------ */
/* truth attitude construction                                               */
/* ------------------------------------------------------------------------ */
static void build_attitude(const sim_config *c, const sim_geometry *g, const pert_t *p, double *coef) {
    int64_t N = g->n_coef;
    int64_t dt = c->knot_dt_ns;
    double t_end = (double)(knot_ns(g, N, dt)) * 1e-9;
    double h = dt * 1e-9;
    /* cubic quasi-interpolant: a_n = (-f(g-h) + 8 f(g) - f(g+h)) / 6 at the support centre g,
     * clamped to the spline interval near the ends */
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; n++) {
        double gc = 0.5 * ((double)knot_ns(g, n + 1, dt) + (double)knot_ns(g, n + 3, dt)) * 1e-9;
        double ts[3] = {gc - h, gc, gc + h};
        double w[3] = {-1.0 / 6.0, 8.0 / 6.0, -1.0 / 6.0};
        if (ts[0] < 0 || ts[2] > t_end) { w[0] = 0; w[1] = 1; w[2] = 0; }
        double qs[3][4];
        for (int i = 0; i < 3; i++) {
            double tt = ts[i] < 0 ? 0 : (ts[i] > t_end ? t_end : ts[i]);
            target_quat(g, p, tt, qs[i]);
        }
        /* local sign continuity with the centre sample */
        for (int i = 0; i < 3; i += 2) {
            double d = qs[i][0] * qs[1][0] + qs[i][1] * qs[1][1] + qs[i][2] * qs[1][2] + qs[i][3] * qs[1][3];
            if (d < 0) for (int k = 0; k < 4; k++) qs[i][k] = -qs[i][k];
        }
        for (int k = 0; k < 4; k++) coef[4 * n + k] = w[0] * qs[0][k] + w[1] * qs[1][k] + w[2] * qs[2][k];
    }
    /* global sign continuity along n */
    for (int64_t n = 1; n < N; n++) {
        double d = 0;
        for (int k = 0; k < 4; k++) d += coef[4 * n + k] * coef[4 * (n - 1) + k];
        if (d < 0) for (int k = 0; k < 4; k++) coef[4 * n + k] = -coef[4 * n + k];
    }
    /* scale so that the mean norm of the (unnormalised) spline is 1 */
    double sum = 0;
    int64_t cnt = 0;
    for (int64_t n = 3; n < N; n += (N > 4000 ? N / 4000 : 1)) {
        double b[4];
        int64_t base = knot_ns(g, n, dt);
        int64_t l = bspline4(g, dt, base, 0.37 * dt, b);
        double s[4] = {0, 0, 0, 0};
        for (int j = 0; j < 4; j++)
            for (int k = 0; k < 4; k++) s[k] += b[j] * coef[4 * (l - 3 + j) + k];
        sum += sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3]);
        cnt++;
    }
    double sc = cnt ? cnt / sum : 1.0;
    for (int64_t i = 0; i < 4 * N; i++) coef[i] *= sc;
}

/* evaluate the truth attitude matrix at t = base + off */
static void attitude_mat(const sim_geometry *g, int64_t dt, const double *coef, int64_t base_ns, double off_ns,
                         double m[3][3]) {
    double b[4];
    int64_t l = bspline4(g, dt, base_ns, off_ns, b);
    double s[4] = {0, 0, 0, 0};
    for (int j = 0; j < 4; j++)
        for (int k = 0; k < 4; k++) s[k] += b[j] * coef[4 * (l - 3 + j) + k];
    double nn = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3]);
    for (int k = 0; k < 4; k++) s[k] /= nn;
    quat2mat(s, m);
}

/* ------------------------------------------------------------------------ */
/* true direction and field angles                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    double p[3], q[3], r[3];
    double par, pma, pmd; /* parallax, mu_alpha*, mu_delta */
} src_geom;

static void source_geom(const double *s5, src_geom *sg) {
    double a = s5[0], d = s5[1];
    double sa = sin(a), ca = cos(a), sd = sin(d), cd = cos(d);
    sg->p[0] = -sa; sg->p[1] = ca; sg->p[2] = 0;
    sg->q[0] = -sd * ca; sg->q[1] = -sd * sa; sg->q[2] = cd;
    sg->r[0] = cd * ca; sg->r[1] = cd * sa; sg->r[2] = sd;
    sg->par = s5[2]; sg->pma = s5[3]; sg->pmd = s5[4];
}

/* proper direction (ICRS) of the source at t = base + off (ns) */
static void proper_direction(const sim_geometry *g, const src_geom *sg, int64_t base_ns, double off_ns, double u[3]) {
    double t_s = (double)base_ns * 1e-9 + off_ns * 1e-9;
    double b[3], v[3];
    ephemeris(g, t_s, b, v);
    double tb_rel_s = (double)(base_ns - g->t_ep_ns) * 1e-9 + off_ns * 1e-9 + v_dot(sg->r, b) * g->au_light_s;
    double tau = tb_rel_s / SIM_YEAR_S;
    double ub[3];
    for (int i = 0; i < 3; i++) ub[i] = sg->r[i] + tau * (sg->p[i] * sg->pma + sg->q[i] * sg->pmd) - sg->par * b[i];
    v_unit(ub);
    for (int i = 0; i < 3; i++) u[i] = ub[i] + v[i] * g->au_light_s;
    v_unit(u);
}

/* field angles: phi, zeta (SRS spherical coordinates) */
static void field_angles(const sim_geometry *g, int64_t dt, const double *coef, const src_geom *sg,
                         int64_t base_ns, double off_ns, double *phi, double *zeta) {
    double u[3], m[3][3];
    proper_direction(g, sg, base_ns, off_ns, u);
    attitude_mat(g, dt, coef, base_ns, off_ns, m);
    double us[3] = {v_dot(m[0], u), v_dot(m[1], u), v_dot(m[2], u)};
    *phi = atan2(us[1], us[0]);
    *zeta = atan2(us[2], sqrt(us[0] * us[0] + us[1] * us[1]));
}

/* ------------------------------------------------------------------------ */
/* observation generation                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n, cap;
    int64_t *t_ns;
    int32_t *src;
    uint8_t *ccd, *fov, *kind;
    float *sigma;
    double *mu;
    double *noise; /* realised R at truth (for tests) */
    uint8_t *gate;
} obs_buf;

static void buf_push(obs_buf *b, int64_t t, int32_t src, int ccd, int fov, int kind, float sig, double mu,
                     double noise, int gate) {
    if (b->n == b->cap) {
        int64_t nc = b->cap ? 2 * b->cap : 4096;
        b->t_ns = realloc(b->t_ns, nc * sizeof(int64_t));
        b->src = realloc(b->src, nc * sizeof(int32_t));
        b->ccd = realloc(b->ccd, nc);
        b->fov = realloc(b->fov, nc);
        b->kind = realloc(b->kind, nc);
        b->sigma = realloc(b->sigma, nc * sizeof(float));
        b->mu = realloc(b->mu, nc * sizeof(double));
        b->noise = realloc(b->noise, nc * sizeof(double));
        b->gate = realloc(b->gate, nc);
        b->cap = nc;
    }
    int64_t i = b->n++;
    b->t_ns[i] = t; b->src[i] = src; b->ccd[i] = (uint8_t)ccd; b->fov[i] = (uint8_t)fov;
    b->kind[i] = (uint8_t)kind; b->sigma[i] = sig; b->mu[i] = mu; b->noise[i] = noise; b->gate[i] = (uint8_t)gate;
}

typedef struct sim_handle {
    sim_config cfg;
    sim_geometry geo;
    pert_t pert;
    double *att_true;       /* N x 4 */
    double *src_true;       /* n_src x 5 */
    double *src_mag;        /* n_src */
    double *cal_true;       /* n_cal */
    int64_t n_cal;
    int nthreads;
    obs_buf *bufs;          /* per thread */
    int32_t *keep;          /* per source: 1 kept */
    int64_t *src_count;     /* observations per source (before filtering) */
    int32_t *src_transits;
    int64_t n_obs;
    int32_t *src_newid;     /* index of the kept source in the output, -1 if dropped */
    int64_t n_src_out;
    double *rev_axes;       /* nominal SRS axes at mid-revolution, 9 per revolution */
    int64_t n_rev;
} sim_handle;

static inline int64_t cal_index_al(const sim_geometry *g, int64_t day, int fov, int ccd) {
    return (day * 2 + fov) * SIM_NCCD + ccd;
}
static inline int64_t cal_index_ac(const sim_geometry *g, int64_t day, int fov, int row) {
    return g->n_cal_days * 2 * SIM_NCCD + (day * 2 + fov) * SIM_NROW + row;
}

/* full geometric calibration, parameter layout: groups (ccd, gate, long interval k) in that
 * order; within an AL group Deta[j in k][f][r] (6 per day) then deta[bin]; all AC groups after
 * all AL groups, Dzeta[f][r] (6 each) */
#define SIM_NCOL 1966
typedef struct {
    int64_t n_j, j_per_k, n_k, n_gate, col_bin, n_bin, al_size, n_groups, n_al;
} gen_layout;
static gen_layout gen_layout_of(const sim_config *c, const sim_geometry *g) {
    gen_layout L;
    L.n_j = g->n_cal_days;
    L.j_per_k = c->cal_j_per_k > 0 ? c->cal_j_per_k : 1;
    L.n_k = (L.n_j + L.j_per_k - 1) / L.j_per_k;
    L.n_gate = c->n_gate > 0 ? c->n_gate : 1;
    L.col_bin = c->cal_col_bin > 0 ? c->cal_col_bin : 1;
    L.n_bin = (SIM_NCOL + L.col_bin - 1) / L.col_bin;
    L.al_size = 6 * L.j_per_k + L.n_bin;
    L.n_groups = (int64_t)SIM_NCCD * L.n_gate * L.n_k;
    L.n_al = L.n_groups * L.al_size;
    return L;
}
static inline int64_t gen_group(const gen_layout *L, int ccd, int gate, int64_t k) {
    return ((int64_t)ccd * L->n_gate + gate) * L->n_k + k;
}
static inline int64_t gen_deta(const gen_layout *L, int ccd, int gate, int64_t j, int fov, int r) {
    return gen_group(L, ccd, gate, j / L->j_per_k) * L->al_size + (j % L->j_per_k) * 6 + fov * 3 + r;
}
static inline int64_t gen_small(const gen_layout *L, int ccd, int gate, int64_t k, int64_t b) {
    return gen_group(L, ccd, gate, k) * L->al_size + 6 * L->j_per_k + b;
}
static inline int64_t gen_dzeta(const gen_layout *L, int ccd, int gate, int64_t k, int fov, int r) {
    return L->n_al + gen_group(L, ccd, gate, k) * 6 + fov * 3 + r;
}
/* shifted Legendre polynomials L*_0..2 at x = (mu - 13.5) / 1966 */
static inline void gen_legendre(double mu, double l[3]) {
    double x = (mu - 13.5) / SIM_NCOL;
    l[0] = 1.0;
    l[1] = 2.0 * x - 1.0;
    l[2] = 6.0 * x * x - 6.0 * x + 1.0;
}
static inline int64_t gen_bin(const gen_layout *L, double mu) {
    int64_t m = (int64_t)floor(mu + 0.5) - 14;
    if (m < 0) m = 0;
    if (m > SIM_NCOL - 1) m = SIM_NCOL - 1;
    return m / L->col_bin;
}
/* the calibration terms of an AL and of an AC observation line (Eq. etazeta) */
static double gen_al_term(const gen_layout *L, const double *cal, int ccd, int gate, int64_t day, int fov,
                          double mu) {
    double l[3];
    gen_legendre(mu, l);
    double v = 0.0;
    for (int r = 0; r < 3; r++) v += cal[gen_deta(L, ccd, gate, day, fov, r)] * l[r];
    return v + cal[gen_small(L, ccd, gate, day / L->j_per_k, gen_bin(L, mu))];
}
static double gen_ac_term(const gen_layout *L, const double *cal, int ccd, int gate, int64_t day, int fov,
                          double mu) {
    double l[3];
    gen_legendre(mu, l);
    double v = 0.0;
    for (int r = 0; r < 3; r++) v += cal[gen_dzeta(L, ccd, gate, day / L->j_per_k, fov, r)] * l[r];
    return v;
}
/* gate of one observation: the source magnitude with a jittered threshold */
static int gen_gate(const sim_config *c, double G, rng_t *rg) {
    if (!c->cal_generic || c->n_gate <= 1) return 0;
    double Gj = G + c->gate_fuzz * rng_gauss(rg);
    if (Gj >= c->gate_g0) return 0;
    int g = 1 + (int)floor((c->gate_g0 - Gj) / c->gate_step);
    return g > c->n_gate - 1 ? c->n_gate - 1 : g;
}

static int64_t day_of(const sim_config *c, const sim_geometry *g, int64_t t_ns) {
    int64_t d = t_ns / c->cal_dt_ns;
    if (d < 0) d = 0;
    if (d >= g->n_cal_days) d = g->n_cal_days - 1;
    return d;
}

static void gen_source(sim_handle *h, int64_t i, obs_buf *ob, int32_t *n_transits) {
    const sim_config *c = &h->cfg;
    const sim_geometry *g = &h->geo;
    const double *coef = h->att_true;
    int64_t dt = c->knot_dt_ns;
    src_geom sg;
    source_geom(&h->src_true[5 * i], &sg);
    double sig_al = c->sigma_al, sig_ac = c->sigma_ac;
    if (c->mag_dependent) {
        sig_al = 50.0 * SIM_UAS * pow(10.0, (h->src_mag[i] - 12.0) / 6.0);
        sig_ac = 5.65 * sig_al;
    }
    rng_t rn;
    rng_seed(&rn, c->seed, 0x5EEDULL + 7, (uint64_t)i);
    /* gates draw from their own stream: the offsets-only data stay as they were */
    rng_t rg;
    rng_seed(&rg, c->seed, 0x6A7EULL, (uint64_t)i);
    const gen_layout GL = gen_layout_of(c, g);
    const int generic = c->cal_generic != 0;
    const double T = 2.0 * SIM_PI / g->spin_rate;
    const double span_s = (double)c->span_ns * 1e-9;
    const int64_t n_rev = h->n_rev;
    const double lim = sin(1.3 * SIM_PI / 180.0);
    const double lim_field = sin(0.5 * SIM_PI / 180.0);
    const double F = g->focal_length;
    const double om_ns = g->spin_rate * 1e-9;
    int32_t ntr = 0;
    for (int64_t k = 0; k < n_rev; k++) {
        double tm = (k + 0.5) * T;
        const double *ax = &h->rev_axes[12 * k];
        double cz = ax[6] * sg.r[0] + ax[7] * sg.r[1] + ax[8] * sg.r[2];
        if (fabs(cz) > lim) continue;
        double cx = ax[0] * sg.r[0] + ax[1] * sg.r[1] + ax[2] * sg.r[2];
        double cy = ax[3] * sg.r[0] + ax[4] * sg.r[1] + ax[5] * sg.r[2];
        double czd = ax[9] * sg.r[0] + ax[10] * sg.r[1] + ax[11] * sg.r[2];
        double phm = atan2(cy, cx);
        for (int fi = 0; fi < 2; fi++) {
            double f = fi == 0 ? 1.0 : -1.0;
            double dph = remainder(phm - f * 0.5 * g->gamma_c, 2.0 * SIM_PI);
            double dts = dph / g->spin_rate;
            /* across-scan pre-filter with the linearly moving spin axis */
            if (fabs(cz + czd * dts) > lim_field) continue;
            double tc = tm + dts;
            if (tc < 0 || tc >= span_s) continue;
            int64_t base = (int64_t)llround(tc * 1e9);
            if (base < 0 || base >= c->span_ns) continue;
            double off = 0, ph, ze;
            int ok = 1;
            for (int it = 0; it < 3; it++) {
                field_angles(g, dt, coef, &sg, base, off, &ph, &ze);
                double eta = remainder(ph - f * 0.5 * g->gamma_c, 2.0 * SIM_PI);
                if (fabs(eta) > 0.2) { ok = 0; break; }
                off += eta / om_ns;
            }
            if (!ok) continue;
            double tcs = (double)base * 1e-9 + off * 1e-9;
            if (tcs < 0 || tcs >= span_s || tcs < k * T || tcs >= (k + 1) * T) continue;
            field_angles(g, dt, coef, &sg, base, off, &ph, &ze);
            if ((ph > 0 ? 1 : -1) != (int)f) continue;
            /* which AC row: zeta = -(X[row] - (mu-mu_c) p - Xc[f]) / F; keep a 30-pixel margin for the
             * across-scan motion during the transit */
            int row = -1;
            for (int r = 0; r < SIM_NROW; r++) {
                double x_row = (r - 3) * 60.2e-3;
                double mu = g->mu_c + (F * ze + x_row - g->x_centre[fi]) / g->p_ac;
                if (mu >= 14.0 + 30.0 && mu <= 1979.0 - 30.0) row = r;
            }
            if (row < 0) continue;
            ntr++;
            /* AL observations on the strips of that row */
            int64_t t_af1 = -1;
            double slope = -om_ns;    /* d eta / d t (rad/ns), refined by the secant */
            double o_start = off - g->eta0[row * SIM_NSTRIP - ((row > SIM_MISSING_ROW) ? 1 : 0)] / om_ns;
            double o_last = 0, eta0_last = 0;
            int have_last = 0;
            for (int s = 0; s < SIM_NSTRIP; s++) {
                if (row == SIM_MISSING_ROW && s == SIM_MISSING_STRIP) continue;
                int ccd = row * SIM_NSTRIP + s - ((row > SIM_MISSING_ROW) ? 1 : 0);
                double eps = 0.0;
                if (!c->noise_free) {
                    eps = sig_al * rng_gauss(&rn);
                    if (rng_uniform(&rn) < c->outlier_frac)
                        eps += (rng_uniform(&rn) < 0.5 ? -1.0 : 1.0) * c->outlier_nsigma * sig_al;
                }
                double eta0 = g->eta0[ccd];
                const int gate = gen_gate(c, h->src_mag[i], &rg);
                double o = have_last ? o_last + (eta0 - eta0_last) / slope : o_start;
                int64_t day = day_of(c, g, base + (int64_t)llround(o));
                double target = generic ? 0.0 : eta0 + h->cal_true[cal_index_al(g, day, fi, ccd)] - eps;
                double o_prev = 0, e_prev = 0, e = 0;
                int converged = 0;
                for (int it = 0; it < 12; it++) {
                    field_angles(g, dt, coef, &sg, base, o, &ph, &ze);
                    if (generic) {
                        /* the line at the AC pixel coordinate of the image at this time */
                        double mu_al = g->mu_c + (F * ze + g->x_fpa[ccd] - g->x_centre[fi]) / g->p_ac;
                        target = eta0 + gen_al_term(&GL, h->cal_true, ccd, gate, day, fi, mu_al) - eps;
                    }
                    e = remainder(ph - f * 0.5 * g->gamma_c, 2.0 * SIM_PI) - target;
                    if (it > 0 && fabs(o - o_prev) > 10.0) {
                        double sl = (e - e_prev) / (o - o_prev);
                        if (sl < 0.5 * (-om_ns) && sl > 2.0 * (-om_ns)) slope = sl;
                    }
                    if (fabs(e) < 1e-15) { converged = 1; break; }
                    o_prev = o; e_prev = e;
                    o += -e / slope;
                    int64_t d2 = day_of(c, g, base + (int64_t)llround(o));
                    if (d2 != day) {
                        day = d2;
                        if (!generic) target = eta0 + h->cal_true[cal_index_al(g, day, fi, ccd)] - eps;
                    }
                }
                (void)converged;
                o_last = o; eta0_last = eta0; have_last = 1;
                int64_t tl = base + (int64_t)llround(o);
                if (tl < 0 || tl >= c->span_ns) continue;
                /* realised residual at truth after rounding to ns */
                field_angles(g, dt, coef, &sg, tl, 0.0, &ph, &ze);
                int64_t dd = day_of(c, g, tl);
                double mu_rec = 0.0, tgt_noiseless;
                if (generic) {
                    mu_rec = g->mu_c + (F * ze + g->x_fpa[ccd] - g->x_centre[fi]) / g->p_ac;
                    tgt_noiseless = eta0 + gen_al_term(&GL, h->cal_true, ccd, gate, dd, fi, mu_rec);
                } else {
                    tgt_noiseless = eta0 + h->cal_true[cal_index_al(g, dd, fi, ccd)];
                }
                double eta_l = remainder(ph - f * 0.5 * g->gamma_c, 2.0 * SIM_PI);
                double R = tgt_noiseless - eta_l;
                (void)e;
                buf_push(ob, tl, (int32_t)i, ccd, fi, 0, (float)sig_al, mu_rec, R, gate);
                if (s == 0) t_af1 = tl;
            }
            /* one AC observation on AF1 of the row */
            if (t_af1 >= 0) {
                int ccd = row * SIM_NSTRIP - ((row > SIM_MISSING_ROW) ? 1 : 0);
                field_angles(g, dt, coef, &sg, t_af1, 0.0, &ph, &ze);
                double eps = 0.0;
                if (!c->noise_free) {
                    eps = sig_ac * rng_gauss(&rn);
                    if (rng_uniform(&rn) < c->outlier_frac)
                        eps += (rng_uniform(&rn) < 0.5 ? -1.0 : 1.0) * c->outlier_nsigma * sig_ac;
                }
                int64_t dd = day_of(c, g, t_af1);
                const int gate = gen_gate(c, h->src_mag[i], &rg);
                double dz, mu;
                if (generic) {
                    /* zeta0(mu) + Dzeta(mu) = zeta + eps, solved for mu by fixed-point steps (the
                     * calibration term changes by < 1e-6 of zeta0's slope per pixel) */
                    mu = g->mu_c + (F * (ze + eps) + g->x_fpa[ccd] - g->x_centre[fi]) / g->p_ac;
                    for (int it = 0; it < 4; it++) {
                        dz = gen_ac_term(&GL, h->cal_true, ccd, gate, dd, fi, mu);
                        mu = g->mu_c + (F * (ze - dz + eps) + g->x_fpa[ccd] - g->x_centre[fi]) / g->p_ac;
                    }
                    dz = gen_ac_term(&GL, h->cal_true, ccd, gate, dd, fi, mu);
                } else {
                    dz = h->cal_true[cal_index_ac(g, dd, fi, row)];
                    /* zeta0(mu) = zeta - dzeta + eps */
                    double z0 = ze - dz + eps;
                    mu = g->mu_c + (F * z0 + g->x_fpa[ccd] - g->x_centre[fi]) / g->p_ac;
                }
                /* realised residual */
                double z0r = -(g->x_fpa[ccd] - (mu - g->mu_c) * g->p_ac - g->x_centre[fi]) / F;
                double R = z0r + dz - ze;
                buf_push(ob, t_af1, (int32_t)i, ccd, fi, 1, (float)sig_ac, mu, R, gate);
            }
        }
    }
    *n_transits = ntr;
}

/* ------------------------------------------------------------------------ */
/* public API                                                                */
/* ------------------------------------------------------------------------ */
/* truth of the full geometric calibration: large-scale AL terms N(0, cal_al_rms) for r = 0 and
 * N(0, cal_l12_rms) for r = 1, 2; small-scale AL terms N(0, cal_small_rms); AC terms on the AF1
 * CCD of each row (the only ones observed across scan) N(0, cal_ac_rms) for r = 0 and
 * N(0, cal_l12_rms) for r = 1, 2.  Made to satisfy the constraints: Eq. cc2 per (CCD, gate,
 * long interval) by removing the least-squares quadratic in the column-centre Legendre values,
 * Eq. cc1 per day over the r = 0 ungated AL terms, Eq. cc3 per field and long interval over the
 * r = 0 ungated AC terms. */
static void gen_truth(sim_handle *h) {
    const sim_config *cfg = &h->cfg;
    const gen_layout L = gen_layout_of(cfg, &h->geo);
    h->n_cal = L.n_al + 6 * L.n_groups;
    h->cal_true = calloc(h->n_cal, sizeof(double));
    double *cal = h->cal_true;
    rng_t r;
    rng_seed(&r, cfg->seed, 0xCA1ULL, 1);
    for (int n = 0; n < SIM_NCCD; n++)
        for (int gt = 0; gt < L.n_gate; gt++)
            for (int64_t j = 0; j < L.n_j; j++)
                for (int f = 0; f < 2; f++)
                    for (int rr = 0; rr < 3; rr++)
                        cal[gen_deta(&L, n, gt, j, f, rr)] = (rr == 0 ? cfg->cal_al_rms : cfg->cal_l12_rms) * rng_gauss(&r);
    /* cc2 weights: sum over each bin's columns of L*_r at the column centres */
    double *w = calloc(3 * L.n_bin, sizeof(double));
    for (int m = 0; m < SIM_NCOL; m++) {
        double l[3];
        gen_legendre(m + 14.0, l);
        for (int rr = 0; rr < 3; rr++) w[rr * L.n_bin + m / L.col_bin] += l[rr];
    }
    double Gm[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double v = 0;
            for (int64_t k = 0; k < L.n_bin; k++) v += w[a * L.n_bin + k] * w[b * L.n_bin + k];
            Gm[a][b] = v;
        }
    for (int n = 0; n < SIM_NCCD; n++)
        for (int gt = 0; gt < L.n_gate; gt++)
            for (int64_t k = 0; k < L.n_k; k++) {
                double *v = &cal[gen_small(&L, n, gt, k, 0)];
                for (int64_t b = 0; b < L.n_bin; b++) v[b] = cfg->cal_small_rms * rng_gauss(&r);
                /* alpha = (W W')^-1 W v by Gaussian elimination on the 3x3 system, v -= W' alpha */
                double A[3][4];
                for (int a = 0; a < 3; a++) {
                    double t = 0;
                    for (int64_t b = 0; b < L.n_bin; b++) t += w[a * L.n_bin + b] * v[b];
                    for (int c2 = 0; c2 < 3; c2++) A[a][c2] = Gm[a][c2];
                    A[a][3] = t;
                }
                for (int p = 0; p < 3; p++)
                    for (int q = p + 1; q < 3; q++) {
                        double fct = A[q][p] / A[p][p];
                        for (int c2 = p; c2 < 4; c2++) A[q][c2] -= fct * A[p][c2];
                    }
                double al[3];
                for (int p = 2; p >= 0; p--) {
                    double t = A[p][3];
                    for (int q = p + 1; q < 3; q++) t -= A[p][q] * al[q];
                    al[p] = t / A[p][p];
                }
                for (int64_t b = 0; b < L.n_bin; b++)
                    v[b] -= al[0] * w[b] + al[1] * w[L.n_bin + b] + al[2] * w[2 * L.n_bin + b];
            }
    free(w);
    for (int n = 0; n < SIM_NCCD; n++) {
        if (h->geo.ccd_strip[n] != 0) continue;
        for (int gt = 0; gt < L.n_gate; gt++)
            for (int64_t k = 0; k < L.n_k; k++)
                for (int f = 0; f < 2; f++)
                    for (int rr = 0; rr < 3; rr++)
                        cal[gen_dzeta(&L, n, gt, k, f, rr)] = (rr == 0 ? cfg->cal_ac_rms : cfg->cal_l12_rms) * rng_gauss(&r);
    }
    for (int64_t j = 0; j < L.n_j; j++) {
        double m = 0;
        for (int f = 0; f < 2; f++)
            for (int n = 0; n < SIM_NCCD; n++) m += cal[gen_deta(&L, n, 0, j, f, 0)];
        m /= 2 * SIM_NCCD;
        for (int f = 0; f < 2; f++)
            for (int n = 0; n < SIM_NCCD; n++) cal[gen_deta(&L, n, 0, j, f, 0)] -= m;
    }
    for (int64_t k = 0; k < L.n_k; k++)
        for (int f = 0; f < 2; f++) {
            double m = 0;
            for (int n = 0; n < SIM_NCCD; n++)
                if (h->geo.ccd_strip[n] == 0) m += cal[gen_dzeta(&L, n, 0, k, f, 0)];
            m /= SIM_NROW;
            for (int n = 0; n < SIM_NCCD; n++)
                if (h->geo.ccd_strip[n] == 0) cal[gen_dzeta(&L, n, 0, k, f, 0)] -= m;
        }
}

sim_handle *sim_create(const sim_config *cfg) {
    sim_handle *h = calloc(1, sizeof(sim_handle));
    h->cfg = *cfg;
    setup_geometry(cfg, &h->geo);
    setup_pert(cfg, &h->pert);
#ifdef _OPENMP
    if (cfg->n_threads > 0) omp_set_num_threads(cfg->n_threads);
    h->nthreads = omp_get_max_threads();
#else
    h->nthreads = 1;
#endif
    int64_t N = h->geo.n_coef;
    h->att_true = malloc(sizeof(double) * 4 * N);
    build_attitude(cfg, &h->geo, &h->pert, h->att_true);
    /* sources */
    int64_t ns = cfg->n_src;
    h->src_true = malloc(sizeof(double) * 5 * ns);
    h->src_mag = malloc(sizeof(double) * ns);
    for (int64_t i = 0; i < ns; i++) {
        rng_t r;
        rng_seed(&r, cfg->seed, 0x50BCEULL, (uint64_t)i);
        double a = cfg->ra_min + (cfg->ra_max - cfg->ra_min) * rng_uniform(&r);
        double smin = sin(cfg->dec_min), smax = sin(cfg->dec_max);
        double d = asin(smin + (smax - smin) * rng_uniform(&r));
        double par = -cfg->parallax_mean * log(1.0 - rng_uniform(&r));
        double pma = cfg->pm_sigma * rng_gauss(&r);
        double pmd = cfg->pm_sigma * rng_gauss(&r);
        h->src_true[5 * i + 0] = a;
        h->src_true[5 * i + 1] = d;
        h->src_true[5 * i + 2] = par;
        h->src_true[5 * i + 3] = pma;
        h->src_true[5 * i + 4] = pmd;
        h->src_mag[i] = 12.0 + 6.0 * rng_uniform(&r);
    }
    /* calibration truth, projected onto the constraints Eq. cc1 and cc3 */
    int64_t nd = h->geo.n_cal_days;
    if (cfg->cal_generic) {
        gen_truth(h);
        return h;
    }
    h->n_cal = nd * 2 * (SIM_NCCD + SIM_NROW);
    h->cal_true = calloc(h->n_cal, sizeof(double));
    {
        rng_t r;
        rng_seed(&r, cfg->seed, 0xCA1ULL, 0);
        for (int64_t d = 0; d < nd; d++) {
            double m = 0;
            for (int f = 0; f < 2; f++)
                for (int n = 0; n < SIM_NCCD; n++) {
                    double v = cfg->cal_al_rms * rng_gauss(&r);
                    h->cal_true[cal_index_al(&h->geo, d, f, n)] = v;
                    m += v;
                }
            m /= 2 * SIM_NCCD;
            for (int f = 0; f < 2; f++)
                for (int n = 0; n < SIM_NCCD; n++) h->cal_true[cal_index_al(&h->geo, d, f, n)] -= m;
            for (int f = 0; f < 2; f++) {
                double ma = 0;
                for (int rr = 0; rr < SIM_NROW; rr++) {
                    double v = cfg->cal_ac_rms * rng_gauss(&r);
                    h->cal_true[cal_index_ac(&h->geo, d, f, rr)] = v;
                    ma += v;
                }
                ma /= SIM_NROW;
                for (int rr = 0; rr < SIM_NROW; rr++) h->cal_true[cal_index_ac(&h->geo, d, f, rr)] -= ma;
            }
        }
    }
    return h;
}

int64_t sim_generate(sim_handle *h) {
    int64_t ns = h->cfg.n_src;
    {
        const double T = 2.0 * SIM_PI / h->geo.spin_rate;
        h->n_rev = (int64_t)ceil((double)h->cfg.span_ns * 1e-9 / T);
        h->rev_axes = malloc(sizeof(double) * 12 * (h->n_rev + 1));
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < h->n_rev; k++) {
            double m[3][3], mp[3][3], mm[3][3];
            double tm = (k + 0.5) * T;
            nominal_axes(&h->geo, tm, m);
            nominal_axes(&h->geo, tm + 60.0, mp);
            nominal_axes(&h->geo, tm - 60.0, mm);
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) h->rev_axes[12 * k + 3 * a + b] = m[a][b];
            for (int b = 0; b < 3; b++) h->rev_axes[12 * k + 9 + b] = (mp[2][b] - mm[2][b]) / 120.0;
        }
    }
    h->bufs = calloc(h->nthreads, sizeof(obs_buf));
    h->src_count = calloc(ns, sizeof(int64_t));
    h->src_transits = calloc(ns, sizeof(int32_t));
    h->keep = calloc(ns, sizeof(int32_t));
    int nt = h->nthreads;
    /* contiguous blocks of sources per thread keep the output sorted by source */
    int64_t chunk = (ns + nt - 1) / nt;
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int64_t i0 = tid * chunk, i1 = i0 + chunk;
        if (i1 > ns) i1 = ns;
        for (int64_t i = i0; i < i1; i++) {
            int64_t before = h->bufs[tid].n;
            int32_t ntr = 0;
            gen_source(h, i, &h->bufs[tid], &ntr);
            h->src_count[i] = h->bufs[tid].n - before;
            h->src_transits[i] = ntr;
        }
    }
    h->src_newid = malloc(sizeof(int32_t) * ns);
    int64_t nobs = 0, nout = 0;
    for (int64_t i = 0; i < ns; i++) {
        int keep = 1;
        if (h->cfg.min_transits > 0 && h->src_transits[i] < h->cfg.min_transits) keep = 0;
        if (h->cfg.max_transits > 0 && h->src_transits[i] > h->cfg.max_transits) keep = 0;
        if (h->src_count[i] == 0) keep = 0;
        h->keep[i] = keep;
        h->src_newid[i] = keep ? (int32_t)nout : -1;
        if (keep) { nout++; nobs += h->src_count[i]; }
    }
    h->n_obs = nobs;
    h->n_src_out = nout;
    return nobs;
}

int64_t sim_n_src_out(const sim_handle *h) { return h->n_src_out; }
int64_t sim_n_coef(const sim_handle *h) { return h->geo.n_coef; }
int64_t sim_n_cal(const sim_handle *h) { return h->n_cal; }
void sim_get_geometry(const sim_handle *h, sim_geometry *g) { *g = h->geo; }

/* copy the kept observations (sorted by source, then time within a transit order) */
void sim_copy_obs(const sim_handle *h, int64_t *t_ns, int32_t *src, uint8_t *ccd, uint8_t *fov, uint8_t *kind,
                  float *sigma, double *mu, double *noise) {
    int nt = h->nthreads;
    int64_t ns = h->cfg.n_src;
    int64_t chunk = (ns + nt - 1) / nt;
    /* output offsets per thread */
    int64_t *off = calloc(nt + 1, sizeof(int64_t));
    for (int tid = 0; tid < nt; tid++) {
        int64_t i0 = tid * chunk, i1 = i0 + chunk;
        if (i1 > ns) i1 = ns;
        int64_t cnt = 0;
        for (int64_t i = i0; i < i1; i++)
            if (h->keep[i]) cnt += h->src_count[i];
        off[tid + 1] = off[tid] + cnt;
    }
#pragma omp parallel for num_threads(nt) schedule(static, 1)
    for (int tid = 0; tid < nt; tid++) {
        const obs_buf *b = &h->bufs[tid];
        int64_t o = off[tid];
        int64_t j = 0;
        int64_t i0 = tid * chunk, i1 = i0 + chunk;
        if (i1 > ns) i1 = ns;
        for (int64_t i = i0; i < i1; i++) {
            int64_t c = h->src_count[i];
            if (h->keep[i]) {
                for (int64_t k = 0; k < c; k++) {
                    int64_t s = j + k;
                    t_ns[o] = b->t_ns[s];
                    src[o] = h->src_newid[i];
                    ccd[o] = b->ccd[s];
                    fov[o] = b->fov[s];
                    kind[o] = b->kind[s];
                    sigma[o] = b->sigma[s];
                    mu[o] = b->mu[s];
                    if (noise) noise[o] = b->noise[s];
                    o++;
                }
            }
            j += c;
        }
    }
    free(off);
}

/* gates of the kept observations, in the order of sim_copy_obs */
void sim_copy_gate(const sim_handle *h, uint8_t *gate) {
    int64_t o = 0;
    int nt = h->nthreads;
    int64_t ns = h->cfg.n_src;
    int64_t chunk = (ns + nt - 1) / nt;
    for (int tid = 0; tid < nt; tid++) {
        const obs_buf *b = &h->bufs[tid];
        int64_t j = 0;
        int64_t i0 = tid * chunk, i1 = i0 + chunk;
        if (i1 > ns) i1 = ns;
        for (int64_t i = i0; i < i1; i++) {
            int64_t c = h->src_count[i];
            if (h->keep[i])
                for (int64_t k = 0; k < c; k++) gate[o++] = b->gate[j + k];
            j += c;
        }
    }
}

/* truth and starting values */
void sim_copy_truth(const sim_handle *h, double *src_true, double *src_mag, double *att_true, double *cal_true,
                    int32_t *n_transits) {
    int64_t ns = h->cfg.n_src;
    for (int64_t i = 0; i < ns; i++) {
        int32_t k = h->src_newid[i];
        if (k < 0) continue;
        memcpy(&src_true[5 * k], &h->src_true[5 * i], 5 * sizeof(double));
        if (src_mag) src_mag[k] = h->src_mag[i];
        if (n_transits) n_transits[k] = h->src_transits[i];
    }
    memcpy(att_true, h->att_true, sizeof(double) * 4 * h->geo.n_coef);
    memcpy(cal_true, h->cal_true, sizeof(double) * h->n_cal);
}

/* starting values: sources truth + N(0, err) in alpha*, delta, zero parallax and proper motion;
 * attitude: every coefficient rotated by an independent small random frame rotation;
 * calibration: zero (nominal). */
void sim_starting_values(const sim_handle *h, double *src0, double *att0, double *cal0) {
    const sim_config *c = &h->cfg;
    int64_t ns = c->n_src;
    for (int64_t i = 0; i < ns; i++) {
        int32_t k = h->src_newid[i];
        if (k < 0) continue;
        rng_t r;
        rng_seed(&r, c->seed, 0x57A27ULL, (uint64_t)i);
        const double *s = &h->src_true[5 * i];
        double da = c->start_src_err * rng_gauss(&r);
        double dd = c->start_src_err * rng_gauss(&r);
        src0[5 * k + 0] = s[0] + da / cos(s[1]);
        src0[5 * k + 1] = s[1] + dd;
        src0[5 * k + 2] = 0.0;
        src0[5 * k + 3] = 0.0;
        src0[5 * k + 4] = 0.0;
    }
    int64_t N = h->geo.n_coef;
    for (int64_t n = 0; n < N; n++) {
        rng_t r;
        rng_seed(&r, c->seed, 0xA770ULL, (uint64_t)n);
        double phi[3] = {c->start_att_err * rng_gauss(&r), c->start_att_err * rng_gauss(&r),
                         c->start_att_err * rng_gauss(&r)};
        /* a0 = a (x) Q(phi): frame rotation followed by a small frame rotation */
        double th = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
        double d[4] = {0, 0, 0, 1};
        if (th > 0) {
            double s = sin(0.5 * th) / th;
            d[0] = phi[0] * s; d[1] = phi[1] * s; d[2] = phi[2] * s; d[3] = cos(0.5 * th);
        }
        const double *a = &h->att_true[4 * n];
        double *o = &att0[4 * n];
        /* quaternion product a*d, components {x,y,z,w} */
        o[0] = a[0] * d[3] + a[1] * d[2] - a[2] * d[1] + a[3] * d[0];
        o[1] = -a[0] * d[2] + a[1] * d[3] + a[2] * d[0] + a[3] * d[1];
        o[2] = a[0] * d[1] - a[1] * d[0] + a[2] * d[3] + a[3] * d[2];
        o[3] = -a[0] * d[0] - a[1] * d[1] - a[2] * d[2] + a[3] * d[3];
    }
    memset(cal0, 0, sizeof(double) * h->n_cal);
}

/* true field angles of a source at a time (for tests of the truth world itself) */
void sim_field_angles(const sim_handle *h, const double *s5, int64_t t_ns, double *phi, double *zeta) {
    src_geom sg;
    source_geom(s5, &sg);
    field_angles(&h->geo, h->cfg.knot_dt_ns, h->att_true, &sg, t_ns, 0.0, phi, zeta);
}

/* nominal and target attitude (for tests) */
void sim_target_quat(const sim_handle *h, double t_s, double q[4]) { target_quat(&h->geo, &h->pert, t_s, q); }

void sim_destroy(sim_handle *h) {
    if (!h) return;
    if (h->bufs) {
        for (int t = 0; t < h->nthreads; t++) {
            obs_buf *b = &h->bufs[t];
            free(b->t_ns); free(b->src); free(b->ccd); free(b->fov); free(b->kind);
            free(b->sigma); free(b->mu); free(b->noise); free(b->gate);
        }
        free(h->bufs);
    }
    free(h->att_true); free(h->src_true); free(h->src_mag); free(h->cal_true);
    free(h->keep); free(h->src_count); free(h->src_transits); free(h->src_newid);
    free(h->rev_axes);
    free(h);
}

int sim_sizeof_config(void) { return (int)sizeof(sim_config); }
int sim_sizeof_geometry(void) { return (int)sizeof(sim_geometry); }
