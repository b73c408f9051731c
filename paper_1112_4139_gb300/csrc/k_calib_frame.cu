// k_calib_frame.cu -- the C block (Sect. 5.3), the frame rotator (Sect. 6.1) and the
// deterministic reductions of the per-source statistics.
#include "agis_internal.cuh"

namespace agis {

// ---------------------------------------------------------------------------------------
// C block: one warp per calibration parameter k over its observations (calibration order):
// N_kk = sum W, b_k = -sum W R (dR/dc_k = 1, Eq. pdC); the 1x1 robust solve of
// Algorithms C.1-C.3 gives d~_k = (b / sqrt(N)) / sqrt(N), or 0 with a rank defect.
// ---------------------------------------------------------------------------------------
// sums != NULL: write (N_kk, b_k) pairs there instead of solving
__global__ void k_cal_accum(int n_cal, const uint32_t* __restrict__ perm_c, const int64_t* __restrict__ cal_off,
                            const ObsRec* __restrict__ rec, double tol, double* __restrict__ dtil,
                            int* __restrict__ rd, double* __restrict__ sums) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n_cal; k += nw) {
        double sw = 0.0, swr = 0.0;
        const int64_t end = cal_off[k + 1];
        int64_t j = cal_off[k] + lane;
        // four independent gathers in flight per lane; the sums keep the order j, j + 32, ...
        for (; j + 3 * kWarp < end; j += 4 * kWarp) {
            const uint32_t p0 = perm_c[j], p1 = perm_c[j + kWarp], p2 = perm_c[j + 2 * kWarp],
                           p3 = perm_c[j + 3 * kWarp];
            const double W0 = rec[p0].W, R0 = rec[p0].R, W1 = rec[p1].W, R1 = rec[p1].R;
            const double W2 = rec[p2].W, R2 = rec[p2].R, W3 = rec[p3].W, R3 = rec[p3].R;
            sw += W0;
            swr += W0 * R0;
            sw += W1;
            swr += W1 * R1;
            sw += W2;
            swr += W2 * R2;
            sw += W3;
            swr += W3 * R3;
        }
        for (; j < end; j += kWarp) {
            const ObsRec* r = rec + perm_c[j];
            const double W = r->W;
            sw += W;
            swr += W * r->R;
        }
        sw = warp_sum(sw);
        swr = warp_sum(swr);
        if (lane == 0) {
            if (sums) {
                sums[2 * (size_t)k] = sw;
                sums[2 * (size_t)k + 1] = -swr;
                continue;
            }
            const double b = -swr;
            if (sw > tol * sw && sw > 0.0) {
                const double u = sqrt(sw);
                dtil[k] = (b / u) / u;
                rd[k] = 0;
            } else {
                dtil[k] = 0.0;
                rd[k] = 1;
            }
        }
    }
}

// the 1x1 robust solves from (N_kk, b_k) pairs (the sums of k_cal_accum, reduced over a
// partition of the sources): same arithmetic as k_cal_accum's own solve
__global__ void k_cal_solve_sums(int n_cal, const double* __restrict__ sums, double tol, double* __restrict__ dtil,
                                 int* __restrict__ rd) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_cal; k += gridDim.x * blockDim.x) {
        const double sw = sums[2 * (size_t)k], b = sums[2 * (size_t)k + 1];
        if (sw > tol * sw && sw > 0.0) {
            const double u = sqrt(sw);
            dtil[k] = (b / u) / u;
            rd[k] = 0;
        } else {
            dtil[k] = 0.0;
            rd[k] = 1;
        }
    }
}

// Constraint projection d = d~ - C (C'C)^-1 C' d~ (Eq. calCon).  The columns of C for
// Eqs. cc1 (per interval: all 124 AL offsets) and cc3 (per interval and field: 7 AC offsets)
// have disjoint supports, so within each column's support d = d~ - mean(d~).  One thread
// per constraint column; then c += d.
__global__ void k_cal_project(int n_days, const double* __restrict__ dtil, double* __restrict__ cal) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 3 * n_days) return;
    int64_t k0;
    int cnt;
    if (g < n_days) {
        k0 = (int64_t)g * 124;
        cnt = 124;
    } else {
        const int h = g - n_days;  // (day, field)
        k0 = (int64_t)n_days * 124 + (int64_t)h * 7;
        cnt = 7;
    }
    double s = 0.0;
    for (int i = 0; i < cnt; i++) s += dtil[k0 + i];
    const double m = s / (double)cnt;
    for (int i = 0; i < cnt; i++) cal[k0 + i] += dtil[k0 + i] - m;
}

void launch_cal(int n_cal, int n_days, const uint32_t* perm_c, const int64_t* cal_off, const ObsRec* rec, double tol,
                double* dtil, int* rd, double* cal, const Shapes& sh, cudaStream_t s) {
    const int wpb = sh.cal_threads / 32;
    int blocks = (n_cal + wpb - 1) / wpb;
    if (blocks > 152 * sh.cal_bps) blocks = 152 * sh.cal_bps;
    if (blocks < 1) blocks = 1;
    k_cal_accum<<<blocks, sh.cal_threads, 0, s>>>(n_cal, perm_c, cal_off, rec, tol, dtil, rd, nullptr);
    k_cal_project<<<(3 * n_days + 127) / 128, 128, 0, s>>>(n_days, dtil, cal);
}

// partitioned sources: the local (N_kk, b_k) sums, and the update from reduced sums
void launch_cal_sums(int n_cal, const uint32_t* perm_c, const int64_t* cal_off, const ObsRec* rec, double* sums,
                     const Shapes& sh, cudaStream_t s) {
    const int wpb = sh.cal_threads / 32;
    int blocks = (n_cal + wpb - 1) / wpb;
    if (blocks > 152 * sh.cal_bps) blocks = 152 * sh.cal_bps;
    if (blocks < 1) blocks = 1;
    k_cal_accum<<<blocks, sh.cal_threads, 0, s>>>(n_cal, perm_c, cal_off, rec, 0.0, nullptr, nullptr, sums);
}
void launch_cal_from_sums(int n_cal, int n_days, const double* sums, double tol, double* dtil, int* rd, double* cal,
                          cudaStream_t s) {
    int blocks = (n_cal + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_cal_solve_sums<<<blocks, 256, 0, s>>>(n_cal, sums, tol, dtil, rd);
    k_cal_project<<<(3 * n_days + 127) / 128, 128, 0, s>>>(n_days, dtil, cal);
}

// ---------------------------------------------------------------------------------------
// Frame rotator
// ---------------------------------------------------------------------------------------
constexpr int kFrameVals = 27;  // 21 upper entries of the 6x6 normals + 6 rhs
__host__ __device__ constexpr int up6(int i, int j) { return i * 6 - i * (i - 1) / 2 + (j - i); }

__device__ __forceinline__ void triad(double a, double d, double* p, double* q, double* r) {
    double sa, ca, sd, cd;
    sincos(a, &sa, &ca);
    sincos(d, &sd, &cd);
    p[0] = -sa; p[1] = ca; p[2] = 0.0;
    q[0] = -sd * ca; q[1] = -sd * sa; q[2] = cd;
    r[0] = cd * ca; r[1] = cd * sa; r[2] = sd;
}

// Per-source observation equations of Eq. cond-mu3 (comparison epoch t = t_ep, unit weights):
//   q'w = dmu_a*,  -p'w = dmu_d,  q'(e + tt w) = Delta alpha*,  -p'(e + tt w) = Delta delta
// with Delta from Eq. fr-Delta1, tt = (t_ep - t_fr) in years.  Each block reduces a fixed
// contiguous range of sources in a fixed order (deterministic).
__global__ void k_frame_normals(int n, const int32_t* __restrict__ subset, const double* __restrict__ src,
                                const double* __restrict__ ref, double tt, double* __restrict__ partial) {
    __shared__ double sh[256];
    double acc[kFrameVals];
#pragma unroll
    for (int i = 0; i < kFrameVals; i++) acc[i] = 0.0;
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int beg = blockIdx.x * per;
    const int end = min(n, beg + per);
    for (int j = beg + threadIdx.x; j < end; j += blockDim.x) {
        const int i = subset ? subset[j] : j;
        const double* s = src + 5 * (size_t)i;
        const double* h = ref + 4 * (size_t)i;
        double p[3], q[3], r[3], ph[3], qh[3], rh[3];
        triad(s[0], s[1], p, q, r);
        triad(h[0], h[1], ph, qh, rh);
        const double dr[3] = {r[0] - rh[0], r[1] - rh[1], r[2] - rh[2]};
        const double da = dot3(p, dr), dd = dot3(q, dr);
        const double dpa = s[3] - h[2], dpd = s[4] - h[3];
        double rows[4][6];
        for (int c = 0; c < 3; c++) {
            rows[0][c] = 0.0; rows[0][3 + c] = q[c];
            rows[1][c] = 0.0; rows[1][3 + c] = -p[c];
            rows[2][c] = q[c]; rows[2][3 + c] = tt * q[c];
            rows[3][c] = -p[c]; rows[3][3 + c] = -tt * p[c];
        }
        const double rhs[4] = {dpa, dpd, da, dd};
        for (int e = 0; e < 4; e++) {
            for (int a = 0; a < 6; a++) {
                for (int c = a; c < 6; c++) acc[up6(a, c)] += rows[e][a] * rows[e][c];
                acc[21 + a] += rows[e][a] * rhs[e];
            }
        }
    }
    for (int v = 0; v < kFrameVals; v++) {
        sh[threadIdx.x] = acc[v];
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[blockIdx.x * kFrameVals + v] = sh[0];
        __syncthreads();
    }
}

// Sum the block partials in order and solve the 6x6 system by Algorithms C.1-C.3.
__global__ void k_frame_solve(int n_part, const double* __restrict__ partial, double tol, double* __restrict__ eo) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double v[kFrameVals];
    for (int i = 0; i < kFrameVals; i++) v[i] = 0.0;
    for (int p = 0; p < n_part; p++)
        for (int i = 0; i < kFrameVals; i++) v[i] += partial[p * kFrameVals + i];
    double U[21];
    for (int j = 0; j < 6; j++) {
        for (int i = 0; i <= j; i++) {
            double s = 0.0;
            for (int k = 0; k < i; k++) s += U[up6(k, i)] * U[up6(k, j)];
            if (i < j) {
                double uii = U[up6(i, i)];
                U[up6(i, j)] = uii > 0.0 ? (v[up6(i, j)] - s) / uii : 0.0;
            } else {
                double d = v[up6(j, j)] - s;
                U[up6(j, j)] = d > tol * v[up6(j, j)] ? sqrt(d) : 0.0;
            }
        }
    }
    double y[6], x[6];
    for (int i = 0; i < 6; i++) {
        double s = v[21 + i];
        for (int k = 0; k < i; k++) s -= U[up6(k, i)] * y[k];
        y[i] = U[up6(i, i)] > 0.0 ? s / U[up6(i, i)] : 0.0;
    }
    for (int i = 5; i >= 0; i--) {
        double s = y[i];
        for (int k = i + 1; k < 6; k++) s -= U[up6(i, k)] * x[k];
        x[i] = U[up6(i, i)] > 0.0 ? s / U[up6(i, i)] : 0.0;
    }
    for (int i = 0; i < 6; i++) eo[i] = x[i];
}

// Q(phi), Eq. qrot
__device__ __forceinline__ void qrot(const double* phi, double* q) {
    const double ang = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
    if (ang > 0.0) {
        const double s = sin(0.5 * ang) / ang;
        q[0] = phi[0] * s; q[1] = phi[1] * s; q[2] = phi[2] * s; q[3] = cos(0.5 * ang);
    } else {
        q[0] = q[1] = q[2] = 0.0; q[3] = 1.0;
    }
}

// f(t) = Q[(t - t_fr) omega] Q(eps), Eq. fr1
__device__ __forceinline__ void frame_f(const double* eo, double dt_years, double* f) {
    const double wt[3] = {dt_years * eo[3], dt_years * eo[4], dt_years * eo[5]};
    double a[4], b[4];
    qrot(wt, a);
    qrot(eo, b);
    qmul(a, b, f);
}

__device__ __forceinline__ void qinv(const double* q, double* r) {
    const double n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    r[0] = -q[0] / n2; r[1] = -q[1] / n2; r[2] = -q[2] / n2; r[3] = q[3] / n2;
}

// frame rotation {S1'v,0} = q^-1 {S0'v,0} q, Eq. quatframerot
__device__ __forceinline__ void frame_rotate(const double* q, const double* v, double* out) {
    double qi[4], vq[4] = {v[0], v[1], v[2], 0.0}, t[4], o[4];
    qinv(q, qi);
    qmul(qi, vq, t);
    qmul(t, q, o);
    out[0] = o[0]; out[1] = o[1]; out[2] = o[2];
}

// Rigorous transformation of the astrometric parameters, Sect. 6.1.2 steps 1-5.
__global__ void k_frame_apply_src(int n_src, double* __restrict__ src, const double* __restrict__ eo, double dt_ep) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_src) return;
    double* s = src + 5 * (size_t)i;
    double f[4];
    frame_f(eo, dt_ep, f);
    double pt[3], qt[3], rt[3];
    triad(s[0], s[1], pt, qt, rt);
    const double w[3] = {eo[3], eo[4], eo[5]};
    double wxr[3] = {w[1] * rt[2] - w[2] * rt[1], w[2] * rt[0] - w[0] * rt[2], w[0] * rt[1] - w[1] * rt[0]};
    double mut[3];
    for (int c = 0; c < 3; c++) mut[c] = pt[c] * s[3] + qt[c] * s[4] - wxr[c];
    double rc[3], muc[3];
    frame_rotate(f, rt, rc);
    frame_rotate(f, mut, muc);
    const double alpha = atan2(rc[1], rc[0]);
    const double delta = atan2(rc[2], sqrt(rc[0] * rc[0] + rc[1] * rc[1]));
    double p[3], q[3], r[3];
    triad(alpha, delta, p, q, r);
    double a = fmod(alpha, 2.0 * 3.141592653589793);
    if (a < 0.0) a += 2.0 * 3.141592653589793;
    s[0] = a;
    s[1] = delta;
    s[3] = dot3(p, muc);
    s[4] = dot3(q, muc);
}

// a_n <- f(t_n)^-1 a_n with t_n the mid-time of the support of B_n (Eqs. fr-q4, RF4).
__global__ void k_frame_apply_att(DevGeo G, double* __restrict__ att, const double* __restrict__ eo) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.n_coef) return;
    const int64_t tbar = (knot_at(G, n) + knot_at(G, n + 4)) / 2;
    const double dt = (double)(tbar - G.t_fr_ns) * 1e-9 / G.year_s;
    double f[4], fi[4], o[4];
    frame_f(eo, dt, f);
    qinv(f, fi);
    double* a = att + 4 * (int64_t)n;
    qmul(fi, a, o);
    a[0] = o[0]; a[1] = o[1]; a[2] = o[2]; a[3] = o[3];
}

// the 27 frame sums of the local sources (the block partials added in order)
__global__ void k_frame_sum(int n_part, const double* __restrict__ partial, double* __restrict__ out) {
    if (blockIdx.x != 0 || threadIdx.x >= kFrameVals) return;
    double v = 0.0;
    for (int p = 0; p < n_part; p++) v += partial[p * kFrameVals + threadIdx.x];
    out[threadIdx.x] = v;
}

void launch_frame_sums(int n, const int32_t* subset, const double* src, const double* ref, const DevGeo& G,
                       double* partial, int n_part, double* sums, cudaStream_t s) {
    const double tt = (double)(G.t_ep_ns - G.t_fr_ns) * 1e-9 / G.year_s;
    k_frame_normals<<<n_part, 256, 0, s>>>(n, subset, src, ref, tt, partial);
    k_frame_sum<<<1, 32, 0, s>>>(n_part, partial, sums);
}
// solve from reduced sums (one part) and apply to the local sources and the attitude
void launch_frame_from_sums(const DevGeo& G, int n_src, double* src, double* att, const double* sums, double tol,
                            double* eo, cudaStream_t s) {
    const double tt = (double)(G.t_ep_ns - G.t_fr_ns) * 1e-9 / G.year_s;
    k_frame_solve<<<1, 32, 0, s>>>(1, sums, tol, eo);
    k_frame_apply_src<<<(n_src + 255) / 256, 256, 0, s>>>(n_src, src, eo, tt);
    k_frame_apply_att<<<(G.n_coef + 255) / 256, 256, 0, s>>>(G, att, eo);
}

void launch_frame(const DevGeo& G, int n, const int32_t* subset, int n_src, double* src, const double* ref,
                  double* att, double* partial, int n_part, double tol, double* eo, cudaStream_t s) {
    const double tt = (double)(G.t_ep_ns - G.t_fr_ns) * 1e-9 / G.year_s;
    k_frame_normals<<<n_part, 256, 0, s>>>(n, subset, src, ref, tt, partial);
    k_frame_solve<<<1, 32, 0, s>>>(n_part, partial, tol, eo);
    k_frame_apply_src<<<(n_src + 255) / 256, 256, 0, s>>>(n_src, src, eo, tt);
    k_frame_apply_att<<<(G.n_coef + 255) / 256, 256, 0, s>>>(G, att, eo);
}

// ---------------------------------------------------------------------------------------
// Deterministic statistics of the S block, in two stages.
// out: [chi2, q, nu, nout, rankdef, d2 x5]
// ---------------------------------------------------------------------------------------
// Stage 1: block b reduces the sources of its fixed contiguous chunk into part[b][10];
// stage 2 (one block) adds the parts in block order, so the sums do not depend on timing.
constexpr int kStatBlocks = 304;
constexpr int kStatThreads = 256;
__global__ void __launch_bounds__(kStatThreads) k_src_stats_part(int n_src, const double* __restrict__ chi2,
                                                                 const double* __restrict__ q,
                                                                 const int* __restrict__ nu,
                                                                 const int* __restrict__ nout,
                                                                 const int* __restrict__ rdf,
                                                                 const double* __restrict__ d,
                                                                 double* __restrict__ part) {
    __shared__ double sh[kStatThreads];
    const int chunk = (n_src + gridDim.x - 1) / gridDim.x;
    const int lo = blockIdx.x * chunk, hi = min(n_src, lo + chunk);
    double acc[10];
    for (int k = 0; k < 10; k++) acc[k] = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        acc[0] += chi2[i];
        acc[1] += q[i];
        acc[2] += (double)nu[i];
        acc[3] += (double)nout[i];
        acc[4] += (double)rdf[i];
        for (int c = 0; c < 5; c++) acc[5 + c] += d[5 * (size_t)i + c] * d[5 * (size_t)i + c];
    }
    for (int k = 0; k < 10; k++) {
        sh[threadIdx.x] = acc[k];
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * 10 + k] = sh[0];
        __syncthreads();
    }
}
__global__ void __launch_bounds__(32) k_src_stats_final(int n_part, const double* __restrict__ part,
                                                        double* __restrict__ out) {
    // lane k < 10 adds statistic k over the parts in order
    if (threadIdx.x < 10) {
        double a = 0.0;
        for (int b = 0; b < n_part; b++) a += part[b * 10 + threadIdx.x];
        out[threadIdx.x] = a;
    }
}

// integer sum in a fixed order (rank defects of segments / calibration parameters)
__global__ void k_int_sum(int n, const int* __restrict__ v, long long* __restrict__ out) {
    __shared__ long long sh[1024];
    long long a = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a += v[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// out: 10 sums; part: kStatBlocks x 10 doubles of scratch
void launch_src_stats(int n_src, const double* chi2, const double* q, const int* nu, const int* nout, const int* rdf,
                      const double* d, double* out, double* part, cudaStream_t s) {
    k_src_stats_part<<<kStatBlocks, kStatThreads, 0, s>>>(n_src, chi2, q, nu, nout, rdf, d, part);
    k_src_stats_final<<<1, 32, 0, s>>>(kStatBlocks, part, out);
}

void launch_int_sum(int n, const int* v, long long* out, cudaStream_t s) { k_int_sum<<<1, 1024, 0, s>>>(n, v, out); }

}  // namespace agis
