// k_source_static.cu -- an S-block entry point that allocates no device memory.
//
// Some callers cannot allocate device memory: code running where the allocator is owned by
// someone else (a host framework with its own pool, or a process that has reserved all
// device memory up front).  agis_source_update_static() runs the same source update as
// agis_source_update() on caller-owned device arrays.  The only scratch it needs lives in
// the file-scope device array below: every GPU that loads this library keeps those 32 MiB
// until the process exits.
//
// Rules for callers:
//  * The first call on a device looks up the device address of the scratch array
//    (cudaGetSymbolAddress) with that device current.  Make that first call before any
//    stream capture on the device.
//  * All calls share the one array, and it keeps the contents of the last call.  Calls
//    whose kernels overlap on the GPU (different streams, or different host threads on the
//    same device) race on it and give wrong results: serialise them.
//  * Every call first checks its inputs on the device (source indices in range and sorted,
//    CCD, field and kind in range, sigma positive and finite, mu finite for AC, finite
//    parameters, at most max_obs_per_source observations per source) and reads the result
//    back before the compute kernel starts: on AGIS_E_INVALID no output has been written.
//    max_obs_per_source must not exceed AGIS_STATIC_MAX_OBS.
//  * Each call synchronises its stream before it returns (the check result and the
//    compute kernel's status are read back).
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "agis_internal.cuh"

namespace agis {
void set_thread_error(const std::string& msg);
}

namespace {

using namespace agis;

constexpr size_t kStaticBytes = (size_t)32 << 20;                 // 32 MiB
constexpr size_t kStaticDoubles = kStaticBytes / sizeof(double);

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];
static __device__ __align__(256) int g_static_ctrl[4];            // [0] work counter, [1] error flags

struct CcdRows {
    int32_t row[AGIS_N_CCD];
};

struct ObsPtrs {
    const int64_t* t_ns;
    const int32_t* src;
    const uint8_t* ccd;
    const uint8_t* fov;
    const uint8_t* kind;
    const float* sigma;
    const double* mu;
};

__device__ __forceinline__ int64_t lower_bound_src(const int32_t* src, int64_t n, int32_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (src[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint64_t skey(double x) {
    const long long b = __double_as_longlong(x);
    return b < 0 ? ~(uint64_t)b : ((uint64_t)b | 0x8000000000000000ull);
}
__device__ __forceinline__ double skey_inv(uint64_t k) {
    const long long b = (k & 0x8000000000000000ull) ? (long long)(k & 0x7fffffffffffffffull) : (long long)(~k);
    return __longlong_as_double(b);
}

// k-th smallest key of the slice (radix select with a 256-bin histogram per warp)
__device__ uint64_t s_select(const double* scr, int n, int k, int* hist, int lane) {
    uint64_t prefix = 0, pmask = 0;
    int kk = k;
    for (int d = 7; d >= 0; d--) {
        const int shift = 8 * d;
        for (int i = 0; i < 8; i++) hist[lane * 8 + i] = 0;
        __syncwarp();
        for (int j = lane; j < n; j += kWarp) {
            const uint64_t key = (uint64_t)__double_as_longlong(scr[(size_t)j * kScr + 6]);
            if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1);
        }
        __syncwarp();
        int c[8], tot = 0;
        for (int i = 0; i < 8; i++) { c[i] = hist[lane * 8 + i]; tot += c[i]; }
        int incl = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, incl > kk);
        const int sl = __ffs(ball) - 1;
        int bin = 0, below = 0;
        if (lane == sl) {
            int acc = incl - tot, bs = 7;
            for (int i = 0; i < 8; i++) {
                if (acc + c[i] > kk) { bs = i; break; }
                acc += c[i];
            }
            bin = lane * 8 + bs;
            below = acc;
        }
        bin = __shfl_sync(0xffffffffu, bin, sl);
        below = __shfl_sync(0xffffffffu, below, sl);
        kk -= below;
        prefix |= (uint64_t)bin << shift;
        pmask |= (uint64_t)0xffu << shift;
        __syncwarp();
    }
    return prefix;
}

__device__ void s_select_pair(const double* scr, int n, int k, int* hist, int lane, double& v0, double& v1) {
    const uint64_t K = s_select(scr, n, k, hist, lane);
    v0 = skey_inv(K);
    if (k + 1 >= n) { v1 = v0; return; }
    int less = 0, eq = 0;
    uint64_t nxt = ~0ull;
    for (int j = lane; j < n; j += kWarp) {
        const uint64_t key = (uint64_t)__double_as_longlong(scr[(size_t)j * kScr + 6]);
        less += key < K;
        eq += key == K;
        if (key > K && key < nxt) nxt = key;
    }
    less = warp_sum_int(less);
    eq = warp_sum_int(eq);
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t v = __shfl_xor_sync(0xffffffffu, nxt, o);
        nxt = v < nxt ? v : nxt;
    }
    v1 = (k + 1 < less + eq) ? v0 : skey_inv(nxt);
}

// normal equations with W = w / (sigma^2 + y), optionally refreshing w from the previous solve
__device__ void s_normals(double* scr, int n, int lane, double y, bool refresh, const double* dp, double yp, int wfn,
                          double* N, double* b, int& nout) {
    for (int i = 0; i < 15; i++) N[i] = 0.0;
    for (int i = 0; i < 5; i++) b[i] = 0.0;
    int cnt = 0;
    for (int j = lane; j < n; j += kWarp) {
        double* e = scr + (size_t)j * kScr;
        const double h = e[0];
        const double A[5] = {e[1], e[2], e[3], e[4], e[5]};
        double w = e[6];
        const double s2 = e[7];
        if (refresh) {
            const double R = h - (A[0] * dp[0] + A[1] * dp[1] + A[2] * dp[2] + A[3] * dp[3] + A[4] * dp[4]);
            w = wfun(R / sqrt(s2 + yp), wfn);
            e[6] = w;
        }
        cnt += (w < 0.2);
        const double W = w / (s2 + y);
        for (int a = 0; a < 5; a++) {
            const double wa = W * A[a];
            for (int c = a; c < 5; c++) N[up5(a, c)] += wa * A[c];
            b[a] += wa * h;
        }
    }
    for (int i = 0; i < 15; i++) N[i] = warp_sum(N[i]);
    for (int i = 0; i < 5; i++) b[i] = warp_sum(b[i]);
    nout = warp_sum_int(cnt);
}

__device__ void s_q(const double* scr, int n, int lane, const double* d, double y, double& Q, double& S2) {
    double q = 0.0, s = 0.0;
    for (int j = lane; j < n; j += kWarp) {
        const double* e = scr + (size_t)j * kScr;
        const double R = e[0] - (e[1] * d[0] + e[2] * d[1] + e[3] * d[2] + e[4] * d[3] + e[5] * d[4]);
        const double den = e[7] + y;
        const double t = e[6] * R * R / den;
        q += t;
        s += t / den;
    }
    Q = warp_sum(q);
    S2 = warp_sum(s);
}

// Input check before any output is written; bits of ctrl[1]: 1 a source with more than cap
// observations, 2 source index out of range, 4 sources not sorted, 8 CCD, field or kind out of
// range, 16 sigma not positive and finite, 32 non-finite mu of an AC observation, 64 a
// non-finite parameter (sources, attitude or calibration).  With sorted sources, observation o
// and observation o - cap belong to the same source exactly when that source has more than
// cap observations.
__global__ void k_static_check(int64_t n_obs, ObsPtrs ob, int32_t n_src, int cap, const double* __restrict__ src,
                               int64_t n_s, const double* __restrict__ att, int64_t n_a,
                               const double* __restrict__ cal, int64_t n_c, int* ctrl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bad = 0;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_obs; o += stride) {
        const int32_t s = ob.src[o];
        if (s < 0 || s >= n_src) bad |= 2;
        if (o > 0 && ob.src[o - 1] > s) bad |= 4;
        if (o >= cap && ob.src[o - cap] == s) bad |= 1;
        const int k = ob.kind[o];
        if (ob.ccd[o] >= AGIS_N_CCD || ob.fov[o] > 1 || k > 1) bad |= 8;
        const float sg = ob.sigma[o];
        if (!(sg > 0.0f) || !isfinite(sg)) bad |= 16;
        if (k == 1 && !isfinite(ob.mu[o])) bad |= 32;
    }
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_s + n_a + n_c; j += stride) {
        const double v = j < n_s ? src[j] : j < n_s + n_a ? att[j - n_s] : cal[j - n_s - n_a];
        if (!isfinite(v)) bad |= 64;
    }
    if (bad) atomicOr(&ctrl[1], bad);
}

// One warp per source: observation pass into the warp's slice of the static scratch, then the
// inner iteration of Sect. 5.1.2 (per-observation form) and the outputs.
__global__ void __launch_bounds__(128) k_source_static(DevGeo G, Settings st, ObsPtrs ob, int64_t n_obs,
                                                       int32_t n_src, CcdRows rows, int64_t cal_t0, int64_t cal_dt,
                                                       int32_t n_days, double* __restrict__ src,
                                                       const double* __restrict__ att, const double* __restrict__ cal,
                                                       double* __restrict__ R_out, double* __restrict__ W_out,
                                                       double* __restrict__ stats, int cap, double* scratch, int* ctrl) {
    __shared__ int hist_all[4 * 256];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int* hist = hist_all + wib * 256;
    const size_t gw = (size_t)blockIdx.x * (blockDim.x >> 5) + wib;
    double* scr = scratch + gw * (size_t)cap * kScr;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(&ctrl[0], 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= n_src) break;
        const int i = idx;
        const int64_t o0 = lower_bound_src(ob.src, n_obs, i);
        const int64_t o1 = lower_bound_src(ob.src, n_obs, i + 1);
        const int n = (int)(o1 - o0);
        if (n < 0 || n > cap) {   // excluded by k_static_check; kept as a guard
            if (lane == 0) atomicOr(&ctrl[1], n < 0 ? 4 : 1);
            continue;
        }
        double s5[5];
        for (int k = 0; k < 5; k++) s5[k] = src[5 * (size_t)i + k];
        if (n == 0) {
            if (lane == 0 && stats)
                for (int k = 0; k < 5; k++) stats[(size_t)k * n_src + i] = 0.0;
            continue;
        }
        SrcGeo S;
        source_geo(s5, S);
        double s2min = 1e300;
        for (int j = lane; j < n; j += kWarp) {
            const int64_t o = o0 + j;
            const int c = ob.ccd[o], f = ob.fov[o], k = ob.kind[o];
            const int64_t t = ob.t_ns[o];
            const int64_t rel = t - cal_t0;
            int64_t day = rel < 0 ? 0 : rel / cal_dt;
            if (day > n_days - 1) day = n_days - 1;
            const int64_t kcal = k == 0 ? (day * 2 + f) * AGIS_N_CCD + c
                                        : (int64_t)n_days * 124 + (day * 2 + f) * AGIS_N_ROW + rows.row[c];
            const uint32_t m = (uint32_t)(c & 63) | ((uint32_t)f << 6) | ((uint32_t)k << 7) | ((uint32_t)kcal << 8);
            ObsOut oo;
            observe<1>(G, S, t, m, k ? ob.mu[o] : 0.0, att, cal, oo);
            const double sg = (double)ob.sigma[o];
            double* e = scr + (size_t)j * kScr;
            e[0] = oo.R;
            e[1] = oo.A[0]; e[2] = oo.A[1]; e[3] = oo.A[2]; e[4] = oo.A[3]; e[5] = oo.A[4];
            e[6] = __longlong_as_double((long long)skey(oo.R / sg));
            e[7] = sg * sg;
            s2min = fmin(s2min, sg * sg);
        }
        s2min = warp_min(s2min);
        __syncwarp();
        if (st.robust) {
            const double p1 = 1.0 / 6.0, p5 = 5.0 / 6.0;
            const double h1 = p1 * (double)(n - 1), h5 = p5 * (double)(n - 1);
            const int lo1 = (int)floor(h1), lo5 = (int)floor(h5);
            double a0, a1, b0, b1;
            s_select_pair(scr, n, lo1, hist, lane, a0, a1);
            s_select_pair(scr, n, lo5, hist, lane, b0, b1);
            const double vs = 0.5 * ((b0 + (h5 - lo5) * (b1 - b0)) - (a0 + (h1 - lo1) * (a1 - a0)));
            __syncwarp();
            for (int j = lane; j < n; j += kWarp) {
                double* e = scr + (size_t)j * kScr;
                const double x = e[0] / sqrt(e[7]);
                e[6] = vs > 0.0 ? wfun(x / vs, st.weight_fn) : 1.0;
            }
        } else {
            for (int j = lane; j < n; j += kWarp) scr[(size_t)j * kScr + 6] = 1.0;
        }
        __syncwarp();
        double d[5] = {0, 0, 0, 0, 0}, U[kU5], N[15], b[5];
        double y = 0.0, Q = 0.0, Q0 = 0.0, S2 = 0.0;
        int nu = 0, nout = 0;
        const int rounds = st.robust ? st.n_rounds + 1 : 1;
        for (int rnd = 0; rnd < rounds; rnd++) {
            const double dprev[5] = {d[0], d[1], d[2], d[3], d[4]};
            const double yprev = y;
            y = 0.0;
            s_normals(scr, n, lane, 0.0, rnd > 0, dprev, yprev, st.weight_fn, N, b, nout);
            nu = n - nout - 5;
            chol5(N, U, st.pivot_tol);
            chol5_solve(U, b, d);
            s_q(scr, n, lane, d, 0.0, Q, S2);
            Q0 = Q;
            if (st.robust && nu > 0 && Q0 > (double)nu) {
                const double tol = 1e-12 * s2min;
                for (int it = 0; it < st.n_eps; it++) {
                    const double dy = (1.0 - Q / (double)nu) * Q / (-S2);
                    y = fmax(0.0, y + dy);
                    s_normals(scr, n, lane, y, false, dprev, yprev, st.weight_fn, N, b, nout);
                    chol5(N, U, st.pivot_tol);
                    chol5_solve(U, b, d);
                    s_q(scr, n, lane, d, y, Q, S2);
                    if (fabs(dy) <= tol) break;
                }
            }
            __syncwarp();
        }
        for (int j = lane; j < n; j += kWarp) {
            const double* e = scr + (size_t)j * kScr;
            const double R = e[0] - (e[1] * d[0] + e[2] * d[1] + e[3] * d[2] + e[4] * d[3] + e[5] * d[4]);
            if (R_out) R_out[o0 + j] = R;
            if (W_out) W_out[o0 + j] = e[6] / (e[7] + y);
        }
        if (lane == 0) {
            double* sp = src + 5 * (size_t)i;
            sp[0] = s5[0] + d[0] / S.cosd;
            sp[1] = s5[1] + d[1];
            sp[2] = s5[2] + d[2];
            sp[3] = s5[3] + d[3];
            sp[4] = s5[4] + d[4];
            if (stats) {
                stats[i] = y;
                stats[(size_t)n_src + i] = Q;
                stats[2 * (size_t)n_src + i] = (double)nu;
                stats[3 * (size_t)n_src + i] = (double)nout;
                stats[4 * (size_t)n_src + i] = nu > 0 ? (Q0 - (double)nu) / sqrt(2.0 * (double)nu) : 0.0;
            }
        }
        __syncwarp();
    }
}

std::mutex g_sym_mutex;
constexpr int kMaxDevices = 64;
void* g_sym_scratch[kMaxDevices] = {nullptr};
void* g_sym_ctrl[kMaxDevices] = {nullptr};

int err(int code, const std::string& msg) {
    set_thread_error(msg);
    return code;
}

}  // namespace

extern "C" int agis_source_update_static(const agis_geometry* geo, const agis_config* cfg, const agis_obs* obs,
                                         int64_t n_obs, double* src, int32_t n_src, const double* att,
                                         const double* cal, double* R_out, double* W_out, double* stats_out,
                                         int32_t max_obs_per_source, void* stream) {
    if (!geo || !cfg || !obs || !src || !att || !cal) return err(AGIS_E_INVALID, "null argument");
    if (n_obs < 0 || n_src < 0) return err(AGIS_E_INVALID, "negative size");
    if (n_obs > 0 && (!obs->t_ns || !obs->src || !obs->ccd || !obs->fov || !obs->kind || !obs->sigma || !obs->mu))
        return err(AGIS_E_INVALID, "null observation array");
    if (cfg->cal_model != 0)
        return err(AGIS_E_INVALID, "the static source update takes the r = 0 calibration offsets only (cal_model 0)");
    if (max_obs_per_source < 1 || max_obs_per_source > AGIS_STATIC_MAX_OBS)
        return err(AGIS_E_INVALID, "max_obs_per_source must be in 1..AGIS_STATIC_MAX_OBS (" +
                                       std::to_string(AGIS_STATIC_MAX_OBS) + ")");
    if (geo->n_coef < 4 || geo->knot_dt_ns <= 0 || geo->cal_dt_ns <= 0 || geo->n_cal_days < 1 ||
        !(geo->year_s > 0) || !(geo->focal_length > 0))
        return err(AGIS_E_INVALID, "bad geometry");
    for (int k = 0; k < AGIS_N_CCD; k++)
        if (geo->ccd_row[k] < 0 || geo->ccd_row[k] >= AGIS_N_ROW) return err(AGIS_E_INVALID, "bad ccd_row");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return err(AGIS_E_CUDA, "cudaGetDevice failed");
    void* scratch = nullptr;
    void* ctrl = nullptr;
    {
        // set-up once per device, with that device current: device addresses of the arrays
        std::lock_guard<std::mutex> lock(g_sym_mutex);
        if (!g_sym_scratch[dev]) {
            void* p = nullptr;
            void* q = nullptr;
            cudaError_t e1 = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e1 != cudaSuccess) return err(AGIS_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e1));
            cudaError_t e2 = cudaGetSymbolAddress(&q, g_static_ctrl);
            if (e2 != cudaSuccess) return err(AGIS_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e2));
            g_sym_scratch[dev] = p;
            g_sym_ctrl[dev] = q;
        }
        scratch = g_sym_scratch[dev];
        ctrl = g_sym_ctrl[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    DevGeo G;
    fill_devgeo(geo, geo->n_coef, G);
    Settings st;
    st.robust = cfg->robust;
    st.n_rounds = cfg->n_rounds;
    st.n_eps = cfg->n_eps;
    st.weight_fn = cfg->weight_fn;
    st.lambda2 = cfg->lambda_att * cfg->lambda_att;
    st.rhs_norm_term = cfg->rhs_norm_term;
    st.pivot_tol = cfg->pivot_tol;
    CcdRows rows;
    for (int k = 0; k < AGIS_N_CCD; k++) rows.row[k] = geo->ccd_row[k];
    ObsPtrs op{obs->t_ns, obs->src, obs->ccd, obs->fov, obs->kind, obs->sigma, obs->mu};
    // as many warps as slices of max_obs_per_source rows fit in the array
    const int cap = max_obs_per_source;
    int n_warps = (int)(kStaticDoubles / ((size_t)cap * kScr));
    if (n_warps > 152 * 16) n_warps = 152 * 16;
    const int blocks = n_warps / 4;
    if (blocks < 1) return err(AGIS_E_INVALID, "max_obs_per_source too large for the static scratch");
    cudaError_t e = cudaMemsetAsync(ctrl, 0, 4 * sizeof(int), s);
    if (e != cudaSuccess) return err(AGIS_E_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    // inputs first, read back before anything is written
    int flags[4] = {0, 0, 0, 0};
    {
        const int64_t n_s = 5 * (int64_t)n_src, n_a = 4 * (int64_t)geo->n_coef,
                      n_c = (int64_t)geo->n_cal_days * (2 * (AGIS_N_CCD + AGIS_N_ROW));
        const int64_t work = n_obs > n_s + n_a + n_c ? n_obs : n_s + n_a + n_c;
        int64_t nb = (work + 255) / 256;
        if (nb > 152 * 8) nb = 152 * 8;
        if (nb < 1) nb = 1;
        k_static_check<<<(int)nb, 256, 0, s>>>(n_obs, op, n_src, max_obs_per_source, src, n_s, att, n_a, cal, n_c,
                                               (int*)ctrl);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(flags, ctrl, sizeof(flags), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return err(AGIS_E_CUDA, std::string("input check: ") + cudaGetErrorString(e));
        const int b = flags[1];
        if (b & 2) return err(AGIS_E_INVALID, "source index out of range");
        if (b & 4) return err(AGIS_E_INVALID, "observations not sorted by source");
        if (b & 8) return err(AGIS_E_INVALID, "ccd, fov or kind out of range");
        if (b & 16) return err(AGIS_E_INVALID, "sigma must be positive and finite");
        if (b & 32) return err(AGIS_E_INVALID, "non-finite mu of an AC observation");
        if (b & 64) return err(AGIS_E_INVALID, "non-finite source, attitude or calibration parameter");
        if (b & 1) return err(AGIS_E_INVALID, "a source has more observations than max_obs_per_source");
    }
    if (n_src > 0)
        k_source_static<<<blocks, 128, 0, s>>>(G, st, op, n_obs, n_src, rows, geo->cal_t0_ns, geo->cal_dt_ns,
                                               geo->n_cal_days, src, att, cal, R_out, W_out, stats_out, cap,
                                               (double*)scratch, (int*)ctrl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return err(AGIS_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    e = cudaMemcpyAsync(flags, ctrl, sizeof(flags), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return err(AGIS_E_CUDA, std::string("static source update: ") + cudaGetErrorString(e));
    if (flags[1] & 1) return err(AGIS_E_INVALID, "a source has more observations than max_obs_per_source");
    return AGIS_OK;
}
