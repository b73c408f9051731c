// agis_api.cu -- the C ABI of include/agis.h: context, device memory, set-up of the
// orderings (source, time / knot interval, calibration parameter) and the block calls.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "agis_internal.cuh"

namespace agis {
void launch_obs_pass(const DevGeo& G, const AttNoise& an, const int64_t* t_ns, const uint32_t* meta, const float* sigma,
                     const double* mu, const int32_t* obs_src, int64_t n_obs, int32_t n_src, const double* src,
                     const double* att, const double* cal, ObsRec* rec, double* geo, double* scratch, uint64_t* skey,
                     const Shapes& sh, cudaStream_t stream);
void launch_source_solve(const Settings& st, const uint32_t* meta, const int64_t* src_off, const int32_t* src_nal,
                         const int32_t* src_order, int32_t n_src, const SrcOutPtrs& out, ObsRec* rec, double* scratch,
                         const uint64_t* skey, int* work_counter, int n_blocks, const Shapes& sh, cudaStream_t stream);
void launch_evaluate(const DevGeo& G, const int64_t* t_ns, const uint32_t* meta, const double* mu,
                     const int32_t* obs_src, int64_t n_obs, const double* src, const double* att, const double* cal,
                     double* R, cudaStream_t stream);
void launch_att_accum(const DevGeo& G, double lambda2, int rhs_norm, const uint32_t* perm_t, const int64_t* ivl_off,
                      int n_iv, const ObsRec* rec, const double* w_att, const double* att, double* blk,
                      const Shapes& sh, cudaStream_t s);
void launch_att_solve(int n_seg, int max_seg_knots, int n_coef, int64_t n_rows, const int64_t* seg_row, const int32_t* seg_l,
                      const int32_t* seg_n, const int32_t* seg_u, const double* blk, double* bandc, double* rhs,
                      double* urow, double* yv, double* x, double tol, int* seg_rd, double* att, float* d_att,
                      double* dx, cudaStream_t s);
void launch_rec_att_correct(const DevGeo& G, int64_t n_obs, ObsRec* rec, const double* dx, cudaStream_t s);
void launch_mix_ac_correct(const DevGeo& G, int64_t n_obs, const MixObs& mo, const float* d_att, cudaStream_t s);
void launch_mix_pass(const DevGeo& G, bool refresh, const int64_t* t_ns, const uint32_t* meta, const float* sigma,
                     const double* mu, const int32_t* obs_src, int64_t n_obs, int32_t n_src, const double* src,
                     const double* att, const double* cal, const MixObs& mo, double* geo, float* d_att,
                     float2* d_cal, int n_coef, int n_cal, const Shapes& sh, cudaStream_t s);
void launch_mix_solve(const Settings& st, const int64_t* src_off, const int32_t* src_nal, const int32_t* src_order,
                      int32_t n_src, const SrcOutPtrs& out, const MixObs& mo, const MixSrcWork& w,
                      const Shapes& sh, cudaStream_t s);
void launch_mix_att_accum(const DevGeo& G, double lambda2, int rhs_norm, const uint32_t* perm_t,
                          const int64_t* ivl_off, int n_iv, const MixObs& mo, const double* att, double* blk,
                          const Shapes& sh, cudaStream_t s);
void launch_mix_cal(int n_cal, int n_days, const uint32_t* perm_c, const int64_t* cal_off, const MixObs& mo,
                    double* dtil, int* rd, double* cal, float2* d_cal, const Shapes& sh, cudaStream_t s);
void launch_mix_rw(int64_t n, const uint32_t* perm, const MixObs& mo, double* R, double* W, cudaStream_t s);
void launch_mix_prop(int32_t n_src, const int64_t* src_off, const MixObs& mo, const double* corr, cudaStream_t s);
void launch_hist_push(int32_t n_src, const double* d, double* hist, cudaStream_t s);
void launch_prop_features(int32_t n_src, const double* hist, const int64_t* src_off, const double* src,
                          double sin_obl, double cos_obl, float* X, double* sigma, cudaStream_t s);
void launch_mlp_forward(const void* packed, const float* X, int n, float* Y, cudaStream_t s);
void launch_prop_apply(int32_t n_src, const float* Y, const double* sigma, double* src, double* corr,
                       cudaStream_t s);
void launch_prop_rec(int32_t n_src, const int64_t* src_off, const double* scratch, ObsRec* rec, const double* corr,
                     cudaStream_t s);
void launch_asi(int32_t n_src, int32_t stride, const double* hist, double lam_max, unsigned long long* keys,
                double* est, const double* d, double* src, double* corr, cudaStream_t s);
void launch_calgen(const DevGeo& G, int64_t n_groups, const ObsRec* rec, const double* mu, const CalGenWork& w,
                   double tol, double* cal, cudaStream_t s);
int calgen_prepare();
void launch_cal_sums(int n_cal, const uint32_t* perm_c, const int64_t* cal_off, const ObsRec* rec, double* sums,
                     const Shapes& sh, cudaStream_t s);
void launch_cal_from_sums(int n_cal, int n_days, const double* sums, double tol, double* dtil, int* rd, double* cal,
                          cudaStream_t s);
void launch_frame_sums(int n, const int32_t* subset, const double* src, const double* ref, const DevGeo& G,
                       double* partial, int n_part, double* sums, cudaStream_t s);
void launch_frame_from_sums(const DevGeo& G, int n_src, double* src, double* att, const double* sums, double tol,
                            double* eo, cudaStream_t s);
void launch_cal(int n_cal, int n_days, const uint32_t* perm_c, const int64_t* cal_off, const ObsRec* rec, double tol,
                double* dtil, int* rd, double* cal, const Shapes& sh, cudaStream_t s);
void launch_frame(const DevGeo& G, int n, const int32_t* subset, int n_src, double* src, const double* ref,
                  double* att, double* partial, int n_part, double tol, double* eo, cudaStream_t s);
void launch_src_stats(int n_src, const double* chi2, const double* q, const int* nu, const int* nout, const int* rdf,
                      const double* d, double* out, double* part, cudaStream_t s);
void launch_int_sum(int n, const int* v, long long* out, cudaStream_t s);
void launch_an_range(int64_t n, const int64_t* t, int64_t t0, unsigned long long* mx, int* neg, cudaStream_t s);
void launch_an_keys(int64_t n, const int64_t* t, const uint32_t* meta, const AttNoise& an, int32_t* key, uint32_t* val,
                    cudaStream_t s);
void launch_an_estimate(int64_t n, const AttNoise& an, int64_t max_run, double* eps2, const uint32_t* perm,
                        const int64_t* off, const ObsRec* rec, const float* sigma, const int32_t* obs_src,
                        const double* eps2_src, int weight_fn, uint64_t* xkey, double* w_att, cudaStream_t s);
void launch_an_estimate_mix(int64_t n, const AttNoise& an, int64_t max_run, double* eps2, const uint32_t* perm,
                            const int64_t* off, const int64_t* t_ns, const uint32_t* meta, const float2* mr,
                            const float* sigma, const int32_t* obs_src, const double* eps2_src, int weight_fn,
                            uint64_t* xkey, float2* ac_att, cudaStream_t s);
void launch_an_sigma_mix(int64_t n, const AttNoise& an, const int64_t* t_ns, const uint32_t* meta, const float* sigma,
                         MixS* ms, cudaStream_t s);
}  // namespace agis

using namespace agis;

// -----------------------------------------------------------------------------------------
// set-up kernels
// -----------------------------------------------------------------------------------------
namespace {

// gate: per observation (full calibration model, n_gate > 0) or NULL
__global__ void k_validate_pack(int64_t n, const int64_t* __restrict__ t, const int32_t* __restrict__ src,
                                const uint8_t* __restrict__ ccd, const uint8_t* __restrict__ fov,
                                const uint8_t* __restrict__ kind, const float* __restrict__ sigma,
                                const double* __restrict__ mu, int32_t n_src, int64_t cal_t0, int64_t cal_dt,
                                int32_t n_days, const int32_t* __restrict__ ccd_row, const uint8_t* __restrict__ gate,
                                int n_gate, uint32_t* __restrict__ meta, int* __restrict__ err) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = src[o];
        const int c = ccd[o], f = fov[o], k = kind[o];
        const float sg = sigma[o];
        int bad = 0;
        if (s < 0 || s >= n_src) bad |= 1;
        if (o > 0 && src[o - 1] > s) bad |= 2;
        if (c >= AGIS_N_CCD || f > 1 || k > 1) bad |= 4;
        if (!(sg > 0.0f) || !isfinite(sg)) bad |= 8;
        if ((k == 1 || n_gate > 0) && !isfinite(mu[o])) bad |= 16;
        const int gt = gate ? gate[o] : 0;
        if (n_gate > 0 && gt >= n_gate) bad |= 64;
        if (bad) atomicOr(err, bad);
        if (n_gate > 0) {
            meta[o] = (uint32_t)(c & 63) | ((uint32_t)f << 6) | ((uint32_t)k << 7) | ((uint32_t)gt << 8);
            continue;
        }
        const int64_t rel = t[o] - cal_t0;
        int64_t day = rel < 0 ? 0 : rel / cal_dt;
        if (day > n_days - 1) day = n_days - 1;
        const int64_t kcal = k == 0 ? (day * 2 + f) * AGIS_N_CCD + c
                                    : (int64_t)n_days * 124 + (day * 2 + f) * AGIS_N_ROW + ccd_row[c < AGIS_N_CCD ? c : 0];
        meta[o] = (uint32_t)(c & 63) | ((uint32_t)f << 6) | ((uint32_t)k << 7) | ((uint32_t)kcal << 8);
    }
}

// internal order: by source, AL before AC within a source (key 2 src + kind, stable sort)
__global__ void k_class_keys(int64_t n, const int32_t* __restrict__ src, const uint8_t* __restrict__ kind,
                             int32_t* __restrict__ key, uint32_t* __restrict__ val) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        key[o] = 2 * src[o] + (kind[o] ? 1 : 0);
        val[o] = (uint32_t)o;
    }
}

// out[o] = in[perm[o]]: the caller's order to the internal order, one array at a time
template <typename T>
__global__ void k_gather(int64_t n, const uint32_t* __restrict__ perm, const T* __restrict__ in, T* __restrict__ out) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x)
        out[o] = in[perm[o]];
}
__global__ void k_gather_mu(int64_t n, const uint32_t* __restrict__ perm, const uint32_t* __restrict__ meta,
                            const double* __restrict__ in, double* __restrict__ out, int all) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x)
        out[o] = (all || meta_kind(meta[o])) ? in[perm[o]] : 0.0;
}

// full calibration model: C-block order keys, AL observations by (cell, bin) with the cell
// (n, g, j) = group * j_per_k + j within k, then AC observations by group
__global__ void k_calgen_keys(DevGeo G, int64_t n, const int64_t* __restrict__ t, const uint32_t* __restrict__ meta,
                              const double* __restrict__ mu, int64_t n_cells, int32_t* __restrict__ key,
                              uint32_t* __restrict__ val) {
    const CalGen& C = G.cg;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t m = meta[o];
        const CalPos p = cal_position(C, t[o], m, mu[o]);
        key[o] = meta_kind(m) == 0 ? (int32_t)((p.grp * C.j_per_k + p.jj) * C.n_bin + p.bin)
                                   : (int32_t)(n_cells * C.n_bin + p.grp);
        val[o] = (uint32_t)o;
    }
}
// offsets of the AL cells (key c * n_bin) and of the AC groups (key n_cells * n_bin + g)
__global__ void k_calgen_off(const int32_t* __restrict__ keys, int64_t n, int64_t n_cells, int64_t n_groups, int nb,
                             int64_t* __restrict__ out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n_cells + n_groups;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = v <= n_cells ? v * nb : n_cells * nb + (v - n_cells);
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)keys[mid] < x) lo = mid + 1; else hi = mid;
        }
        out[v] = lo;
    }
}

// out[perm[o]] = in[o]: internal order back to the caller's order
__global__ void k_scatter(int64_t n, const uint32_t* __restrict__ perm, const double* __restrict__ in,
                          double* __restrict__ out) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x)
        out[perm[o]] = in[o];
}

// AL observations of each source from the offsets of the (source, kind) groups
__global__ void k_src_nal(int32_t n_src, const int64_t* __restrict__ goff, int32_t* __restrict__ nal) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += gridDim.x * blockDim.x)
        nal[i] = (int32_t)(goff[2 * (size_t)i + 1] - goff[2 * (size_t)i]);
}

__global__ void k_check_finite(int64_t n, const double* __restrict__ v, int* __restrict__ err, int code) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) atomicOr(err, code);
}

// first index with key >= v in a sorted array (one thread per v)
template <typename K>
__global__ void k_lower_bound(const K* __restrict__ keys, int64_t n, int64_t n_out, int64_t* __restrict__ out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_out; v += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if ((int64_t)keys[mid] < v) lo = mid + 1; else hi = mid;
        }
        out[v] = lo;
    }
}

__global__ void k_interval_keys(DevGeo G, int64_t n, const int64_t* __restrict__ t, int32_t* __restrict__ key,
                                uint32_t* __restrict__ val) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        key[o] = left_index(G, t[o]) - 3;
        val[o] = (uint32_t)o;
    }
}

__global__ void k_cal_keys(int64_t n, const uint32_t* __restrict__ meta, int32_t* __restrict__ key,
                           uint32_t* __restrict__ val) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        key[o] = (int32_t)meta_cal(meta[o]);
        val[o] = (uint32_t)o;
    }
}

__global__ void k_src_counts(int32_t n_src, const int64_t* __restrict__ off, int32_t* __restrict__ negcount,
                             int32_t* __restrict__ idx) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += gridDim.x * blockDim.x) {
        negcount[i] = -(int32_t)(off[i + 1] - off[i]);
        idx[i] = i;
    }
}

__global__ void k_rec_rw(int64_t n, const uint32_t* __restrict__ perm, const ObsRec* __restrict__ rec,
                         double* __restrict__ R, double* __restrict__ W) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        if (R) R[perm[o]] = rec[o].R;
        if (W) W[perm[o]] = rec[o].W;
    }
}

__global__ void k_src_stats_out(int32_t n_src, const double* __restrict__ eps2, const double* __restrict__ q,
                                const int* __restrict__ nu, const int* __restrict__ nout,
                                const double* __restrict__ dsig, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += gridDim.x * blockDim.x) {
        out[i] = eps2[i];
        out[(size_t)n_src + i] = q[i];
        out[2 * (size_t)n_src + i] = (double)nu[i];
        out[3 * (size_t)n_src + i] = (double)nout[i];
        out[4 * (size_t)n_src + i] = dsig[i];
    }
}

int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

// -----------------------------------------------------------------------------------------
// context
// -----------------------------------------------------------------------------------------
struct agis_ctx {
    std::string err;
    agis_geometry geo;
    agis_config cfg;
    DevGeo G;
    Settings st;
    cudaStream_t stream = nullptr;
    int device = 0;
    int n_sm = 152;
    int64_t n_obs = 0;
    int32_t n_src = 0, n_coef = 0, n_cal = 0, n_days = 0;
    std::vector<void*> allocs;
    // observations (source order)
    int64_t* t_ns = nullptr;
    uint32_t* meta = nullptr;
    float* sigma = nullptr;
    double* mu = nullptr;
    int32_t* obs_src = nullptr;
    uint32_t* perm_in = nullptr;  // internal observation -> index in the caller's arrays
    int32_t* src_nal = nullptr;   // AL observations of each source (they come first)
    int64_t* src_off = nullptr;
    int32_t* src_order = nullptr;
    // state
    double* src = nullptr;
    double* ref = nullptr;
    double* att = nullptr;
    double* cal = nullptr;
    // S block
    ObsRec* rec = nullptr;
    // mixed-precision form: records, updates since the last S block, refresh bookkeeping
    bool mixed = false;
    MixObs mo{};
    float* d_att = nullptr;
    double* datt64 = nullptr;     // FP64 form, block Gauss-Seidel: this iteration's attitude update
    float2* d_cal = nullptr;
    MixSrcWork mw{};
    bool mix_stale = true;   // the records do not describe the current state: evaluate in full
    int mix_since = 0;       // source updates since the last full evaluation
    double* scratch = nullptr;   // n_obs x 8 doubles, source order
    uint64_t* skey = nullptr;    // n_obs sort keys of h / sigma (the robust scale's selects), source order
    double* sgeo = nullptr;      // n_src x 16
    int cap = 0, n_sblocks = 0;
    int* work = nullptr;
    SrcOutPtrs so{};
    double* sstats = nullptr;     // 10
    double* sstat_part = nullptr; // 304 x 10 partial sums of the source statistics
    // A block
    uint32_t* perm_t = nullptr;
    int64_t* ivl_off = nullptr;
    int n_iv = 0;
    double* blk = nullptr;
    int n_seg = 0;
    int max_seg_knots = 0;   // the largest segment's coefficients (band rows / 4)
    int64_t n_rows = 0;
    int64_t* seg_row = nullptr;
    int32_t *seg_l = nullptr, *seg_n = nullptr, *seg_u = nullptr;
    double *bandc = nullptr, *rhs = nullptr, *urow = nullptr, *yv = nullptr, *xs = nullptr;
    int* seg_rd = nullptr;
    long long* isum = nullptr;    // [0] A rank defect, [1] C rank defect
    // C block (full calibration model: its own order, offsets and work arrays)
    bool cal_generic = false;
    int64_t cg_groups = 0;
    CalGenWork cgw{};
    uint32_t* perm_c = nullptr;
    int64_t* cal_off = nullptr;
    double* dtil = nullptr;
    int* cal_rd = nullptr;
    // exchange buffers of a source partition: calibration sums (2 per parameter), frame sums
    // (27); the attitude's are the interval blocks blk
    double* xcal = nullptr;
    double* xframe = nullptr;
    bool x_att_ready = false, x_cal_ready = false, x_frame_ready = false;
    // frame rotator
    double* fpart = nullptr;
    int n_fpart = 0;
    double* eo = nullptr;
    int32_t* subset = nullptr;
    int32_t subset_cap = 0;
    double* evalR = nullptr;
    double* tmpR = nullptr;
    double* tmpW = nullptr;
    // host read-back (pinned)
    double* hstat = nullptr;      // 10 S, 6 frame at 16, 4 ASI estimate at 24
    long long* hisum = nullptr;   // 2
    bool have_s = false;
    bool have_s_out = false;    // the S block's hand-over (R, W) exists and no state was set since
    bool a_since_c = false;     // an A update not yet seen by a C update (block Gauss-Seidel)
    // events 0-13 on the stream; 14, 15 the C block's start and end on the second stream
    static constexpr int kEvents = 16;
    cudaEvent_t ev[kEvents];
    cudaStream_t stream_c = nullptr;   // the C block beside the A block (S[AC] and [SAC] orders)
    double ktimes[5] = {0, 0, 0, 0, 0};
    // per-block graphs: 0 S observation pass (FP64 model, or the mixed form's linearized
    // correction), 1 A, 2 C, 3 frame, 4 mixed S pass with the full FP64 model, 5 S solves,
    // 6 learned proposal, 7 ASI extrapolation
    static constexpr int kGraphs = 8;
    cudaGraphExec_t graph_execs[kGraphs] = {};
    cudaGraph_t graphs[kGraphs] = {};
    // learned proposal: the last four source updates, the network, the state before the
    // iteration that carries a proposal (for the rollback)
    double* hist = nullptr;         // n_src x 4 x 5, oldest first
    int hist_count = 0;             // source updates since agis_init / the last agis_set_*
    void* prop_packed = nullptr;
    float* prop_params = nullptr;
    float* prop_X = nullptr;
    float* prop_Y = nullptr;
    double* prop_sigma = nullptr;
    double* prop_corr = nullptr;    // correction in tangent units (proposal or ASI)
    int prop_every = 0;
    int since_prop = 1 << 30;
    bool prop_pending = false;
    double chi2_before_prop = 0.0;
    double *snap_src = nullptr, *snap_att = nullptr, *snap_cal = nullptr, *snap_hist = nullptr;
    int snap_hist_count = 0;
    // accelerated simple iteration: sample stride (0 off), clamp of lambda, the sample's keys
    // and the estimate [median, lambda, factor, count]
    int asi_stride = 0;
    double asi_lam_max = 0.9;
    unsigned long long* asi_keys = nullptr;
    double* asi_est = nullptr;
    // excess attitude noise (FP64 form; an.eps2 null: off): bucket length, eps_a^2 [3 x n_b],
    // the (component, bucket) order and its run offsets, the x_l keys in that order, and the
    // attitude weights (source order)
    int64_t an_bucket_ns = 0;
    int64_t an_max_run = 0;         // observations in the longest (component, bucket) run
    AttNoise an;
    double* an_eps2 = nullptr;
    uint32_t* an_perm = nullptr;
    int64_t* an_off = nullptr;
    uint64_t* an_x = nullptr;
    double* an_w = nullptr;
    // launch shapes (defaults until agis_autotune or agis_set_tuning)
    Shapes sh;
    bool graphs_ready = false;
    bool own_stream = false;
    double* tmpS = nullptr;
};

namespace {

int fail(agis_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_check(agis_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return AGIS_OK;
    if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? AGIS_E_OOM : AGIS_E_CUDA;
}

template <typename T>
int dalloc(agis_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaMalloc");
    c->allocs.push_back(q);
    *p = (T*)q;
    return AGIS_OK;
}

// frees an array of dalloc before agis_destroy
void dfree(agis_ctx* c, void* p) {
    if (!p) return;
    for (size_t i = 0; i < c->allocs.size(); i++)
        if (c->allocs[i] == p) {
            c->allocs.erase(c->allocs.begin() + (long)i);
            cudaFree(p);
            return;
        }
}

// device temporary of the set-up, freed at the end of its scope
struct TmpDev {
    void* p = nullptr;
    ~TmpDev() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
    }
    template <typename T>
    int alloc(agis_ctx* c, T** out, size_t count) {
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return cuda_check(c, e, "cudaMalloc (set-up)");
        *out = (T*)p;
        return AGIS_OK;
    }
};

#define AGIS_TRY(x)                    \
    do {                               \
        int _r = (x);                  \
        if (_r != AGIS_OK) return _r;  \
    } while (0)
#define AGIS_CU(c, x, what) AGIS_TRY(cuda_check((c), (x), (what)))

// radix sort of (key, value) pairs, stable: the order within equal keys is the source order
int sort_pairs(agis_ctx* c, int32_t* keys_in, int32_t* keys_out, uint32_t* vals_in, uint32_t* vals_out, int64_t n,
               int end_bit) {
    size_t tmp_bytes = 0;
    AGIS_CU(c, cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys_in, keys_out, vals_in, vals_out, n, 0, end_bit,
                                               c->stream),
            "cub sort (size)");
    void* tmp = nullptr;
    AGIS_CU(c, cudaMalloc(&tmp, tmp_bytes + 16), "cudaMalloc (sort)");
    cudaError_t e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys_in, keys_out, vals_in, vals_out, n, 0,
                                                    end_bit, c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    AGIS_CU(c, e, "cub sort");
    AGIS_CU(c, e2, "cub sort (sync)");
    return AGIS_OK;
}

int bits_for(int64_t v) {
    int b = 1;
    while (b < 31 && ((int64_t)1 << b) <= v) b++;
    return b;
}

// overlapping attitude segments of Sect. 5.2.2 (same construction as the paper: cross-over
// knots every seg_len intervals, 2L overlapping intervals, segment K updates a_n up to
// n = x - floor(M/2))
void build_segments(int n_coef, int seg_len, int L, std::vector<int32_t>& sl, std::vector<int32_t>& sn,
                    std::vector<int32_t>& su, std::vector<int64_t>& srow) {
    const int M = 4;
    const int K = n_coef - M + 1;
    const int S = seg_len;
    const int nseg = std::max(1, (K + S - 1) / S);
    srow.push_back(0);
    for (int k = 0; k < nseg; k++) {
        const int x0 = (M - 1) + k * S, x1 = (M - 1) + (k + 1) * S;
        const int l_lo = std::max(M - 1, x0 - L);
        const int l_hi = std::min(n_coef - 1, x1 + L - 1);
        const int u_lo = k == 0 ? 0 : x0 - M / 2 + 1;
        const int u_hi = k == nseg - 1 ? n_coef - 1 : x1 - M / 2;
        sl.push_back(l_lo); sl.push_back(l_hi);
        sn.push_back(l_lo - (M - 1)); sn.push_back(l_hi);
        su.push_back(u_lo); su.push_back(u_hi);
        srow.push_back(srow.back() + 4 * (int64_t)(l_hi - (l_lo - (M - 1)) + 1));
    }
}

void record(agis_ctx* c, int i) { cudaEventRecord(c->ev[i], c->stream); }
double elapsed(agis_ctx* c, int a, int b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1.0;
    }
    return ms;
}

// --- the block sequences (enqueue only; no host synchronisation) ---------------------------
// mixed form: does the next source update start with a full FP64 evaluation?
bool s_refresh_due(const agis_ctx* c) {
    return c->mixed && (c->mix_stale || c->mix_since >= c->cfg.refresh_every);
}
void s_done(agis_ctx* c, bool refresh) {
    if (!c->mixed) return;
    c->mix_stale = false;
    c->mix_since = refresh ? 1 : c->mix_since + 1;
}

// S block in two parts: the observation pass (timed separately) and the per-source solves
void enqueue_s_pass(agis_ctx* c, bool refresh) {
    if (c->mixed) {
        launch_mix_pass(c->G, refresh, c->t_ns, c->meta, c->sigma, c->mu, c->obs_src, c->n_obs, c->n_src, c->src,
                        c->att, c->cal, c->mo, c->sgeo, c->d_att, c->d_cal, c->n_coef, c->n_cal, c->sh,
                        c->stream);
        // excess attitude noise: sigma~ of the previous estimate into the records (Eq. W)
        if (c->an.eps2) launch_an_sigma_mix(c->n_obs, c->an, c->t_ns, c->meta, c->sigma, c->mo.s, c->stream);
    } else
        launch_obs_pass(c->G, c->an, c->t_ns, c->meta, c->sigma, c->mu, c->obs_src, c->n_obs, c->n_src, c->src, c->att,
                        c->cal, c->rec, c->sgeo, c->scratch, c->skey, c->sh, c->stream);
}
void enqueue_s_solve(agis_ctx* c) {
    if (c->mixed)
        launch_mix_solve(c->st, c->src_off, c->src_nal, c->src_order, c->n_src, c->so, c->mo, c->mw, c->sh,
                         c->stream);
    else
        launch_source_solve(c->st, c->meta, c->src_off, c->src_nal, c->src_order, c->n_src, c->so, c->rec, c->scratch,
                            c->skey, c->work, c->n_sblocks, c->sh, c->stream);
    // excess attitude noise from the residuals of this source update, and the attitude weights
    if (c->an.eps2 && c->mixed)
        launch_an_estimate_mix(c->n_obs, c->an, c->an_max_run, c->an_eps2, c->an_perm, c->an_off, c->t_ns, c->meta,
                               c->mo.r, c->sigma, c->obs_src, c->so.eps2, c->st.weight_fn, c->an_x,
                               reinterpret_cast<float2*>(c->an_w), c->stream);
    else if (c->an.eps2)
        launch_an_estimate(c->n_obs, c->an, c->an_max_run, c->an_eps2, c->an_perm, c->an_off, c->rec, c->sigma,
                           c->obs_src, c->so.eps2, c->st.weight_fn, c->an_x, c->an_w, c->stream);
    launch_src_stats(c->n_src, c->so.chi2, c->so.q, c->so.nu, c->so.nout, c->so.rankdef, c->so.d, c->sstats,
                     c->sstat_part, c->stream);
    launch_hist_push(c->n_src, c->so.d, c->hist, c->stream);
    // block Gauss-Seidel, FP64 form: the attitude update C will see is this iteration's (none
    // until an A block runs)
    if (c->datt64) cudaMemsetAsync(c->datt64, 0, sizeof(double) * 4 * (size_t)c->n_coef, c->stream);
}
// learned proposal after the S block: features, network, sources += correction, and the
// residuals that A and C read -= A correction
void enqueue_proposal(agis_ctx* c) {
    launch_prop_features(c->n_src, c->hist, c->src_off, c->src, c->G.sin_obl, c->G.cos_obl, c->prop_X,
                         c->prop_sigma, c->stream);
    launch_mlp_forward(c->prop_packed, c->prop_X, c->n_src, c->prop_Y, c->stream);
    launch_prop_apply(c->n_src, c->prop_Y, c->prop_sigma, c->src, c->prop_corr, c->stream);
    if (c->mixed)
        launch_mix_prop(c->n_src, c->src_off, c->mo, c->prop_corr, c->stream);
    else
        launch_prop_rec(c->n_src, c->src_off, c->scratch, c->rec, c->prop_corr, c->stream);
}
// ASI after the S block: lambda from the sample's parallax-update ratios, sources +=
// (f - 1) d, and the residuals that A and C read -= A (f - 1) d
void enqueue_asi(agis_ctx* c) {
    launch_asi(c->n_src, c->asi_stride, c->hist, c->asi_lam_max, c->asi_keys, c->asi_est, c->so.d, c->src,
               c->prop_corr, c->stream);
    if (c->mixed)
        launch_mix_prop(c->n_src, c->src_off, c->mo, c->prop_corr, c->stream);
    else
        launch_prop_rec(c->n_src, c->src_off, c->scratch, c->rec, c->prop_corr, c->stream);
}
void enqueue_a(agis_ctx* c) {
    if (c->mixed) {
        // with the excess attitude noise the attitude update reads its own (W, W R) pairs
        MixObs mo = c->mo;
        if (c->an.eps2) mo.ac = reinterpret_cast<float2*>(c->an_w);
        launch_mix_att_accum(c->G, c->st.lambda2, c->st.rhs_norm_term, c->perm_t, c->ivl_off, c->n_iv, mo,
                             c->att, c->blk, c->sh, c->stream);
    } else
        launch_att_accum(c->G, c->st.lambda2, c->st.rhs_norm_term, c->perm_t, c->ivl_off, c->n_iv,
                         c->rec, c->an.eps2 ? c->an_w : nullptr, c->att, c->blk, c->sh, c->stream);
    launch_att_solve(c->n_seg, c->max_seg_knots, c->n_coef, c->n_rows, c->seg_row, c->seg_l, c->seg_n, c->seg_u, c->blk, c->bandc,
                     c->rhs, c->urow, c->yv, c->xs, c->st.pivot_tol, c->seg_rd, c->att, c->mixed ? c->d_att : nullptr,
                     c->datt64, c->stream);
    launch_int_sum(c->n_seg, c->seg_rd, c->isum, c->stream);
}
void enqueue_c(agis_ctx* c, bool with_att = true) {
    // block Gauss-Seidel (Eq. precond): the residuals C reads take the attitude update (once
    // per A update: a repeated manual C update does not add it again)
    if (c->cfg.block_order == 1 && with_att) {
        if (c->mixed)
            launch_mix_ac_correct(c->G, c->n_obs, c->mo, c->d_att, c->stream);
        else
            launch_rec_att_correct(c->G, c->n_obs, c->rec, c->datt64, c->stream);
    }
    if (c->cal_generic) {
        launch_calgen(c->G, c->cg_groups, c->rec, c->mu, c->cgw, c->st.pivot_tol, c->cal, c->stream);
        launch_int_sum((int)(c->cg_groups * (c->G.cg.j_per_k + 2)), c->cgw.rd, c->isum + 1, c->stream);
        return;
    }
    if (c->mixed)
        launch_mix_cal(c->n_cal, c->n_days, c->perm_c, c->cal_off, c->mo, c->dtil, c->cal_rd, c->cal, c->d_cal,
                       c->sh, c->stream);
    else
        launch_cal(c->n_cal, c->n_days, c->perm_c, c->cal_off, c->rec, c->st.pivot_tol, c->dtil,
                   c->cal_rd, c->cal, c->sh, c->stream);
    launch_int_sum(c->n_cal, c->cal_rd, c->isum + 1, c->stream);
}
void enqueue_frame(agis_ctx* c, const int32_t* subset, int n) {
    launch_frame(c->G, n, subset, c->n_src, c->src, c->ref, c->att, c->fpart, c->n_fpart, c->st.pivot_tol, c->eo,
                 c->stream);
}

void fill_s_stats(agis_ctx* c, const double* h, agis_block_stats* out) {
    if (!out) return;
    std::memset(out, 0, sizeof(*out));
    out->chi2 = h[0];
    out->q_sum = h[1];
    out->nu_sum = (int64_t)llround(h[2]);
    out->n_out = (int64_t)llround(h[3]);
    out->rank_defect = (int64_t)llround(h[4]);
    for (int k = 0; k < 5; k++) out->d_rms[k] = c->n_src > 0 ? std::sqrt(h[5 + k] / c->n_src) : 0.0;
}

}  // namespace

// -----------------------------------------------------------------------------------------
// ABI
// -----------------------------------------------------------------------------------------
// --- launch-shape autotuner --------------------------------------------------------------
namespace {
struct ShapeCand {
    int a, b;
};
void knob_get(const Shapes& sh, int k, int& a, int& b) {
    switch (k) {
        case AGIS_KNOB_OBS_PASS: a = sh.obs_threads; b = sh.obs_bps; break;
        case AGIS_KNOB_SRC_BATCH: a = sh.src_batch; b = 0; break;
        case AGIS_KNOB_MIX_SUMS: a = sh.sums_warps; b = sh.sums_bps; break;
        case AGIS_KNOB_MIX_SOLVE5: a = sh.solve5_threads; b = 0; break;
        case AGIS_KNOB_ATT_ACCUM: a = 0; b = sh.att_bps; break;
        default: a = sh.cal_threads; b = sh.cal_bps; break;
    }
}
void knob_set(Shapes& sh, int k, int a, int b) {
    switch (k) {
        case AGIS_KNOB_OBS_PASS: sh.obs_threads = a; sh.obs_bps = b; break;
        case AGIS_KNOB_SRC_BATCH: sh.src_batch = a; break;
        case AGIS_KNOB_MIX_SUMS: sh.sums_warps = a; sh.sums_bps = b; break;
        case AGIS_KNOB_MIX_SOLVE5: sh.solve5_threads = a; break;
        case AGIS_KNOB_ATT_ACCUM: sh.att_bps = b; break;
        default: sh.cal_threads = a; sh.cal_bps = b; break;
    }
}
bool knob_valid(int k, int a, int b) {
    const bool bps = b >= 1 && b <= 64;
    switch (k) {
        case AGIS_KNOB_OBS_PASS: return (a == 128 || a == 256) && bps;
        case AGIS_KNOB_SRC_BATCH: return a >= 0 && a <= 32;
        case AGIS_KNOB_MIX_SUMS: return (a == 2 || a == 4 || a == 8) && bps;
        case AGIS_KNOB_MIX_SOLVE5: return a == 64 || a == 128 || a == 256;
        case AGIS_KNOB_ATT_ACCUM: return b == 0 || bps;
        case AGIS_KNOB_CAL_ACCUM: return (a == 128 || a == 256) && bps;
        default: return false;
    }
}
// candidate shapes of a knob, the default first (empty: the knob does not apply to the form)
std::vector<ShapeCand> knob_candidates(int k, bool mixed) {
    switch (k) {
        case AGIS_KNOB_OBS_PASS:
            if (mixed) return {{256, 64}, {256, 32}, {256, 16}, {256, 8}, {128, 64}, {128, 32}, {128, 16}};
            return {{256, 64}, {256, 16}, {256, 8}, {128, 32}, {128, 16}};
        case AGIS_KNOB_SRC_BATCH:
            if (mixed) return {};
            return {{0, 0}, {1, 0}, {2, 0}, {4, 0}, {8, 0}, {16, 0}};
        case AGIS_KNOB_MIX_SUMS:
            if (!mixed) return {};
            return {{4, 16}, {2, 32}, {8, 8}, {4, 8}, {2, 16}, {8, 4}};
        case AGIS_KNOB_MIX_SOLVE5:
            if (!mixed) return {};
            return {{128, 0}, {64, 0}, {256, 0}};
        case AGIS_KNOB_ATT_ACCUM:
            if (mixed) return {{0, 0}, {0, 32}, {0, 16}, {0, 8}};
            return {{0, 0}, {0, 16}, {0, 8}, {0, 4}};
        default:
            return {{256, 16}, {256, 8}, {128, 16}, {128, 32}, {256, 4}};
    }
}
}  // namespace

extern "C" {

int agis_abi_version(void) { return AGIS_ABI_VERSION; }

void agis_default_config(agis_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->robust = 1;
    cfg->n_rounds = 4;
    cfg->n_eps = 3;
    cfg->weight_fn = 0;
    cfg->lambda_att = 1e-3;
    cfg->rhs_norm_term = 0;
    cfg->seg_len = 2880;
    cfg->seg_overlap = 12;
    cfg->frame_each_iter = 1;
    cfg->block_mask = 7;
    cfg->use_graph = 1;
    cfg->pivot_tol = 1e-12;
    cfg->max_obs_per_source = 0;
    cfg->precision = 0;
    cfg->refresh_every = 8;
}

static thread_local std::string g_init_err = "no error";
const char* agis_last_error(const agis_ctx* ctx) { return ctx ? ctx->err.c_str() : g_init_err.c_str(); }

void agis_destroy(agis_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int b = 0; b < agis_ctx::kGraphs; b++) {
        if (c->graph_execs[b]) cudaGraphExecDestroy(c->graph_execs[b]);
        if (c->graphs[b]) cudaGraphDestroy(c->graphs[b]);
    }
    for (void* p : c->allocs) cudaFree(p);
    if (c->hstat) cudaFreeHost(c->hstat);
    if (c->hisum) cudaFreeHost(c->hisum);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->stream_c) cudaStreamDestroy(c->stream_c);
    for (int i = 0; i < agis_ctx::kEvents; i++)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    delete c;
}

int agis_init(const agis_geometry* geo, const agis_config* cfg, const agis_obs* obs, int64_t n_obs, const double* src0,
              const double* src_ref, int32_t n_src, const double* att0, int32_t n_coef, const double* cal0,
              int32_t n_cal, void* stream, agis_ctx** out) {
    if (!out) return AGIS_E_INVALID;
    *out = nullptr;
    agis_ctx* c = new agis_ctx();
    for (int i = 0; i < agis_ctx::kEvents; i++) c->ev[i] = nullptr;
    auto bail = [&](int code) {
        g_init_err = c->err;
        agis_destroy(c);
        return code;
    };
    if (!geo || !cfg || !obs || !src0 || !att0 || !cal0) return bail(fail(c, AGIS_E_INVALID, "null argument"));
    if (n_obs < 0 || n_src < 0) return bail(fail(c, AGIS_E_INVALID, "negative size"));
    if (n_obs >= ((int64_t)1 << 32)) return bail(fail(c, AGIS_E_INVALID, "more than 2^32-1 observations"));
    if (n_coef < 4 || n_coef != geo->n_coef) return bail(fail(c, AGIS_E_INVALID, "n_coef < 4 or != geo->n_coef"));
    if (cfg->cal_model != 0 && cfg->cal_model != 1) return bail(fail(c, AGIS_E_INVALID, "cal_model must be 0 or 1"));
    CalGen cg{};
    if (cfg->cal_model == 1) {
        if (cfg->n_gate < 1 || cfg->n_gate > AGIS_MAX_GATE || cfg->cal_j_per_k < 1 || cfg->cal_col_bin < 1 ||
            cfg->cal_col_bin > AGIS_N_COL || geo->n_cal_days < 1)
            return bail(fail(c, AGIS_E_INVALID, "full calibration: n_gate 1..AGIS_MAX_GATE, cal_j_per_k >= 1, "
                                                "cal_col_bin 1..AGIS_N_COL"));
        if (cfg->precision != 0)
            return bail(fail(c, AGIS_E_INVALID, "the full calibration model needs the FP64 form (precision 0)"));
        cg.on = 1;
        cg.n_gate = cfg->n_gate;
        cg.j_per_k = cfg->cal_j_per_k;
        cg.col_bin = cfg->cal_col_bin;
        cg.n_bin = (AGIS_N_COL + cfg->cal_col_bin - 1) / cfg->cal_col_bin;
        cg.n_j = geo->n_cal_days;
        cg.n_k = (geo->n_cal_days + cfg->cal_j_per_k - 1) / cfg->cal_j_per_k;
        cg.al_size = 6 * cg.j_per_k + cg.n_bin;
        const int64_t n_groups = (int64_t)AGIS_N_CCD * cg.n_gate * cg.n_k;
        cg.n_al = n_groups * cg.al_size;
        cg.t0 = geo->cal_t0_ns;
        cg.dt = geo->cal_dt_ns;
        cg.inv_ncol = 1.0 / (double)AGIS_N_COL;
        if ((int64_t)n_cal != cg.n_al + 6 * n_groups)
            return bail(fail(c, AGIS_E_INVALID, "n_cal != 62 n_gate n_k (6 j_per_k + n_bin + 6) (full calibration)"));
        if ((n_groups * cg.j_per_k + 1) * cg.n_bin + n_groups >= ((int64_t)1 << 31))
            return bail(fail(c, AGIS_E_INVALID, "full calibration layout too large for the C-block order keys"));
    } else if (geo->n_cal_days < 1 || n_cal != geo->n_cal_days * 2 * (AGIS_N_CCD + AGIS_N_ROW)) {
        return bail(fail(c, AGIS_E_INVALID, "n_cal != n_cal_days * 138"));
    }
    if (geo->knot_dt_ns <= 0 || geo->cal_dt_ns <= 0 || !(geo->year_s > 0) || !(geo->focal_length > 0))
        return bail(fail(c, AGIS_E_INVALID, "non-positive interval, year or focal length"));
    if (n_obs > 0 && (!obs->t_ns || !obs->src || !obs->ccd || !obs->fov || !obs->kind || !obs->sigma || !obs->mu))
        return bail(fail(c, AGIS_E_INVALID, "null observation array"));
    if (cfg->seg_len < 1 || cfg->seg_overlap < 0 || cfg->n_rounds < 0 || cfg->n_eps < 0)
        return bail(fail(c, AGIS_E_INVALID, "bad segmentation or iteration counts"));
    if (cfg->precision != 0 && cfg->precision != 1) return bail(fail(c, AGIS_E_INVALID, "precision must be 0 or 1"));
    if (cfg->precision == 1 && cfg->refresh_every < 1)
        return bail(fail(c, AGIS_E_INVALID, "refresh_every must be at least 1"));
    if (cfg->block_order < 0 || cfg->block_order > 2)
        return bail(fail(c, AGIS_E_INVALID, "block_order must be 0 (S[AC]), 1 (SAC) or 2 ([SAC])"));
    for (int i = 0; i < AGIS_N_CCD; i++)
        if (geo->ccd_row[i] < 0 || geo->ccd_row[i] >= AGIS_N_ROW) return bail(fail(c, AGIS_E_INVALID, "bad ccd_row"));
    c->geo = *geo;
    c->cfg = *cfg;
    c->n_obs = n_obs;
    c->n_src = n_src;
    c->n_coef = n_coef;
    c->n_cal = n_cal;
    c->n_days = geo->n_cal_days;
    c->stream = (cudaStream_t)stream;
    if (!c->stream) {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(c, AGIS_E_CUDA, "cudaStreamCreate"));
        c->own_stream = true;
    }
    if (cuda_check(c, cudaGetDevice(&c->device), "cudaGetDevice") != AGIS_OK) return bail(AGIS_E_CUDA);
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    // device geometry
    DevGeo& G = c->G;
    fill_devgeo(geo, n_coef, G);
    G.cg = cg;
    c->cal_generic = cg.on != 0;
    Settings& st = c->st;
    st.robust = cfg->robust;
    st.n_rounds = cfg->n_rounds;
    st.n_eps = cfg->n_eps;
    st.weight_fn = cfg->weight_fn;
    st.lambda2 = cfg->lambda_att * cfg->lambda_att;
    st.rhs_norm_term = cfg->rhs_norm_term;
    st.pivot_tol = cfg->pivot_tol;
    st.handover_h = cfg->block_order == 2 ? 1 : 0;
    for (int i = 0; i < agis_ctx::kEvents; i++) cudaEventCreate(&c->ev[i]);
    if (cudaStreamCreateWithFlags(&c->stream_c, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(c, AGIS_E_CUDA, "cudaStreamCreate (C block)"));
    if (cudaMallocHost(&c->hstat, 32 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->hisum, 4 * sizeof(long long)) != cudaSuccess)
        return bail(fail(c, AGIS_E_OOM, "pinned host buffer"));
    const int64_t n = n_obs;
    // ---- observations: copied in the caller's order, validated, then reordered
    int* derr = nullptr;
    int32_t* d_ccdrow = nullptr;
    int rc = AGIS_OK;
    TmpDev tb_t, tb_src, tb_sig, tb_mu, tb_8, tb_meta, tb_gate;
    uint8_t* gate_in = nullptr;
    if (c->cal_generic && obs->gate && n > 0 && (rc = tb_gate.alloc(c, &gate_in, n))) return bail(rc);
    int64_t* t_in = nullptr;
    int32_t* src_in = nullptr;
    float* sig_in = nullptr;
    double* mu_in = nullptr;
    uint8_t* tmp8 = nullptr;
    uint32_t* meta_in = nullptr;
    if ((rc = dalloc(c, &derr, 1)) || (rc = dalloc(c, &d_ccdrow, AGIS_N_CCD)) || (rc = tb_t.alloc(c, &t_in, n)) ||
        (rc = tb_src.alloc(c, &src_in, n)) || (rc = tb_sig.alloc(c, &sig_in, n)) || (rc = tb_mu.alloc(c, &mu_in, n)) ||
        (rc = tb_8.alloc(c, &tmp8, 3 * (size_t)n + 16)) || (rc = tb_meta.alloc(c, &meta_in, n)))
        return bail(rc);
    cudaStream_t s = c->stream;
#define CP(dst, srcp, bytes)                                                                          \
    if (cuda_check(c, cudaMemcpyAsync((dst), (srcp), (bytes), cudaMemcpyDefault, s), "copy inputs")) \
        return bail(AGIS_E_CUDA);
    if (n > 0) {
        CP(t_in, obs->t_ns, n * sizeof(int64_t));
        CP(src_in, obs->src, n * sizeof(int32_t));
        CP(tmp8, obs->ccd, n);
        CP(tmp8 + n, obs->fov, n);
        CP(tmp8 + 2 * n, obs->kind, n);
        CP(sig_in, obs->sigma, n * sizeof(float));
        CP(mu_in, obs->mu, n * sizeof(double));
        if (gate_in) CP(gate_in, obs->gate, n);
    }
    CP(d_ccdrow, geo->ccd_row, AGIS_N_CCD * sizeof(int32_t));
    cudaMemsetAsync(derr, 0, sizeof(int), s);
    if (n > 0) {
        k_validate_pack<<<grid_for(n, 256), 256, 0, s>>>(n, t_in, src_in, tmp8, tmp8 + n, tmp8 + 2 * n, sig_in, mu_in,
                                                         n_src, geo->cal_t0_ns, geo->cal_dt_ns, geo->n_cal_days,
                                                         d_ccdrow, gate_in, c->cal_generic ? cg.n_gate : 0, meta_in,
                                                         derr);
    }
    // ---- state
    if ((rc = dalloc(c, &c->src, 5 * (size_t)n_src)) || (rc = dalloc(c, &c->att, 4 * (size_t)n_coef)) ||
        (rc = dalloc(c, &c->cal, n_cal)))
        return bail(rc);
    CP(c->src, src0, 5 * (size_t)n_src * sizeof(double));
    CP(c->att, att0, 4 * (size_t)n_coef * sizeof(double));
    CP(c->cal, cal0, (size_t)n_cal * sizeof(double));
    if (src_ref) {
        if ((rc = dalloc(c, &c->ref, 4 * (size_t)n_src))) return bail(rc);
        CP(c->ref, src_ref, 4 * (size_t)n_src * sizeof(double));
    }
    k_check_finite<<<grid_for(5 * (int64_t)n_src, 256), 256, 0, s>>>(5 * (int64_t)n_src, c->src, derr, 32);
    k_check_finite<<<grid_for(4 * (int64_t)n_coef, 256), 256, 0, s>>>(4 * (int64_t)n_coef, c->att, derr, 32);
    k_check_finite<<<grid_for(n_cal, 256), 256, 0, s>>>(n_cal, c->cal, derr, 32);
    int herr = 0;
    if (cuda_check(c, cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s), "validate") ||
        cuda_check(c, cudaStreamSynchronize(s), "validate (sync)"))
        return bail(AGIS_E_CUDA);
    if (herr) {
        static const char* what[7] = {"source index out of range", "observations not sorted by source",
                                      "ccd, fov or kind out of range", "sigma not positive and finite",
                                      "mu of an AC observation (or of any, full calibration) not finite",
                                      "non-finite starting value (src0, att0 or cal0)", "gate out of range"};
        std::string msg = "invalid input:";
        for (int b = 0; b < 7; b++)
            if (herr & (1 << b)) msg += std::string(" ") + what[b] + ";";
        return bail(fail(c, AGIS_E_INVALID, msg));
    }
    // ---- internal order: by source, AL before AC (the per-class passes of the S block then
    // sweep contiguous ranges)
    // (each array is gathered into its internal copy and its caller-order copy released
    // before the next, which keeps the set-up's peak memory near 60 bytes per observation)
    if ((rc = dalloc(c, &c->perm_in, n)) || (rc = dalloc(c, &c->src_nal, n_src))) return bail(rc);
    {
        TmpDev tk_in, tk_out, tv_in, tg;
        int32_t *k_in = nullptr, *k_out = nullptr;
        uint32_t* v_in = nullptr;
        int64_t* goff = nullptr;
        if ((rc = tk_in.alloc(c, &k_in, n)) || (rc = tk_out.alloc(c, &k_out, n)) || (rc = tv_in.alloc(c, &v_in, n)) ||
            (rc = tg.alloc(c, &goff, 2 * (size_t)n_src + 1)))
            return bail(rc);
        if (n > 0) {
            k_class_keys<<<grid_for(n, 256), 256, 0, s>>>(n, src_in, tmp8 + 2 * n, k_in, v_in);
            if ((rc = sort_pairs(c, k_in, k_out, v_in, c->perm_in, n, bits_for(2 * (int64_t)n_src)))) return bail(rc);
        }
        k_lower_bound<int32_t><<<grid_for(2 * (int64_t)n_src + 1, 256), 256, 0, s>>>(k_out, n,
                                                                                      2 * (int64_t)n_src + 1, goff);
        k_src_nal<<<grid_for(n_src, 256), 256, 0, s>>>(n_src, goff, c->src_nal);
        if (cuda_check(c, cudaStreamSynchronize(s), "reorder")) return bail(AGIS_E_CUDA);
    }
    tb_8.release();
    const uint32_t* pin = c->perm_in;
    if ((rc = dalloc(c, &c->t_ns, n))) return bail(rc);
    k_gather<int64_t><<<grid_for(n, 256), 256, 0, s>>>(n, pin, t_in, c->t_ns);
    if (cuda_check(c, cudaStreamSynchronize(s), "reorder")) return bail(AGIS_E_CUDA);
    tb_t.release();
    if ((rc = dalloc(c, &c->meta, n))) return bail(rc);
    k_gather<uint32_t><<<grid_for(n, 256), 256, 0, s>>>(n, pin, meta_in, c->meta);
    if ((rc = dalloc(c, &c->mu, n))) return bail(rc);
    k_gather_mu<<<grid_for(n, 256), 256, 0, s>>>(n, pin, c->meta, mu_in, c->mu, c->cal_generic ? 1 : 0);
    if (cuda_check(c, cudaStreamSynchronize(s), "reorder")) return bail(AGIS_E_CUDA);
    tb_mu.release();
    tb_meta.release();
    if ((rc = dalloc(c, &c->sigma, n))) return bail(rc);
    k_gather<float><<<grid_for(n, 256), 256, 0, s>>>(n, pin, sig_in, c->sigma);
    if ((rc = dalloc(c, &c->obs_src, n))) return bail(rc);
    k_gather<int32_t><<<grid_for(n, 256), 256, 0, s>>>(n, pin, src_in, c->obs_src);
    if (cuda_check(c, cudaStreamSynchronize(s), "reorder")) return bail(AGIS_E_CUDA);
    tb_sig.release();
    tb_src.release();
    // ---- source offsets, largest-first order, scratch capacity
    if ((rc = dalloc(c, &c->src_off, (size_t)n_src + 1)) || (rc = dalloc(c, &c->src_order, n_src))) return bail(rc);
    k_lower_bound<int32_t><<<grid_for(n_src + 1, 256), 256, 0, s>>>(c->obs_src, n, (int64_t)n_src + 1, c->src_off);
    std::vector<int64_t> hoff((size_t)n_src + 1);
    if (cuda_check(c, cudaMemcpyAsync(hoff.data(), c->src_off, hoff.size() * 8, cudaMemcpyDeviceToHost, s), "offsets") ||
        cuda_check(c, cudaStreamSynchronize(s), "offsets (sync)"))
        return bail(AGIS_E_CUDA);
    int64_t maxn = 0;
    for (int32_t i = 0; i < n_src; i++) maxn = std::max(maxn, hoff[i + 1] - hoff[i]);
    if (cfg->max_obs_per_source > 0) {
        if (maxn > cfg->max_obs_per_source)
            return bail(fail(c, AGIS_E_INVALID, "a source has more observations than max_obs_per_source"));
        maxn = cfg->max_obs_per_source;
    }
    c->cap = (int)std::max<int64_t>(maxn, 32);
    {
        TmpDev tk_in, tk_out, ti_in;
        int32_t *k_in = nullptr, *k_out = nullptr, *i_in = nullptr;
        if ((rc = tk_in.alloc(c, &k_in, n_src)) || (rc = tk_out.alloc(c, &k_out, n_src)) ||
            (rc = ti_in.alloc(c, &i_in, n_src)))
            return bail(rc);
        k_src_counts<<<grid_for(n_src, 256), 256, 0, s>>>(n_src, c->src_off, k_in, i_in);
        if (n_src > 0 && (rc = sort_pairs(c, k_in, k_out, (uint32_t*)i_in, (uint32_t*)c->src_order, n_src, 32)))
            return bail(rc);
    }
    // ---- time order by knot interval
    c->n_iv = n_coef - 3;
    {
        TmpDev tk_in, tk_out, tv_in;
        int32_t *k_in = nullptr, *k_out = nullptr;
        uint32_t* v_in = nullptr;
        if ((rc = tk_in.alloc(c, &k_in, n)) || (rc = tk_out.alloc(c, &k_out, n)) || (rc = tv_in.alloc(c, &v_in, n)) ||
            (rc = dalloc(c, &c->perm_t, n)) || (rc = dalloc(c, &c->ivl_off, (size_t)c->n_iv + 1)))
            return bail(rc);
        if (n > 0) {
            k_interval_keys<<<grid_for(n, 256), 256, 0, s>>>(G, n, c->t_ns, k_in, v_in);
            if ((rc = sort_pairs(c, k_in, k_out, v_in, c->perm_t, n, bits_for(c->n_iv)))) return bail(rc);
        }
        k_lower_bound<int32_t><<<grid_for(c->n_iv + 1, 256), 256, 0, s>>>(k_out, n, (int64_t)c->n_iv + 1, c->ivl_off);
        // calibration order
        if (c->cal_generic) {
            const int64_t ng = (int64_t)AGIS_N_CCD * cg.n_gate * cg.n_k, ncell = ng * cg.j_per_k;
            const int nb = cg.n_bin;
            c->cg_groups = ng;
            CalGenWork& w = c->cgw;
            uint32_t* perm = nullptr;
            int64_t* off = nullptr;
            double* cc2 = nullptr;
            if ((rc = dalloc(c, &perm, n)) || (rc = dalloc(c, &off, (size_t)(ncell + ng + 1))) ||
                (rc = dalloc(c, &w.V, (size_t)ncell * 6 * nb)) || (rc = dalloc(c, &w.E, (size_t)ncell * nb)) ||
                (rc = dalloc(c, &w.bs, (size_t)ncell * nb)) || (rc = dalloc(c, &w.cw, (size_t)ncell * 18)) ||
                (rc = dalloc(c, &w.S, (size_t)ng * nb * nb)) || (rc = dalloc(c, &w.r, (size_t)ng * nb)) ||
                (rc = dalloc(c, &w.Et, (size_t)ng * nb)) || (rc = dalloc(c, &w.H, (size_t)ng * 3 * nb)) ||
                (rc = dalloc(c, &w.v, (size_t)ng * nb)) || (rc = dalloc(c, &w.idx, (size_t)ng * nb)) ||
                (rc = dalloc(c, &cc2, 3 * (size_t)nb)) || (rc = dalloc(c, &w.d, (size_t)n_cal)) ||
                (rc = dalloc(c, &w.rd, (size_t)(ncell + 2 * ng))))
                return bail(rc);
            // cc2 weights: sum of L*_r((m + 14 - 13.5) / n_col) over the columns m of each bin
            std::vector<double> hw(3 * (size_t)nb, 0.0);
            for (int m = 0; m < AGIS_N_COL; m++) {
                const double x = (m + 0.5) / (double)AGIS_N_COL;
                const int b = m / cg.col_bin;
                hw[b] += 1.0;
                hw[(size_t)nb + b] += 2.0 * x - 1.0;
                hw[2 * (size_t)nb + b] += 6.0 * x * x - 6.0 * x + 1.0;
            }
            CP(cc2, hw.data(), hw.size() * sizeof(double));
            if (cuda_check(c, cudaMemsetAsync(w.d, 0, (size_t)n_cal * 8, s), "calibration work")) return bail(AGIS_E_CUDA);
            if (n > 0) {
                k_calgen_keys<<<grid_for(n, 256), 256, 0, s>>>(G, n, c->t_ns, c->meta, c->mu, ncell, k_in, v_in);
                if ((rc = sort_pairs(c, k_in, k_out, v_in, perm, n, bits_for((ncell + 1) * nb + ng)))) return bail(rc);
            }
            k_calgen_off<<<grid_for(ncell + ng + 1, 256), 256, 0, s>>>(k_out, n, ncell, ng, nb, off);
            w.perm = perm;
            w.off = off;
            w.cc2w = cc2;
            if (calgen_prepare() != 0) return bail(fail(c, AGIS_E_CUDA, "shared-memory attribute (calibration)"));
        } else {
            if ((rc = dalloc(c, &c->perm_c, n)) || (rc = dalloc(c, &c->cal_off, (size_t)n_cal + 1))) return bail(rc);
            if (n > 0) {
                k_cal_keys<<<grid_for(n, 256), 256, 0, s>>>(n, c->meta, k_in, v_in);
                if ((rc = sort_pairs(c, k_in, k_out, v_in, c->perm_c, n, bits_for(n_cal)))) return bail(rc);
            }
            k_lower_bound<int32_t><<<grid_for(n_cal + 1, 256), 256, 0, s>>>(k_out, n, (int64_t)n_cal + 1, c->cal_off);
        }
        if (cuda_check(c, cudaStreamSynchronize(s), "orders")) return bail(AGIS_E_CUDA);
    }
    c->n_sblocks = c->n_sm * 8;
    c->mixed = cfg->precision == 1;
    if (c->mixed) {
        if ((rc = dalloc(c, &c->mo.s, n)) || (rc = dalloc(c, &c->mo.r, n)) || (rc = dalloc(c, &c->mo.ac, n)) ||
            (rc = dalloc(c, &c->mo.t, n)) || (rc = dalloc(c, &c->d_att, 4 * (size_t)n_coef)) ||
            (rc = dalloc(c, &c->d_cal, n_cal)) || (rc = dalloc(c, &c->mw.scale, n_src)) ||
            (rc = dalloc(c, &c->mw.round, n_src)) || (rc = dalloc(c, &c->mw.fin, n_src)) ||
            (rc = dalloc(c, &c->mw.sums, n_src)))
            return bail(rc);
    } else {
        if ((rc = dalloc(c, &c->rec, n)) || (rc = dalloc(c, &c->scratch, (size_t)n * kScr)) ||
            (rc = dalloc(c, &c->skey, n)))
            return bail(rc);
        if (cfg->block_order == 1) {
            if ((rc = dalloc(c, &c->datt64, 4 * (size_t)n_coef))) return bail(rc);
            cudaMemsetAsync(c->datt64, 0, sizeof(double) * 4 * (size_t)n_coef, s);
        }
    }
    if ((rc = dalloc(c, &c->sgeo, 16 * (size_t)n_src)) ||
        (rc = dalloc(c, &c->work, 4)) || (rc = dalloc(c, &c->so.d, 5 * (size_t)n_src)) ||
        (rc = dalloc(c, &c->so.eps2, n_src)) || (rc = dalloc(c, &c->so.q, n_src)) ||
        (rc = dalloc(c, &c->so.dsig, n_src)) || (rc = dalloc(c, &c->so.chi2, n_src)) ||
        (rc = dalloc(c, &c->so.cov, 25 * (size_t)n_src)) || (rc = dalloc(c, &c->so.nu, n_src)) ||
        (rc = dalloc(c, &c->so.nout, n_src)) || (rc = dalloc(c, &c->so.rankdef, n_src)) ||
        (rc = dalloc(c, &c->sstats, 16)) || (rc = dalloc(c, &c->sstat_part, 512 * 10)))
        return bail(rc);
    c->so.src = c->src;
    // the orbital longitude tabulated over the knot range with one step of margin either
    // side (observations outside take sincospi)
    {
        const int64_t step = (int64_t)1 << kOrbShift;
        const int64_t span = (int64_t)std::max(n_coef - 3, 1) * geo->knot_dt_ns;
        const int32_t n_tab = (int32_t)((span + 2 * step) / step + 1);
        std::vector<double> tab(2 * (size_t)n_tab);
        G.orb_t0 = geo->knot0_ns - step;
        G.orb_n = n_tab;
        fill_orbit_table(G, G.orb_t0, n_tab, tab.data());
        double* dtab = nullptr;
        if ((rc = dalloc(c, &dtab, tab.size()))) return bail(rc);
        if (cuda_check(c, cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, s),
                       "orbit table") != AGIS_OK ||
            cuda_check(c, cudaStreamSynchronize(s), "orbit table (sync)") != AGIS_OK)
            return bail(AGIS_E_CUDA);
        G.orb_tab = dtab;
    }
    if ((rc = dalloc(c, &c->hist, 20 * (size_t)n_src))) return bail(rc);
    cudaMemsetAsync(c->hist, 0, sizeof(double) * 20 * (size_t)n_src, s);
    // ---- segments and band storage
    {
        std::vector<int32_t> sl, sn, su;
        std::vector<int64_t> srow;
        build_segments(n_coef, cfg->seg_len, cfg->seg_overlap, sl, sn, su, srow);
        c->n_seg = (int)(srow.size() - 1);
        c->n_rows = srow.back();
        for (size_t q = 0; q + 1 < srow.size(); q++)
            c->max_seg_knots = std::max(c->max_seg_knots, (int)((srow[q + 1] - srow[q]) / 4));
        if ((rc = dalloc(c, &c->seg_row, srow.size())) || (rc = dalloc(c, &c->seg_l, sl.size())) ||
            (rc = dalloc(c, &c->seg_n, sn.size())) || (rc = dalloc(c, &c->seg_u, su.size())) ||
            (rc = dalloc(c, &c->blk, (size_t)c->n_iv * kBlkVals)) || (rc = dalloc(c, &c->bandc, 16 * (size_t)c->n_rows)) ||
            (rc = dalloc(c, &c->rhs, c->n_rows)) || (rc = dalloc(c, &c->urow, 16 * (size_t)c->n_rows)) ||
            (rc = dalloc(c, &c->yv, c->n_rows)) || (rc = dalloc(c, &c->xs, c->n_rows)) ||
            (rc = dalloc(c, &c->seg_rd, c->n_seg)) || (rc = dalloc(c, &c->isum, 4)))
            return bail(rc);
        CP(c->seg_row, srow.data(), srow.size() * sizeof(int64_t));
        CP(c->seg_l, sl.data(), sl.size() * sizeof(int32_t));
        CP(c->seg_n, sn.data(), sn.size() * sizeof(int32_t));
        CP(c->seg_u, su.data(), su.size() * sizeof(int32_t));
    }
    if ((rc = dalloc(c, &c->dtil, n_cal)) || (rc = dalloc(c, &c->cal_rd, n_cal))) return bail(rc);
    c->n_fpart = std::min(1024, std::max(1, (n_src + 255) / 256));
    if ((rc = dalloc(c, &c->fpart, (size_t)c->n_fpart * 27)) || (rc = dalloc(c, &c->eo, 8))) return bail(rc);
    if (cuda_check(c, cudaStreamSynchronize(s), "init") || cuda_check(c, cudaGetLastError(), "init kernels"))
        return bail(AGIS_E_CUDA);
#undef CP
    *out = c;
    return AGIS_OK;
}

int agis_source_update(agis_ctx* c, agis_block_stats* out) {
    if (!c) return AGIS_E_INVALID;
    const bool refresh = s_refresh_due(c);
    record(c, 0);
    enqueue_s_pass(c, refresh);
    record(c, 13);
    enqueue_s_solve(c);
    record(c, 1);
    AGIS_CU(c, cudaMemcpyAsync(c->hstat, c->sstats, 10 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "stats");
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "source update");
    AGIS_CU(c, cudaGetLastError(), "source update kernels");
    s_done(c, refresh);
    c->hist_count++;
    c->have_s = true;
    c->have_s_out = true;
    c->a_since_c = false;   // the source update reset the attitude update C would see
    fill_s_stats(c, c->hstat, out);
    c->ktimes[0] = elapsed(c, 0, 1);
    if (out) {
        out->elapsed_ms = c->ktimes[0];
        out->pass_ms = elapsed(c, 0, 13);
        out->full_eval = (!c->mixed || refresh) ? 1 : 0;
    }
    if (!std::isfinite(c->hstat[0])) return fail(c, AGIS_E_NONFINITE, "non-finite chi^2 after the source update");
    return AGIS_OK;
}

int agis_attitude_update(agis_ctx* c, agis_block_stats* out) {
    if (!c) return AGIS_E_INVALID;
    if (!c->have_s) return fail(c, AGIS_E_INVALID, "attitude update needs a source update first");
    record(c, 2);
    enqueue_a(c);
    c->a_since_c = true;
    record(c, 3);
    AGIS_CU(c, cudaMemcpyAsync(c->hisum, c->isum, sizeof(long long), cudaMemcpyDeviceToHost, c->stream), "stats");
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "attitude update");
    AGIS_CU(c, cudaGetLastError(), "attitude update kernels");
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->rank_defect = c->hisum[0];
        out->elapsed_ms = elapsed(c, 2, 3);
    }
    c->ktimes[2] = elapsed(c, 2, 3);
    return AGIS_OK;
}

int agis_calibration_update(agis_ctx* c, agis_block_stats* out) {
    if (!c) return AGIS_E_INVALID;
    if (!c->have_s) return fail(c, AGIS_E_INVALID, "calibration update needs a source update first");
    record(c, 4);
    enqueue_c(c, c->a_since_c);
    c->a_since_c = false;
    record(c, 5);
    AGIS_CU(c, cudaMemcpyAsync(c->hisum + 1, c->isum + 1, sizeof(long long), cudaMemcpyDeviceToHost, c->stream),
            "stats");
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "calibration update");
    AGIS_CU(c, cudaGetLastError(), "calibration update kernels");
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->rank_defect = c->hisum[1];
        out->elapsed_ms = elapsed(c, 4, 5);
    }
    c->ktimes[3] = elapsed(c, 4, 5);
    return AGIS_OK;
}

int agis_frame_rotate(agis_ctx* c, const int32_t* subset, int32_t n_subset, double eps_omega_out[6]) {
    if (!c) return AGIS_E_INVALID;
    if (!c->ref) return fail(c, AGIS_E_INVALID, "no frame-rotator reference given at agis_init");
    const int32_t* dsub = nullptr;
    int nn = c->n_src;
    if (subset) {
        if (n_subset < 0) return fail(c, AGIS_E_INVALID, "negative subset size");
        if (n_subset > c->subset_cap) {
            int rc = dalloc(c, &c->subset, (size_t)n_subset);
            if (rc) return rc;
            c->subset_cap = n_subset;
        }
        std::vector<int32_t> h(subset, subset + n_subset);
        for (int32_t v : h)
            if (v < 0 || v >= c->n_src) return fail(c, AGIS_E_INVALID, "subset index out of range");
        AGIS_CU(c, cudaMemcpyAsync(c->subset, h.data(), n_subset * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream),
                "subset");
        dsub = c->subset;
        nn = n_subset;
    }
    record(c, 6);
    enqueue_frame(c, dsub, nn);
    record(c, 7);
    AGIS_CU(c, cudaMemcpyAsync(c->hstat + 16, c->eo, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "frame");
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "frame rotator");
    AGIS_CU(c, cudaGetLastError(), "frame rotator kernels");
    if (eps_omega_out)
        for (int i = 0; i < 6; i++) eps_omega_out[i] = c->hstat[16 + i];
    c->ktimes[4] = elapsed(c, 6, 7);
    c->have_s = false;  // the residuals of the last S block refer to the unrotated frame
    return AGIS_OK;
}

int agis_iterate(agis_ctx* c, int32_t n_iter, agis_iter_stats* per_iter, int32_t* n_done) {
    if (!c) return AGIS_E_INVALID;
    if (n_done) *n_done = 0;
    if (n_iter < 0) return fail(c, AGIS_E_INVALID, "negative iteration count");
    const bool do_frame = c->cfg.frame_each_iter && c->ref;
    const int mask = c->cfg.block_mask;
    if (!(mask & 1) && (mask & 6) && !c->have_s)
        return fail(c, AGIS_E_INVALID, "A/C blocks without an S block need a prior source update");
    const bool graph = c->cfg.use_graph != 0;
    // one graph per block, so that the blocks can be timed by events between the launches
    if (graph && !c->graphs_ready) {
        for (int b = 0; b < agis_ctx::kGraphs; b++) {
            if (b == 4 && !c->mixed) continue;
            if (b == 6 && !c->prop_packed) continue;
            if (b == 7 && !c->asi_keys) continue;
            AGIS_CU(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            if (b == 0) enqueue_s_pass(c, false);
            if (b == 4) enqueue_s_pass(c, true);
            if (b == 5) enqueue_s_solve(c);
            if (b == 1) enqueue_a(c);
            if (b == 2) enqueue_c(c);
            if (b == 3 && c->ref) enqueue_frame(c, nullptr, c->n_src);
            if (b == 6) enqueue_proposal(c);
            if (b == 7) enqueue_asi(c);
            AGIS_CU(c, cudaStreamEndCapture(c->stream, &c->graphs[b]), "end capture");
            AGIS_CU(c, cudaGraphInstantiate(&c->graph_execs[b], c->graphs[b], 0), "instantiate graph");
        }
        c->graphs_ready = true;
    }
    auto run_block = [&](int b) -> int {
        if (graph) return cuda_check(c, cudaGraphLaunch(c->graph_execs[b], c->stream), "graph launch");
        if (b == 0) enqueue_s_pass(c, false);
        if (b == 4) enqueue_s_pass(c, true);
        if (b == 5) enqueue_s_solve(c);
        if (b == 1) enqueue_a(c);
        if (b == 2) enqueue_c(c);
        if (b == 3) enqueue_frame(c, nullptr, c->n_src);
        if (b == 6) enqueue_proposal(c);
        if (b == 7) enqueue_asi(c);
        return cuda_check(c, cudaGetLastError(), "block launch");
    };
    const bool proposals = c->prop_every > 0 && (mask & 1);
    const bool asi = c->asi_stride > 0 && (mask & 1);
    auto snapshot = [&](bool save) -> int {
        const size_t ns = 5 * (size_t)c->n_src, na = 4 * (size_t)c->n_coef, nc = (size_t)c->n_cal,
                     nh = 20 * (size_t)c->n_src;
        double *s0 = save ? c->snap_src : c->src, *s1 = save ? c->src : c->snap_src;
        double *a0 = save ? c->snap_att : c->att, *a1 = save ? c->att : c->snap_att;
        double *c0 = save ? c->snap_cal : c->cal, *c1 = save ? c->cal : c->snap_cal;
        double *h0 = save ? c->snap_hist : c->hist, *h1 = save ? c->hist : c->snap_hist;
        AGIS_CU(c, cudaMemcpyAsync(s0, s1, ns * 8, cudaMemcpyDeviceToDevice, c->stream), "snapshot");
        AGIS_CU(c, cudaMemcpyAsync(a0, a1, na * 8, cudaMemcpyDeviceToDevice, c->stream), "snapshot");
        AGIS_CU(c, cudaMemcpyAsync(c0, c1, nc * 8, cudaMemcpyDeviceToDevice, c->stream), "snapshot");
        AGIS_CU(c, cudaMemcpyAsync(h0, h1, nh * 8, cudaMemcpyDeviceToDevice, c->stream), "snapshot");
        if (save) {
            c->snap_hist_count = c->hist_count;
        } else {
            c->hist_count = c->snap_hist_count;
            c->mix_stale = true;   // the records describe the state that is being discarded
        }
        return AGIS_OK;
    };
    // one S block; returns its chi^2 (synchronises)
    bool refresh = false;
    auto run_s = [&](double& chi2) -> int {
        refresh = s_refresh_due(c);
        AGIS_TRY(run_block(refresh ? 4 : 0));
        AGIS_CU(c, cudaEventRecord(c->ev[12], c->stream), "event");
        AGIS_TRY(run_block(5));
        s_done(c, refresh);
        c->hist_count++;
        AGIS_CU(c, cudaMemcpyAsync(c->hstat, c->sstats, 10 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                "stats");
        AGIS_CU(c, cudaStreamSynchronize(c->stream), "source update");
        chi2 = c->hstat[0];
        return AGIS_OK;
    };
    auto run_acf = [&]() -> int {
        if (mask & 2) AGIS_TRY(run_block(1));
        if (mask & 4) AGIS_TRY(run_block(2));
        if (do_frame) AGIS_TRY(run_block(3));
        return AGIS_OK;
    };
    for (int32_t k = 0; k < n_iter; k++) {
        int prop_state = 0;
        const bool plan = proposals && !c->prop_pending && c->hist_count >= 3 && c->since_prop >= c->prop_every;
        if (plan) AGIS_TRY(snapshot(true));
        AGIS_CU(c, cudaEventRecord(c->ev[8], c->stream), "event");
        double chi2 = 0.0;
        if (mask & 1) AGIS_TRY(run_s(chi2));
        if (c->prop_pending) {
            c->prop_pending = false;
            if (!(chi2 <= c->chi2_before_prop)) {
                // the proposal did not lower the robust chi^2: back to the state before the
                // iteration that carried it, which is redone without it, then this S again
                AGIS_TRY(snapshot(false));
                double chi2_redo = 0.0;
                AGIS_TRY(run_s(chi2_redo));
                AGIS_TRY(run_acf());
                AGIS_TRY(run_s(chi2));
                prop_state = 2;
            }
        }
        if (plan && prop_state == 0) {
            AGIS_TRY(run_block(6));
            c->prop_pending = true;
            c->chi2_before_prop = chi2;
            c->since_prop = 0;
            prop_state = 1;
        }
        // ASI needs the updates of two S blocks; not on top of a proposal
        const bool asi_now = asi && prop_state != 1 && c->hist_count >= 2;
        if (asi_now) {
            AGIS_TRY(run_block(7));
            AGIS_CU(c, cudaMemcpyAsync(c->hstat + 24, c->asi_est, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                       c->stream),
                    "stats");
        }
        AGIS_CU(c, cudaEventRecord(c->ev[9], c->stream), "event");
        // S[AC] and [SAC]: A and C read the same hand-over and write disjoint state, so the C
        // graph runs on a second stream beside the A graph (Sect. 4.6: A and C are independent
        // given S); block Gauss-Seidel SAC keeps C after A
        const bool c_beside = graph && (mask & 2) && (mask & 4) && c->cfg.block_order != 1;
        if (c_beside) {
            AGIS_CU(c, cudaStreamWaitEvent(c->stream_c, c->ev[9], 0), "fork");
            AGIS_CU(c, cudaEventRecord(c->ev[14], c->stream_c), "event");
            AGIS_CU(c, cudaGraphLaunch(c->graph_execs[2], c->stream_c), "graph launch");
            AGIS_CU(c, cudaEventRecord(c->ev[15], c->stream_c), "event");
        }
        if (mask & 2) AGIS_TRY(run_block(1));
        AGIS_CU(c, cudaEventRecord(c->ev[10], c->stream), "event");
        if (c_beside) AGIS_CU(c, cudaStreamWaitEvent(c->stream, c->ev[15], 0), "join");
        else if (mask & 4) AGIS_TRY(run_block(2));
        if (do_frame) AGIS_TRY(run_block(3));
        AGIS_CU(c, cudaEventRecord(c->ev[11], c->stream), "event");
        c->since_prop++;
        AGIS_CU(c, cudaMemcpyAsync(c->hisum, c->isum, 2 * sizeof(long long), cudaMemcpyDeviceToHost, c->stream),
                "stats");
        if (do_frame)
            AGIS_CU(c, cudaMemcpyAsync(c->hstat + 16, c->eo, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                    "stats");
        AGIS_CU(c, cudaStreamSynchronize(c->stream), "iteration");
        if (mask & 1) {
            c->have_s = !do_frame;
            c->have_s_out = true;
        }
        c->a_since_c = false;
        if (per_iter) {
            agis_iter_stats& it = per_iter[k];
            std::memset(&it, 0, sizeof(it));
            if (mask & 1) fill_s_stats(c, c->hstat, &it.s);
            it.a.rank_defect = (mask & 2) ? c->hisum[0] : 0;
            it.c.rank_defect = (mask & 4) ? c->hisum[1] : 0;
            if (do_frame)
                for (int i = 0; i < 6; i++) it.frame[i] = c->hstat[16 + i];
            it.s.elapsed_ms = elapsed(c, 8, 9);
            it.s.pass_ms = prop_state == 0 ? elapsed(c, 8, 12) : -1.0;
            it.s.full_eval = (mask & 1) && (!c->mixed || refresh) ? 1 : 0;
            it.a.elapsed_ms = elapsed(c, 9, 10);
            it.c.elapsed_ms = c_beside ? elapsed(c, 14, 15) : elapsed(c, 10, 11);
            it.elapsed_ms = elapsed(c, 8, 11);
            it.proposal = prop_state;
            it.asi_factor = 1.0;
            if (asi_now) {
                it.asi_lambda = c->hstat[24];
                it.asi_factor = c->hstat[26];
                it.asi_n = (int32_t)llround(c->hstat[27]);
            }
        }
        if ((mask & 1) && !std::isfinite(chi2)) return fail(c, AGIS_E_NONFINITE, "non-finite chi^2");
        if (n_done) *n_done = k + 1;
    }
    return AGIS_OK;
}

int agis_evaluate(agis_ctx* c, double* R_out) {
    if (!c || !R_out) return AGIS_E_INVALID;
    if (!c->evalR) AGIS_TRY(dalloc(c, &c->evalR, (size_t)c->n_obs));
    if (!c->tmpR) AGIS_TRY(dalloc(c, &c->tmpR, (size_t)c->n_obs));
    launch_evaluate(c->G, c->t_ns, c->meta, c->mu, c->obs_src, c->n_obs, c->src, c->att, c->cal, c->evalR, c->stream);
    k_scatter<<<grid_for(c->n_obs, 256), 256, 0, c->stream>>>(c->n_obs, c->perm_in, c->evalR, c->tmpR);
    AGIS_CU(c, cudaMemcpyAsync(R_out, c->tmpR, c->n_obs * sizeof(double), cudaMemcpyDefault, c->stream), "copy R");
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "evaluate");
    return cuda_check(c, cudaGetLastError(), "evaluate kernels");
}

static int get_copy(agis_ctx* c, void* dst, const void* src, size_t bytes) {
    if (!c || !dst) return AGIS_E_INVALID;
    AGIS_CU(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream), "copy");
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "copy (sync)");
    return AGIS_OK;
}

int agis_get_sources(agis_ctx* c, double* o) { return c ? get_copy(c, o, c->src, 5 * (size_t)c->n_src * 8) : AGIS_E_INVALID; }
int agis_get_attitude(agis_ctx* c, double* o) { return c ? get_copy(c, o, c->att, 4 * (size_t)c->n_coef * 8) : AGIS_E_INVALID; }
int agis_get_calibration(agis_ctx* c, double* o) { return c ? get_copy(c, o, c->cal, (size_t)c->n_cal * 8) : AGIS_E_INVALID; }

static int set_copy(agis_ctx* c, void* dst, const void* src, size_t bytes) {
    if (!c || !src) return AGIS_E_INVALID;
    AGIS_CU(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream), "copy");
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "copy (sync)");
    c->have_s = false;
    c->have_s_out = false;
    c->mix_stale = true;
    c->hist_count = 0;
    c->prop_pending = false;
    AGIS_CU(c, cudaMemsetAsync(c->hist, 0, sizeof(double) * 20 * (size_t)c->n_src, c->stream), "history");
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "history (sync)");
    return AGIS_OK;
}
int agis_set_sources(agis_ctx* c, const double* v) { return c ? set_copy(c, c->src, v, 5 * (size_t)c->n_src * 8) : AGIS_E_INVALID; }
int agis_set_attitude(agis_ctx* c, const double* v) { return c ? set_copy(c, c->att, v, 4 * (size_t)c->n_coef * 8) : AGIS_E_INVALID; }
int agis_set_calibration(agis_ctx* c, const double* v) { return c ? set_copy(c, c->cal, v, (size_t)c->n_cal * 8) : AGIS_E_INVALID; }

int agis_get_residuals(agis_ctx* c, double* R_out, double* W_out) {
    if (!c) return AGIS_E_INVALID;
    if (!c->have_s_out) return fail(c, AGIS_E_INVALID, "no source update since the last state change");
    if (!c->tmpR) AGIS_TRY(dalloc(c, &c->tmpR, (size_t)c->n_obs));
    if (!c->tmpW) AGIS_TRY(dalloc(c, &c->tmpW, (size_t)c->n_obs));
    if (c->mixed)
        launch_mix_rw(c->n_obs, c->perm_in, c->mo, c->tmpR, c->tmpW, c->stream);
    else
        k_rec_rw<<<grid_for(c->n_obs, 256), 256, 0, c->stream>>>(c->n_obs, c->perm_in, c->rec, c->tmpR, c->tmpW);
    if (R_out) AGIS_CU(c, cudaMemcpyAsync(R_out, c->tmpR, c->n_obs * 8, cudaMemcpyDefault, c->stream), "copy R");
    if (W_out) AGIS_CU(c, cudaMemcpyAsync(W_out, c->tmpW, c->n_obs * 8, cudaMemcpyDefault, c->stream), "copy W");
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "residuals");
    return AGIS_OK;
}

int agis_get_source_stats(agis_ctx* c, double* stats_out, double* cov_out) {
    if (!c) return AGIS_E_INVALID;
    if (stats_out) {
        if (!c->tmpS) AGIS_TRY(dalloc(c, &c->tmpS, 5 * (size_t)c->n_src));
        double* buf = c->tmpS;
        k_src_stats_out<<<grid_for(c->n_src, 256), 256, 0, c->stream>>>(c->n_src, c->so.eps2, c->so.q, c->so.nu,
                                                                       c->so.nout, c->so.dsig, buf);
        AGIS_TRY(get_copy(c, stats_out, buf, 5 * (size_t)c->n_src * 8));
    }
    if (cov_out) AGIS_TRY(get_copy(c, cov_out, c->so.cov, 25 * (size_t)c->n_src * 8));
    return AGIS_OK;
}

static void drop_graphs(agis_ctx* c) {
    for (int b = 0; b < agis_ctx::kGraphs; b++) {
        if (c->graph_execs[b]) cudaGraphExecDestroy(c->graph_execs[b]);
        if (c->graphs[b]) cudaGraphDestroy(c->graphs[b]);
        c->graph_execs[b] = nullptr;
        c->graphs[b] = nullptr;
    }
    c->graphs_ready = false;
}

int agis_set_proposal(agis_ctx* c, const float* params, int32_t every) {
    if (!c) return AGIS_E_INVALID;
    if (!params) {
        c->prop_every = 0;
        c->prop_pending = false;
        return AGIS_OK;
    }
    if (every < 5) return fail(c, AGIS_E_INVALID, "proposal period below 5 iterations");
    if (c->cfg.block_order == 2)
        return fail(c, AGIS_E_INVALID, "the learned proposal needs block order S[AC] or SAC");
    if (c->an.eps2) return fail(c, AGIS_E_INVALID, "the learned proposal does not combine with the excess attitude noise");
    if (!c->prop_packed) {
        void* packed = nullptr;
        AGIS_TRY(dalloc(c, reinterpret_cast<uint8_t**>(&packed), AGIS_MLP_PACKED_BYTES));
        c->prop_packed = packed;
        AGIS_TRY(dalloc(c, &c->prop_params, AGIS_MLP_N_PARAMS));
        AGIS_TRY(dalloc(c, &c->prop_X, (size_t)AGIS_MLP_N_IN * c->n_src));
        AGIS_TRY(dalloc(c, &c->prop_Y, (size_t)AGIS_MLP_N_OUT * c->n_src));
        AGIS_TRY(dalloc(c, &c->prop_sigma, c->n_src));
        if (!c->prop_corr) AGIS_TRY(dalloc(c, &c->prop_corr, 5 * (size_t)c->n_src));
        AGIS_TRY(dalloc(c, &c->snap_src, 5 * (size_t)c->n_src));
        AGIS_TRY(dalloc(c, &c->snap_att, 4 * (size_t)c->n_coef));
        AGIS_TRY(dalloc(c, &c->snap_cal, c->n_cal));
        AGIS_TRY(dalloc(c, &c->snap_hist, 20 * (size_t)c->n_src));
    }
    AGIS_CU(c, cudaMemcpyAsync(c->prop_params, params, sizeof(float) * AGIS_MLP_N_PARAMS, cudaMemcpyDefault,
                               c->stream),
            "proposal parameters");
    AGIS_TRY(agis_mlp_pack(c->prop_params, c->prop_packed, c->stream) == AGIS_OK
                 ? AGIS_OK
                 : fail(c, AGIS_E_CUDA, "packing the proposal network"));
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "proposal parameters (sync)");
    c->prop_every = every;
    c->prop_pending = false;
    c->since_prop = 1 << 30;
    drop_graphs(c);   // captured again with the proposal graph
    return AGIS_OK;
}

int agis_set_asi(agis_ctx* c, int32_t stride, double lambda_max) {
    if (!c) return AGIS_E_INVALID;
    if (stride <= 0) {
        c->asi_stride = 0;
        return AGIS_OK;
    }
    if (!(lambda_max >= 0.0 && lambda_max < 1.0)) return fail(c, AGIS_E_INVALID, "lambda_max outside [0, 1)");
    if (c->cfg.block_order == 2) return fail(c, AGIS_E_INVALID, "ASI needs block order S[AC] or SAC");
    if (c->an.eps2) return fail(c, AGIS_E_INVALID, "ASI does not combine with the excess attitude noise");
    if (!c->asi_keys) {
        const size_t n_s = std::max<size_t>(1, ((size_t)c->n_src + stride - 1) / stride);
        AGIS_TRY(dalloc(c, &c->asi_keys, std::max<size_t>(n_s, (size_t)c->n_src)));
        AGIS_TRY(dalloc(c, &c->asi_est, 4));
        if (!c->prop_corr) AGIS_TRY(dalloc(c, &c->prop_corr, 5 * (size_t)c->n_src));
    }
    c->asi_stride = stride;
    c->asi_lam_max = lambda_max;
    drop_graphs(c);   // the stride and the clamp are captured in the ASI graph
    return AGIS_OK;
}

// --- excess attitude noise (Sect. 5.2.5) --------------------------------------------------

int agis_set_attnoise(agis_ctx* c, int64_t bucket_ns) {
    if (!c) return AGIS_E_INVALID;
    if (bucket_ns < 0) return fail(c, AGIS_E_INVALID, "bucket_ns below 0");
    if (bucket_ns > 0) {
        if (c->cfg.block_order == 2)
            return fail(c, AGIS_E_INVALID, "the excess attitude noise needs block order S[AC] or SAC");
        if (c->asi_stride > 0 || c->prop_every > 0)
            return fail(c, AGIS_E_INVALID, "the excess attitude noise does not combine with ASI or the proposal");
    }
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "set_attnoise (sync)");
    drop_graphs(c);   // the estimate and the adjusted variances are captured in the graphs
    dfree(c, c->an_eps2);
    dfree(c, c->an_perm);
    dfree(c, c->an_off);
    dfree(c, c->an_x);
    dfree(c, c->an_w);
    c->an_eps2 = nullptr;
    c->an_perm = nullptr;
    c->an_off = nullptr;
    c->an_x = nullptr;
    c->an_w = nullptr;
    c->an = AttNoise{};
    c->an_bucket_ns = 0;
    c->an_max_run = 0;
    // mixed form: the records' sigma may hold sigma~; the next source update starts with a
    // full evaluation, which rewrites it
    c->mix_stale = true;
    if (bucket_ns == 0 || c->n_obs == 0) return AGIS_OK;
    const int64_t n = c->n_obs;
    cudaStream_t s = c->stream;
    // number of buckets from the last observation; none may precede the first bucket
    int64_t n_b = 0;
    {
        TmpDev tm;
        unsigned long long* mx = nullptr;
        AGIS_TRY(tm.alloc(c, &mx, 2));
        int* neg = reinterpret_cast<int*>(mx + 1);
        AGIS_CU(c, cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned long long), s), "set_attnoise (memset)");
        launch_an_range(n, c->t_ns, c->G.knot0_ns, mx, neg, s);
        unsigned long long h[2] = {0, 0};
        AGIS_CU(c, cudaMemcpyAsync(h, mx, sizeof(h), cudaMemcpyDeviceToHost, s), "set_attnoise (range)");
        AGIS_CU(c, cudaStreamSynchronize(s), "set_attnoise (range sync)");
        if (h[1] != 0ull)
            return fail(c, AGIS_E_INVALID, "an observation precedes knot0_ns, the start of the first bucket");
        n_b = (int64_t)(h[0] / (unsigned long long)bucket_ns) + 1;
    }
    if (3 * n_b >= (int64_t)1 << 30) return fail(c, AGIS_E_INVALID, "more than 2^30 / 3 attitude-noise buckets");
    AttNoise an;
    an.t0 = c->G.knot0_ns;
    an.dt = bucket_ns;
    an.n_b = (int32_t)n_b;
    AGIS_TRY(dalloc(c, &c->an_eps2, 3 * (size_t)n_b));
    AGIS_TRY(dalloc(c, &c->an_perm, (size_t)n));
    AGIS_TRY(dalloc(c, &c->an_off, 3 * (size_t)n_b + 1));
    AGIS_TRY(dalloc(c, &c->an_x, (size_t)n));
    AGIS_TRY(dalloc(c, &c->an_w, (size_t)n));
    AGIS_CU(c, cudaMemsetAsync(c->an_eps2, 0, sizeof(double) * 3 * (size_t)n_b, s), "set_attnoise (memset)");
    {
        TmpDev tk_in, tk_out, tv_in;
        int32_t *k_in = nullptr, *k_out = nullptr;
        uint32_t* v_in = nullptr;
        AGIS_TRY(tk_in.alloc(c, &k_in, n));
        AGIS_TRY(tk_out.alloc(c, &k_out, n));
        AGIS_TRY(tv_in.alloc(c, &v_in, n));
        launch_an_keys(n, c->t_ns, c->meta, an, k_in, v_in, s);
        AGIS_TRY(sort_pairs(c, k_in, k_out, v_in, c->an_perm, n, bits_for(3 * n_b)));
        k_lower_bound<int32_t><<<grid_for(3 * n_b + 1, 256), 256, 0, s>>>(k_out, n, 3 * n_b + 1, c->an_off);
        std::vector<int64_t> hoff(3 * (size_t)n_b + 1);
        AGIS_CU(c, cudaMemcpyAsync(hoff.data(), c->an_off, hoff.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                "set_attnoise (offsets)");
        AGIS_CU(c, cudaStreamSynchronize(s), "set_attnoise (order)");
        for (size_t r = 0; r + 1 < hoff.size(); r++) c->an_max_run = std::max(c->an_max_run, hoff[r + 1] - hoff[r]);
    }
    an.eps2 = c->an_eps2;
    c->an = an;
    c->an_bucket_ns = bucket_ns;
    return AGIS_OK;
}

int agis_get_attnoise(agis_ctx* c, double* eps2_a, int32_t* n_buckets) {
    if (!c || !n_buckets) return AGIS_E_INVALID;
    *n_buckets = c->an.n_b;
    if (eps2_a && c->an.n_b > 0) {
        AGIS_CU(c, cudaMemcpyAsync(eps2_a, c->an_eps2, sizeof(double) * 3 * (size_t)c->an.n_b, cudaMemcpyDeviceToHost,
                                   c->stream),
                "get_attnoise");
        AGIS_CU(c, cudaStreamSynchronize(c->stream), "get_attnoise (sync)");
    }
    return AGIS_OK;
}

// --- launch-shape autotuner (ABI functions below) ---------------------------------------

int agis_autotune(agis_ctx* c, int32_t max_iter, int32_t* n_done, agis_tune_entry* out) {
    if (!c || max_iter < 0) return AGIS_E_INVALID;
    if (n_done) *n_done = 0;
    const int mask = c->cfg.block_mask;
    if (!(mask & 1)) return fail(c, AGIS_E_INVALID, "the autotuner times iterations with the S block");
    struct KnobState {
        std::vector<ShapeCand> cand;
        std::vector<double> ms;
        size_t next = 0;
    };
    KnobState ks[AGIS_N_KNOBS];
    for (int k = 0; k < AGIS_N_KNOBS; k++) {
        ks[k].cand = knob_candidates(k, c->mixed);
        if ((k == AGIS_KNOB_ATT_ACCUM && !(mask & 2)) || (k == AGIS_KNOB_CAL_ACCUM && !(mask & 4)))
            ks[k].cand.clear();
        ks[k].ms.assign(ks[k].cand.size(), -1.0);
    }
    // the timed blocks and the knobs each one rates, in order: S pass, S solves, A, C
    const int groups[4][3] = {{AGIS_KNOB_OBS_PASS, -1, -1},
                              {AGIS_KNOB_SRC_BATCH, AGIS_KNOB_MIX_SUMS, AGIS_KNOB_MIX_SOLVE5},
                              {AGIS_KNOB_ATT_ACCUM, -1, -1},
                              {AGIS_KNOB_CAL_ACCUM, -1, -1}};
    auto open_knob = [&](int g) -> int {
        for (int j = 0; j < 3; j++) {
            const int k = groups[g][j];
            if (k >= 0 && ks[k].next < ks[k].cand.size()) return k;
        }
        return -1;
    };
    const int saved_graph = c->cfg.use_graph, saved_prop = c->prop_every, saved_asi = c->asi_stride;
    c->cfg.use_graph = 0;
    c->prop_every = 0;
    c->asi_stride = 0;
    Shapes best = c->sh;
    int it = 0, rc = AGIS_OK;
    for (; it < max_iter; it++) {
        int kk[4];
        bool any = false;
        Shapes trial = best;
        for (int g = 0; g < 4; g++) {
            kk[g] = open_knob(g);
            if (kk[g] < 0) continue;
            any = true;
            const ShapeCand& sc = ks[kk[g]].cand[ks[kk[g]].next];
            knob_set(trial, kk[g], sc.a, sc.b);
        }
        if (!any) break;
        c->sh = trial;
        agis_iter_stats st;
        rc = agis_iterate(c, 1, &st, nullptr);
        if (rc != AGIS_OK) break;
        const double t[4] = {st.s.pass_ms, st.s.elapsed_ms - st.s.pass_ms, st.a.elapsed_ms, st.c.elapsed_ms};
        const bool valid[4] = {!c->mixed || st.s.full_eval == 0, true, true, true};
        for (int g = 0; g < 4; g++) {
            if (kk[g] < 0 || !valid[g] || !(t[g] >= 0.0)) continue;
            KnobState& k = ks[kk[g]];
            k.ms[k.next++] = t[g];
            if (k.next == k.cand.size()) {
                size_t arg = 0;
                for (size_t j = 1; j < k.ms.size(); j++)
                    if (k.ms[j] < k.ms[arg]) arg = j;
                knob_set(best, kk[g], k.cand[arg].a, k.cand[arg].b);
            }
        }
    }
    c->sh = best;
    c->cfg.use_graph = saved_graph;
    c->prop_every = saved_prop;
    c->asi_stride = saved_asi;
    drop_graphs(c);
    if (n_done) *n_done = it;
    if (out) {
        for (int k = 0; k < AGIS_N_KNOBS; k++) {
            agis_tune_entry& e = out[k];
            e.knob = k;
            knob_get(best, k, e.a, e.b);
            e.n_tried = (int32_t)ks[k].next;
            e.best_ms = -1.0;
            for (size_t j = 0; j < ks[k].next; j++)
                if (e.best_ms < 0.0 || ks[k].ms[j] < e.best_ms) e.best_ms = ks[k].ms[j];
            e.default_ms = ks[k].next > 0 ? ks[k].ms[0] : -1.0;
        }
    }
    return rc;
}

int agis_get_tuning(const agis_ctx* c, agis_tune_entry* out) {
    if (!c || !out) return AGIS_E_INVALID;
    for (int k = 0; k < AGIS_N_KNOBS; k++) {
        out[k].knob = k;
        knob_get(c->sh, k, out[k].a, out[k].b);
        out[k].n_tried = 0;
        out[k].best_ms = -1.0;
        out[k].default_ms = -1.0;
    }
    return AGIS_OK;
}

int agis_set_tuning(agis_ctx* c, const agis_tune_entry* in, int32_t n) {
    if (!c || n < 0 || (n > 0 && !in)) return AGIS_E_INVALID;
    Shapes sh = c->sh;
    for (int32_t i = 0; i < n; i++) {
        const int k = in[i].knob;
        if (k < 0 || k >= AGIS_N_KNOBS || !knob_valid(k, in[i].a, in[i].b))
            return fail(c, AGIS_E_INVALID, "launch shape outside the knob's range");
        knob_set(sh, k, in[i].a, in[i].b);
    }
    c->sh = sh;
    drop_graphs(c);
    return AGIS_OK;
}

int agis_get_proposal_features(agis_ctx* c, float* X, double* sigma) {
    if (!c || !X || !sigma) return AGIS_E_INVALID;
    launch_prop_features(c->n_src, c->hist, c->src_off, c->src, c->G.sin_obl, c->G.cos_obl, X, sigma, c->stream);
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "proposal features");
    return cuda_check(c, cudaGetLastError(), "proposal features");
}

int agis_copy_sources_device(agis_ctx* c, double* dst) {
    if (!c || !dst) return AGIS_E_INVALID;
    AGIS_CU(c, cudaMemcpyAsync(dst, c->src, 5 * (size_t)c->n_src * 8, cudaMemcpyDeviceToDevice, c->stream), "copy");
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "copy (sync)");
    return AGIS_OK;
}

int agis_get_sizes(const agis_ctx* c, int64_t* n_obs, int32_t* n_src, int32_t* n_coef, int32_t* n_cal) {
    if (!c) return AGIS_E_INVALID;
    if (n_obs) *n_obs = c->n_obs;
    if (n_src) *n_src = c->n_src;
    if (n_coef) *n_coef = c->n_coef;
    if (n_cal) *n_cal = c->n_cal;
    return AGIS_OK;
}

int agis_get_kernel_times(const agis_ctx* c, double* ms) {
    if (!c || !ms) return AGIS_E_INVALID;
    for (int i = 0; i < 5; i++) ms[i] = c->ktimes[i];
    return AGIS_OK;
}

}  // extern "C"

// --- source partitions: local sums, exchange, solve from the reduced sums --------------------
namespace {
int x_size(const agis_ctx* c, int which, int64_t* n) {
    switch (which) {
        case AGIS_X_ATTITUDE: *n = (int64_t)c->n_iv * kBlkVals; return AGIS_OK;
        case AGIS_X_CALIBRATION: *n = 2 * (int64_t)c->n_cal; return AGIS_OK;
        case AGIS_X_FRAME: *n = 27; return AGIS_OK;
        default: return AGIS_E_INVALID;
    }
}
double* x_buf(agis_ctx* c, int which) {
    return which == AGIS_X_ATTITUDE ? c->blk : which == AGIS_X_CALIBRATION ? c->xcal : c->xframe;
}
int x_check(agis_ctx* c, int which) {
    if (c->mixed) return fail(c, AGIS_E_INVALID, "the exchange of partial sums needs the FP64 form (precision 0)");
    if (which == AGIS_X_CALIBRATION && c->cal_generic)
        return fail(c, AGIS_E_INVALID, "the exchange of calibration sums needs the offsets model (cal_model 0)");
    if (which == AGIS_X_FRAME && !c->ref) return fail(c, AGIS_E_INVALID, "no frame-rotator reference");
    int64_t n = 0;
    if (x_size(c, which, &n) != AGIS_OK) return fail(c, AGIS_E_INVALID, "unknown exchange buffer");
    return AGIS_OK;
}
}  // namespace

int agis_exchange_size(const agis_ctx* c, int32_t which, int64_t* n_doubles) {
    if (!c || !n_doubles) return AGIS_E_INVALID;
    return x_size(c, which, n_doubles);
}

int agis_accumulate(agis_ctx* c, int32_t which) {
    if (!c) return AGIS_E_INVALID;
    AGIS_TRY(x_check(c, which));
    if (which != AGIS_X_FRAME && !c->have_s)
        return fail(c, AGIS_E_INVALID, "the attitude and calibration sums need a source update first");
    if (which == AGIS_X_ATTITUDE) {
        launch_att_accum(c->G, c->st.lambda2, c->st.rhs_norm_term, c->perm_t, c->ivl_off, c->n_iv, c->rec,
                         c->an.eps2 ? c->an_w : nullptr, c->att, c->blk, c->sh, c->stream);
        c->x_att_ready = true;
    } else if (which == AGIS_X_CALIBRATION) {
        if (!c->xcal) AGIS_TRY(dalloc(c, &c->xcal, 2 * (size_t)c->n_cal));
        // block Gauss-Seidel: the residuals C reads take the attitude update (once per A update)
        if (c->cfg.block_order == 1 && c->a_since_c) {
            launch_rec_att_correct(c->G, c->n_obs, c->rec, c->datt64, c->stream);
            c->a_since_c = false;
        }
        launch_cal_sums(c->n_cal, c->perm_c, c->cal_off, c->rec, c->xcal, c->sh, c->stream);
        c->x_cal_ready = true;
    } else {
        if (!c->xframe) AGIS_TRY(dalloc(c, &c->xframe, 27));
        launch_frame_sums(c->n_src, nullptr, c->src, c->ref, c->G, c->fpart, c->n_fpart, c->xframe, c->stream);
        c->x_frame_ready = true;
    }
    AGIS_CU(c, cudaGetLastError(), "accumulate");
    return cuda_check(c, cudaStreamSynchronize(c->stream), "accumulate (sync)");
}

int agis_get_exchange(agis_ctx* c, int32_t which, double* out) {
    if (!c || !out) return AGIS_E_INVALID;
    AGIS_TRY(x_check(c, which));
    int64_t n = 0;
    x_size(c, which, &n);
    double* b = x_buf(c, which);
    if (!b) return fail(c, AGIS_E_INVALID, "no sums accumulated yet");
    AGIS_CU(c, cudaMemcpyAsync(out, b, (size_t)n * 8, cudaMemcpyDefault, c->stream), "get exchange");
    return cuda_check(c, cudaStreamSynchronize(c->stream), "get exchange (sync)");
}

int agis_set_exchange(agis_ctx* c, int32_t which, const double* in) {
    if (!c || !in) return AGIS_E_INVALID;
    AGIS_TRY(x_check(c, which));
    int64_t n = 0;
    x_size(c, which, &n);
    if (which == AGIS_X_CALIBRATION && !c->xcal) AGIS_TRY(dalloc(c, &c->xcal, 2 * (size_t)c->n_cal));
    if (which == AGIS_X_FRAME && !c->xframe) AGIS_TRY(dalloc(c, &c->xframe, 27));
    AGIS_CU(c, cudaMemcpyAsync(x_buf(c, which), in, (size_t)n * 8, cudaMemcpyDefault, c->stream), "set exchange");
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "set exchange (sync)");
    if (which == AGIS_X_ATTITUDE) c->x_att_ready = true;
    if (which == AGIS_X_CALIBRATION) c->x_cal_ready = true;
    if (which == AGIS_X_FRAME) c->x_frame_ready = true;
    return AGIS_OK;
}

int agis_solve_exchange(agis_ctx* c, int32_t which, agis_block_stats* out, double eps_omega_out[6]) {
    if (!c) return AGIS_E_INVALID;
    AGIS_TRY(x_check(c, which));
    if (out) std::memset(out, 0, sizeof(*out));
    record(c, 0);
    if (which == AGIS_X_ATTITUDE) {
        if (!c->x_att_ready) return fail(c, AGIS_E_INVALID, "no attitude sums accumulated or set");
        launch_att_solve(c->n_seg, c->max_seg_knots, c->n_coef, c->n_rows, c->seg_row, c->seg_l, c->seg_n, c->seg_u,
                         c->blk, c->bandc, c->rhs, c->urow, c->yv, c->xs, c->st.pivot_tol, c->seg_rd, c->att, nullptr,
                         c->datt64, c->stream);
        launch_int_sum(c->n_seg, c->seg_rd, c->isum, c->stream);
        c->x_att_ready = false;
        c->a_since_c = true;
    } else if (which == AGIS_X_CALIBRATION) {
        if (!c->x_cal_ready) return fail(c, AGIS_E_INVALID, "no calibration sums accumulated or set");
        launch_cal_from_sums(c->n_cal, c->n_days, c->xcal, c->st.pivot_tol, c->dtil, c->cal_rd, c->cal, c->stream);
        launch_int_sum(c->n_cal, c->cal_rd, c->isum + 1, c->stream);
        c->x_cal_ready = false;
        c->a_since_c = false;
    } else {
        if (!c->x_frame_ready) return fail(c, AGIS_E_INVALID, "no frame sums accumulated or set");
        launch_frame_from_sums(c->G, c->n_src, c->src, c->att, c->xframe, c->st.pivot_tol, c->eo, c->stream);
        c->x_frame_ready = false;
        c->have_s = false;   // the residuals of the last S block refer to the unrotated frame
    }
    record(c, 1);
    AGIS_CU(c, cudaGetLastError(), "solve");
    AGIS_CU(c, cudaMemcpyAsync(c->hisum, c->isum, 2 * sizeof(long long), cudaMemcpyDeviceToHost, c->stream), "stats");
    AGIS_CU(c, cudaMemcpyAsync(c->hstat + 16, c->eo, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "stats");
    AGIS_CU(c, cudaStreamSynchronize(c->stream), "solve (sync)");
    if (out) {
        out->rank_defect = which == AGIS_X_ATTITUDE ? c->hisum[0] : which == AGIS_X_CALIBRATION ? c->hisum[1] : 0;
        out->elapsed_ms = elapsed(c, 0, 1);
    }
    if (which == AGIS_X_FRAME && eps_omega_out)
        for (int i = 0; i < 6; i++) eps_omega_out[i] = c->hstat[16 + i];
    return AGIS_OK;
}

namespace agis {
// message returned by agis_last_error(NULL) for calls that have no context
void set_thread_error(const std::string& msg) { g_init_err = msg; }
}  // namespace agis
