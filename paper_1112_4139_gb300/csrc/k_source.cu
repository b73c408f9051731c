// k_source.cu -- the observation pass in source order and the S block (Sect. 5.1).
//
// One warp per source (persistent warps take sources from a work counter, largest first).
// The warp evaluates every observation of the source once (residual h_l, design row A_l,
// attitude partial g_l), keeps (h, A, w, sigma^2) in a per-warp scratch slice that stays in
// L2 during the inner iteration, and runs the inner iteration of Sect. 5.1.2 with
// butterfly (xor-shuffle) reductions, so every lane holds the same 5x5 system and solves it
// redundantly.  At the end it writes the hand-over record (t, R = h - A d, W, g, meta) that
// the time-ordered attitude pass and the calibration pass gather.
#include "agis_internal.cuh"

namespace agis {



// k-th smallest (0-based) of the keys[0..n) (order-preserving maps of h / sigma, one 8-byte key
// per observation, contiguous) by a radix select of 8-bit digits with a 256-bin shared-memory
// histogram per warp.  A pass whose chosen digit holds a single key ends the select: one more
// pass finds that key (on continuous data about 4 passes instead of 8).
__device__ uint64_t warp_select(const uint64_t* __restrict__ keys, int n, int k, int* hist, int lane) {
    uint64_t prefix = 0, pmask = 0;
    int kk = k;
    for (int d = 7; d >= 0; d--) {
        int shift = 8 * d;
#pragma unroll
        for (int i = 0; i < 8; i++) hist[lane * 8 + i] = 0;
        __syncwarp();
        for (int j = lane; j < n; j += kWarp) {
            const uint64_t key = keys[j];
            if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1);
        }
        __syncwarp();
        int c[8];
        int tot = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) { c[i] = hist[lane * 8 + i]; tot += c[i]; }
        // inclusive scan across lanes
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int excl = incl - tot;
        unsigned ball = __ballot_sync(0xffffffffu, incl > kk);
        int src_lane = __ffs(ball) - 1;
        int bin = 0, below = 0, cnt = 0;
        if (lane == src_lane) {
            int acc = excl;
            int bsel = 7;
#pragma unroll
            for (int i = 0; i < 8; i++) {
                if (acc + c[i] > kk) { bsel = i; break; }
                acc += c[i];
            }
            bin = lane * 8 + bsel;
            below = acc;
            cnt = hist[bin];
        }
        bin = __shfl_sync(0xffffffffu, bin, src_lane);
        below = __shfl_sync(0xffffffffu, below, src_lane);
        cnt = __shfl_sync(0xffffffffu, cnt, src_lane);
        kk -= below;
        prefix |= (uint64_t)bin << shift;
        pmask |= (uint64_t)0xffu << shift;
        __syncwarp();
        if (cnt == 1 && d > 0) {
            // the only key with this prefix is the k-th smallest
            uint64_t found = 0;
            for (int j = lane; j < n; j += kWarp) {
                const uint64_t key = keys[j];
                if ((key & pmask) == prefix) found = key;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint64_t v = __shfl_xor_sync(0xffffffffu, found, o);
                found = v > found ? v : found;
            }
            return found;
        }
    }
    return prefix;
}

// the (k)-th and (k+1)-th smallest values (k+1 capped at n-1)
__device__ void warp_select_pair(const uint64_t* __restrict__ keys, int n, int k, int* hist, int lane, double& v0,
                                 double& v1) {
    uint64_t K = warp_select(keys, n, k, hist, lane);
    v0 = dkey_inv(K);
    if (k + 1 >= n) { v1 = v0; return; }
    int less = 0, eq = 0;
    uint64_t nxt = ~0ull;
    for (int j = lane; j < n; j += kWarp) {
        const uint64_t key = keys[j];
        less += key < K;
        eq += key == K;
        if (key > K && key < nxt) nxt = key;
    }
    less = warp_sum_int(less);
    eq = warp_sum_int(eq);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t v = __shfl_xor_sync(0xffffffffu, nxt, o);
        nxt = v < nxt ? v : nxt;
    }
    v1 = (k + 1 < less + eq) ? v0 : dkey_inv(nxt);
}

struct Sys5 {
    double N[15];
    double b[5];
};

// normal equations with W = w / (sigma^2 + y); optionally refresh w from the previous solve
__device__ __forceinline__ void pass_normals(double* scr, int n, int lane, double y, bool refresh, const double* dp,
                                             double yp, int wfn, Sys5& S, int& nout) {
#pragma unroll
    for (int i = 0; i < 15; i++) S.N[i] = 0.0;
#pragma unroll
    for (int i = 0; i < 5; i++) S.b[i] = 0.0;
    int cnt = 0;
    for (int j = lane; j < n; j += kWarp) {
        double* e = scr + (size_t)j * kScr;
        double h = e[0];
        double A[5] = {e[1], e[2], e[3], e[4], e[5]};
        double w = e[6];
        double s2 = e[7];
        if (refresh) {
            double R = h - (A[0] * dp[0] + A[1] * dp[1] + A[2] * dp[2] + A[3] * dp[3] + A[4] * dp[4]);
            w = wfun(R / sqrt(s2 + yp), wfn);
            e[6] = w;
        }
        cnt += (w < 0.2);
        double W = w / (s2 + y);
#pragma unroll
        for (int a = 0; a < 5; a++) {
            double wa = W * A[a];
#pragma unroll
            for (int c = a; c < 5; c++) S.N[up5(a, c)] += wa * A[c];
            S.b[a] += wa * h;
        }
    }
#pragma unroll
    for (int i = 0; i < 15; i++) S.N[i] = warp_sum(S.N[i]);
#pragma unroll
    for (int i = 0; i < 5; i++) S.b[i] = warp_sum(S.b[i]);
    nout = warp_sum_int(cnt);
}

// Q(y) = sum w R^2 / (s2 + y) and S2 = sum w R^2 / (s2 + y)^2 for R = h - A d
__device__ __forceinline__ void pass_q(const double* scr, int n, int lane, const double* d, double y, double& Q,
                                       double& S2) {
    double q = 0.0, s = 0.0;
    for (int j = lane; j < n; j += kWarp) {
        const double* e = scr + (size_t)j * kScr;
        double R = e[0] - (e[1] * d[0] + e[2] * d[1] + e[3] * d[2] + e[4] * d[3] + e[5] * d[4]);
        double den = e[7] + y;
        double t = e[6] * R * R / den;
        q += t;
        s += t / den;
    }
    Q = warp_sum(q);
    S2 = warp_sum(s);
}

// Weight of one row in the class-sum path.  mode 0 (initial downweighting): w = wfun(x / vs)
// with x = h / sigma_c, evaluated as h * rx with rx = 1 / (sigma_c vs) (rx = 0: vs = 0, w = 1);
// mode 1 (later rounds): w = wfun(R / sqrt(sigma_c^2 + y_prev)) with R = h - A d_prev; mode 2
// (plain weights): w = 1.
__device__ __forceinline__ double class_w(int mode, double h, const double* A, const double* dp, double rx,
                                          double inv_sd, int wfn) {
    if (mode == 2) return 1.0;
    if (mode == 0) return rx > 0.0 ? wfun(h * rx, wfn) : 1.0;
    double Ad = A[0] * dp[0];
    Ad = fma(A[1], dp[1], Ad);
    Ad = fma(A[2], dp[2], Ad);
    Ad = fma(A[3], dp[3], Ad);
    Ad = fma(A[4], dp[4], Ad);
    return wfun((h - Ad) * inv_sd, wfn);
}

// Per-class inputs of one round of a source: sigma_c, rx = 1 / (sigma_c vs), 1 / sqrt(s2_c + y)
struct RoundIn {
    double rx[2], isd[2];
};
__device__ __forceinline__ RoundIn round_in(const double* s2c, double y, double vs) {
    RoundIn r;
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const double sig = sqrt(s2c[c]);
        r.rx[c] = vs > 0.0 ? 1.0 / (sig * vs) : 0.0;
        r.isd[c] = 1.0 / sqrt(s2c[c] + y);
    }
    return r;
}

// Lane partial sums of one class over its contiguous range [lo, hi) of the source's rows (AL
// rows come first), with the weights of class_w, written to column `lane` of the warp's
// reduction buffer red[21][kRedStride] (15 AA, 5 Ah, hh); the last round (store) keeps w in
// the scratch row for the hand-over records.
constexpr int kRedVals = 42;      // both classes
constexpr int kRedStride = 33;    // doubles per value row (odd: the column sums read distinct banks)
__device__ __forceinline__ void pass_class1(double* scr, int lo, int hi, int lane, int mode, double rx,
                                            const double* dp, double inv_sd, int wfn, bool store, double* red,
                                            int& nout) {
    double AA[15], Ah[5];
#pragma unroll
    for (int i = 0; i < 15; i++) AA[i] = 0.0;
#pragma unroll
    for (int i = 0; i < 5; i++) Ah[i] = 0.0;
    double hs = 0.0;
    int cnt = 0;
    for (int j = lo + lane; j < hi; j += kWarp) {
        double* e = scr + (size_t)j * kScr;
        const double h = e[0];
        const double A[5] = {e[1], e[2], e[3], e[4], e[5]};
        const double w = class_w(mode, h, A, dp, rx, inv_sd, wfn);
        if (store) e[6] = w;
        cnt += (w < 0.2);
#pragma unroll
        for (int a = 0; a < 5; a++) {
            const double wa = w * A[a];
#pragma unroll
            for (int b = a; b < 5; b++) AA[up5(a, b)] += wa * A[b];
            Ah[a] += wa * h;
        }
        hs += w * h * h;
    }
#pragma unroll
    for (int i = 0; i < 15; i++) red[i * kRedStride + lane] = AA[i];
#pragma unroll
    for (int i = 0; i < 5; i++) red[(15 + i) * kRedStride + lane] = Ah[i];
    red[20 * kRedStride + lane] = hs;
    nout = warp_sum_int(cnt);
}

// both classes: the 42 lane partials go to the warp's reduction buffer, and lane v adds the
// 32 partials of value v in lane order (31 additions per value instead of 5 per value in every
// lane for butterflies); the sums go to the warp's shared-memory slot S, so that they do not
// occupy registers during the 5x5 algebra
__device__ __forceinline__ void pass_class(double* scr, int n, int nal, int lane, int mode, const RoundIn& ri,
                                           const double* dp, int wfn, bool store, ClassSums& S, int& nout,
                                           double* red) {
    int nc[2];
    for (int c = 0; c < 2; c++)
        pass_class1(scr, c ? nal : 0, c ? n : nal, lane, mode, ri.rx[c], dp, ri.isd[c], wfn, store,
                    red + c * 21 * kRedStride, nc[c]);
    __syncwarp();
    for (int v = lane; v < kRedVals; v += kWarp) {
        const double* col = red + v * kRedStride;
        double t = col[0];
#pragma unroll
        for (int k = 1; k < kWarp; k++) t += col[k];
        const int c = v / 21, i = v % 21;
        if (i < 15) S.AA[c][i] = t;
        else if (i < 20) S.Ah[c][i - 15] = t;
        else S.hh[c] = t;
    }
    __syncwarp();
    nout = nc[0] + nc[1];
}

// Per-source geometry for the observation pass: p, q, r (Eq. normal-triad), parameters, cos(delta).
__global__ void k_src_geo(int32_t n_src, const double* __restrict__ src, double* __restrict__ geo) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += gridDim.x * blockDim.x) {
        SrcGeo S;
        source_geo(src + 5 * (size_t)i, S);
        double* g = geo + 16 * (size_t)i;
        for (int k = 0; k < 3; k++) { g[k] = S.p[k]; g[3 + k] = S.q[k]; g[6 + k] = S.r[k]; }
        g[9] = S.par; g[10] = S.pma; g[11] = S.pmd; g[12] = S.cosd;
        // slots 13-15: p and q rounded to FP32 (six floats)
        float* gf = reinterpret_cast<float*>(g + 13);
        for (int k = 0; k < 3; k++) { gf[k] = (float)S.p[k]; gf[3 + k] = (float)S.q[k]; }
    }
}

// Observation pass, one thread per observation (source order): residual h, design row A and
// attitude partial g at the current parameters.  Scratch row: h, A[5], key(h/sigma), sigma^2;
// with the excess attitude noise on, sigma~^2 = sigma^2 + eps_a^2(t) in place of sigma^2 (Eq. W).
__global__ void __launch_bounds__(256) k_obs_forward(DevGeo G, AttNoise an, int64_t n_obs, const int64_t* __restrict__ t_ns,
                                                     const uint32_t* __restrict__ meta,
                                                     const float* __restrict__ sigma, const double* __restrict__ mu,
                                                     const int32_t* __restrict__ obs_src,
                                                     const double* __restrict__ geo, const double* __restrict__ att,
                                                     const double* __restrict__ cal, double* __restrict__ scr,
                                                     uint64_t* __restrict__ skey, ObsRec* __restrict__ rec) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_obs; o += (int64_t)gridDim.x * blockDim.x) {
        const double* g = geo + 16 * (size_t)obs_src[o];
        SrcGeo S;
        for (int k = 0; k < 3; k++) { S.p[k] = g[k]; S.q[k] = g[3 + k]; S.r[k] = g[6 + k]; }
        S.par = g[9]; S.pma = g[10]; S.pmd = g[11]; S.cosd = g[12];
        const int64_t t = t_ns[o];
        const uint32_t m = meta[o];
        const double muv = (G.cg.on || meta_kind(m)) ? mu[o] : 0.0;
        ObsOut ob;
        observe<1>(G, S, t, m, muv, att, cal, ob);
        const double sg = (double)sigma[o];
        double s2 = sg * sg, x = ob.R * rcp_pos(sg);
        if (an.eps2) {
            s2 = s2 + an.eps2[an_index(an, t, m)];
            x = ob.R * rsqrt(s2);
        }
        double* e = scr + (size_t)o * kScr;
        e[0] = ob.R;
        e[1] = ob.A[0]; e[2] = ob.A[1]; e[3] = ob.A[2]; e[4] = ob.A[3]; e[5] = ob.A[4];
        skey[o] = dkey(x);
        e[7] = s2;
        ObsRec* r = rec + o;
        r->t_ns = t;
        r->meta = m;
        r->pad = 0;
        r->g[0] = ob.g[0]; r->g[1] = ob.g[1]; r->g[2] = ob.g[2]; r->g[3] = ob.g[3];
    }
}

// General path for one source (any sigma per observation): per-observation passes for every
// excess-noise step.  Whole warp; the robust sigma vs is given.
__device__ __noinline__ void solve_general(const Settings& st, int i, int64_t o0, int n, const double* s5, double cosd,
                                           double* scr, double s2min, double vs, const SrcOutPtrs& out,
                                           ObsRec* __restrict__ rec, int lane) {
    if (st.robust) {
        for (int j = lane; j < n; j += kWarp) {
            double* e = scr + (size_t)j * kScr;
            const double x = e[0] / sqrt(e[7]);
            e[6] = vs > 0.0 ? wfun(x / vs, st.weight_fn) : 1.0;
        }
    } else {
        for (int j = lane; j < n; j += kWarp) scr[(size_t)j * kScr + 6] = 1.0;
    }
    __syncwarp();
    double d[5] = {0, 0, 0, 0, 0};
    double U[kU5];
    double y = 0.0, Q = 0.0, Q0 = 0.0;
    int nu = 0, nout = 0, rd = 0;
    const int rounds = st.robust ? st.n_rounds + 1 : 1;
    for (int rnd = 0; rnd < rounds; rnd++) {
        Sys5 sy;
        double dprev[5] = {d[0], d[1], d[2], d[3], d[4]};
        const double yprev = y;
        y = 0.0;
        pass_normals(scr, n, lane, 0.0, rnd > 0, dprev, yprev, st.weight_fn, sy, nout);
        nu = n - nout - 5;
        rd = chol5(sy.N, U, st.pivot_tol);
        chol5_solve(U, sy.b, d);
        double S2;
        pass_q(scr, n, lane, d, 0.0, Q, S2);
        Q0 = Q;
        if (st.robust && nu > 0 && Q0 > (double)nu) {
            const double tol = 1e-12 * s2min;
            for (int it = 0; it < st.n_eps; it++) {
                double dy = (1.0 - Q / (double)nu) * Q / (-S2);
                y = fmax(0.0, y + dy);
                pass_normals(scr, n, lane, y, false, dprev, yprev, st.weight_fn, sy, nout);
                rd = chol5(sy.N, U, st.pivot_tol);
                chol5_solve(U, sy.b, d);
                pass_q(scr, n, lane, d, y, Q, S2);
                if (fabs(dy) <= tol) break;
            }
        }
        __syncwarp();
    }
    double chi = 0.0;
    for (int j = lane; j < n; j += kWarp) {
        const double* e = scr + (size_t)j * kScr;
        double R = e[0] - (e[1] * d[0] + e[2] * d[1] + e[3] * d[2] + e[4] * d[3] + e[5] * d[4]);
        double W = e[6] / (e[7] + y);
        ObsRec* r = rec + (o0 + j);
        r->R = st.handover_h ? e[0] : R;
        r->W = W;
        chi += W * R * R;
    }
    chi = warp_sum(chi);
    if (lane == 0) {
        double* sp = out.src + 5 * (size_t)i;
        sp[0] = s5[0] + d[0] / cosd;
        sp[1] = s5[1] + d[1];
        sp[2] = s5[2] + d[2];
        sp[3] = s5[3] + d[3];
        sp[4] = s5[4] + d[4];
        for (int k = 0; k < 5; k++) out.d[5 * (size_t)i + k] = d[k];
        for (int c = 0; c < 5; c++) {
            double e[5] = {0, 0, 0, 0, 0};
            e[c] = 1.0;
            double x[5];
            chol5_solve(U, e, x);
            for (int k = 0; k < 5; k++) out.cov[25 * (size_t)i + 5 * k + c] = x[k];
        }
        out.eps2[i] = y;
        out.q[i] = Q;
        out.nu[i] = nu;
        out.nout[i] = nout;
        out.dsig[i] = nu > 0 ? (Q0 - (double)nu) / sqrt(2.0 * (double)nu) : 0.0;
        out.chi2[i] = chi;
        out.rankdef[i] = rd;
    }
    __syncwarp();
}

// Per-source solve, batched: a warp takes `batch` consecutive sources of the largest-first
// order.  The warp sweeps each source's observations cooperatively (robust sigma, per-class
// sums, hand-over records); lane k keeps source k's state and class sums, so the 5x5
// algebra of the excess-noise steps runs for the whole batch in parallel instead of
// redundantly in every lane.  Sources whose observations do not have one sigma per class use
// the general per-observation path.
constexpr int kSolveWarps = 2;
__global__ void __launch_bounds__(32 * kSolveWarps, 1) k_source_solve(
    Settings st, const uint32_t* __restrict__ meta, const int64_t* __restrict__ src_off,
    const int32_t* __restrict__ src_nal, const int32_t* __restrict__ src_order, int32_t n_src, int batch,
    SrcOutPtrs out, ObsRec* __restrict__ rec, double* __restrict__ scratch, const uint64_t* __restrict__ skey,
    int* work_counter) {
    __shared__ int hist_all[kSolveWarps * 256];
    __shared__ ClassSums sums_all[kSolveWarps][kWarp];
    __shared__ double red_all[kSolveWarps][kRedVals * kRedStride];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int* hist = hist_all + wib * 256;
    ClassSums* sums = sums_all[wib];
    double* red = red_all[wib];
    const int rounds = st.robust ? st.n_rounds + 1 : 1;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(work_counter, batch);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_src) break;
        const int nb = min(batch, n_src - base);
        // ---- this lane's source
        const bool mine = lane < nb;
        const int my_i = mine ? src_order[base + lane] : 0;
        const int64_t my_o0 = mine ? src_off[my_i] : 0;
        const int my_n = mine ? (int)(src_off[my_i + 1] - my_o0) : 0;
        const int my_nal = mine ? src_nal[my_i] : 0;
        double s5[5] = {0, 0, 0, 0, 0};
        if (mine)
            for (int k = 0; k < 5; k++) s5[k] = out.src[5 * (size_t)my_i + k];
        const double cosd = cos(s5[1]);
        double my_s2c[2] = {1.0, 1.0}, my_s2min = 1.0, my_vs = 0.0;
        bool my_uniform = false;
        // ---- per source: sigma per class, robust sigma
        for (int k = 0; k < nb; k++) {
            const int64_t o0 = __shfl_sync(0xffffffffu, my_o0, k);
            const int n = __shfl_sync(0xffffffffu, my_n, k);
            if (n == 0) continue;
            double* scr = scratch + (size_t)o0 * kScr;
            double s2min = 1e300;
            double s2lo[2] = {1e300, 1e300}, s2hi[2] = {-1e300, -1e300};
            for (int j = lane; j < n; j += kWarp) {
                const double s2 = scr[(size_t)j * kScr + 7];
                const int c = meta_kind(meta[o0 + j]);
                s2lo[c] = fmin(s2lo[c], s2);
                s2hi[c] = fmax(s2hi[c], s2);
                s2min = fmin(s2min, s2);
            }
            s2min = warp_min(s2min);
            for (int c = 0; c < 2; c++) {
                s2lo[c] = warp_min(s2lo[c]);
                s2hi[c] = -warp_min(-s2hi[c]);
            }
            const bool uni = (s2lo[0] == s2hi[0] || s2lo[0] == 1e300) && (s2lo[1] == s2hi[1] || s2lo[1] == 1e300);
            __syncwarp();
            double vs = 0.0;
            if (st.robust) {
                const double p1 = 1.0 / 6.0, p5 = 5.0 / 6.0;
                const double h1 = p1 * (double)(n - 1), h5 = p5 * (double)(n - 1);
                const int lo1 = (int)floor(h1), lo5 = (int)floor(h5);
                double a0, a1, b0, b1;
                warp_select_pair(skey + o0, n, lo1, hist, lane, a0, a1);
                warp_select_pair(skey + o0, n, lo5, hist, lane, b0, b1);
                vs = 0.5 * ((b0 + (h5 - lo5) * (b1 - b0)) - (a0 + (h1 - lo1) * (a1 - a0)));
                __syncwarp();
            }
            __syncwarp();
            if (lane == k) {
                my_uniform = uni;
                my_s2c[0] = s2lo[0] == 1e300 ? 1.0 : s2lo[0];
                my_s2c[1] = s2lo[1] == 1e300 ? 1.0 : s2lo[1];
                my_s2min = s2min;
                my_vs = vs;
            }
        }
        // ---- inner iteration, class-sum path (lane k solves source k)
        double d[5] = {0, 0, 0, 0, 0};
        double U[kU5];
        for (int q = 0; q < kU5; q++) U[q] = 0.0;
        double y = 0.0, Q = 0.0, Q0 = 0.0, S2 = 0.0;
        int nu = 0, nout = 0, rd = 0;
        for (int rnd = 0; rnd < rounds; rnd++) {
            const int mode = !st.robust ? 2 : (rnd == 0 ? 0 : 1);
            for (int k = 0; k < nb; k++) {
                const int n = __shfl_sync(0xffffffffu, my_n, k);
                const int uni = __shfl_sync(0xffffffffu, (int)my_uniform, k);
                if (n == 0 || !uni) continue;
                const int64_t o0 = __shfl_sync(0xffffffffu, my_o0, k);
                const int nal = __shfl_sync(0xffffffffu, my_nal, k);
                double dk[5];
                for (int a = 0; a < 5; a++) dk[a] = __shfl_sync(0xffffffffu, d[a], k);
                const double yk = __shfl_sync(0xffffffffu, y, k);
                const double s2c[2] = {__shfl_sync(0xffffffffu, my_s2c[0], k), __shfl_sync(0xffffffffu, my_s2c[1], k)};
                const double vsk = __shfl_sync(0xffffffffu, my_vs, k);
                const RoundIn ri = round_in(s2c, yk, vsk);
                double* scr = scratch + (size_t)o0 * kScr;
                int no = 0;
                pass_class(scr, n, nal, lane, mode, ri, dk, st.weight_fn, rnd == rounds - 1, sums[k], no, red);
                if (lane == k) nout = no;
            }
            __syncwarp();
            if (mine && my_n > 0 && my_uniform) {
                nu = my_n - nout - 5;
                y = 0.0;
                class_solve(sums[lane], my_s2c, 0.0, st.pivot_tol, U, d, rd, Q, S2);
                Q0 = Q;
                if (st.robust && nu > 0 && Q0 > (double)nu) {
                    const double tol = 1e-12 * my_s2min;
                    for (int it = 0; it < st.n_eps; it++) {
                        const double dy = (1.0 - Q / (double)nu) * Q / (-S2);
                        y = fmax(0.0, y + dy);
                        class_solve(sums[lane], my_s2c, y, st.pivot_tol, U, d, rd, Q, S2);
                        if (fabs(dy) <= tol) break;
                    }
                }
            }
            __syncwarp();
        }
        // ---- hand-over records and per-source results
        double my_chi = 0.0;
        for (int k = 0; k < nb; k++) {
            const int n = __shfl_sync(0xffffffffu, my_n, k);
            const int uni = __shfl_sync(0xffffffffu, (int)my_uniform, k);
            if (n == 0 || !uni) continue;
            const int64_t o0 = __shfl_sync(0xffffffffu, my_o0, k);
            const int nal = __shfl_sync(0xffffffffu, my_nal, k);
            double dk[5];
            for (int a = 0; a < 5; a++) dk[a] = __shfl_sync(0xffffffffu, d[a], k);
            const double yk = __shfl_sync(0xffffffffu, y, k);
            const double iw[2] = {1.0 / (__shfl_sync(0xffffffffu, my_s2c[0], k) + yk),
                                  1.0 / (__shfl_sync(0xffffffffu, my_s2c[1], k) + yk)};
            const double* scr = scratch + (size_t)o0 * kScr;
            double chi = 0.0;
            for (int j = lane; j < n; j += kWarp) {
                const double* e = scr + (size_t)j * kScr;
                const double R = e[0] - (e[1] * dk[0] + e[2] * dk[1] + e[3] * dk[2] + e[4] * dk[3] + e[5] * dk[4]);
                const double W = e[6] * (j < nal ? iw[0] : iw[1]);
                ObsRec* r = rec + (o0 + j);
                r->R = st.handover_h ? e[0] : R;
                r->W = W;
                chi += W * R * R;
            }
            chi = warp_sum(chi);
            if (lane == k) my_chi = chi;
        }
        if (mine && (my_n == 0 || my_uniform)) {
            const int i = my_i;
            if (my_n == 0) {
                for (int k = 0; k < 5; k++) out.d[5 * (size_t)i + k] = 0.0;
                for (int k = 0; k < 25; k++) out.cov[25 * (size_t)i + k] = 0.0;
                out.eps2[i] = out.q[i] = out.dsig[i] = out.chi2[i] = 0.0;
                out.nu[i] = out.nout[i] = out.rankdef[i] = 0;
            } else {
                double* sp = out.src + 5 * (size_t)i;
                sp[0] = s5[0] + d[0] / cosd;
                sp[1] = s5[1] + d[1];
                sp[2] = s5[2] + d[2];
                sp[3] = s5[3] + d[3];
                sp[4] = s5[4] + d[4];
                for (int k = 0; k < 5; k++) out.d[5 * (size_t)i + k] = d[k];
                for (int c = 0; c < 5; c++) {
                    double e[5] = {0, 0, 0, 0, 0};
                    e[c] = 1.0;
                    double x[5];
                    chol5_solve(U, e, x);
                    for (int k = 0; k < 5; k++) out.cov[25 * (size_t)i + 5 * k + c] = x[k];
                }
                out.eps2[i] = y;
                out.q[i] = Q;
                out.nu[i] = nu;
                out.nout[i] = nout;
                out.dsig[i] = nu > 0 ? (Q0 - (double)nu) / sqrt(2.0 * (double)nu) : 0.0;
                out.chi2[i] = my_chi;
                out.rankdef[i] = rd;
            }
        }
        __syncwarp();
        // ---- sources without one sigma per class: general path, one at a time
        for (int k = 0; k < nb; k++) {
            const int n = __shfl_sync(0xffffffffu, my_n, k);
            const int uni = __shfl_sync(0xffffffffu, (int)my_uniform, k);
            if (n == 0 || uni) continue;
            const int i = __shfl_sync(0xffffffffu, my_i, k);
            const int64_t o0 = __shfl_sync(0xffffffffu, my_o0, k);
            double sk[5];
            for (int a = 0; a < 5; a++) sk[a] = __shfl_sync(0xffffffffu, s5[a], k);
            const double ck = __shfl_sync(0xffffffffu, cosd, k);
            const double s2m = __shfl_sync(0xffffffffu, my_s2min, k);
            const double vsk = __shfl_sync(0xffffffffu, my_vs, k);
            solve_general(st, i, o0, n, sk, ck, scratch + (size_t)o0 * kScr, s2m, vsk, out, rec, lane);
        }
    }
}

// Residuals at the current parameters, one thread per observation (no update).
__global__ void k_evaluate(DevGeo G, const int64_t* __restrict__ t_ns, const uint32_t* __restrict__ meta,
                           const double* __restrict__ mu, const int32_t* __restrict__ obs_src, int64_t n_obs,
                           const double* __restrict__ src, const double* __restrict__ att,
                           const double* __restrict__ cal, double* __restrict__ R) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_obs; o += (int64_t)gridDim.x * blockDim.x) {
        SrcGeo S;
        source_geo(src + 5 * (size_t)obs_src[o], S);
        uint32_t m = meta[o];
        ObsOut ob;
        observe<0>(G, S, t_ns[o], m, (G.cg.on || meta_kind(m)) ? mu[o] : 0.0, att, cal, ob);
        R[o] = ob.R;
    }
}

// the observation pass of the S block: source geometry, then the model at every observation
void launch_obs_pass(const DevGeo& G, const AttNoise& an, const int64_t* t_ns, const uint32_t* meta, const float* sigma,
                     const double* mu, const int32_t* obs_src, int64_t n_obs, int32_t n_src, const double* src,
                     const double* att, const double* cal, ObsRec* rec, double* geo, double* scratch,
                     uint64_t* skey, const Shapes& sh, cudaStream_t stream) {
    k_src_geo<<<(n_src + 255) / 256 > 0 ? (n_src + 255) / 256 : 1, 256, 0, stream>>>(n_src, src, geo);
    const int th = sh.obs_threads;
    int64_t fb = (n_obs + th - 1) / th;
    if (fb > 152 * (int64_t)sh.obs_bps) fb = 152 * (int64_t)sh.obs_bps;
    if (fb < 1) fb = 1;
    k_obs_forward<<<(int)fb, th, 0, stream>>>(G, an, n_obs, t_ns, meta, sigma, mu, obs_src, geo, att, cal, scratch, skey,
                                              rec);
}

// the per-source solves of the S block on the scratch rows of the observation pass
void launch_source_solve(const Settings& st, const uint32_t* meta, const int64_t* src_off, const int32_t* src_nal,
                         const int32_t* src_order, int32_t n_src, const SrcOutPtrs& out, ObsRec* rec, double* scratch,
                         const uint64_t* skey, int* work_counter, int n_blocks, const Shapes& sh, cudaStream_t stream) {
    cudaMemsetAsync(work_counter, 0, sizeof(int), stream);
    // batch size: 32 sources per warp when there are enough sources to keep ~16 warps per SM
    // busy, unless the autotuner chose one
    int batch = n_src / (152 * 16);
    batch = batch < 1 ? 1 : (batch > 32 ? 32 : batch);
    if (sh.src_batch > 0) batch = sh.src_batch;
    int warps = (n_src + batch - 1) / batch;
    int blocks = (warps + kSolveWarps - 1) / kSolveWarps;
    if (blocks > n_blocks * 4) blocks = n_blocks * 4;
    if (blocks < 1) blocks = 1;
    k_source_solve<<<blocks, 32 * kSolveWarps, 0, stream>>>(st, meta, src_off, src_nal, src_order, n_src, batch, out,
                                                            rec, scratch, skey, work_counter);
}

void launch_src_geo(int32_t n_src, const double* src, double* geo, cudaStream_t s) {
    k_src_geo<<<(n_src + 255) / 256 > 0 ? (n_src + 255) / 256 : 1, 256, 0, s>>>(n_src, src, geo);
}

void launch_evaluate(const DevGeo& G, const int64_t* t_ns, const uint32_t* meta, const double* mu,
                     const int32_t* obs_src, int64_t n_obs, const double* src, const double* att, const double* cal,
                     double* R, cudaStream_t stream) {
    int blocks = (int)((n_obs + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    k_evaluate<<<blocks, 256, 0, stream>>>(G, t_ns, meta, mu, obs_src, n_obs, src, att, cal, R);
}

}  // namespace agis
