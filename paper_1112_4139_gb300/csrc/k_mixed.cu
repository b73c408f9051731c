// k_mixed.cu -- the mixed-precision form of the observation pass and of the S, A and C
// accumulations.
//
// Each observation keeps two 32-byte records (source order, see MixS / MixT).  A full FP64
// evaluation of the model (k_mix_forward) refreshes R and the FP32 partials every few
// source updates; in between, R follows the first-order identity behind Eq. precond2:
// after the A and C blocks k_mix_correct adds (dR/da) d_a + (dR/dc) d_c, and the source
// solve subtracts A d.  R itself stays FP64, so the updates solve for corrections of an FP64
// residual (iterative refinement): FP32 rounding of the normal equations changes the rate
// of convergence, not the point it converges to.  The 5x5 and band Cholesky factorisations
// and the frame rotator stay FP64.
#include "agis_internal.cuh"

namespace agis {

void launch_src_geo(int32_t n_src, const double* src, double* geo, cudaStream_t s);
void launch_cal_project(int n_days, const double* dtil, double* cal, double* d_cal, cudaStream_t s);

namespace {

int grid_of(int64_t n, int per_block, int cap) {
    int64_t b = (n + per_block - 1) / per_block;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

// B_{l-3..l}(t) in FP32: closed form on regular intervals (the offset from the knot is an
// exact integer number of ns before its conversion), Algorithm B.1 in FP64 near the end knots.
__device__ __forceinline__ void bspline4f(const DevGeo& G, int64_t t, int l, float b[4]) {
    if (l >= 5 && l <= G.n_coef - 3) {
        const float u = (float)(t - knot_at(G, l)) * (float)G.inv_knot_dt;
        const float v = 1.0f - u;
        const float u2 = u * u, u3 = u2 * u;
        b[0] = v * v * v * (1.0f / 6.0f);
        b[1] = (3.0f * u3 - 6.0f * u2 + 4.0f) * (1.0f / 6.0f);
        b[2] = (-3.0f * u3 + 3.0f * u2 + 3.0f * u + 1.0f) * (1.0f / 6.0f);
        b[3] = u3 * (1.0f / 6.0f);
        return;
    }
    double bd[4];
    bspline4(G, t, l, bd);
    for (int j = 0; j < 4; j++) b[j] = (float)bd[j];
}

__device__ __forceinline__ float wfun_f(float z, int fn) {
    const float a = fabsf(z);
    if (fn == 0) {
        if (a <= 2.0f) return 1.0f;
        if (a < 3.0f) {
            const float t = a - 2.0f;
            return 1.0f - 1.773735f * t * t + 1.141615f * t * t * t;
        }
        return expf(-a * (1.0f / 3.0f));
    }
    if (a <= 2.0f) return 1.0f;
    return 2.0f * (2.0f * a - 2.0f) / (a * a);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void arow(const MixS& r, float A[5]) {
    A[0] = r.Ap; A[1] = r.Aq; A[2] = r.Aw; A[3] = r.Ap * r.tau; A[4] = r.Aq * r.tau;
}
__device__ __forceinline__ float adot(const float A[5], const float* d) {
    return A[0] * d[0] + A[1] * d[1] + A[2] * d[2] + A[3] * d[3] + A[4] * d[4];
}
// A d in FP64 with the FP32 design row of the normal equations (A[3], A[4] rounded as there)
__device__ __forceinline__ double adot_d(const MixS& r, const double* d) {
    return (double)r.Ap * d[0] + (double)r.Aq * d[1] + (double)r.Aw * d[2] + (double)(r.Ap * r.tau) * d[3] +
           (double)(r.Aq * r.tau) * d[4];
}

// ---- order statistics of x = R / sigma over a source (4-pass radix select on FP32 keys)
__device__ __forceinline__ uint32_t fkey(float x) {
    const uint32_t b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ uint32_t xkey(const MixS* rs, int j) {
    return fkey((float)rs[j].R / fabsf(rs[j].sig));
}

__device__ uint32_t mix_select(const MixS* rs, int n, int k, int* hist, int lane) {
    uint32_t prefix = 0, pmask = 0;
    int kk = k;
    for (int dgt = 3; dgt >= 0; dgt--) {
        const int shift = 8 * dgt;
#pragma unroll
        for (int i = 0; i < 8; i++) hist[lane * 8 + i] = 0;
        __syncwarp();
        for (int j = lane; j < n; j += kWarp) {
            const uint32_t key = xkey(rs, j);
            if ((key & pmask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1);
        }
        __syncwarp();
        int c[8], tot = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) { c[i] = hist[lane * 8 + i]; tot += c[i]; }
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, incl > kk);
        const int sl = __ffs(ball) - 1;
        int bin = 0, below = 0;
        if (lane == sl) {
            int acc = incl - tot, bs = 7;
#pragma unroll
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
        prefix |= (uint32_t)bin << shift;
        pmask |= 0xffu << shift;
        __syncwarp();
    }
    return prefix;
}

__device__ void mix_select_pair(const MixS* rs, int n, int k, int* hist, int lane, float& v0, float& v1) {
    const uint32_t K = mix_select(rs, n, k, hist, lane);
    v0 = fkey_inv(K);
    if (k + 1 >= n) { v1 = v0; return; }
    int less = 0, eq = 0;
    uint32_t nxt = 0xffffffffu;
    for (int j = lane; j < n; j += kWarp) {
        const uint32_t key = xkey(rs, j);
        less += key < K;
        eq += key == K;
        if (key > K && key < nxt) nxt = key;
    }
    less = warp_sum_int(less);
    eq = warp_sum_int(eq);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint32_t v = __shfl_xor_sync(0xffffffffu, nxt, o);
        nxt = v < nxt ? v : nxt;
    }
    v1 = (k + 1 < less + eq) ? v0 : fkey_inv(nxt);
}

// Robust sigma of x = R / sigma: half the distance between the 1/6 and 5/6 quantiles
// (intersextile range, type-7 interpolation), Sect. 5.1.2.
__device__ float mix_robust_sigma(const MixS* rs, int n, int* hist, int lane) {
    const double h1 = (1.0 / 6.0) * (double)(n - 1), h5 = (5.0 / 6.0) * (double)(n - 1);
    const int lo1 = (int)floor(h1), lo5 = (int)floor(h5);
    float a0, a1, b0, b1;
    mix_select_pair(rs, n, lo1, hist, lane, a0, a1);
    mix_select_pair(rs, n, lo5, hist, lane, b0, b1);
    return 0.5f * ((b0 + (float)(h5 - lo5) * (b1 - b0)) - (a0 + (float)(h1 - lo1) * (a1 - a0)));
}

// ---- class sums of one source in FP32, both classes in one sweep.  The sums are shifted to
// the previous round's solution dp: h' = R - A dp, so that Q(y) = hh - 2 d'Ah + d'AA d is
// formed from a residual that is already small (no cancellation in FP32).
//   mode 0: w = wfun(x / vs), x = R / sigma (initial downweighting; dp = 0)
//   mode 1: w = wfun(h' / sqrt(sigma^2 + y_prev))
//   mode 2: keep the stored w
__device__ void mix_pass_class(MixS* rs, int n, int lane, int mode, float vs, const float* sigc, const float* dp,
                               const float* isd, int wfn, ClassSums& S, int& nout) {
    float AA[2][15], Ah[2][5], hh[2] = {0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < 2; c++) {
#pragma unroll
        for (int i = 0; i < 15; i++) AA[c][i] = 0.0f;
#pragma unroll
        for (int i = 0; i < 5; i++) Ah[c][i] = 0.0f;
    }
    int cnt = 0;
    for (int j = lane; j < n; j += kWarp) {
        const MixS r = rs[j];
        float A[5];
        arow(r, A);
        const bool ac = r.sig < 0.0f;
        const float m1 = ac ? 1.0f : 0.0f, m0 = 1.0f - m1;
        const float h = (float)r.R - adot(A, dp);
        float w;
        if (mode == 0) {
            w = vs > 0.0f ? wfun_f(((float)r.R / (ac ? sigc[1] : sigc[0])) / vs, wfn) : 1.0f;
            rs[j].W = w;
        } else if (mode == 1) {
            w = wfun_f(h * (ac ? isd[1] : isd[0]), wfn);
            rs[j].W = w;
        } else {
            w = r.W;
        }
        cnt += (w < 0.2f);
        const float w0 = w * m0, w1 = w * m1;
#pragma unroll
        for (int a = 0; a < 5; a++) {
            const float wa0 = w0 * A[a], wa1 = w1 * A[a];
#pragma unroll
            for (int b = a; b < 5; b++) {
                AA[0][up5(a, b)] = fmaf(wa0, A[b], AA[0][up5(a, b)]);
                AA[1][up5(a, b)] = fmaf(wa1, A[b], AA[1][up5(a, b)]);
            }
            Ah[0][a] = fmaf(wa0, h, Ah[0][a]);
            Ah[1][a] = fmaf(wa1, h, Ah[1][a]);
        }
        hh[0] = fmaf(w0 * h, h, hh[0]);
        hh[1] = fmaf(w1 * h, h, hh[1]);
    }
#pragma unroll
    for (int c = 0; c < 2; c++) {
#pragma unroll
        for (int i = 0; i < 15; i++) AA[c][i] = warp_sum_f(AA[c][i]);
#pragma unroll
        for (int i = 0; i < 5; i++) Ah[c][i] = warp_sum_f(Ah[c][i]);
        hh[c] = warp_sum_f(hh[c]);
    }
    nout = warp_sum_int(cnt);
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < 2; c++) {
#pragma unroll
            for (int i = 0; i < 15; i++) S.AA[c][i] = AA[c][i];
#pragma unroll
            for (int i = 0; i < 5; i++) S.Ah[c][i] = Ah[c][i];
            S.hh[c] = hh[c];
        }
    }
    __syncwarp();
}

// ---- general path (sigma varies within a class): per-observation sweeps for every
// excess-noise step, FP32 sums shifted to the previous round's solution.
__device__ __forceinline__ void mix_gen_normals(MixS* rs, int n, int lane, float y, bool refresh, const float* dp,
                                                float yp, int wfn, double* N, double* b, int& nout) {
    float Nf[15], bf[5];
#pragma unroll
    for (int i = 0; i < 15; i++) Nf[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < 5; i++) bf[i] = 0.0f;
    int cnt = 0;
    for (int j = lane; j < n; j += kWarp) {
        const MixS r = rs[j];
        float A[5];
        arow(r, A);
        const float s2 = r.sig * r.sig;
        const float h = (float)r.R - adot(A, dp);
        float w = r.W;
        if (refresh) {
            w = wfun_f(h / sqrtf(s2 + yp), wfn);
            rs[j].W = w;
        }
        cnt += (w < 0.2f);
        const float W = w / (s2 + y);
#pragma unroll
        for (int a = 0; a < 5; a++) {
            const float wa = W * A[a];
#pragma unroll
            for (int c = a; c < 5; c++) Nf[up5(a, c)] = fmaf(wa, A[c], Nf[up5(a, c)]);
            bf[a] = fmaf(wa, h, bf[a]);
        }
    }
#pragma unroll
    for (int i = 0; i < 15; i++) N[i] = (double)warp_sum_f(Nf[i]);
#pragma unroll
    for (int i = 0; i < 5; i++) b[i] = (double)warp_sum_f(bf[i]);
    nout = warp_sum_int(cnt);
}

// Q(y) = sum w R^2 / (sigma^2 + y) and S2 = sum w R^2 / (sigma^2 + y)^2 for R = h' - A delta
__device__ __forceinline__ void mix_gen_q(const MixS* rs, int n, int lane, const float* dp, const float* dl, float y,
                                          double& Q, double& S2) {
    float q = 0.0f, s = 0.0f;
    for (int j = lane; j < n; j += kWarp) {
        const MixS r = rs[j];
        float A[5];
        arow(r, A);
        const float R = ((float)r.R - adot(A, dp)) - adot(A, dl);
        const float den = r.sig * r.sig + y;
        const float t = r.W * R * R / den;
        q += t;
        s += t / den;
    }
    Q = (double)warp_sum_f(q);
    S2 = (double)warp_sum_f(s);
}

__device__ __noinline__ void mix_solve_general(const Settings& st, int i, int n, const double* s5, double cosd,
                                               MixS* rs, double s2min, float vs, const SrcOutPtrs& out, int lane) {
    if (st.robust) {
        for (int j = lane; j < n; j += kWarp) {
            const MixS r = rs[j];
            rs[j].W = vs > 0.0f ? wfun_f(((float)r.R / fabsf(r.sig)) / vs, st.weight_fn) : 1.0f;
        }
    } else {
        for (int j = lane; j < n; j += kWarp) rs[j].W = 1.0f;
    }
    __syncwarp();
    double d[5] = {0, 0, 0, 0, 0};
    double U[15];
    double y = 0.0, Q = 0.0, Q0 = 0.0, S2 = 0.0;
    int nu = 0, nout = 0, rd = 0;
    const int rounds = st.robust ? st.n_rounds + 1 : 1;
    for (int rnd = 0; rnd < rounds; rnd++) {
        const float dpf[5] = {(float)d[0], (float)d[1], (float)d[2], (float)d[3], (float)d[4]};
        const float yp = (float)y;
        double N[15], b[5], dl[5];
        y = 0.0;
        mix_gen_normals(rs, n, lane, 0.0f, rnd > 0, dpf, yp, st.weight_fn, N, b, nout);
        nu = n - nout - 5;
        rd = chol5(N, U, st.pivot_tol);
        chol5_solve(U, b, dl);
        float dlf[5] = {(float)dl[0], (float)dl[1], (float)dl[2], (float)dl[3], (float)dl[4]};
        mix_gen_q(rs, n, lane, dpf, dlf, 0.0f, Q, S2);
        Q0 = Q;
        if (st.robust && nu > 0 && Q0 > (double)nu) {
            const double tol = 1e-12 * s2min;
            for (int it = 0; it < st.n_eps; it++) {
                const double dy = (1.0 - Q / (double)nu) * Q / (-S2);
                y = fmax(0.0, y + dy);
                mix_gen_normals(rs, n, lane, (float)y, false, dpf, yp, st.weight_fn, N, b, nout);
                rd = chol5(N, U, st.pivot_tol);
                chol5_solve(U, b, dl);
                for (int a = 0; a < 5; a++) dlf[a] = (float)dl[a];
                mix_gen_q(rs, n, lane, dpf, dlf, (float)y, Q, S2);
                if (fabs(dy) <= tol) break;
            }
        }
        for (int a = 0; a < 5; a++) d[a] = (double)dpf[a] + dl[a];
        __syncwarp();
    }
    double chi = 0.0;
    for (int j = lane; j < n; j += kWarp) {
        const MixS v = rs[j];
        const double R = v.R - adot_d(v, d);
        const float W = v.W / (v.sig * v.sig + (float)y);
        rs[j].R = R;
        rs[j].W = W;
        chi += (double)W * R * R;
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
        out.q[i] = chi;
        out.nu[i] = nu;
        out.nout[i] = nout;
        out.dsig[i] = nu > 0 ? (Q0 - (double)nu) / sqrt(2.0 * (double)nu) : 0.0;
        out.chi2[i] = chi;
        out.rankdef[i] = rd;
    }
    __syncwarp();
}

}  // namespace

// ---------------------------------------------------------------------------------------
// full FP64 evaluation into the records (one thread per observation, source order)
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mix_forward(DevGeo G, int64_t n_obs, const int64_t* __restrict__ t_ns,
                                                     const uint32_t* __restrict__ meta,
                                                     const float* __restrict__ sigma, const double* __restrict__ mu,
                                                     const int32_t* __restrict__ obs_src,
                                                     const double* __restrict__ geo, const double* __restrict__ att,
                                                     const double* __restrict__ cal, MixS* __restrict__ ms,
                                                     MixT* __restrict__ mt) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_obs; o += (int64_t)gridDim.x * blockDim.x) {
        const double* gp = geo + 16 * (size_t)obs_src[o];
        SrcGeo S;
        for (int k = 0; k < 3; k++) { S.p[k] = gp[k]; S.q[k] = gp[3 + k]; S.r[k] = gp[6 + k]; }
        S.par = gp[9]; S.pma = gp[10]; S.pmd = gp[11]; S.cosd = gp[12];
        const int64_t t = t_ns[o];
        const uint32_t m = meta[o];
        ObsOut ob;
        observe<true>(G, S, t, m, meta_kind(m) ? mu[o] : 0.0, att, cal, ob);
        MixS a;
        a.R = ob.R;
        a.Ap = (float)ob.A[0];
        a.Aq = (float)ob.A[1];
        a.Aw = (float)ob.A[2];
        a.tau = (float)ob.tau;
        a.sig = meta_kind(m) ? -sigma[o] : sigma[o];
        a.W = 0.0f;
        ms[o] = a;
        MixT b;
        for (int k = 0; k < 4; k++) b.g[k] = (float)ob.g[k];
        b.meta = m;
        b.pad = 0;
        b.t_ns = t;
        mt[o] = b;
    }
}

// R += sum_j B_j g . d_a[l-3+j] + d_c[k]  (dR/da_n = g B_n, dR/dc_k = 1; Eqs. dfadq, pdC)
__global__ void __launch_bounds__(256) k_mix_correct(DevGeo G, int64_t n_obs, MixS* __restrict__ ms,
                                                     const MixT* __restrict__ mt, const float4* __restrict__ d_att,
                                                     const double* __restrict__ d_cal) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_obs; o += (int64_t)gridDim.x * blockDim.x) {
        const MixT r = mt[o];
        const int l = left_index(G, r.t_ns);
        float B[4];
        bspline4f(G, r.t_ns, l, B);
        const float4* da = d_att + (l - 3);
        float corr = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const float4 v = __ldg(da + j);
            corr = fmaf(B[j], r.g[0] * v.x + r.g[1] * v.y + r.g[2] * v.z + r.g[3] * v.w, corr);
        }
        ms[o].R += (double)corr + __ldg(d_cal + meta_cal(r.meta));
    }
}

// ---------------------------------------------------------------------------------------
// per-source solve: batches of sources per warp as in the FP64 form; lane k solves source
// k's 5x5 systems in FP64 from the FP32 class sums
// ---------------------------------------------------------------------------------------
constexpr int kMixWarps = 2;
__global__ void __launch_bounds__(32 * kMixWarps) k_mix_solve(Settings st, const int64_t* __restrict__ src_off,
                                                              const int32_t* __restrict__ src_order, int32_t n_src,
                                                              int batch, SrcOutPtrs out, MixS* __restrict__ ms,
                                                              int* work_counter) {
    __shared__ int hist_all[kMixWarps * 256];
    __shared__ ClassSums sums_all[kMixWarps][kWarp];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int* hist = hist_all + wib * 256;
    ClassSums* sums = sums_all[wib];
    const int rounds = st.robust ? st.n_rounds + 1 : 1;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(work_counter, batch);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_src) break;
        const int nb = min(batch, n_src - base);
        const bool mine = lane < nb;
        const int my_i = mine ? src_order[base + lane] : 0;
        const int64_t my_o0 = mine ? src_off[my_i] : 0;
        const int my_n = mine ? (int)(src_off[my_i + 1] - my_o0) : 0;
        double s5[5] = {0, 0, 0, 0, 0};
        if (mine)
            for (int k = 0; k < 5; k++) s5[k] = out.src[5 * (size_t)my_i + k];
        const double cosd = cos(s5[1]);
        double my_s2c[2] = {1.0, 1.0}, my_s2min = 1.0;
        float my_vs = 0.0f;
        bool my_uniform = false;
        // ---- per source: sigma per class (one value per class selects the class-sum path)
        for (int k = 0; k < nb; k++) {
            const int64_t o0 = __shfl_sync(0xffffffffu, my_o0, k);
            const int n = __shfl_sync(0xffffffffu, my_n, k);
            if (n == 0) continue;
            const MixS* rs = ms + o0;
            float lo[2] = {3.0e38f, 3.0e38f}, hi[2] = {0.0f, 0.0f};
            for (int j = lane; j < n; j += kWarp) {
                const float sg = rs[j].sig;
                const float a = fabsf(sg);
                if (sg < 0.0f) { lo[1] = fminf(lo[1], a); hi[1] = fmaxf(hi[1], a); }
                else { lo[0] = fminf(lo[0], a); hi[0] = fmaxf(hi[0], a); }
            }
#pragma unroll
            for (int c = 0; c < 2; c++)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
                    hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
                }
            const bool has0 = hi[0] > 0.0f, has1 = hi[1] > 0.0f;
            const bool uni = (!has0 || lo[0] == hi[0]) && (!has1 || lo[1] == hi[1]);
            const float vs = st.robust ? mix_robust_sigma(rs, n, hist, lane) : 0.0f;
            if (lane == k) {
                my_uniform = uni;
                my_s2c[0] = has0 ? (double)lo[0] * (double)lo[0] : 1.0;
                my_s2c[1] = has1 ? (double)lo[1] * (double)lo[1] : 1.0;
                const float smin = fminf(lo[0], lo[1]);
                my_s2min = (double)smin * (double)smin;
                my_vs = vs;
            }
        }
        // ---- inner iteration, class-sum path
        double d[5] = {0, 0, 0, 0, 0};
        double U[15];
        for (int q = 0; q < 15; q++) U[q] = 0.0;
        double y = 0.0, Q = 0.0, Q0 = 0.0, S2 = 0.0;
        int nu = 0, nout = 0, rd = 0;
        for (int rnd = 0; rnd < rounds; rnd++) {
            // the shift: the previous round's solution rounded to FP32 (it is applied as such)
            double dp[5];
            for (int a = 0; a < 5; a++) dp[a] = (double)(float)d[a];
            for (int k = 0; k < nb; k++) {
                const int n = __shfl_sync(0xffffffffu, my_n, k);
                const int uni = __shfl_sync(0xffffffffu, (int)my_uniform, k);
                if (n == 0 || !uni) continue;
                const int64_t o0 = __shfl_sync(0xffffffffu, my_o0, k);
                float dk[5];
                for (int a = 0; a < 5; a++) dk[a] = (float)__shfl_sync(0xffffffffu, dp[a], k);
                const double yk = __shfl_sync(0xffffffffu, y, k);
                const double s2c[2] = {__shfl_sync(0xffffffffu, my_s2c[0], k), __shfl_sync(0xffffffffu, my_s2c[1], k)};
                const float vsk = __shfl_sync(0xffffffffu, my_vs, k);
                const float sigc[2] = {(float)sqrt(s2c[0]), (float)sqrt(s2c[1])};
                const float isd[2] = {(float)(1.0 / sqrt(s2c[0] + yk)), (float)(1.0 / sqrt(s2c[1] + yk))};
                MixS* rs = ms + o0;
                int no = 0;
                if (!st.robust) {
                    if (rnd == 0) {
                        for (int j = lane; j < n; j += kWarp) rs[j].W = 1.0f;
                        __syncwarp();
                    }
                    mix_pass_class(rs, n, lane, 2, 0.0f, sigc, dk, isd, st.weight_fn, sums[k], no);
                } else {
                    mix_pass_class(rs, n, lane, rnd == 0 ? 0 : 1, vsk, sigc, dk, isd, st.weight_fn, sums[k], no);
                }
                if (lane == k) nout = no;
            }
            __syncwarp();
            if (mine && my_n > 0 && my_uniform) {
                double dl[5];
                nu = my_n - nout - 5;
                y = 0.0;
                class_solve(sums[lane], my_s2c, 0.0, st.pivot_tol, U, dl, rd, Q, S2);
                Q0 = Q;
                if (st.robust && nu > 0 && Q0 > (double)nu) {
                    const double tol = 1e-12 * my_s2min;
                    for (int it = 0; it < st.n_eps; it++) {
                        const double dy = (1.0 - Q / (double)nu) * Q / (-S2);
                        y = fmax(0.0, y + dy);
                        class_solve(sums[lane], my_s2c, y, st.pivot_tol, U, dl, rd, Q, S2);
                        if (fabs(dy) <= tol) break;
                    }
                }
                for (int a = 0; a < 5; a++) d[a] = dp[a] + dl[a];
            }
            __syncwarp();
        }
        // ---- residuals after the update (FP64) and the statistical weights
        double my_chi = 0.0;
        for (int k = 0; k < nb; k++) {
            const int n = __shfl_sync(0xffffffffu, my_n, k);
            const int uni = __shfl_sync(0xffffffffu, (int)my_uniform, k);
            if (n == 0 || !uni) continue;
            const int64_t o0 = __shfl_sync(0xffffffffu, my_o0, k);
            double dk[5];
            for (int a = 0; a < 5; a++) dk[a] = __shfl_sync(0xffffffffu, d[a], k);
            const double yk = __shfl_sync(0xffffffffu, y, k);
            const float iw[2] = {(float)(1.0 / (__shfl_sync(0xffffffffu, my_s2c[0], k) + yk)),
                                 (float)(1.0 / (__shfl_sync(0xffffffffu, my_s2c[1], k) + yk))};
            MixS* rs = ms + o0;
            double chi = 0.0;
            for (int j = lane; j < n; j += kWarp) {
                const MixS v = rs[j];
                const double R = v.R - adot_d(v, dk);
                const float W = v.W * iw[v.sig < 0.0f ? 1 : 0];
                rs[j].R = R;
                rs[j].W = W;
                chi += (double)W * R * R;
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
                out.q[i] = my_chi;  // Q at the final (d, eps^2), from the FP64 residuals
                out.nu[i] = nu;
                out.nout[i] = nout;
                out.dsig[i] = nu > 0 ? (Q0 - (double)nu) / sqrt(2.0 * (double)nu) : 0.0;
                out.chi2[i] = my_chi;
                out.rankdef[i] = rd;
            }
        }
        __syncwarp();
        // ---- sources without one sigma per class
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
            const float vsk = __shfl_sync(0xffffffffu, my_vs, k);
            mix_solve_general(st, i, n, sk, ck, ms + o0, s2m, vsk, out, lane);
        }
    }
}

// ---------------------------------------------------------------------------------------
// A block accumulation with FP32 arithmetic (same staging as the FP64 form): per knot
// interval the 16x16 block W (B B') (x) (g g' + 4 lambda^2 s s') and the right-hand side
// -W B (x) (R g [- 2 lambda^2 D s]) (Eqs. normAmod, dDldan).
//
// The sums are compensated (Knuth's TwoSum: hi + lo carries the sum to about 2^-48 relative)
// because the attitude normals are nearly singular along the coefficient vector itself:
// the observation terms vanish along it (g is orthogonal to q) and only the norm term of
// relative size 4 lambda^2 ~ 4e-6 fixes it, which plain FP32 accumulation (2^-24 per
// addition, growing with the number of terms) does not resolve.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float p) {
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

__host__ __device__ constexpr int mtri16(int i, int j) { return i * 16 - i * (i - 1) / 2 + (j - i); }
__host__ __device__ constexpr int mtri4(int i, int j) { return i * 4 - i * (i - 1) / 2 + (j - i); }
constexpr int kMStage = 28;  // B[4], M[10], r[4], BB[10]

__global__ void __launch_bounds__(128) k_mix_att_accum(DevGeo G, float lambda2, int rhs_norm,
                                                       const uint32_t* __restrict__ perm_t,
                                                       const int64_t* __restrict__ ivl_off, int n_iv,
                                                       const MixS* __restrict__ ms, const MixT* __restrict__ mt,
                                                       const double* __restrict__ att, double* __restrict__ blk) {
    __shared__ float stage_all[4][kWarp * kMStage];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float* stg = stage_all[wib];
    int oi[5], oj[5];
#pragma unroll
    for (int k = 0; k < 5; k++) {
        const int o = lane + 32 * k;
        oi[k] = -1; oj[k] = -1;
        if (o < 136) {
            int i = 0;
            while (o >= mtri16(i, 15) + 1) i++;
            oi[k] = i;
            oj[k] = i + (o - mtri16(i, i));
        } else if (o < kBlkVals) {
            oi[k] = o - 136;
        }
    }
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int iv = blockIdx.x * (blockDim.x >> 5) + wib; iv < n_iv; iv += nwarps) {
        const int l = iv + 3;
        const double* ad = att + 4 * (int64_t)(l - 3);
        float a[16];
#pragma unroll
        for (int k = 0; k < 16; k++) a[k] = (float)ad[k];
        float acc[5] = {0, 0, 0, 0, 0}, lo[5] = {0, 0, 0, 0, 0};
        const int64_t beg = ivl_off[iv], end = ivl_off[iv + 1];
        for (int64_t base = beg; base < end; base += kWarp) {
            const int64_t j = base + lane;
            float* st = stg + lane * kMStage;
            if (j < end) {
                const uint32_t o = perm_t[j];
                const MixT rt = mt[o];
                const MixS rs = ms[o];
                const float W = rs.W;
                const float Rf = (float)rs.R;
                float B[4];
                bspline4f(G, rt.t_ns, l, B);
                float s[4];
#pragma unroll
                for (int c = 0; c < 4; c++) s[c] = B[0] * a[c] + B[1] * a[4 + c] + B[2] * a[8 + c] + B[3] * a[12 + c];
                const float l4 = 4.0f * lambda2;
#pragma unroll
                for (int c = 0; c < 4; c++)
#pragma unroll
                    for (int e = c; e < 4; e++) st[4 + mtri4(c, e)] = W * (rt.g[c] * rt.g[e] + l4 * s[c] * s[e]);
                float D = 0.0f;
                if (rhs_norm) {
                    // 1 - |s|^2 cancels: form it in FP64
                    double Bd[4];
                    bspline4(G, rt.t_ns, l, Bd);
                    double sd2 = 0.0;
                    for (int c = 0; c < 4; c++) {
                        const double v = Bd[0] * ad[c] + Bd[1] * ad[4 + c] + Bd[2] * ad[8 + c] + Bd[3] * ad[12 + c];
                        sd2 += v * v;
                    }
                    D = (float)(1.0 - sd2);
                }
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    float v = Rf * rt.g[c];
                    if (rhs_norm) v -= 2.0f * lambda2 * D * s[c];
                    st[14 + c] = W * v;
                    st[c] = B[c];
                }
#pragma unroll
                for (int c = 0; c < 4; c++)
#pragma unroll
                    for (int e = c; e < 4; e++) st[18 + mtri4(c, e)] = B[c] * B[e];
            } else {
#pragma unroll
                for (int c = 0; c < kMStage; c++) st[c] = 0.0f;
            }
            __syncwarp();
            const int cnt = (int)((end - base) < kWarp ? (end - base) : kWarp);
            for (int q = 0; q < cnt; q++) {
                const float* sq = stg + q * kMStage;
#pragma unroll
                for (int k = 0; k < 5; k++) {
                    if (oi[k] < 0) continue;
                    const int i = oi[k];
                    if (oj[k] >= 0) {
                        const int jj = oj[k];
                        const int bi = i >> 2, ci = i & 3, bj = jj >> 2, cj = jj & 3;
                        const int mi = ci <= cj ? mtri4(ci, cj) : mtri4(cj, ci);
                        two_sum_acc(acc[k], lo[k], __fmul_rn(sq[18 + mtri4(bi, bj)], sq[4 + mi]));
                    } else {
                        two_sum_acc(acc[k], lo[k], -__fmul_rn(sq[i >> 2], sq[14 + (i & 3)]));
                    }
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int k = 0; k < 5; k++) {
            const int o = lane + 32 * k;
            if (o < kBlkVals) blk[(int64_t)iv * kBlkVals + o] = (double)acc[k] + (double)lo[k];
        }
    }
}

// C block sums from the records (calibration order): N_kk = sum W, b_k = -sum W R; the 1x1
// robust solve gives d~_k = (b / sqrt(N)) / sqrt(N), or 0 with a rank defect.
__global__ void k_mix_cal_accum(int n_cal, const uint32_t* __restrict__ perm_c, const int64_t* __restrict__ cal_off,
                                const MixS* __restrict__ ms, double* __restrict__ dtil, int* __restrict__ rd) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n_cal; k += nw) {
        double sw = 0.0, swr = 0.0;
        for (int64_t j = cal_off[k] + lane; j < cal_off[k + 1]; j += kWarp) {
            const MixS r = ms[perm_c[j]];
            const double W = (double)r.W;
            sw += W;
            swr += W * r.R;
        }
        sw = warp_sum(sw);
        swr = warp_sum(swr);
        if (lane == 0) {
            if (sw > 0.0) {
                const double u = sqrt(sw);
                dtil[k] = (-swr / u) / u;
                rd[k] = 0;
            } else {
                dtil[k] = 0.0;
                rd[k] = 1;
            }
        }
    }
}

__global__ void k_mix_rw(int64_t n, const MixS* __restrict__ ms, double* __restrict__ R, double* __restrict__ W) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        if (R) R[o] = ms[o].R;
        if (W) W[o] = (double)ms[o].W;
    }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
void launch_mix_s(const DevGeo& G, const Settings& st, bool refresh, const int64_t* t_ns, const uint32_t* meta,
                  const float* sigma, const double* mu, const int32_t* obs_src, int64_t n_obs, const int64_t* src_off,
                  const int32_t* src_order, int32_t n_src, const double* att, const double* cal, const SrcOutPtrs& out,
                  MixS* ms, MixT* mt, double* geo, float* d_att, double* d_cal, int n_coef, int n_cal, int* work,
                  cudaStream_t s) {
    if (refresh) {
        launch_src_geo(n_src, out.src, geo, s);
        k_mix_forward<<<grid_of(n_obs, 256, 152 * 64), 256, 0, s>>>(G, n_obs, t_ns, meta, sigma, mu, obs_src, geo,
                                                                     att, cal, ms, mt);
    } else {
        k_mix_correct<<<grid_of(n_obs, 256, 152 * 64), 256, 0, s>>>(G, n_obs, ms, mt,
                                                                     reinterpret_cast<const float4*>(d_att), d_cal);
    }
    cudaMemsetAsync(d_att, 0, sizeof(float) * 4 * (size_t)n_coef, s);
    cudaMemsetAsync(d_cal, 0, sizeof(double) * (size_t)n_cal, s);
    cudaMemsetAsync(work, 0, sizeof(int), s);
    int batch = n_src / (152 * 16);
    batch = batch < 1 ? 1 : (batch > 32 ? 32 : batch);
    const int warps = (n_src + batch - 1) / batch;
    k_mix_solve<<<grid_of(warps, kMixWarps, 152 * 32), 32 * kMixWarps, 0, s>>>(st, src_off, src_order, n_src, batch,
                                                                                out, ms, work);
}

void launch_mix_att_accum(const DevGeo& G, double lambda2, int rhs_norm, const uint32_t* perm_t,
                          const int64_t* ivl_off, int n_iv, const MixS* ms, const MixT* mt, const double* att,
                          double* blk, cudaStream_t s) {
    k_mix_att_accum<<<grid_of(n_iv, 4, 152 * 32), 128, 0, s>>>(G, (float)lambda2, rhs_norm, perm_t, ivl_off, n_iv,
                                                               ms, mt, att, blk);
}

void launch_mix_cal(int n_cal, int n_days, const uint32_t* perm_c, const int64_t* cal_off, const MixS* ms,
                    double* dtil, int* rd, double* cal, double* d_cal, cudaStream_t s) {
    k_mix_cal_accum<<<grid_of(n_cal, 8, 152 * 16), 256, 0, s>>>(n_cal, perm_c, cal_off, ms, dtil, rd);
    launch_cal_project(n_days, dtil, cal, d_cal, s);
}

void launch_mix_rw(int64_t n, const MixS* ms, double* R, double* W, cudaStream_t s) {
    k_mix_rw<<<grid_of(n, 256, 152 * 32), 256, 0, s>>>(n, ms, R, W);
}

}  // namespace agis
