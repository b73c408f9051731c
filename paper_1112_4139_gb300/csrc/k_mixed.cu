// k_mixed.cu -- the mixed-precision form of the observation pass and of the S, A and C
// blocks.
//
// Each observation keeps two 32-byte records (source order, see MixS / MixT).  A full FP64
// evaluation of the model (k_mix_forward) refreshes R and the FP32 partials every few
// source updates; in between, R follows the first-order identity behind Eq. precond2:
// k_mix_correct adds (dR/da) d_a + (dR/dc) d_c for the A and C updates since the last source
// update, and the source update subtracts A d.  R is kept to about 48 bits as a float pair,
// so the updates solve for corrections of an accurately known residual (iterative
// refinement): FP32 rounding of the normal equations changes the rate of convergence, not
// the point it converges to.  The 5x5 and band Cholesky factorisations and the frame
// rotator stay FP64.  Every per-observation operation runs on the FP32 pipe.
//
// S block: k_mix_scale_sums (sigma per class, robust scale, round-0 class sums), then per
// weight round k_mix_solve5 (one thread per source: the 5x5 algebra of the excess-noise
// steps in FP64) and k_mix_sums (the next round's sums), then k_mix_final (R <- R - A d and
// W).  Sources whose sigma varies within a class take k_mix_general (all rounds in one warp
// with per-observation sweeps).
#include "agis_internal.cuh"

namespace agis {

void launch_src_geo(int32_t n_src, const double* src, double* geo, cudaStream_t s);

// pivots below this fraction of N_jj are not resolved by FP32 normals: they count as zero
// in the mixed form (App. C robust Cholesky with a tolerance for FP32 accumulation)
constexpr double kMixPivotTol = 64.0 / 16777216.0;

namespace {

int grid_of(int64_t n, int per_block, int cap) {
    int64_t b = (n + per_block - 1) / per_block;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

// ---- float-pair arithmetic (Knuth's TwoSum, FMA-based exact product) ----------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// (hi, lo) += (xh, xl)
__device__ __forceinline__ void pair_add(float& hi, float& lo, float xh, float xl) {
    float s, e;
    two_sum(hi, xh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, xl));
    fast_two_sum(s, e, hi, lo);
}
__device__ __forceinline__ void split_pair(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}
// A d for the FP32 row A and d given as float pairs, as a float pair
__device__ __forceinline__ void row_dot_pair(const float A[5], const float* dh, const float* dl, float& sh,
                                             float& sl) {
    sh = 0.0f;
    sl = 0.0f;
#pragma unroll
    for (int k = 0; k < 5; k++) {
        const float p = __fmul_rn(A[k], dh[k]);
        const float e = __fmaf_rn(A[k], dh[k], -p);
        float s, t;
        two_sum(sh, p, s, t);
        sh = s;
        sl = __fadd_rn(sl, __fadd_rn(t, __fmaf_rn(A[k], dl[k], e)));
    }
    fast_two_sum(sh, sl, sh, sl);
}

// B_{l-3..l} at offset u (units of the knot interval) from tau_l, in FP32: closed form on
// regular intervals, Algorithm B.1 with the knots relative to tau_l near the end knots.
__device__ __forceinline__ void bspline4_lu(const DevGeo& G, int l, float u, float b[4]) {
    if (l >= 5 && l <= G.n_coef - 3) {
        const float v = 1.0f - u;
        const float u2 = u * u, u3 = u2 * u;
        b[0] = v * v * v * (1.0f / 6.0f);
        b[1] = (3.0f * u3 - 6.0f * u2 + 4.0f) * (1.0f / 6.0f);
        b[2] = (-3.0f * u3 + 3.0f * u2 + 3.0f * u + 1.0f) * (1.0f / 6.0f);
        b[3] = u3 * (1.0f / 6.0f);
        return;
    }
    const int K = G.n_coef - 3;
    auto kc = [K](int k) { k -= 3; return k < 0 ? 0 : (k > K ? K : k); };
    const int k0 = kc(l);
    float R[3], L[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        R[i] = (float)(kc(l + i + 1) - k0) - u;
        L[i] = u - (float)(kc(l - i) - k0);
    }
    b[0] = 1.0f; b[1] = b[2] = b[3] = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j <= i; j++) {
            const float den = R[j] + L[i - j];
            const float w = den != 0.0f ? b[j] / den : 0.0f;
            b[j] = s + R[j] * w;
            s = L[i - j] * w;
        }
        b[i + 1] = s;
    }
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

// Weight of one observation in a round.  Round 0 (robust): w = wfun(x / vs), x = R / sigma_c;
// later rounds: w = wfun(h' / sqrt(sigma_c^2 + y_prev)) with h' = R - A d_prev; plain: w = 1.
// The same function serves the sums and the final pass, so both see identical weights.
__device__ __forceinline__ float round_weight(const SrcRound& in, float Rh, float hp, int cls, int wfn) {
    if (in.mode == 2) return 1.0f;
    if (in.mode == 0) return in.vs > 0.0f ? wfun_f((Rh / (cls ? in.sigc[1] : in.sigc[0])) / in.vs, wfn) : 1.0f;
    return wfun_f(hp * (cls ? in.isd[1] : in.isd[0]), wfn);
}

// ---- order statistics of x = R / sigma over a source (4-pass radix select on FP32 keys) ----
__device__ __forceinline__ uint32_t fkey(float x) {
    const uint32_t b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ uint32_t xkey(const MixS* rs, const float2* rr, int j) {
    return fkey(rr[j].x / fabsf(rs[j].sig));
}

// keys of one source: from a shared-memory copy when the source fits, else recomputed
struct KeySrc {
    const uint32_t* sk;
    const MixS* rs;
    const float2* rr;
    __device__ __forceinline__ uint32_t operator()(int j) const { return sk ? sk[j] : xkey(rs, rr, j); }
};

// the ka-th and kb-th smallest keys (0-based), by a 4-pass radix select with 8-bit digits in
// which both selections share each sweep over the keys
__device__ void select2(const KeySrc& key, int n, int ka, int kb, int* hist, int lane, uint32_t& Ka, uint32_t& Kb) {
    uint32_t pre[2] = {0, 0}, pmask = 0;
    int kk[2] = {ka, kb};
    for (int dgt = 3; dgt >= 0; dgt--) {
        const int shift = 8 * dgt;
#pragma unroll
        for (int i = 0; i < 16; i++) hist[lane * 16 + i] = 0;
        __syncwarp();
        for (int j = lane; j < n; j += kWarp) {
            const uint32_t k = key(j);
            const uint32_t bin = (k >> shift) & 255u;
            if ((k & pmask) == pre[0]) atomicAdd(&hist[bin], 1);
            if ((k & pmask) == pre[1]) atomicAdd(&hist[256 + bin], 1);
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int* h = hist + 256 * q;
            int c[8], tot = 0;
#pragma unroll
            for (int i = 0; i < 8; i++) { c[i] = h[lane * 8 + i]; tot += c[i]; }
            int incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const unsigned ball = __ballot_sync(0xffffffffu, incl > kk[q]);
            const int sl = __ffs(ball) - 1;
            int bin = 0, below = 0;
            if (lane == sl) {
                int acc = incl - tot, bs = 7;
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    if (acc + c[i] > kk[q]) { bs = i; break; }
                    acc += c[i];
                }
                bin = lane * 8 + bs;
                below = acc;
            }
            bin = __shfl_sync(0xffffffffu, bin, sl);
            below = __shfl_sync(0xffffffffu, below, sl);
            kk[q] -= below;
            pre[q] |= (uint32_t)bin << shift;
        }
        pmask |= 0xffu << shift;
        __syncwarp();
    }
    Ka = pre[0];
    Kb = pre[1];
}

// the next value after K in sorted order (K itself when the (k+1)-th smallest equals it)
__device__ __forceinline__ float next_value(const KeySrc& key, int n, int k, uint32_t K, int lane) {
    if (k + 1 >= n) return fkey_inv(K);
    int le = 0;
    uint32_t nxt = 0xffffffffu;
    for (int j = lane; j < n; j += kWarp) {
        const uint32_t v = key(j);
        le += v <= K;
        if (v > K && v < nxt) nxt = v;
    }
    le = warp_sum_int(le);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint32_t v = __shfl_xor_sync(0xffffffffu, nxt, o);
        nxt = v < nxt ? v : nxt;
    }
    return (k + 1 < le) ? fkey_inv(K) : fkey_inv(nxt);
}

// Robust scale of x = R / sigma: half the intersextile range (type-7 interpolation), Sect. 5.1.2.
__device__ float mix_robust_sigma(const KeySrc& key, int n, int* hist, int lane) {
    const double h1 = (1.0 / 6.0) * (double)(n - 1), h5 = (5.0 / 6.0) * (double)(n - 1);
    const int lo1 = (int)floor(h1), lo5 = (int)floor(h5);
    uint32_t K1, K5;
    select2(key, n, lo1, lo5, hist, lane, K1, K5);
    const float a0 = fkey_inv(K1), a1 = next_value(key, n, lo1, K1, lane);
    const float b0 = fkey_inv(K5), b1 = next_value(key, n, lo5, K5, lane);
    return 0.5f * ((b0 + (float)(h5 - lo5) * (b1 - b0)) - (a0 + (float)(h1 - lo1) * (a1 - a0)));
}

// Class sums of one source for one round (whole warp), shifted to the previous solution:
// h' = R - A dp, so that Q(y) = hh - 2 d'Ah + d'AA d is formed without cancellation.  The AL
// rows of a source come first (rows [0, nal)), the AC rows after them.
__device__ __forceinline__ void class_sums(const MixS* rs, const float2* rr, int n, int nal, int lane,
                                           const SrcRound& in, int wfn, RoundSums* out) {
    float* o = reinterpret_cast<float*>(out);
    int cnt = 0;
#pragma unroll 1
    for (int c = 0; c < 2; c++) {
        float AA[15], Ah[5], hh = 0.0f;
#pragma unroll
        for (int i = 0; i < 15; i++) AA[i] = 0.0f;
#pragma unroll
        for (int i = 0; i < 5; i++) Ah[i] = 0.0f;
        const int lo = c ? nal : 0, hi = c ? n : nal;
        auto add = [&](const MixS& r, float Rh) {
            float A[5];
            arow(r, A);
            const float hp = Rh - adot(A, in.dp);
            const float w = round_weight(in, Rh, hp, c, wfn);
            cnt += (w < 0.2f);
#pragma unroll
            for (int a = 0; a < 5; a++) {
                const float wa = w * A[a];
#pragma unroll
                for (int b = a; b < 5; b++) AA[up5(a, b)] = fmaf(wa, A[b], AA[up5(a, b)]);
                Ah[a] = fmaf(wa, hp, Ah[a]);
            }
            hh = fmaf(w * hp, hp, hh);
        };
        // two records per lane in flight; the sums keep the order j, j + 32, ...
        int j = lo + lane;
        for (; j + kWarp < hi; j += 2 * kWarp) {
            const MixS r0 = rs[j], r1 = rs[j + kWarp];
            const float R0 = rr[j].x, R1 = rr[j + kWarp].x;
            add(r0, R0);
            add(r1, R1);
        }
        if (j < hi) add(rs[j], rr[j].x);
#pragma unroll
        for (int i = 0; i < 15; i++) AA[i] = warp_sum_f(AA[i]);
#pragma unroll
        for (int i = 0; i < 5; i++) Ah[i] = warp_sum_f(Ah[i]);
        hh = warp_sum_f(hh);
        // lanes write disjoint parts of the 176-byte record
#pragma unroll
        for (int i = 0; i < 15; i++)
            if (lane == i) o[c * 15 + i] = AA[i];
#pragma unroll
        for (int i = 0; i < 5; i++)
            if (lane == 15 + i) o[30 + c * 5 + i] = Ah[i];
        if (lane == 20) o[40 + c] = hh;
    }
    cnt = warp_sum_int(cnt);
    if (lane == 21) out->nout = cnt;
}

// ---- general path (sigma varies within a class): per-observation sweeps for every
// excess-noise step, FP32 sums shifted to the previous round's solution.
__device__ __forceinline__ void gen_normals(const MixS* rs, const float2* rr, float2* ac, int n, int lane, float y,
                                            bool refresh, const float* dp, float yp, int wfn, double* N, double* b,
                                            int& nout) {
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
        const float h = rr[j].x - adot(A, dp);
        float w = ac[j].x;
        if (refresh) {
            w = wfun_f(h / sqrtf(s2 + yp), wfn);
            ac[j].x = w;
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

__device__ __forceinline__ void gen_q(const MixS* rs, const float2* rr, const float2* ac, int n, int lane,
                                      const float* dp, const float* dl, float y, double& Q, double& S2) {
    float q = 0.0f, s = 0.0f;
    for (int j = lane; j < n; j += kWarp) {
        const MixS r = rs[j];
        float A[5];
        arow(r, A);
        const float R = (rr[j].x - adot(A, dp)) - adot(A, dl);
        const float den = r.sig * r.sig + y;
        const float t = ac[j].x * R * R / den;
        q += t;
        s += t / den;
    }
    Q = (double)warp_sum_f(q);
    S2 = (double)warp_sum_f(s);
}

// R <- R - A d (float-pair arithmetic), the A/C inputs (W, W Rh), and the chi^2 term
__device__ __forceinline__ float apply_update(const MixS& v, float2 R, const float* dh, const float* dl, float W,
                                              float2* rr, float2* ac, int handover_h) {
    float A[5];
    arow(v, A);
    float sh, sl;
    const float h = R.x;
    row_dot_pair(A, dh, dl, sh, sl);
    pair_add(R.x, R.y, -sh, -sl);
    *rr = R;
    *ac = make_float2(W, W * (handover_h ? h : R.x));
    return W * R.x * R.x;
}

__device__ __forceinline__ void write_source(const SrcOutPtrs& out, int i, const double* d, const double* U, double y,
                                             double Q0, int nu, int nout, int rd) {
    double* sp = out.src + 5 * (size_t)i;
    const double cosd = cos(sp[1]);
    sp[0] += d[0] / cosd;
    sp[1] += d[1];
    sp[2] += d[2];
    sp[3] += d[3];
    sp[4] += d[4];
    for (int k = 0; k < 5; k++) out.d[5 * (size_t)i + k] = d[k];
    for (int c = 0; c < 5; c++) {
        double e[5] = {0, 0, 0, 0, 0};
        e[c] = 1.0;
        double x[5];
        chol5_solve(U, e, x);
        for (int k = 0; k < 5; k++) out.cov[25 * (size_t)i + 5 * k + c] = x[k];
    }
    out.eps2[i] = y;
    out.nu[i] = nu;
    out.nout[i] = nout;
    out.dsig[i] = nu > 0 ? (Q0 - (double)nu) / sqrt(2.0 * (double)nu) : 0.0;
    out.rankdef[i] = rd;
}

__device__ __noinline__ void mix_solve_general(const Settings& st, int i, int n, const MixS* rs, float2* rr,
                                               float2* ac, double s2min, float vs, const SrcOutPtrs& out, int lane) {
    const double tol_piv = fmax(st.pivot_tol, kMixPivotTol);
    if (st.robust) {
        for (int j = lane; j < n; j += kWarp)
            ac[j].x = vs > 0.0f ? wfun_f((rr[j].x / fabsf(rs[j].sig)) / vs, st.weight_fn) : 1.0f;
    } else {
        for (int j = lane; j < n; j += kWarp) ac[j].x = 1.0f;
    }
    __syncwarp();
    double d[5] = {0, 0, 0, 0, 0};
    double U[kU5];
    double y = 0.0, Q = 0.0, Q0 = 0.0, S2 = 0.0;
    int nu = 0, nout = 0, rd = 0;
    const int rounds = st.robust ? st.n_rounds + 1 : 1;
    for (int rnd = 0; rnd < rounds; rnd++) {
        const float dpf[5] = {(float)d[0], (float)d[1], (float)d[2], (float)d[3], (float)d[4]};
        const float yp = (float)y;
        double N[15], b[5], dl[5];
        y = 0.0;
        gen_normals(rs, rr, ac, n, lane, 0.0f, rnd > 0, dpf, yp, st.weight_fn, N, b, nout);
        nu = n - nout - 5;
        rd = chol5(N, U, tol_piv);
        chol5_solve(U, b, dl);
        float dlf[5] = {(float)dl[0], (float)dl[1], (float)dl[2], (float)dl[3], (float)dl[4]};
        gen_q(rs, rr, ac, n, lane, dpf, dlf, 0.0f, Q, S2);
        Q0 = Q;
        if (st.robust && nu > 0 && Q0 > (double)nu) {
            const double tol = 1e-12 * s2min;
            for (int it = 0; it < st.n_eps; it++) {
                const double dy = (1.0 - Q / (double)nu) * Q / (-S2);
                y = fmax(0.0, y + dy);
                gen_normals(rs, rr, ac, n, lane, (float)y, false, dpf, yp, st.weight_fn, N, b, nout);
                rd = chol5(N, U, tol_piv);
                chol5_solve(U, b, dl);
                for (int a = 0; a < 5; a++) dlf[a] = (float)dl[a];
                gen_q(rs, rr, ac, n, lane, dpf, dlf, (float)y, Q, S2);
                if (fabs(dy) <= tol) break;
            }
        }
        for (int a = 0; a < 5; a++) d[a] = (double)dpf[a] + dl[a];
        __syncwarp();
    }
    float dh[5], dlo[5];
    for (int a = 0; a < 5; a++) split_pair(d[a], dh[a], dlo[a]);
    float chi = 0.0f;
    for (int j = lane; j < n; j += kWarp) {
        const MixS v = rs[j];
        chi += apply_update(v, rr[j], dh, dlo, ac[j].x / (v.sig * v.sig + (float)y), rr + j, ac + j, st.handover_h);
    }
    const double chid = warp_sum((double)chi);
    if (lane == 0) {
        write_source(out, i, d, U, y, Q0, nu, nout, rd);
        out.q[i] = chid;
        out.chi2[i] = chid;
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
                                                     const double* __restrict__ cal, MixObs mo) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_obs; o += (int64_t)gridDim.x * blockDim.x) {
        const double* gp = geo + 16 * (size_t)obs_src[o];
        SrcGeo S;
        for (int k = 0; k < 3; k++) { S.p[k] = gp[k]; S.q[k] = gp[3 + k]; S.r[k] = gp[6 + k]; }
        S.par = gp[9]; S.pma = gp[10]; S.pmd = gp[11]; S.cosd = gp[12];
        const float* gf = reinterpret_cast<const float*>(gp + 13);
        for (int k = 0; k < 3; k++) { S.pf[k] = gf[k]; S.qf[k] = gf[3 + k]; }
        const int64_t t = t_ns[o];
        const uint32_t m = meta[o];
        ObsOut ob;
        observe<2>(G, S, t, m, (G.cg.on || meta_kind(m)) ? mu[o] : 0.0, att, cal, ob);
        MixS a;
        float2 R;
        split_pair(ob.R, R.x, R.y);
        a.Ap = ob.Af[0];
        a.Aq = ob.Af[1];
        a.Aw = ob.Af[2];
        a.tau = ob.tauf;
        a.sig = meta_kind(m) ? -sigma[o] : sigma[o];
        mo.s[o] = a;
        mo.r[o] = R;
        MixT b;
        for (int k = 0; k < 4; k++) b.g[k] = ob.gf[k];
        b.meta = m;
        b.l = left_index(G, t);
        b.u = (float)((double)(t - knot_at(G, b.l)) * G.inv_knot_dt);
        b.pad = 0;
        mo.t[o] = b;
    }
}

// R += sum_j B_j g . d_a[l-3+j] + d_c[k]  (dR/da_n = g B_n, dR/dc_k = 1; Eqs. dfadq, pdC)
__global__ void __launch_bounds__(256) k_mix_correct(DevGeo G, int64_t n_obs, float2* __restrict__ mr,
                                                     const MixT* __restrict__ mt, const float4* __restrict__ d_att,
                                                     const float2* __restrict__ d_cal) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_obs; o += (int64_t)gridDim.x * blockDim.x) {
        const MixT r = mt[o];
        float B[4];
        bspline4_lu(G, r.l, r.u, B);
        const float4* da = d_att + (r.l - 3);
        float corr = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const float4 v = __ldg(da + j);
            corr = fmaf(B[j], r.g[0] * v.x + r.g[1] * v.y + r.g[2] * v.z + r.g[3] * v.w, corr);
        }
        const float2 dc = __ldg(d_cal + meta_cal(r.meta));
        float2 R = mr[o];
        pair_add(R.x, R.y, dc.x, dc.y);
        pair_add(R.x, R.y, corr, 0.0f);
        mr[o] = R;
    }
}

// Block Gauss-Seidel (Sect. 4.6, Eq. precond): before the C block the (W, W R) pairs take
// this iteration's attitude update d_att to first order, W R += W sum_j B_j g . d_a[l-3+j]
__global__ void __launch_bounds__(256) k_mix_ac_correct(DevGeo G, int64_t n_obs, float2* __restrict__ mac,
                                                        const MixT* __restrict__ mt,
                                                        const float4* __restrict__ d_att) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_obs; o += (int64_t)gridDim.x * blockDim.x) {
        const MixT r = mt[o];
        float B[4];
        bspline4_lu(G, r.l, r.u, B);
        const float4* da = d_att + (r.l - 3);
        float corr = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const float4 v = __ldg(da + j);
            corr = fmaf(B[j], r.g[0] * v.x + r.g[1] * v.y + r.g[2] * v.z + r.g[3] * v.w, corr);
        }
        float2 a = mac[o];
        a.y = fmaf(a.x, corr, a.y);
        mac[o] = a;
    }
}

// ---------------------------------------------------------------------------------------
// S block
// ---------------------------------------------------------------------------------------
constexpr int kScaleWarps = 4;
constexpr int kKeyCap = 1536;  // keys of a source kept in shared memory (6 KB per warp)

// sigma per class, robust scale and the round-0 class sums; one warp per source (largest first)
__global__ void __launch_bounds__(32 * kScaleWarps) k_mix_scale_sums(Settings st, const int64_t* __restrict__ src_off,
                                                                     const int32_t* __restrict__ src_nal,
                                                                     const int32_t* __restrict__ src_order,
                                                                     int32_t n_src, MixObs mo, MixSrcWork w) {
    __shared__ int hist_all[kScaleWarps][512];
    __shared__ uint32_t keys_all[kScaleWarps][kKeyCap];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int* hist = hist_all[wib];
    uint32_t* skeys = keys_all[wib];
    const int nw = gridDim.x * kScaleWarps;
    for (int q = blockIdx.x * kScaleWarps + wib; q < n_src; q += nw) {
        const int i = src_order[q];
        const int64_t o0 = src_off[i];
        const int n = (int)(src_off[i + 1] - o0);
        if (n == 0) {
            if (lane == 0) {
                SrcScale sc;
                sc.s2c[0] = sc.s2c[1] = sc.s2min = 1.0;
                sc.vs = 0.0f;
                sc.flags = 2;
                w.scale[i] = sc;
            }
            continue;
        }
        const MixS* rs = mo.s + o0;
        const float2* rr = mo.r + o0;
        const bool in_smem = n <= kKeyCap;
        float lo[2] = {3.0e38f, 3.0e38f}, hi[2] = {0.0f, 0.0f};
        auto scan = [&](int jj, float sg, float Rh) {
            if (in_smem) skeys[jj] = fkey(Rh / fabsf(sg));
            if (sg < 0.0f) {
                lo[1] = fminf(lo[1], -sg);
                hi[1] = fmaxf(hi[1], -sg);
            } else {
                lo[0] = fminf(lo[0], sg);
                hi[0] = fmaxf(hi[0], sg);
            }
        };
        int j = lane;
        for (; j + kWarp < n; j += 2 * kWarp) {   // two records in flight per lane
            const float sg0 = rs[j].sig, sg1 = rs[j + kWarp].sig;
            const float R0 = rr[j].x, R1 = rr[j + kWarp].x;
            scan(j, sg0, R0);
            scan(j + kWarp, sg1, R1);
        }
        if (j < n) scan(j, rs[j].sig, rr[j].x);
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
                hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
            }
        __syncwarp();
        const bool has0 = hi[0] > 0.0f, has1 = hi[1] > 0.0f;
        const bool uni = (!has0 || lo[0] == hi[0]) && (!has1 || lo[1] == hi[1]);
        const KeySrc key{in_smem ? skeys : nullptr, rs, rr};
        SrcRound in;
        for (int a = 0; a < 5; a++) in.dp[a] = 0.0f;
        in.isd[0] = in.isd[1] = 0.0f;
        in.sigc[0] = has0 ? lo[0] : 1.0f;
        in.sigc[1] = has1 ? lo[1] : 1.0f;
        in.vs = st.robust ? mix_robust_sigma(key, n, hist, lane) : 0.0f;
        in.mode = st.robust ? 0 : 2;
        in.pad = 0;
        if (lane == 0) {
            SrcScale sc;
            sc.s2c[0] = has0 ? (double)lo[0] * (double)lo[0] : 1.0;
            sc.s2c[1] = has1 ? (double)lo[1] * (double)lo[1] : 1.0;
            const float smin = fminf(lo[0], lo[1]);
            sc.s2min = (double)smin * (double)smin;
            sc.vs = in.vs;
            sc.flags = uni ? 1 : 0;
            w.scale[i] = sc;
            w.round[i] = in;
        }
        if (uni) class_sums(rs, rr, n, src_nal[i], lane, in, st.weight_fn, w.sums + i);
        __syncwarp();
    }
}

// class sums of round r >= 1 (weights and shift from the previous round's solution)
constexpr int kSumWarps = 4;
template <int kW>
__global__ void __launch_bounds__(32 * kW) k_mix_sums(Settings st, const int64_t* __restrict__ src_off,
                                                             const int32_t* __restrict__ src_nal,
                                                             const int32_t* __restrict__ src_order, int32_t n_src,
                                                             MixObs mo, MixSrcWork w) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * kW;
    for (int q = blockIdx.x * kW + (threadIdx.x >> 5); q < n_src; q += nw) {
        const int i = src_order[q];
        if (w.scale[i].flags != 1) continue;
        const int64_t o0 = src_off[i];
        const int n = (int)(src_off[i + 1] - o0);
        const SrcRound in = w.round[i];
        class_sums(mo.s + o0, mo.r + o0, n, src_nal[i], lane, in, st.weight_fn, w.sums + i);
    }
}

// the 5x5 algebra of one round, one thread per source: N(y), b(y), Q(y) from the class sums,
// y = 0 first, then the rational steps of the excess variance; d = d_prev + delta.  Writes the
// FP32 inputs of the next round, or after the last round the final update and the outputs.
__global__ void __launch_bounds__(256) k_mix_solve5(Settings st, int last, const int64_t* __restrict__ src_off,
                                                    int32_t n_src, SrcOutPtrs out, MixSrcWork w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_src) return;
    const SrcScale sc = w.scale[i];
    if (sc.flags & 2) {
        if (last) {
            for (int k = 0; k < 5; k++) out.d[5 * (size_t)i + k] = 0.0;
            for (int k = 0; k < 25; k++) out.cov[25 * (size_t)i + k] = 0.0;
            out.eps2[i] = out.q[i] = out.dsig[i] = out.chi2[i] = 0.0;
            out.nu[i] = out.nout[i] = out.rankdef[i] = 0;
        }
        return;
    }
    if (!(sc.flags & 1)) return;
    const int n = (int)(src_off[i + 1] - src_off[i]);
    const RoundSums& rsum = w.sums[i];
    ClassSums S;
    for (int c = 0; c < 2; c++) {
        for (int k = 0; k < 15; k++) S.AA[c][k] = rsum.AA[c][k];
        for (int k = 0; k < 5; k++) S.Ah[c][k] = rsum.Ah[c][k];
        S.hh[c] = rsum.hh[c];
    }
    const int nout = rsum.nout;
    SrcRound in = w.round[i];
    const double tol_piv = fmax(st.pivot_tol, kMixPivotTol);
    double U[kU5], dl[5], Q, S2;
    int rd;
    const int nu = n - nout - 5;
    double y = 0.0;
    class_solve(S, sc.s2c, 0.0, tol_piv, U, dl, rd, Q, S2);
    const double Q0 = Q;
    if (st.robust && nu > 0 && Q0 > (double)nu) {
        const double tol = 1e-12 * sc.s2min;
        for (int it = 0; it < st.n_eps; it++) {
            const double dy = (1.0 - Q / (double)nu) * Q / (-S2);
            y = fmax(0.0, y + dy);
            class_solve(S, sc.s2c, y, tol_piv, U, dl, rd, Q, S2);
            if (fabs(dy) <= tol) break;
        }
    }
    double d[5];
    for (int a = 0; a < 5; a++) d[a] = (double)in.dp[a] + dl[a];
    if (!last) {
        for (int a = 0; a < 5; a++) in.dp[a] = (float)d[a];
        for (int c = 0; c < 2; c++) in.isd[c] = (float)(1.0 / sqrt(sc.s2c[c] + y));
        in.mode = 1;
        w.round[i] = in;
    } else {
        SrcFinal f;
        for (int a = 0; a < 5; a++) split_pair(d[a], f.dh[a], f.dl[a]);
        for (int c = 0; c < 2; c++) f.iw[c] = (float)(1.0 / (sc.s2c[c] + y));
        w.fin[i] = f;
        write_source(out, i, d, U, y, Q0, nu, nout, rd);
    }
}

// R <- R - A d (float pairs), W = w / (sigma_c^2 + eps^2) with the last round's weights, chi^2
template <int kW>
__global__ void __launch_bounds__(32 * kW) k_mix_final(Settings st, const int64_t* __restrict__ src_off,
                                                              const int32_t* __restrict__ src_order, int32_t n_src,
                                                              SrcOutPtrs out, MixObs mo, MixSrcWork w) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * kW;
    for (int q = blockIdx.x * kW + (threadIdx.x >> 5); q < n_src; q += nw) {
        const int i = src_order[q];
        if (w.scale[i].flags != 1) continue;
        const int64_t o0 = src_off[i];
        const int n = (int)(src_off[i + 1] - o0);
        const SrcRound in = w.round[i];
        const SrcFinal f = w.fin[i];
        const MixS* rs = mo.s + o0;
        float2* rr = mo.r + o0;
        float2* ac = mo.ac + o0;
        float chi = 0.0f;
        auto fin = [&](int jj, const MixS& v, float2 R) {
            float A[5];
            arow(v, A);
            const int cls = v.sig < 0.0f ? 1 : 0;
            const float wgt = round_weight(in, R.x, R.x - adot(A, in.dp), cls, st.weight_fn);
            chi += apply_update(v, R, f.dh, f.dl, wgt * (cls ? f.iw[1] : f.iw[0]), rr + jj, ac + jj, st.handover_h);
        };
        int j = lane;
        for (; j + kWarp < n; j += 2 * kWarp) {
            const MixS v0 = rs[j], v1 = rs[j + kWarp];
            const float2 R0 = rr[j], R1 = rr[j + kWarp];
            fin(j, v0, R0);
            fin(j + kWarp, v1, R1);
        }
        if (j < n) fin(j, rs[j], rr[j]);
        chi = warp_sum_f(chi);
        if (lane == 0) {
            out.chi2[i] = chi;
            out.q[i] = chi;  // Q at the final (d, eps^2)
        }
    }
}

__global__ void __launch_bounds__(32 * kSumWarps) k_mix_general(Settings st, const int64_t* __restrict__ src_off,
                                                                int32_t n_src, SrcOutPtrs out, MixObs mo,
                                                                MixSrcWork w) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * kSumWarps;
    for (int i = blockIdx.x * kSumWarps + (threadIdx.x >> 5); i < n_src; i += nw) {
        const SrcScale sc = w.scale[i];
        if (sc.flags != 0) continue;
        const int64_t o0 = src_off[i];
        const int n = (int)(src_off[i + 1] - o0);
        mix_solve_general(st, i, n, mo.s + o0, mo.r + o0, mo.ac + o0, sc.s2min, sc.vs, out, lane);
    }
}

// ---------------------------------------------------------------------------------------
// A block accumulation (Eqs. normAmod, dDldan), one warp per knot interval.  Each lane
// sums its own observations in FP32 registers: the 100 distinct products BB'[p] M[m] of
// the 16x16 block (p, m over the 10 upper entries of the 4x4 matrices B B' and
// M = W (g g' + 4 lambda^2 s s')) and the 16 products B r.  The 32 lane partials are then
// added with TwoSum (compensated), because the attitude normals are nearly singular along
// the coefficient vector: the observation terms vanish along it (g is orthogonal to q) and
// only the norm term of relative size 4 lambda^2 fixes it.
// ---------------------------------------------------------------------------------------
constexpr int kAccVals = 116;
constexpr int kAccPad = 117;
constexpr int kAttWarps = 2;
// Observations in flight per lane: the records of the next kAttStages observations of a lane
// are copied into shared memory by cp.async while the current one is summed, and the
// time-order indices one round further ahead are held in registers, so that neither the
// index nor the record gather waits on the arithmetic (the kernel holds 116 accumulators per
// lane and runs at 8 warps per SM, too few to hide a dependent gather by occupancy).
constexpr int kAttStages = 4;
struct __align__(16) AttStage {
    MixT t;
    float2 ac;
    float2 pad;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void att_stage_load(AttStage* st, const MixT* mt, const float2* mac, uint32_t o) {
    cp_async16(&st->t, mt + o);
    cp_async16(reinterpret_cast<char*>(&st->t) + 16, reinterpret_cast<const char*>(mt + o) + 16);
    cp_async8(&st->ac, mac + o);
}

__host__ __device__ constexpr int mtri4(int i, int j) { return i * 4 - i * (i - 1) / 2 + (j - i); }
__host__ __device__ constexpr int mtri16(int i, int j) { return i * 16 - i * (i - 1) / 2 + (j - i); }
static_assert(mtri16(15, 15) == 135 && mtri16(1, 1) == 16, "upper-triangle index of the 16x16 block");

// One knot interval per group of kAttLanes lanes (kWarp / kAttLanes intervals per warp):
// each lane sums its share of the interval's observations in FP32, and each output of the
// 16x16 block is then the compensated sum of the group's kAttLanes lane partials.  The
// attitude normals are nearly singular along the coefficient vector (only the 4 lambda^2
// norm term, 4e-6 relative, fixes that direction), so the uncompensated per-lane sums must
// stay short: a whole warp per interval.  With 8 lanes per interval (about 34 observations
// per lane on 1-h knots) the rounding of the lane sums swamped the norm term and the update
// along the coefficient vector was lost.
constexpr int kAttLanes = 32;
constexpr int kAttGroups = kWarp / kAttLanes;

__global__ void __launch_bounds__(32 * kAttWarps) k_mix_att_accum(DevGeo G, float lambda2, int rhs_norm,
                                                                  const uint32_t* __restrict__ perm_t,
                                                                  const int64_t* __restrict__ ivl_off, int n_iv,
                                                                  const float2* __restrict__ mac,
                                                                  const MixT* __restrict__ mt,
                                                                  const double* __restrict__ att,
                                                                  double* __restrict__ blk) {
    __shared__ float red_all[kAttWarps][kWarp * kAccPad];
    __shared__ AttStage stage_all[kAttWarps][kAttStages][kWarp];
    __shared__ int16_t src_tab[kBlkVals];  // accumulator of each block output (>= 100: right-hand side)
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int sub = lane & (kAttLanes - 1);
    const int grp = lane / kAttLanes;
    const unsigned gmask = kAttLanes == kWarp ? 0xffffffffu : ((1u << (kAttLanes % kWarp)) - 1u) << (grp * kAttLanes);
    float* red = red_all[wib];
    for (int o = threadIdx.x; o < kBlkVals; o += blockDim.x) {
        int v;
        if (o < 136) {
            int i = 0;
            while (o >= mtri16(i, 15) + 1) i++;
            const int jj = i + (o - mtri16(i, i));
            const int bi = i >> 2, ci = i & 3, bj = jj >> 2, cj = jj & 3;
            const int m = ci <= cj ? mtri4(ci, cj) : mtri4(cj, ci);
            v = mtri4(bi, bj) * 10 + m;
        } else {
            v = 100 + (o - 136);
        }
        src_tab[o] = (int16_t)v;
    }
    __syncthreads();
    const int nwarps = gridDim.x * kAttWarps;
    const float l4 = 4.0f * lambda2;
    for (int iv0 = (blockIdx.x * kAttWarps + wib) * kAttGroups; iv0 < n_iv; iv0 += nwarps * kAttGroups) {
        const int iv = iv0 + grp;
        const bool have = iv < n_iv;
        const int l = iv + 3;
        // the 16 coefficients of the interval: two conversions per lane, then broadcast in the group
        const float af0 = have ? (float)att[4 * (int64_t)(l - 3) + sub] : 0.0f;
        const float af1 = have ? (float)att[4 * (int64_t)(l - 3) + kAttLanes + sub] : 0.0f;
        float a[16];
#pragma unroll
        for (int k = 0; k < 16; k++)
            a[k] = __shfl_sync(0xffffffffu, k < kAttLanes ? af0 : af1, grp * kAttLanes + (k & (kAttLanes - 1)));
        // accumulators as pairs: acc2[k] = (acc[2k], acc[2k+1]); two-wide FP32 FMAs (each lane
        // of the pair rounds like fmaf) halve the FMA instructions of the issue-bound loop
        float2 acc2[kAccVals / 2];
#pragma unroll
        for (int k = 0; k < kAccVals / 2; k++) acc2[k] = make_float2(0.0f, 0.0f);
        const int64_t beg = have ? ivl_off[iv] : 0, end = have ? ivl_off[iv + 1] : 0;
        // prologue: this lane's first kAttStages observations into the stages, and the indices
        // of the next kAttStages into registers
        uint32_t pnext[kAttStages];
#pragma unroll
        for (int q = 0; q < kAttStages; q++) {
            const int64_t j = beg + sub + kAttLanes * q;
            if (j < end) att_stage_load(&stage_all[wib][q][lane], mt, mac, perm_t[j]);
            cp_async_commit();
        }
#pragma unroll
        for (int q = 0; q < kAttStages; q++) {
            const int64_t j = beg + sub + kAttLanes * (q + kAttStages);
            pnext[q] = j < end ? perm_t[j] : 0u;
        }
        // the group's lanes run the same rounds (their own interval's length)
        for (int64_t base = beg; base < end; base += kAttLanes * kAttStages) {
#pragma unroll
          for (int q = 0; q < kAttStages; q++) {
            const int64_t j = base + kAttLanes * q + sub;
            cp_async_wait<kAttStages - 1>();  // the oldest outstanding group: this stage
            AttStage& sg = stage_all[wib][q][lane];
            const MixT rt = sg.t;
            const float2 WR = sg.ac;          // (W, W R)
            __syncwarp(gmask);
            // refill the stage with this lane's observation kAttStages rounds ahead
            const int64_t jn = j + kAttLanes * kAttStages;
            if (jn < end) {
                att_stage_load(&sg, mt, mac, pnext[q]);
                const int64_t jf = jn + kAttLanes * kAttStages;
                pnext[q] = jf < end ? perm_t[jf] : 0u;
            }
            cp_async_commit();
            if (j >= end) continue;
            float B[4];
            bspline4_lu(G, l, rt.u, B);
            float s[4];
#pragma unroll
            for (int c = 0; c < 4; c++) s[c] = B[0] * a[c] + B[1] * a[4 + c] + B[2] * a[8 + c] + B[3] * a[12 + c];
            const float W = WR.x;
            float M[10], r[4], BB[10];
#pragma unroll
            for (int c = 0; c < 4; c++)
#pragma unroll
                for (int e = c; e < 4; e++) {
                    M[mtri4(c, e)] = W * (rt.g[c] * rt.g[e] + l4 * s[c] * s[e]);
                    BB[mtri4(c, e)] = B[c] * B[e];
                }
            float D = 0.0f;
            if (rhs_norm) D = 1.0f - (s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3]);
#pragma unroll
            for (int c = 0; c < 4; c++) {
                r[c] = WR.y * rt.g[c];
                if (rhs_norm) r[c] -= W * (2.0f * lambda2 * D * s[c]);
            }
#pragma unroll
            for (int p = 0; p < 10; p++) {
                const float2 bb = make_float2(BB[p], BB[p]);
#pragma unroll
                for (int m = 0; m < 10; m += 2)
                    acc2[(p * 10 + m) / 2] = __ffma2_rn(bb, make_float2(M[m], M[m + 1]), acc2[(p * 10 + m) / 2]);
            }
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const float2 bv = make_float2(B[b], B[b]);
#pragma unroll
                for (int c = 0; c < 4; c += 2)
                    acc2[(100 + 4 * b + c) / 2] = __ffma2_rn(bv, make_float2(r[c], r[c + 1]), acc2[(100 + 4 * b + c) / 2]);
            }
          }
        }
        cp_async_wait<0>();
        // compensated reduction of the group's lane partials through shared memory
#pragma unroll
        for (int k = 0; k < kAccVals / 2; k++) {
            red[lane * kAccPad + 2 * k] = acc2[k].x;
            red[lane * kAccPad + 2 * k + 1] = acc2[k].y;
        }
        __syncwarp();
        if (have) {
            const float* gred = red + grp * kAttLanes * kAccPad;
            for (int o = sub; o < kBlkVals; o += kAttLanes) {
                const int src = src_tab[o];
                float hi = 0.0f, lo = 0.0f;
#pragma unroll
                for (int q = 0; q < kAttLanes; q++) {
                    float s_, e_;
                    two_sum(hi, gred[q * kAccPad + src], s_, e_);
                    hi = s_;
                    lo = __fadd_rn(lo, e_);
                }
                const double v = (double)hi + (double)lo;
                blk[(int64_t)iv * kBlkVals + o] = src >= 100 ? -v : v;
            }
        }
        __syncwarp();
    }
}

// C block sums from the records (calibration order): N_kk = sum W, b_k = -sum W R; the 1x1
// robust solve gives d~_k = (b / sqrt(N)) / sqrt(N), or 0 with a rank defect.
__global__ void k_mix_cal_accum(int n_cal, const uint32_t* __restrict__ perm_c, const int64_t* __restrict__ cal_off,
                                const float2* __restrict__ mac, double* __restrict__ dtil, int* __restrict__ rd) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n_cal; k += nw) {
        float sw = 0.0f, swr = 0.0f;
        const int64_t end = cal_off[k + 1];
        int64_t j = cal_off[k] + lane;
        // four independent gathers in flight per lane; the sums keep the order j, j + 32, ...
        for (; j + 3 * kWarp < end; j += 4 * kWarp) {
            const uint32_t p0 = perm_c[j], p1 = perm_c[j + kWarp], p2 = perm_c[j + 2 * kWarp],
                           p3 = perm_c[j + 3 * kWarp];
            const float2 a0 = mac[p0], a1 = mac[p1], a2 = mac[p2], a3 = mac[p3];   // (W, W R)
            sw += a0.x;
            swr += a0.y;
            sw += a1.x;
            swr += a1.y;
            sw += a2.x;
            swr += a2.y;
            sw += a3.x;
            swr += a3.y;
        }
        for (; j < end; j += kWarp) {
            const float2 a = mac[perm_c[j]];
            sw += a.x;
            swr += a.y;
        }
        const double swd = warp_sum((double)sw);
        const double swrd = warp_sum((double)swr);
        if (lane == 0) {
            if (swd > 0.0) {
                const double u = sqrt(swd);
                dtil[k] = (-swrd / u) / u;
                rd[k] = 0;
            } else {
                dtil[k] = 0.0;
                rd[k] = 1;
            }
        }
    }
}

// constraint projection as in the FP64 form (Eq. calCon: disjoint groups, d = d~ - mean d~);
// c += d, and the update is accumulated as a float pair for the next linearized pass
__global__ void k_mix_cal_project(int n_days, const double* __restrict__ dtil, double* __restrict__ cal,
                                  float2* __restrict__ d_cal) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 3 * n_days) return;
    int64_t k0;
    int cnt;
    if (g < n_days) {
        k0 = (int64_t)g * 124;
        cnt = 124;
    } else {
        k0 = (int64_t)n_days * 124 + (int64_t)(g - n_days) * 7;
        cnt = 7;
    }
    double s = 0.0;
    for (int i = 0; i < cnt; i++) s += dtil[k0 + i];
    const double m = s / (double)cnt;
    for (int i = 0; i < cnt; i++) {
        const double dk = dtil[k0 + i] - m;
        cal[k0 + i] += dk;
        const float2 p = d_cal[k0 + i];
        float hi, lo;
        split_pair((double)p.x + (double)p.y + dk, hi, lo);
        d_cal[k0 + i] = make_float2(hi, lo);
    }
}

// R <- R - A c for a learned proposal c added to the sources (float-pair arithmetic)
__global__ void k_mix_prop(int32_t n_src, const int64_t* __restrict__ src_off, MixObs mo,
                           const double* __restrict__ corr) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n_src; i += nw) {
        float ch[5], cl[5];
        for (int a = 0; a < 5; a++) split_pair(corr[5 * (size_t)i + a], ch[a], cl[a]);
        for (int64_t o = src_off[i] + lane; o < src_off[i + 1]; o += kWarp) {
            const MixS v = mo.s[o];
            float A[5];
            arow(v, A);
            float sh, sl;
            row_dot_pair(A, ch, cl, sh, sl);
            float2 R = mo.r[o];
            pair_add(R.x, R.y, -sh, -sl);
            mo.r[o] = R;
            const float W = mo.ac[o].x;
            mo.ac[o] = make_float2(W, W * R.x);
        }
    }
}

__global__ void k_mix_rw(int64_t n, const uint32_t* __restrict__ perm, const float2* __restrict__ mr,
                         const float2* __restrict__ mac, double* __restrict__ R, double* __restrict__ W) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        if (R) R[perm[o]] = (double)mr[o].x + (double)mr[o].y;
        if (W) W[perm[o]] = (double)mac[o].x;
    }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
// the observation pass of the mixed S block: the full FP64 model (refresh) or the linearized
// correction by the A and C updates since the last source update; both leave d_att, d_cal zero
void launch_mix_pass(const DevGeo& G, bool refresh, const int64_t* t_ns, const uint32_t* meta, const float* sigma,
                     const double* mu, const int32_t* obs_src, int64_t n_obs, int32_t n_src, const double* src,
                     const double* att, const double* cal, const MixObs& mo, double* geo, float* d_att,
                     float2* d_cal, int n_coef, int n_cal, const Shapes& sh, cudaStream_t s) {
    if (refresh) {
        launch_src_geo(n_src, src, geo, s);
        k_mix_forward<<<grid_of(n_obs, 256, 152 * 64), 256, 0, s>>>(G, n_obs, t_ns, meta, sigma, mu, obs_src, geo,
                                                                     att, cal, mo);
    } else {
        k_mix_correct<<<grid_of(n_obs, sh.obs_threads, 152 * sh.obs_bps), sh.obs_threads, 0, s>>>(G, n_obs, mo.r, mo.t,
                                                                     reinterpret_cast<const float4*>(d_att), d_cal);
    }
    cudaMemsetAsync(d_att, 0, sizeof(float) * 4 * (size_t)n_coef, s);
    cudaMemsetAsync(d_cal, 0, sizeof(float2) * (size_t)n_cal, s);
}

void launch_mix_solve(const Settings& st, const int64_t* src_off, const int32_t* src_nal, const int32_t* src_order,
                      int32_t n_src, const SrcOutPtrs& out, const MixObs& mo, const MixSrcWork& w,
                      const Shapes& sh, cudaStream_t s) {
    const int rounds = st.robust ? st.n_rounds + 1 : 1;
    const int W = sh.sums_warps;
    const int warp_blocks = grid_of(n_src, W, 152 * sh.sums_bps);
    const int t5 = sh.solve5_threads;
    const int thread_blocks = (n_src + t5 - 1) / t5 > 0 ? (n_src + t5 - 1) / t5 : 1;
    k_mix_scale_sums<<<grid_of(n_src, kScaleWarps, 152 * 8), 32 * kScaleWarps, 0, s>>>(st, src_off, src_nal,
                                                                                       src_order, n_src, mo, w);
    auto sums = [&]() {
        if (W == 2) k_mix_sums<2><<<warp_blocks, 64, 0, s>>>(st, src_off, src_nal, src_order, n_src, mo, w);
        else if (W == 8) k_mix_sums<8><<<warp_blocks, 256, 0, s>>>(st, src_off, src_nal, src_order, n_src, mo, w);
        else k_mix_sums<4><<<warp_blocks, 128, 0, s>>>(st, src_off, src_nal, src_order, n_src, mo, w);
    };
    for (int r = 0; r < rounds; r++) {
        if (r > 0) sums();
        k_mix_solve5<<<thread_blocks, t5, 0, s>>>(st, r == rounds - 1, src_off, n_src, out, w);
    }
    if (W == 2) k_mix_final<2><<<warp_blocks, 64, 0, s>>>(st, src_off, src_order, n_src, out, mo, w);
    else if (W == 8) k_mix_final<8><<<warp_blocks, 256, 0, s>>>(st, src_off, src_order, n_src, out, mo, w);
    else k_mix_final<4><<<warp_blocks, 128, 0, s>>>(st, src_off, src_order, n_src, out, mo, w);
    k_mix_general<<<grid_of(n_src, kSumWarps, 152 * 4), 32 * kSumWarps, 0, s>>>(st, src_off, n_src, out, mo, w);
}

void launch_mix_att_accum(const DevGeo& G, double lambda2, int rhs_norm, const uint32_t* perm_t,
                          const int64_t* ivl_off, int n_iv, const MixObs& mo, const double* att, double* blk,
                          const Shapes& sh, cudaStream_t s) {
    const int bps = sh.att_bps > 0 ? sh.att_bps : 64;
    k_mix_att_accum<<<grid_of((n_iv + kAttGroups - 1) / kAttGroups, kAttWarps, 152 * bps), 32 * kAttWarps, 0, s>>>(G, (float)lambda2, rhs_norm, perm_t,
                                                                                 ivl_off, n_iv, mo.ac, mo.t, att, blk);
}

void launch_mix_cal(int n_cal, int n_days, const uint32_t* perm_c, const int64_t* cal_off, const MixObs& mo,
                    double* dtil, int* rd, double* cal, float2* d_cal, const Shapes& sh, cudaStream_t s) {
    k_mix_cal_accum<<<grid_of(n_cal, sh.cal_threads / 32, 152 * sh.cal_bps), sh.cal_threads, 0, s>>>(
        n_cal, perm_c, cal_off, mo.ac, dtil, rd);
    k_mix_cal_project<<<(3 * n_days + 127) / 128, 128, 0, s>>>(n_days, dtil, cal, d_cal);
}

void launch_mix_ac_correct(const DevGeo& G, int64_t n_obs, const MixObs& mo, const float* d_att, cudaStream_t s) {
    k_mix_ac_correct<<<grid_of(n_obs, 256, 152 * 32), 256, 0, s>>>(G, n_obs, mo.ac, mo.t,
                                                                    reinterpret_cast<const float4*>(d_att));
}

void launch_mix_prop(int32_t n_src, const int64_t* src_off, const MixObs& mo, const double* corr, cudaStream_t s) {
    k_mix_prop<<<grid_of(n_src, 8, 152 * 16), 256, 0, s>>>(n_src, src_off, mo, corr);
}

void launch_mix_rw(int64_t n, const uint32_t* perm, const MixObs& mo, double* R, double* W, cudaStream_t s) {
    k_mix_rw<<<grid_of(n, 256, 152 * 32), 256, 0, s>>>(n, perm, mo.r, mo.ac, R, W);
}

}  // namespace agis
