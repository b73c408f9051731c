// k_learned.cu -- the learned iteration proposal: update history, features, the network's
// forward on tensor cores (BF16 mma.sync, FP32 accumulation), its training gradient and
// Adam step, and the application of a proposal to the sources and to the residuals that
// the A and C blocks read.  Not part of the paper (its analogue is the accelerated simple
// iteration of Sect. 4.7); the definitions are those of include/agis.h.
#include <cuda_bf16.h>

#include <string>

#include "agis_internal.cuh"

namespace agis {

namespace {

constexpr int kIn = AGIS_MLP_N_IN, kH = AGIS_MLP_N_HIDDEN, kOut = AGIS_MLP_N_OUT;
// packed layout (32-bit words; rows padded so that the fragment loads of a warp hit
// distinct shared-memory banks)
constexpr int kS1 = 20, kS2 = 36, kS3 = 36;           // row strides (words) of W1, W2, W3
constexpr int kW1 = 0, kW2 = kW1 + kH * kS1, kW3 = kW2 + kH * kS2, kB1 = kW3 + 8 * kS3;
constexpr int kB2 = kB1 + kH, kB3 = kB2 + kH, kPackedWords = kB3 + 8;
static_assert(kPackedWords * 4 == AGIS_MLP_PACKED_BYTES, "packed size");
// flat FP32 parameter offsets
constexpr int pW1 = 0, pB1 = pW1 + kH * kIn, pW2 = pB1 + kH, pB2 = pW2 + kH * kH, pW3 = pB2 + kH,
              pB3 = pW3 + kOut * kH, pN = pB3 + kOut;
static_assert(pN == AGIS_MLP_N_PARAMS, "parameter count");

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// D = A B + D for one 16x8x16 tile: A 16x16 (row), B 16x8 (col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

int grid_of(int64_t n, int per_block, int cap) {
    int64_t b = (n + per_block - 1) / per_block;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

// FP32 parameters -> packed BF16 weights (zero padding) and FP32 biases
__global__ void k_mlp_pack(const float* __restrict__ p, uint32_t* __restrict__ out) {
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < kPackedWords; w += gridDim.x * blockDim.x) {
        uint32_t v = 0;
        if (w < kW2) {
            const int r = w / kS1, k = 2 * (w % kS1);
            const float a = k < kIn ? p[pW1 + r * kIn + k] : 0.0f, b = k + 1 < kIn ? p[pW1 + r * kIn + k + 1] : 0.0f;
            v = (k < 32) ? pack2(a, b) : 0u;
        } else if (w < kW3) {
            const int r = (w - kW2) / kS2, k = 2 * ((w - kW2) % kS2);
            v = k < kH ? pack2(p[pW2 + r * kH + k], p[pW2 + r * kH + k + 1]) : 0u;
        } else if (w < kB1) {
            const int r = (w - kW3) / kS3, k = 2 * ((w - kW3) % kS3);
            v = (r < kOut && k < kH) ? pack2(p[pW3 + r * kH + k], p[pW3 + r * kH + k + 1]) : 0u;
        } else if (w < kB2) {
            v = __float_as_uint(p[pB1 + (w - kB1)]);
        } else if (w < kB3) {
            v = __float_as_uint(p[pB2 + (w - kB2)]);
        } else {
            const int o = w - kB3;
            v = __float_as_uint(o < kOut ? p[pB3 + o] : 0.0f);
        }
        out[w] = v;
    }
}

// Forward on tensor cores: each warp takes 16 rows at a time.  Fragment layouts of
// mma.m16n8k16 (PTX ISA): A row r = lane/4 (+8), k = 2 (lane%4) (+1, +8); B n = lane/4,
// k = 2 (lane%4) (+1, +8); C row lane/4 (+8), n = 2 (lane%4) (+1).  The C tiles of n-blocks
// 2t and 2t+1 form, after bias, ReLU and rounding, the A tile of k-block t of the next layer.
constexpr int kFwdWarps = 4;
__global__ void __launch_bounds__(32 * kFwdWarps) k_mlp_fwd_tc(const uint32_t* __restrict__ packed,
                                                                const float* __restrict__ X, int n,
                                                                float* __restrict__ Y) {
    __shared__ uint32_t sp[kPackedWords];
    for (int w = threadIdx.x; w < kPackedWords; w += blockDim.x) sp[w] = packed[w];
    __syncthreads();
    const float* b1 = reinterpret_cast<const float*>(sp + kB1);
    const float* b2 = reinterpret_cast<const float*>(sp + kB2);
    const float* b3 = reinterpret_cast<const float*>(sp + kB3);
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int nt = (n + 15) / 16;
    for (int tile = blockIdx.x * kFwdWarps + (threadIdx.x >> 5); tile < nt; tile += gridDim.x * kFwdWarps) {
        const int r0 = tile * 16 + g, r1 = r0 + 8;
        auto xin = [&](int r, int k) -> uint32_t {
            if (r >= n || k >= kIn) return 0u;
            const float2 v = *reinterpret_cast<const float2*>(X + (size_t)r * kIn + k);
            return pack2(v.x, v.y);
        };
        uint32_t a1[2][4];
#pragma unroll
        for (int t = 0; t < 2; t++) {
            a1[t][0] = xin(r0, 16 * t + 2 * q);
            a1[t][1] = xin(r1, 16 * t + 2 * q);
            a1[t][2] = xin(r0, 16 * t + 8 + 2 * q);
            a1[t][3] = xin(r1, 16 * t + 8 + 2 * q);
        }
        float h[8][4];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            const uint32_t* wr = sp + kW1 + (8 * j + g) * kS1;
#pragma unroll
            for (int t = 0; t < 2; t++) mma16816(c, a1[t], wr[8 * t + q], wr[8 * t + 4 + q]);
            const float bb0 = b1[8 * j + 2 * q], bb1 = b1[8 * j + 2 * q + 1];
            h[j][0] = fmaxf(c[0] + bb0, 0.f); h[j][1] = fmaxf(c[1] + bb1, 0.f);
            h[j][2] = fmaxf(c[2] + bb0, 0.f); h[j][3] = fmaxf(c[3] + bb1, 0.f);
        }
        uint32_t a2[4][4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            a2[t][0] = pack2(h[2 * t][0], h[2 * t][1]);
            a2[t][1] = pack2(h[2 * t][2], h[2 * t][3]);
            a2[t][2] = pack2(h[2 * t + 1][0], h[2 * t + 1][1]);
            a2[t][3] = pack2(h[2 * t + 1][2], h[2 * t + 1][3]);
        }
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            const uint32_t* wr = sp + kW2 + (8 * j + g) * kS2;
#pragma unroll
            for (int t = 0; t < 4; t++) mma16816(c, a2[t], wr[8 * t + q], wr[8 * t + 4 + q]);
            const float bb0 = b2[8 * j + 2 * q], bb1 = b2[8 * j + 2 * q + 1];
            h[j][0] = fmaxf(c[0] + bb0, 0.f); h[j][1] = fmaxf(c[1] + bb1, 0.f);
            h[j][2] = fmaxf(c[2] + bb0, 0.f); h[j][3] = fmaxf(c[3] + bb1, 0.f);
        }
#pragma unroll
        for (int t = 0; t < 4; t++) {
            a2[t][0] = pack2(h[2 * t][0], h[2 * t][1]);
            a2[t][1] = pack2(h[2 * t][2], h[2 * t][3]);
            a2[t][2] = pack2(h[2 * t + 1][0], h[2 * t + 1][1]);
            a2[t][3] = pack2(h[2 * t + 1][2], h[2 * t + 1][3]);
        }
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        const uint32_t* wr = sp + kW3 + g * kS3;
#pragma unroll
        for (int t = 0; t < 4; t++) mma16816(c, a2[t], wr[8 * t + q], wr[8 * t + 4 + q]);
        const int col = 2 * q;
        if (r0 < n) {
            if (col < kOut) Y[(size_t)r0 * kOut + col] = c[0] + b3[col];
            if (col + 1 < kOut) Y[(size_t)r0 * kOut + col + 1] = c[1] + b3[col + 1];
        }
        if (r1 < n) {
            if (col < kOut) Y[(size_t)r1 * kOut + col] = c[2] + b3[col];
            if (col + 1 < kOut) Y[(size_t)r1 * kOut + col + 1] = c[3] + b3[col + 1];
        }
    }
}

// Loss and gradient of the BF16-rounded forward (FP32 arithmetic on the CUDA cores): every
// lane takes one row; the weight gradients of a warp's 32 rows are outer-product sums over
// the rows kept in shared memory, added into a per-block gradient with shared atomics and
// then into the global gradient.
constexpr int kGradWarps = 4;
constexpr int kRowF = kIn + 4 * kH + kOut;            // per row: x, h1, h2, dh2, dh1, dy
constexpr size_t kGradSmem = (size_t)(2 * pN + kGradWarps * 32 * kRowF + 1) * sizeof(float);

__global__ void __launch_bounds__(32 * kGradWarps) k_mlp_loss_grad(const float* __restrict__ p,
                                                                    const float* __restrict__ X,
                                                                    const float* __restrict__ T,
                                                                    const int32_t* __restrict__ idx, int n,
                                                                    float* __restrict__ grad,
                                                                    float* __restrict__ loss) {
    extern __shared__ float sm[];
    float* W = sm;                                     // rounded weights and FP32 biases, flat layout
    float* G = sm + pN;                                // block gradient
    float* rowbuf = sm + 2 * pN + (threadIdx.x >> 5) * 32 * kRowF;
    float* Lsum = sm + 2 * pN + kGradWarps * 32 * kRowF;
    for (int i = threadIdx.x; i < pN; i += blockDim.x) {
        const bool is_w = (i < pB1) || (i >= pW2 && i < pB2) || (i >= pW3 && i < pB3);
        W[i] = is_w ? bf16r(p[i]) : p[i];
        G[i] = 0.0f;
    }
    if (threadIdx.x == 0) *Lsum = 0.0f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float inv_n = 1.0f / (float)n;
    float lpart = 0.0f;
    const int ntile = (n + 31) / 32;
    for (int tile = blockIdx.x * kGradWarps + (threadIdx.x >> 5); tile < ntile; tile += gridDim.x * kGradWarps) {
        const int rb_ = tile * 32 + lane;
        const bool valid = rb_ < n;
        const int64_t r = valid ? (idx ? (int64_t)idx[rb_] : (int64_t)rb_) : 0;
        float* xs = rowbuf + lane * kRowF;
        float* h1 = xs + kIn;
        float* h2 = h1 + kH;
        float* dh2 = h2 + kH;
        float* dh1 = dh2 + kH;
        float* dy = dh1 + kH;
        for (int k = 0; k < kIn; k++) xs[k] = valid ? bf16r(X[r * kIn + k]) : 0.0f;
        for (int i = 0; i < kH; i++) {
            float z = W[pB1 + i];
            for (int k = 0; k < kIn; k++) z = fmaf(W[pW1 + i * kIn + k], xs[k], z);
            h1[i] = bf16r(fmaxf(z, 0.0f));
        }
        for (int i = 0; i < kH; i++) {
            float z = W[pB2 + i];
            for (int k = 0; k < kH; k++) z = fmaf(W[pW2 + i * kH + k], h1[k], z);
            h2[i] = bf16r(fmaxf(z, 0.0f));
        }
        for (int o = 0; o < kOut; o++) {
            float y = W[pB3 + o];
            for (int k = 0; k < kH; k++) y = fmaf(W[pW3 + o * kH + k], h2[k], y);
            const float e = valid ? y - T[r * kOut + o] : 0.0f;
            lpart = fmaf(e, e, lpart);
            dy[o] = 2.0f * e * inv_n;
        }
        for (int i = 0; i < kH; i++) {
            float s = 0.0f;
            for (int o = 0; o < kOut; o++) s = fmaf(dy[o], W[pW3 + o * kH + i], s);
            dh2[i] = h2[i] > 0.0f ? s : 0.0f;
        }
        for (int k = 0; k < kH; k++) {
            float s = 0.0f;
            for (int i = 0; i < kH; i++) s = fmaf(dh2[i], W[pW2 + i * kH + k], s);
            dh1[k] = h1[k] > 0.0f ? s : 0.0f;
        }
        __syncwarp();
        // weight gradients over the 32 rows of the tile, each lane owning entries lane + 32 m
        const float* rb = rowbuf;
        for (int e = lane; e < kOut * kH; e += 32) {           // W3
            const int o = e / kH, k = e % kH;
            float s = 0.0f;
            for (int q = 0; q < 32; q++) s = fmaf(rb[q * kRowF + kIn + 4 * kH + o], rb[q * kRowF + kIn + kH + k], s);
            atomicAdd(&G[pW3 + e], s);
        }
        for (int e = lane; e < kH * kH; e += 32) {             // W2
            const int i = e / kH, k = e % kH;
            float s = 0.0f;
            for (int q = 0; q < 32; q++) s = fmaf(rb[q * kRowF + kIn + 2 * kH + i], rb[q * kRowF + kIn + k], s);
            atomicAdd(&G[pW2 + e], s);
        }
        for (int e = lane; e < kH * kIn; e += 32) {            // W1
            const int i = e / kIn, k = e % kIn;
            float s = 0.0f;
            for (int q = 0; q < 32; q++) s = fmaf(rb[q * kRowF + kIn + 3 * kH + i], rb[q * kRowF + k], s);
            atomicAdd(&G[pW1 + e], s);
        }
        for (int e = lane; e < 2 * kH + kOut; e += 32) {      // biases
            int off, src;
            if (e < kH) { off = pB1 + e; src = kIn + 3 * kH + e; }
            else if (e < 2 * kH) { off = pB2 + e - kH; src = kIn + 2 * kH + e - kH; }
            else { off = pB3 + e - 2 * kH; src = kIn + 4 * kH + e - 2 * kH; }
            float s = 0.0f;
            for (int q = 0; q < 32; q++) s += rb[q * kRowF + src];
            atomicAdd(&G[off], s);
        }
        __syncwarp();
    }
    lpart = warp_sum_f32(lpart);
    if (lane == 0) atomicAdd(Lsum, lpart);
    __syncthreads();
    for (int i = threadIdx.x; i < pN; i += blockDim.x) atomicAdd(&grad[i], G[i]);
    if (threadIdx.x == 0) atomicAdd(loss, *Lsum * inv_n);
}

__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int t, float lr, float b1, float b2, float eps) {
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pN; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ---------------------------------------------------------------------------------------
// proposal: history, features, application
// ---------------------------------------------------------------------------------------
// shift the per-source history of the last four updates (oldest first) and append d
__global__ void k_hist_push(int32_t n_src, const double* __restrict__ d, double* __restrict__ hist) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += gridDim.x * blockDim.x) {
        double* h = hist + 20 * (size_t)i;
#pragma unroll
        for (int k = 0; k < 15; k++) h[k] = h[k + 5];
#pragma unroll
        for (int k = 0; k < 5; k++) h[15 + k] = d[5 * (size_t)i + k];
    }
}

__global__ void k_prop_features(int32_t n_src, const double* __restrict__ hist, const int64_t* __restrict__ src_off,
                                const double* __restrict__ src, double sin_obl, double cos_obl,
                                float* __restrict__ X, double* __restrict__ sigma) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += gridDim.x * blockDim.x) {
        const double* h = hist + 20 * (size_t)i;
        double s2 = 0.0;
        for (int k = 0; k < 20; k++) s2 += h[k] * h[k];
        const double sg = sqrt(s2 / 20.0);
        const double inv = sg > 0.0 ? 1.0 / sg : 1.0;
        float* x = X + (size_t)kIn * i;
        for (int k = 0; k < 20; k++) x[k] = (float)(h[k] * inv);
        const double nobs = (double)(src_off[i + 1] - src_off[i]);
        x[20] = (float)(log10(nobs > 1.0 ? nobs : 1.0) - 2.5);
        double sa, ca, sd, cd;
        sincos(src[5 * (size_t)i], &sa, &ca);
        sincos(src[5 * (size_t)i + 1], &sd, &cd);
        x[21] = (float)(-sin_obl * cd * sa + cos_obl * sd);
        sigma[i] = sg;
    }
}

// sources += sigma * y (alpha* turned into alpha with cos(delta)); the correction is kept in
// tangent units for the residual update
__global__ void k_prop_apply(int32_t n_src, const float* __restrict__ Y, const double* __restrict__ sigma,
                             double* __restrict__ src, double* __restrict__ corr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += gridDim.x * blockDim.x) {
        double* s = src + 5 * (size_t)i;
        double c[5];
        for (int k = 0; k < 5; k++) {
            const double y = (double)Y[(size_t)kOut * i + k];
            c[k] = isfinite(y) ? sigma[i] * y : 0.0;
        }
        s[0] += c[0] / cos(s[1]);
        for (int k = 1; k < 5; k++) s[k] += c[k];
        for (int k = 0; k < 5; k++) corr[5 * (size_t)i + k] = c[k];
    }
}

__global__ void k_prop_targets(int32_t n, const double* __restrict__ xk, const double* __restrict__ xr,
                               const double* __restrict__ sigma, float* __restrict__ T) {
    const double pi = 3.141592653589793;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double* a = xk + 5 * (size_t)i;
        const double* b = xr + 5 * (size_t)i;
        const double inv = sigma[i] > 0.0 ? 1.0 / sigma[i] : 1.0;
        double da = b[0] - a[0];
        da = da - 2.0 * pi * floor((da + pi) / (2.0 * pi));
        T[(size_t)kOut * i] = (float)(da * cos(a[1]) * inv);
        for (int k = 1; k < 5; k++) T[(size_t)kOut * i + k] = (float)((b[k] - a[k]) * inv);
    }
}

// FP64 form: R <- R - A c on the hand-over records (A from the observation pass's scratch)
__global__ void k_prop_rec(int32_t n_src, const int64_t* __restrict__ src_off, const double* __restrict__ scratch,
                           ObsRec* __restrict__ rec, const double* __restrict__ corr) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n_src; i += nw) {
        const double* c = corr + 5 * (size_t)i;
        const double c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3], c4 = c[4];
        for (int64_t o = src_off[i] + lane; o < src_off[i + 1]; o += kWarp) {
            const double* e = scratch + (size_t)o * kScr;
            rec[o].R -= e[1] * c0 + e[2] * c1 + e[3] * c2 + e[4] * c3 + e[5] * c4;
        }
    }
}

// ---------------------------------------------------------------------------------------
// accelerated simple iteration (Sect. 4.7)
// ---------------------------------------------------------------------------------------
// order-preserving map of a double onto uint64 (negative values: all bits flipped; others:
// sign bit set), and back
__device__ __forceinline__ unsigned long long ord_key(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(unsigned long long k) {
    const unsigned long long u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)u);
}

constexpr int kAsiThreads = 1024;

// One block.  r_j = d1[i] / d0[i] for the parallax of sample source i = j * stride (rows
// of ld doubles, parallax at 2); the lower median of the finite ratios by an exact radix
// select over their order-preserving keys, 8 digits of 8 bits.  out: [median, lambda
// clamped to [0, lam_max], 1 / (1 - lambda), count of ratios].
__global__ void __launch_bounds__(kAsiThreads) k_asi_lambda(int32_t n_src, int32_t stride,
                                                            const double* __restrict__ d0p,
                                                            const double* __restrict__ d1p, int ld, double lam_max,
                                                            unsigned long long* __restrict__ keys,
                                                            double* __restrict__ out) {
    __shared__ unsigned int bins[256];
    __shared__ unsigned int s_count;
    __shared__ unsigned long long s_prefix, s_mask;
    __shared__ unsigned int s_rank;
    const int n_s = (n_src + stride - 1) / stride;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    unsigned int cnt = 0;
    for (int j = threadIdx.x; j < n_s; j += kAsiThreads) {
        const size_t row = (size_t)ld * j * stride + 2;
        const double d0 = d0p[row], d1 = d1p[row];
        const double r = d0 != 0.0 ? d1 / d0 : 0.0;
        const bool ok = d0 != 0.0 && isfinite(r);
        keys[j] = ok ? ord_key(r) : ~0ull;   // invalid ratios sort after every finite one
        cnt += ok ? 1u : 0u;
    }
    atomicAdd(&s_count, cnt);
    if (threadIdx.x == 0) {
        s_prefix = 0ull;
        s_mask = 0ull;
    }
    __syncthreads();
    const unsigned int n_ok = s_count;
    if (n_ok == 0) {
        if (threadIdx.x == 0) {
            out[0] = 0.0;
            out[1] = 0.0;
            out[2] = 1.0;
            out[3] = 0.0;
        }
        return;
    }
    if (threadIdx.x == 0) s_rank = (n_ok - 1) / 2;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += kAsiThreads) bins[b] = 0;
        __syncthreads();
        const unsigned long long prefix = s_prefix, mask = s_mask;
        for (int j = threadIdx.x; j < n_s; j += kAsiThreads) {
            const unsigned long long k = keys[j];
            if ((k & mask) == prefix) atomicAdd(&bins[(unsigned int)(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int rank = s_rank, b = 0;
            for (; b < 255; b++) {
                if (rank < bins[b]) break;
                rank -= bins[b];
            }
            s_rank = rank;
            s_prefix = prefix | ((unsigned long long)b << shift);
            s_mask = mask | (255ull << shift);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double med = key_value(s_prefix);
        const double lam = fmin(fmax(med, 0.0), lam_max);
        out[0] = med;
        out[1] = lam;
        out[2] = 1.0 / (1.0 - lam);
        out[3] = (double)n_ok;
    }
}

// sources += (f - 1) d (alpha* turned into alpha with cos(delta)); the correction is kept in
// tangent units for the residual update
__global__ void k_asi_apply(int32_t n_src, const double* __restrict__ d, const double* __restrict__ est,
                            double* __restrict__ src, double* __restrict__ corr) {
    const double g = est[2] - 1.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += gridDim.x * blockDim.x) {
        double* s = src + 5 * (size_t)i;
        double c[5];
        for (int k = 0; k < 5; k++) {
            const double v = g * d[5 * (size_t)i + k];
            c[k] = isfinite(v) ? v : 0.0;
        }
        s[0] += c[0] / cos(s[1]);
        for (int k = 1; k < 5; k++) s[k] += c[k];
        for (int k = 0; k < 5; k++) corr[5 * (size_t)i + k] = c[k];
    }
}

// host launchers
void launch_asi(int32_t n_src, int32_t stride, const double* hist, double lam_max, unsigned long long* keys,
                double* est, const double* d, double* src, double* corr, cudaStream_t s) {
    // the history holds the last four updates, oldest first: the previous at 10, the latest at 15
    k_asi_lambda<<<1, kAsiThreads, 0, s>>>(n_src, stride, hist + 10, hist + 15, 20, lam_max, keys, est);
    k_asi_apply<<<grid_of(n_src, 256, 152 * 16), 256, 0, s>>>(n_src, d, est, src, corr);
}
void launch_hist_push(int32_t n_src, const double* d, double* hist, cudaStream_t s) {
    k_hist_push<<<grid_of(n_src, 256, 152 * 16), 256, 0, s>>>(n_src, d, hist);
}
void launch_prop_features(int32_t n_src, const double* hist, const int64_t* src_off, const double* src,
                          double sin_obl, double cos_obl, float* X, double* sigma, cudaStream_t s) {
    k_prop_features<<<grid_of(n_src, 256, 152 * 16), 256, 0, s>>>(n_src, hist, src_off, src, sin_obl, cos_obl, X,
                                                                  sigma);
}
void launch_mlp_forward(const void* packed, const float* X, int n, float* Y, cudaStream_t s) {
    k_mlp_fwd_tc<<<grid_of((n + 15) / 16, kFwdWarps, 152 * 8), 32 * kFwdWarps, 0, s>>>(
        (const uint32_t*)packed, X, n, Y);
}
void launch_prop_apply(int32_t n_src, const float* Y, const double* sigma, double* src, double* corr,
                       cudaStream_t s) {
    k_prop_apply<<<grid_of(n_src, 256, 152 * 16), 256, 0, s>>>(n_src, Y, sigma, src, corr);
}
void launch_prop_rec(int32_t n_src, const int64_t* src_off, const double* scratch, ObsRec* rec, const double* corr,
                     cudaStream_t s) {
    k_prop_rec<<<grid_of(n_src, 8, 152 * 16), 256, 0, s>>>(n_src, src_off, scratch, rec, corr);
}

}  // namespace agis

// ---------------------------------------------------------------------------------------
// C ABI of the network kernels (device pointers)
// ---------------------------------------------------------------------------------------
namespace agis {
void set_thread_error(const std::string& msg);
}

extern "C" {

static int mlp_launch_status(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return AGIS_OK;
    agis::set_thread_error(std::string(what) + ": " + cudaGetErrorString(e));
    return AGIS_E_CUDA;
}

int agis_mlp_pack(const float* params, void* packed, void* stream) {
    if (!params || !packed) { agis::set_thread_error("agis_mlp_pack: null pointer"); return AGIS_E_INVALID; }
    agis::k_mlp_pack<<<8, 512, 0, (cudaStream_t)stream>>>(params, (uint32_t*)packed);
    return mlp_launch_status("agis_mlp_pack");
}

int agis_mlp_forward(const void* packed, const float* X, int32_t n, float* Y, void* stream) {
    if (!packed || n < 0 || (n > 0 && (!X || !Y))) {
        agis::set_thread_error("agis_mlp_forward: null pointer or n < 0");
        return AGIS_E_INVALID;
    }
    if (n == 0) return AGIS_OK;
    agis::launch_mlp_forward(packed, X, n, Y, (cudaStream_t)stream);
    return mlp_launch_status("agis_mlp_forward");
}

int agis_mlp_loss_grad(const float* params, const float* X, const float* T, const int32_t* idx, int32_t n,
                       float* grad, float* loss, void* stream) {
    if (!params || !grad || !loss || n < 1 || !X || !T) {
        agis::set_thread_error("agis_mlp_loss_grad: null pointer or n < 1");
        return AGIS_E_INVALID;
    }
    if (cudaFuncSetAttribute(agis::k_mlp_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)agis::kGradSmem) != cudaSuccess)
        return mlp_launch_status("agis_mlp_loss_grad (shared memory)");
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(grad, 0, sizeof(float) * agis::pN, s);
    cudaMemsetAsync(loss, 0, sizeof(float), s);
    const int tiles = (n + 31) / 32;
    agis::k_mlp_loss_grad<<<agis::grid_of(tiles, agis::kGradWarps, 152), 32 * agis::kGradWarps, agis::kGradSmem, s>>>(
        params, X, T, idx, n, grad, loss);
    return mlp_launch_status("agis_mlp_loss_grad");
}

int agis_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t t, float lr, float beta1, float beta2,
                  float eps, void* stream) {
    if (!params || !grad || !m || !v || t < 1) {
        agis::set_thread_error("agis_mlp_adam: null pointer or t < 1");
        return AGIS_E_INVALID;
    }
    agis::k_mlp_adam<<<12, 512, 0, (cudaStream_t)stream>>>(params, grad, m, v, t, lr, beta1, beta2, eps);
    return mlp_launch_status("agis_mlp_adam");
}

int agis_proposal_targets(const double* src_k, const double* src_ref, const double* sigma, int32_t n, float* T,
                          void* stream) {
    if (n < 0 || (n > 0 && (!src_k || !src_ref || !sigma || !T))) {
        agis::set_thread_error("agis_proposal_targets: null pointer or n < 0");
        return AGIS_E_INVALID;
    }
    if (n == 0) return AGIS_OK;
    agis::k_prop_targets<<<agis::grid_of(n, 256, 152 * 16), 256, 0, (cudaStream_t)stream>>>(n, src_k, src_ref, sigma,
                                                                                             T);
    return mlp_launch_status("agis_proposal_targets");
}

int agis_asi_estimate(const double* d_prev, const double* d_cur, int32_t n_src, int32_t stride, double lambda_max,
                      void* scratch, double* est, void* stream) {
    if (!d_prev || !d_cur || !scratch || !est || n_src < 1 || stride < 1 || !(lambda_max >= 0.0 && lambda_max < 1.0)) {
        agis::set_thread_error("agis_asi_estimate: invalid argument");
        return AGIS_E_INVALID;
    }
    agis::k_asi_lambda<<<1, agis::kAsiThreads, 0, (cudaStream_t)stream>>>(
        n_src, stride, d_prev, d_cur, 5, lambda_max, (unsigned long long*)scratch, est);
    return mlp_launch_status("agis_asi_estimate");
}

}  // extern "C"
