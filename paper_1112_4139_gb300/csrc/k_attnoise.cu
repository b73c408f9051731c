// k_attnoise.cu -- excess attitude noise (Sect. 5.2.5, Eqs. excess, W, wl, e09), both forms.
//
// The excess noise of observation l is split into a source part and an attitude part,
// eps_l^2 = eps_i^2 + eps_a^2(t_l), with one attitude function per component (AL, AC in the
// preceding field, AC in the following field) that is constant on time buckets.  After the
// source update every observation gets x_l = R_l^2 - sigma_l^2 - eps_i^2, and each bucket j
// of each component gets
//     eps_a^2(j) = max(0, F_0.68 of the x_l of that bucket and component)          (Eq. e09)
// with F the quantile by linear interpolation between order statistics (0 for an empty
// bucket).  The attitude update then weighs each observation with W_l = w(R_l / sqrt(v)) / v,
// v = sigma_l^2 + eps_a^2(t_l) + eps_i^2 (Eqs. W, wl), and the next source update uses
// sigma~_l^2 = sigma_l^2 + eps_a^2(t_l) (in the observation pass).
//
// Layout: a permutation of the observations sorted once by (component, bucket) makes every
// bucket a contiguous run; x_l is written in that order as an order-preserving 64-bit key.
// The two order statistics around 0.68 (n - 1) of a run are selected exactly by a radix
// select (passes of 8 bits, counts in shared memory), so the estimate does not depend on
// timing or launch shape: one warp per run of up to kWarpRun keys (no block barriers; a pass
// whose chosen digit holds a single key ends the select, about 4 passes instead of 8 on
// continuous data), one block per longer run.
//
// Mixed form: x_l and the attitude weights come from the float-pair residuals (R = hi + lo in
// FP64, as exact as the FP64 form's to about 48 bits); the attitude update reads the pairs
// (W_l, W_l R_l) in FP32 like its other inputs, and the source update reads sigma~_l as the
// FP32 sigma of the observation records (k_an_sigma_mix, after every observation pass).
#include "agis_internal.cuh"

namespace agis {

constexpr int kSelThreads = 256;
constexpr int kSelWarps = 8;      // warps per block of the warp-per-run kernel
constexpr int kWarpRun = 4096;    // longest run of the warp-per-run kernel

// largest t - t0 over the observations, and a flag for any t < t0
__global__ void k_an_range(int64_t n, const int64_t* __restrict__ t, int64_t t0, unsigned long long* __restrict__ mx,
                           int* __restrict__ neg) {
    unsigned long long m = 0;
    int bad = 0;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t[o] - t0;
        if (r < 0)
            bad = 1;
        else if ((unsigned long long)r > m)
            m = (unsigned long long)r;
    }
    for (int s = 16; s > 0; s >>= 1) {
        const unsigned long long mo = __shfl_xor_sync(0xffffffffu, m, s);
        m = mo > m ? mo : m;
        bad |= __shfl_xor_sync(0xffffffffu, bad, s);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(mx, m);
        if (bad) atomicOr(neg, 1);
    }
}

// sort keys of the one-time (component, bucket) order
__global__ void k_an_keys(int64_t n, const int64_t* __restrict__ t, const uint32_t* __restrict__ meta, AttNoise an,
                          int32_t* __restrict__ key, uint32_t* __restrict__ val) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        key[o] = (int32_t)an_index(an, t[o], meta[o]);
        val[o] = (uint32_t)o;
    }
}

// x_l = R_l^2 - sigma_l^2 - eps_i^2 in (component, bucket) order, as keys.  The products and
// differences are rounded one by one (no contraction into a fused multiply-add), in the order
// of the definition.
__global__ void k_an_values(int64_t n, const uint32_t* __restrict__ perm, const ObsRec* __restrict__ rec,
                            const float* __restrict__ sigma, const int32_t* __restrict__ obs_src,
                            const double* __restrict__ eps2_src, uint64_t* __restrict__ xkey) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t o = perm[p];
        const double R = rec[o].R;
        const double s = (double)sigma[o];
        const double x = __dadd_rn(__dadd_rn(__dmul_rn(R, R), -__dmul_rn(s, s)), -eps2_src[obs_src[o]]);
        xkey[p] = dkey(x);
    }
}

// linear interpolation between the order statistics a = x_(k) and b = x_(k+1) at weight
// gamma, from the nearer end, each operation rounded on its own; clamped at 0 (Eq. e09)
__device__ __forceinline__ double quantile_clamped(uint64_t ka, uint64_t kb, double gamma) {
    const double a = dkey_inv(ka), b = dkey_inv(kb);
    const double diff = __dadd_rn(b, -a);
    const double val = gamma >= 0.5 ? __dadd_rn(b, -__dmul_rn(diff, __dadd_rn(1.0, -gamma)))
                                    : __dadd_rn(a, __dmul_rn(diff, gamma));
    return val > 0.0 ? val : 0.0;
}

// eps_a^2 of the runs longer than kWarpRun: one block per run (grid-stride over runs)
__global__ void __launch_bounds__(kSelThreads) k_an_select(int n_run, const int64_t* __restrict__ off,
                                                           const uint64_t* __restrict__ xkey, double q,
                                                           double* __restrict__ eps2) {
    __shared__ unsigned long long hist[256];
    __shared__ int sh_bin;
    __shared__ long long sh_below;
    __shared__ unsigned long long sh_cle, sh_nxt;
    const int lane = threadIdx.x & 31;
    for (int run = blockIdx.x; run < n_run; run += gridDim.x) {
        const int64_t lo = off[run];
        const int64_t n = off[run + 1] - lo;
        if (n <= kWarpRun) continue;   // the warp-per-run kernel's (the same for the whole block)
        const uint64_t* v = xkey + lo;
        // virtual index h = q (n - 1): order statistics k = floor(h) and k + 1, weight h - k
        const double h = q * (double)(n - 1);
        const double fl = floor(h);
        const int64_t k = (int64_t)fl;
        // radix select of the k-th smallest key (0-based), most significant byte first
        uint64_t prefix = 0;
        long long kk = k;
        for (int d = 7; d >= 0; d--) {
            const int shift = 8 * d;
            const uint64_t hmask = d == 7 ? 0ull : (~0ull << (shift + 8));
            for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0ull;
            __syncthreads();
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
                const uint64_t key = v[j];
                if (((key ^ prefix) & hmask) == 0ull) atomicAdd(&hist[(key >> shift) & 255u], 1ull);
            }
            __syncthreads();
            if (threadIdx.x < 32) {
                unsigned long long c[8], sum = 0;
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    c[i] = hist[lane * 8 + i];
                    sum += c[i];
                }
                unsigned long long incl = sum;
                for (int s = 1; s < 32; s <<= 1) {
                    const unsigned long long up = __shfl_up_sync(0xffffffffu, incl, s);
                    if (lane >= s) incl += up;
                }
                const unsigned long long excl = incl - sum;
                if ((unsigned long long)kk >= excl && (unsigned long long)kk < incl) {
                    unsigned long long below = excl;
                    for (int i = 0; i < 8; i++) {
                        if ((unsigned long long)kk < below + c[i]) {
                            sh_bin = lane * 8 + i;
                            sh_below = (long long)below;
                            break;
                        }
                        below += c[i];
                    }
                }
            }
            __syncthreads();
            prefix |= (uint64_t)sh_bin << shift;
            kk -= sh_below;
        }
        // the next order statistic: the same key if more than k + 1 keys are <= it, else the
        // smallest key above it
        if (threadIdx.x == 0) {
            sh_cle = 0ull;
            sh_nxt = ~0ull;
        }
        __syncthreads();
        unsigned long long cle = 0, nxt = ~0ull;
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
            const uint64_t key = v[j];
            if (key <= prefix)
                cle++;
            else if (key < nxt)
                nxt = key;
        }
        for (int s = 16; s > 0; s >>= 1) {
            cle += __shfl_xor_sync(0xffffffffu, cle, s);
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, nxt, s);
            nxt = o < nxt ? o : nxt;
        }
        if (lane == 0) {
            atomicAdd(&sh_cle, cle);
            atomicMin(&sh_nxt, nxt);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint64_t k1 = (k + 1 < n && sh_cle <= (unsigned long long)(k + 1)) ? sh_nxt : prefix;
            eps2[run] = quantile_clamped(prefix, k1, h - fl);
        }
        __syncthreads();
    }
}

// eps_a^2 of the runs of up to kWarpRun keys (empty runs included): one warp per run
__global__ void __launch_bounds__(32 * kSelWarps) k_an_select_warp(int n_run, const int64_t* __restrict__ off,
                                                                   const uint64_t* __restrict__ xkey, double q,
                                                                   double* __restrict__ eps2) {
    __shared__ unsigned int hist_all[kSelWarps][256];
    const int lane = threadIdx.x & 31;
    unsigned int* hist = hist_all[threadIdx.x >> 5];
    const int n_warps = gridDim.x * kSelWarps;
    for (int run = blockIdx.x * kSelWarps + (threadIdx.x >> 5); run < n_run; run += n_warps) {
        const int64_t lo = off[run];
        const int64_t n64 = off[run + 1] - lo;
        if (n64 > kWarpRun) continue;   // the block kernel's
        const int n = (int)n64;
        if (n == 0) {
            if (lane == 0) eps2[run] = 0.0;
            continue;
        }
        const uint64_t* v = xkey + lo;
        const double h = q * (double)(n - 1);
        const double fl = floor(h);
        const int k = (int)fl;
        uint64_t prefix = 0;
        int kk = k;
        for (int d = 7; d >= 0; d--) {
            const int shift = 8 * d;
            const uint64_t hmask = d == 7 ? 0ull : (~0ull << (shift + 8));
            for (int b = lane; b < 256; b += 32) hist[b] = 0u;
            __syncwarp();
            for (int j = lane; j < n; j += 32) {
                const uint64_t key = v[j];
                if (((key ^ prefix) & hmask) == 0ull) atomicAdd(&hist[(key >> shift) & 255u], 1u);
            }
            __syncwarp();
            unsigned int c[8], sum = 0;
#pragma unroll
            for (int i = 0; i < 8; i++) {
                c[i] = hist[lane * 8 + i];
                sum += c[i];
            }
            unsigned int incl = sum;
            for (int s = 1; s < 32; s <<= 1) {
                const unsigned int up = __shfl_up_sync(0xffffffffu, incl, s);
                if (lane >= s) incl += up;
            }
            const unsigned int excl = incl - sum;
            const bool holds = (unsigned int)kk >= excl && (unsigned int)kk < incl;
            int bin = 0, below = 0, cnt = 0;
            if (holds) {
                unsigned int bl = excl;
                for (int i = 0; i < 8; i++) {
                    if ((unsigned int)kk < bl + c[i]) {
                        bin = lane * 8 + i;
                        below = (int)bl;
                        cnt = (int)c[i];
                        break;
                    }
                    bl += c[i];
                }
            }
            const int src = __ffs(__ballot_sync(0xffffffffu, holds)) - 1;
            bin = __shfl_sync(0xffffffffu, bin, src);
            below = __shfl_sync(0xffffffffu, below, src);
            cnt = __shfl_sync(0xffffffffu, cnt, src);
            prefix |= (uint64_t)bin << shift;
            kk -= below;
            __syncwarp();   // the histogram is read before the next pass clears it
            if (cnt == 1 && d > 0) {
                // one key carries this prefix down to digit d: it is the k-th
                uint64_t cand = ~0ull;
                for (int j = lane; j < n; j += 32) {
                    const uint64_t key = v[j];
                    if (((key ^ prefix) >> shift) == 0ull && key < cand) cand = key;
                }
                for (int s = 16; s > 0; s >>= 1) {
                    const uint64_t o = __shfl_xor_sync(0xffffffffu, cand, s);
                    cand = o < cand ? o : cand;
                }
                prefix = cand;
                break;
            }
        }
        // the next order statistic, as in the block kernel
        unsigned int cle = 0;
        uint64_t nxt = ~0ull;
        for (int j = lane; j < n; j += 32) {
            const uint64_t key = v[j];
            if (key <= prefix)
                cle++;
            else if (key < nxt)
                nxt = key;
        }
        for (int s = 16; s > 0; s >>= 1) {
            cle += __shfl_xor_sync(0xffffffffu, cle, s);
            const uint64_t o = __shfl_xor_sync(0xffffffffu, nxt, s);
            nxt = o < nxt ? o : nxt;
        }
        if (lane == 0) {
            const uint64_t k1 = (k + 1 < n && cle <= (unsigned int)(k + 1)) ? nxt : prefix;
            eps2[run] = quantile_clamped(prefix, k1, h - fl);
        }
    }
}

// attitude weights W_l = w(R_l / sqrt(v)) / v, v = (sigma_l^2 + eps_a^2(t_l)) + eps_i^2
__global__ void k_an_weights(int64_t n, AttNoise an, const ObsRec* __restrict__ rec, const float* __restrict__ sigma,
                             const int32_t* __restrict__ obs_src, const double* __restrict__ eps2_src, int weight_fn,
                             double* __restrict__ w_att) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = rec[o].t_ns;
        const uint32_t m = rec[o].meta;
        const double R = rec[o].R;
        const double s = (double)sigma[o];
        const double v = __dadd_rn(__dadd_rn(__dmul_rn(s, s), an.eps2[an_index(an, t, m)]), eps2_src[obs_src[o]]);
        w_att[o] = wfun(R / sqrt(v), weight_fn) / v;
    }
}

static int an_grid(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return b < 1 ? 1 : (int)b;
}

void launch_an_range(int64_t n, const int64_t* t, int64_t t0, unsigned long long* mx, int* neg, cudaStream_t s) {
    k_an_range<<<an_grid(n), 256, 0, s>>>(n, t, t0, mx, neg);
}

void launch_an_keys(int64_t n, const int64_t* t, const uint32_t* meta, const AttNoise& an, int32_t* key, uint32_t* val,
                    cudaStream_t s) {
    k_an_keys<<<an_grid(n), 256, 0, s>>>(n, t, meta, an, key, val);
}

// eps_a^2 from the residuals of the source update just made, then the attitude weights.
// an.eps2 and eps2 are the same array (written here); max_run: the longest run (the block
// kernel runs only when some run is longer than kWarpRun).
// mixed form: x_l from the float-pair residual R = hi + lo
__global__ void k_an_values_mix(int64_t n, const uint32_t* __restrict__ perm, const float2* __restrict__ mr,
                                const float* __restrict__ sigma, const int32_t* __restrict__ obs_src,
                                const double* __restrict__ eps2_src, uint64_t* __restrict__ xkey) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t o = perm[p];
        const float2 r = mr[o];
        const double R = (double)r.x + (double)r.y;
        const double s = (double)sigma[o];
        const double x = __dadd_rn(__dadd_rn(__dmul_rn(R, R), -__dmul_rn(s, s)), -eps2_src[obs_src[o]]);
        xkey[p] = dkey(x);
    }
}

// mixed form: the attitude update's pairs (W_l, W_l R_l), W_l = w(R_l / sqrt(v)) / v
__global__ void k_an_weights_mix(int64_t n, AttNoise an, const int64_t* __restrict__ t_ns,
                                 const uint32_t* __restrict__ meta, const float2* __restrict__ mr,
                                 const float* __restrict__ sigma, const int32_t* __restrict__ obs_src,
                                 const double* __restrict__ eps2_src, int weight_fn, float2* __restrict__ ac_att) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const float2 r = mr[o];
        const double R = (double)r.x + (double)r.y;
        const double s = (double)sigma[o];
        const double v = __dadd_rn(__dadd_rn(__dmul_rn(s, s), an.eps2[an_index(an, t_ns[o], meta[o])]),
                                   eps2_src[obs_src[o]]);
        const double W = wfun(R / sqrt(v), weight_fn) / v;
        ac_att[o] = make_float2((float)W, (float)(W * R));
    }
}

// mixed form: sigma~_l = sqrt(sigma_l^2 + eps_a^2(t_l)) into the observation records (sign:
// + AL, - AC, as the records keep it); eps2 null restores sigma_l
__global__ void k_an_sigma_mix(int64_t n, AttNoise an, const int64_t* __restrict__ t_ns,
                               const uint32_t* __restrict__ meta, const float* __restrict__ sigma,
                               MixS* __restrict__ ms) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t m = meta[o];
        const double s = (double)sigma[o];
        const double v = an.eps2 ? __dadd_rn(__dmul_rn(s, s), an.eps2[an_index(an, t_ns[o], m)]) : s * s;
        const float sg = (float)sqrt(v);
        ms[o].sig = meta_kind(m) ? -sg : sg;
    }
}

void launch_an_estimate(int64_t n, const AttNoise& an, int64_t max_run, double* eps2, const uint32_t* perm,
                        const int64_t* off, const ObsRec* rec, const float* sigma, const int32_t* obs_src,
                        const double* eps2_src, int weight_fn, uint64_t* xkey, double* w_att, cudaStream_t s) {
    if (n == 0 || an.n_b == 0) return;
    k_an_values<<<an_grid(n), 256, 0, s>>>(n, perm, rec, sigma, obs_src, eps2_src, xkey);
    const int n_run = 3 * an.n_b;
    const int wblocks = (n_run + kSelWarps - 1) / kSelWarps;
    k_an_select_warp<<<wblocks < 152 * 16 ? wblocks : 152 * 16, 32 * kSelWarps, 0, s>>>(n_run, off, xkey, 0.68, eps2);
    if (max_run > kWarpRun) {
        const int blocks = n_run < 152 * 8 ? n_run : 152 * 8;
        k_an_select<<<blocks, kSelThreads, 0, s>>>(n_run, off, xkey, 0.68, eps2);
    }
    k_an_weights<<<an_grid(n), 256, 0, s>>>(n, an, rec, sigma, obs_src, eps2_src, weight_fn, w_att);
}


void launch_an_estimate_mix(int64_t n, const AttNoise& an, int64_t max_run, double* eps2, const uint32_t* perm,
                            const int64_t* off, const int64_t* t_ns, const uint32_t* meta, const float2* mr,
                            const float* sigma, const int32_t* obs_src, const double* eps2_src, int weight_fn,
                            uint64_t* xkey, float2* ac_att, cudaStream_t s) {
    if (n == 0 || an.n_b == 0) return;
    k_an_values_mix<<<an_grid(n), 256, 0, s>>>(n, perm, mr, sigma, obs_src, eps2_src, xkey);
    const int n_run = 3 * an.n_b;
    const int wblocks = (n_run + kSelWarps - 1) / kSelWarps;
    k_an_select_warp<<<wblocks < 152 * 16 ? wblocks : 152 * 16, 32 * kSelWarps, 0, s>>>(n_run, off, xkey, 0.68, eps2);
    if (max_run > kWarpRun) {
        const int blocks = n_run < 152 * 8 ? n_run : 152 * 8;
        k_an_select<<<blocks, kSelThreads, 0, s>>>(n_run, off, xkey, 0.68, eps2);
    }
    k_an_weights_mix<<<an_grid(n), 256, 0, s>>>(n, an, t_ns, meta, mr, sigma, obs_src, eps2_src, weight_fn, ac_att);
}

void launch_an_sigma_mix(int64_t n, const AttNoise& an, const int64_t* t_ns, const uint32_t* meta, const float* sigma,
                         MixS* ms, cudaStream_t s) {
    if (n == 0) return;
    k_an_sigma_mix<<<an_grid(n), 256, 0, s>>>(n, an, t_ns, meta, sigma, ms);
}

}  // namespace agis
