// k_attitude.cu -- the A block (Sect. 5.2): per-knot-interval partial normals from the
// time-ordered observations, assembly of the banded normals of each overlapping segment,
// and the segmented robust banded Cholesky (App. C restricted to the envelope).
#include "agis_internal.cuh"

namespace agis {

// linear index of the upper entry (i <= j) of a 16x16 symmetric matrix
__host__ __device__ constexpr int tri16(int i, int j) { return i * 16 - i * (i - 1) / 2 + (j - i); }
// 4x4 symmetric upper storage
__host__ __device__ constexpr int tri4(int i, int j) { return i * 4 - i * (i - 1) / 2 + (j - i); }

constexpr int kStage = 28;  // staged per observation: B[4], M[10], r[4], BB[10]
constexpr int kAccFP64 = 116;  // distinct products: BB[p] M[m] (10 x 10) and B[b] r[c] (4 x 4)

// One warp per knot interval l (left index), iv = l - 3.  For each observation
// dR/da = B (x) g and dD/da = -2 B (x) s (Eqs. dfadq, dDldan), so its contribution to the
// 16x16 block of the interval is W (B B') (x) (g g' + 4 lambda^2 s s') (Eq. normAmod) and
// to the right-hand side -W B (x) (R g [- 2 lambda^2 D s]).  The 136 upper entries of the
// block hold only 100 distinct products (the 10 upper entries of B B' times those of the
// symmetric 4x4 M), so the lanes accumulate those 100 and the 16 right-hand-side products
// (4 per lane) and expand them into the 152 outputs at the end.
__global__ void __launch_bounds__(128) k_att_accum(DevGeo G, double lambda2, int rhs_norm,
                                                   const uint32_t* __restrict__ perm_t,
                                                   const int64_t* __restrict__ ivl_off, int n_iv,
                                                   const ObsRec* __restrict__ rec, const double* __restrict__ att,
                                                   double* __restrict__ blk) {
    __shared__ double stage_all[4][kWarp * kStage];
    __shared__ double red_all[4][kAccFP64];
    __shared__ int16_t src_tab[kBlkVals];  // accumulator of each block output
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    double* stg = stage_all[wib];
    double* red = red_all[wib];
    for (int o = threadIdx.x; o < kBlkVals; o += blockDim.x) {
        int v;
        if (o < 136) {
            int i = 0;
            while (o >= tri16(i, 15) + 1) i++;
            const int jj = i + (o - tri16(i, i));
            const int bi = i >> 2, ci = i & 3, bj = jj >> 2, cj = jj & 3;
            v = tri4(bi, bj) * 10 + (ci <= cj ? tri4(ci, cj) : tri4(cj, ci));
        } else {
            v = 100 + (o - 136);
        }
        src_tab[o] = (int16_t)v;
    }
    __syncthreads();
    // this lane's accumulators s = lane + 32 k (k < 3: BB[p] M[m]; k = 3: lanes 0-3 BB M,
    // lanes 4-19 B[b] r[c] of the right-hand side, lanes 20-31 none): the staged factors
    int fa[4], fb[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int sidx = lane + 32 * k;
        fa[k] = sidx < 100 ? 18 + sidx / 10 : (sidx < kAccFP64 ? (sidx - 100) >> 2 : 0);
        fb[k] = sidx < 100 ? 4 + sidx % 10 : 14 + ((sidx - 100) & 3);
    }
    const bool k3 = lane < 20;              // accumulator 3 in use
    const bool k3_rhs = lane >= 4 && k3;    // ... and it is a right-hand-side product
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int iv = blockIdx.x * (blockDim.x >> 5) + wib; iv < n_iv; iv += nwarps) {
        const int l = iv + 3;
        double a[16];
#pragma unroll
        for (int k = 0; k < 16; k++) a[k] = att[4 * (int64_t)(l - 3) + k];
        double acc[4] = {0, 0, 0, 0};
        const int64_t beg = ivl_off[iv], end = ivl_off[iv + 1];
        for (int64_t base = beg; base < end; base += kWarp) {
            const int64_t j = base + lane;
            double* st = stg + lane * kStage;
            if (j < end) {
                const ObsRec r = rec[perm_t[j]];
                double B[4];
                bspline4(G, r.t_ns, l, B);
                double s[4];
#pragma unroll
                for (int c = 0; c < 4; c++) s[c] = B[0] * a[c] + B[1] * a[4 + c] + B[2] * a[8 + c] + B[3] * a[12 + c];
                const double W = r.W;
                const double l4 = 4.0 * lambda2;
#pragma unroll
                for (int c = 0; c < 4; c++) {
#pragma unroll
                    for (int e = c; e < 4; e++) st[4 + tri4(c, e)] = W * (r.g[c] * r.g[e] + l4 * s[c] * s[e]);
                }
                double D = 1.0 - (s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3]);
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    double v = r.R * r.g[c];
                    if (rhs_norm) v -= 2.0 * lambda2 * D * s[c];
                    st[14 + c] = W * v;
                    st[c] = B[c];
                }
#pragma unroll
                for (int c = 0; c < 4; c++) {
#pragma unroll
                    for (int e = c; e < 4; e++) st[18 + tri4(c, e)] = B[c] * B[e];
                }
            } else {
#pragma unroll
                for (int c = 0; c < kStage; c++) st[c] = 0.0;
            }
            __syncwarp();
            const int cnt = (int)((end - base) < kWarp ? (end - base) : kWarp);
            for (int q = 0; q < cnt; q++) {
                const double* sq = stg + q * kStage;
#pragma unroll
                for (int k = 0; k < 3; k++) acc[k] += sq[fa[k]] * sq[fb[k]];
                if (k3) acc[3] += sq[fa[3]] * sq[fb[3]];
            }
            __syncwarp();
        }
#pragma unroll
        for (int k = 0; k < 3; k++) red[lane + 32 * k] = acc[k];
        if (k3) red[lane + 96] = k3_rhs ? -acc[3] : acc[3];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 5; k++) {
            const int o = lane + 32 * k;
            if (o < kBlkVals) blk[(int64_t)iv * kBlkVals + o] = red[src_tab[o]];
        }
        __syncwarp();
    }
}

// Band of every segment in column layout: bandc[(row0 + c)*16 + k] = N[c-k][c] (k = 0..15)
// and rhs[row0 + c], summed over the knot intervals of the segment only.
__global__ void k_att_assemble(int n_seg, const int64_t* __restrict__ seg_row, const int32_t* __restrict__ seg_l,
                               const int32_t* __restrict__ seg_n, const double* __restrict__ blk,
                               double* __restrict__ bandc, double* __restrict__ rhs) {
    const int64_t total = seg_row[n_seg] * 16;
    const int64_t avg_rows = (seg_row[n_seg] + n_seg - 1) / n_seg > 0 ? (seg_row[n_seg] + n_seg - 1) / n_seg : 1;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t >> 4;
        const int k = (int)(t & 15);
        // the segment of this row: the segments are of nearly equal length, so a guess from
        // the average length and a step or two of correction replace a binary search
        int sg = (int)(row / avg_rows);
        if (sg > n_seg - 1) sg = n_seg - 1;
        while (sg > 0 && seg_row[sg] > row) sg--;
        while (sg < n_seg - 1 && seg_row[sg + 1] <= row) sg++;
        const int c = (int)(row - seg_row[sg]);
        const int l_lo = seg_l[2 * sg], l_hi = seg_l[2 * sg + 1];
        const int n_lo = seg_n[2 * sg];
        const int v = c - k;
        double val = 0.0;
        if (v >= 0) {
            const int nc = n_lo + (c >> 2), cc = c & 3;
            const int nv = n_lo + (v >> 2), cv = v & 3;
            int lb = nc > nv ? nc : nv;
            int le = (nc < nv ? nc : nv) + 3;
            if (lb < l_lo) lb = l_lo;
            if (le > l_hi) le = l_hi;
            for (int l = lb; l <= le; l++) {
                const int i = 4 * (nv - l + 3) + cv, j = 4 * (nc - l + 3) + cc;
                val += blk[(int64_t)(l - 3) * kBlkVals + tri16(i, j)];
            }
        }
        bandc[t] = val;
        if (k == 0) {
            const int nc = n_lo + (c >> 2), cc = c & 3;
            double r = 0.0;
            int lb = nc < l_lo ? l_lo : nc;
            int le = nc + 3 > l_hi ? l_hi : nc + 3;
            for (int l = lb; l <= le; l++) r += blk[(int64_t)(l - 3) * kBlkVals + 136 + 4 * (nc - l + 3) + cc];
            rhs[row] = r;
        }
    }
}

// Two segments per warp, one per 16-lane half: right-looking robust Cholesky (Algorithm C.1
// on the envelope) with forward substitution (C.2) fused, then back substitution (C.3).
// Lane b of a half holds column b of the sliding window W[a][b] = N[r+a][r+b] (a <= b); the
// window moves one row per step by a shuffle within the half, and the column entering at
// lane 15 comes from a shared-memory double buffer filled one block of 16 columns ahead.
// The pivot's reciprocal is formed once per row and stored in place of U_rr for C.3.
constexpr int kSolveSegWarps = 2;
__global__ void __launch_bounds__(32 * kSolveSegWarps) k_att_solve(int n_seg, const int64_t* __restrict__ seg_row,
                                                  const double* __restrict__ bandc, const double* __restrict__ rhs,
                                                  double* __restrict__ urow, double* __restrict__ yv,
                                                  double* __restrict__ x, double tol, int* __restrict__ seg_rd) {
    __shared__ double colbuf_all[kSolveSegWarps][2][2][16][17];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int half = lane >> 4;
    const int b = lane & 15;
    double (*colbuf)[16][17] = colbuf_all[wib][half];
    const int sg = (blockIdx.x * kSolveSegWarps + wib) * 2 + half;
    const bool seg_ok = sg < n_seg;
    const int64_t base = seg_ok ? seg_row[sg] : 0;
    const int64_t n = seg_ok ? seg_row[sg + 1] - base : 0;
    const int64_t n_other = __shfl_xor_sync(0xffffffffu, n, 16);
    const int64_t n_max = n > n_other ? n : n_other;
    if (n_max == 0) return;
    const unsigned FULL = 0xffffffffu;
    double pre[17];
    auto load_block = [&](int64_t kb) {
        const int64_t c = 16 * kb + b;
        const bool ok = c < n;
#pragma unroll
        for (int a = 0; a < 16; a++) pre[a] = ok ? bandc[(base + c) * 16 + a] : 0.0;
        pre[16] = ok ? rhs[base + c] : 0.0;
    };
    auto store_block = [&](int64_t kb) {
#pragma unroll
        for (int a = 0; a < 17; a++) colbuf[kb & 1][b][a] = pre[a];
        __syncwarp();
    };
    double w[16];
#pragma unroll
    for (int a = 0; a < 16; a++) w[a] = (a <= b && b < n) ? bandc[(base + b) * 16 + (b - a)] : 0.0;
    double dg = b < n ? bandc[(base + b) * 16] : 0.0;
    double z = b < n ? rhs[base + b] : 0.0;
    load_block(1);
    store_block(1);
    load_block(2);
    int rd = 0;
    for (int64_t r = 0; r < n_max; r++) {
        if (r >= 16 && (r & 15) == 0) {
            const int64_t m = r >> 4;
            store_block(m + 1);
            load_block(m + 2);
        }
        const bool live = r < n;
        const double piv = __shfl_sync(FULL, w[0], 0, 16);
        const double dg0 = __shfl_sync(FULL, dg, 0, 16);
        const double urr = piv > tol * dg0 ? sqrt(piv) : 0.0;
        const double inv = urr > 0.0 ? 1.0 / urr : 0.0;
        if (live) rd += urr == 0.0;
        double myU = (b == 0) ? urr : w[0] * inv;
        if (r + b >= n && b > 0) myU = 0.0;
        const double zr = __shfl_sync(FULL, z, 0, 16);
        const double yr = zr * inv;
        if (live) {
            urow[(base + r) * 16 + b] = (b == 0) ? inv : myU;
            if (b == 0) yv[base + r] = yr;
        }
        if (b >= 1) z -= myU * yr;
#pragma unroll
        for (int a = 1; a < 16; a++) {
            const double ua = __shfl_sync(FULL, myU, a, 16);
            if (a <= b) w[a] -= ua * myU;
        }
#pragma unroll
        for (int a = 0; a < 15; a++) w[a] = __shfl_down_sync(FULL, w[a + 1], 1, 16);
        w[15] = 0.0;
        z = __shfl_down_sync(FULL, z, 1, 16);
        dg = __shfl_down_sync(FULL, dg, 1, 16);
        if (b == 15) {
            const int64_t c = r + 16;
            if (c < n) {
                const double* col = colbuf[(c >> 4) & 1][c & 15];
#pragma unroll
                for (int a = 0; a < 16; a++) w[a] = col[15 - a];
                dg = col[0];
                z = col[16];
            } else {
#pragma unroll
                for (int a = 0; a < 16; a++) w[a] = 0.0;
                dg = 0.0;
                z = 0.0;
            }
        }
    }
    // back substitution: lane b of the half holds x_{r+b} (b >= 1); slot 0 of a U row holds 1/U_rr
    double xw = 0.0;
    for (int64_t k = 0; k < n_max; k++) {
        const int64_t r = n - 1 - k;
        const bool live = r >= 0;
        const double ur = live ? urow[(base + r) * 16 + b] : 0.0;
        double part = (b >= 1) ? ur * xw : 0.0;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o, 16);
        const double inv = __shfl_sync(FULL, ur, 0, 16);
        const double xr = live ? (yv[base + r] - part) * inv : 0.0;
        if (live && b == 0) x[base + r] = xr;
        xw = __shfl_up_sync(FULL, xw, 1, 16);
        if (b == 1) xw = xr;
    }
    if (b == 0 && seg_ok) seg_rd[sg] = rd;
}

// a_n += x for the coefficients each segment owns (n in [u_lo, u_hi]); one thread per
// coefficient.  The mixed form also accumulates the update in d_att (FP32).
__global__ void k_att_apply(int n_coef, int n_seg, const int32_t* __restrict__ seg_u, const int32_t* __restrict__ seg_n,
                            const int64_t* __restrict__ seg_row, const double* __restrict__ x,
                            double* __restrict__ att, float* __restrict__ d_att) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < n_coef; n += gridDim.x * blockDim.x) {
        int lo = 0, hi = n_seg - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (seg_u[2 * mid] <= n) lo = mid; else hi = mid - 1;
        }
        const int sg = lo;
        const int64_t r0 = seg_row[sg] + 4 * (int64_t)(n - seg_n[2 * sg]);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            att[4 * (int64_t)n + c] += x[r0 + c];
            if (d_att) d_att[4 * (int64_t)n + c] += (float)x[r0 + c];
        }
    }
}

void launch_att_accum(const DevGeo& G, double lambda2, int rhs_norm, const uint32_t* perm_t, const int64_t* ivl_off,
                      int n_iv, const ObsRec* rec, const double* att, double* blk, const Shapes& sh, cudaStream_t s) {
    int warps = n_iv;
    int blocks = (warps + 3) / 4;
    const int bps = sh.att_bps > 0 ? sh.att_bps : 32;
    if (blocks > 152 * bps) blocks = 152 * bps;
    if (blocks < 1) blocks = 1;
    k_att_accum<<<blocks, 128, 0, s>>>(G, lambda2, rhs_norm, perm_t, ivl_off, n_iv, rec, att, blk);
}

// d_att (mixed form only, else null) accumulates the applied update in FP32
void launch_att_solve(int n_seg, int n_coef, int64_t n_rows, const int64_t* seg_row, const int32_t* seg_l,
                      const int32_t* seg_n, const int32_t* seg_u, const double* blk, double* bandc, double* rhs,
                      double* urow, double* yv, double* x, double tol, int* seg_rd, double* att, float* d_att,
                      cudaStream_t s) {
    int64_t total = n_rows * 16;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    k_att_assemble<<<blocks, 256, 0, s>>>(n_seg, seg_row, seg_l, seg_n, blk, bandc, rhs);
    const int seg_warps = (n_seg + 1) / 2;
    k_att_solve<<<(seg_warps + kSolveSegWarps - 1) / kSolveSegWarps, 32 * kSolveSegWarps, 0, s>>>(
        n_seg, seg_row, bandc, rhs, urow, yv, x, tol, seg_rd);
    k_att_apply<<<(n_coef + 255) / 256, 256, 0, s>>>(n_coef, n_seg, seg_u, seg_n, seg_row, x, att, d_att);
}

}  // namespace agis
