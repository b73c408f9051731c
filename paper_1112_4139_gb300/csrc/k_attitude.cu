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
// (4 per lane) and expand them into the 152 outputs at the end.  W is the weight of the
// source update, or w_att[o] (Eqs. W, wl) when the excess attitude noise is estimated.
__global__ void __launch_bounds__(128) k_att_accum(DevGeo G, double lambda2, int rhs_norm,
                                                   const uint32_t* __restrict__ perm_t,
                                                   const int64_t* __restrict__ ivl_off, int n_iv,
                                                   const ObsRec* __restrict__ rec,
                                                   const double* __restrict__ w_att,
                                                   const double* __restrict__ att, double* __restrict__ blk) {
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
                const uint32_t o = perm_t[j];
                const ObsRec r = rec[o];
                double B[4];
                bspline4(G, r.t_ns, l, B);
                double s[4];
#pragma unroll
                for (int c = 0; c < 4; c++) s[c] = B[0] * a[c] + B[1] * a[4 + c] + B[2] * a[8 + c] + B[3] * a[12 + c];
                const double W = w_att ? w_att[o] : r.W;
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
// and rhs[row0 + c], summed over the knot intervals of the segment only.  One warp per run of
// kAsmKnots consecutive knots of a segment: the interval blocks those knots touch (a
// contiguous range of blk) are copied into shared memory once, coalesced, and every band
// entry of the run is summed from there over its intervals in increasing order.
constexpr int kAsmKnots = 8;
constexpr int kAsmWarps = 4;
__global__ void __launch_bounds__(32 * kAsmWarps) k_att_assemble(int n_seg, int runs_per_seg,
                                                                 const int64_t* __restrict__ seg_row,
                                                                 const int32_t* __restrict__ seg_l,
                                                                 const int32_t* __restrict__ seg_n,
                                                                 const double* __restrict__ blk,
                                                                 double* __restrict__ bandc, double* __restrict__ rhs) {
    __shared__ double stage_all[kAsmWarps][(kAsmKnots + 3) * kBlkVals];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    double* st = stage_all[wib];
    const int64_t n_units = (int64_t)n_seg * runs_per_seg;
    for (int64_t u = (int64_t)blockIdx.x * kAsmWarps + wib; u < n_units; u += (int64_t)gridDim.x * kAsmWarps) {
        const int sg = (int)(u / runs_per_seg);
        const int run = (int)(u % runs_per_seg);
        const int64_t row0 = seg_row[sg];
        const int n_knots = (int)((seg_row[sg + 1] - row0) / 4);
        const int k0 = run * kAsmKnots;
        if (k0 >= n_knots) continue;
        const int k1 = min(k0 + kAsmKnots, n_knots);
        const int l_lo = seg_l[2 * sg], l_hi = seg_l[2 * sg + 1];
        const int n_lo = seg_n[2 * sg];
        // intervals touched by the knots n_lo + k0 .. n_lo + k1 - 1 (l = n .. n + 3), within the segment
        const int lmin = max(n_lo + k0, l_lo), lmax = min(n_lo + k1 - 1 + 3, l_hi);
        const int nb = lmax - lmin + 1;
        __syncwarp();
        if (nb > 0) {
            const double* src = blk + (int64_t)(lmin - 3) * kBlkVals;
            for (int e = lane; e < nb * kBlkVals; e += kWarp) st[e] = src[e];
        }
        __syncwarp();
        const int n_ent = (k1 - k0) * 4 * 16;
        for (int e = lane; e < n_ent; e += kWarp) {
            const int c = 4 * k0 + (e >> 4);
            const int k = e & 15;
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
                    val += st[(l - lmin) * kBlkVals + tri16(i, j)];
                }
            }
            bandc[(row0 + c) * 16 + k] = val;
        }
        for (int c = 4 * k0 + lane; c < 4 * k1; c += kWarp) {
            const int nc = n_lo + (c >> 2), cc = c & 3;
            double r = 0.0;
            int lb = nc < l_lo ? l_lo : nc;
            int le = nc + 3 > l_hi ? l_hi : nc + 3;
            for (int l = lb; l <= le; l++) r += st[(l - lmin) * kBlkVals + 136 + 4 * (nc - l + 3) + cc];
            rhs[row0 + c] = r;
        }
    }
}

// Robust factorisation of each segment's band (Algorithm C.1 on the envelope, in the
// square-root-free form N = V' D V with V unit upper triangular: U = sqrt(D) V, the same pivot
// test on D and the same zeroed rows for a failing pivot) with the forward substitution (C.2)
// fused, then the back substitution (C.3).  Without the square root the per-row chain that
// bounds the recurrence (pivot, reciprocal, V_{r,r+1}, the next pivot's update) is about a
// third as long.  One segment per group of 8 lanes, four per warp.  The 16x16 window W[a][b] = N'[r+a][r+b] (a <= b) of the
// partly reduced matrix lives in shared memory, addressed by absolute row and column modulo
// 16, so that moving the window by one row moves no data.  Per row the 120 window entries
// below the pivot row are updated 15 per lane (every lane the same count, so one FP64
// instruction of the warp does useful work in all its lanes), and the column that enters
// the window comes from a ring filled by cp.async kColAhead rows ahead, each lane copying
// and later consuming the same two entries.  Every entry receives the same FMAs in the
// same order whatever the lane mapping, and the back substitution sums its 15 products in a
// fixed tree.  Row r of urow holds 1/D_r and V_{r, r+1..r+15}; yv holds w_r / D_r.
constexpr int kSegLanes = 8;
constexpr int kSegsPerWarp = kWarp / kSegLanes;
constexpr int kSolveSegWarps = 2;
constexpr int kColAhead = 8;
struct __align__(16) SegWin {
    double Wf[256];              // W[row mod 16][col mod 16] at row * 16 + (col + row) mod 16 (a
                                 // diagonal skew: a column's entries fall in distinct banks)
    double z[16];                // partly reduced right-hand side per row slot
    double dg[16];               // original diagonal per row slot (the pivot test of C.1)
    double U[16];                // the current row of V: U[b] = V_{r, r+b} (b >= 1)
    double xs[16];               // back substitution: x of the rows r+1 .. r+15 by slot
    double ring[kColAhead][18];  // incoming columns: 16 band values, rhs, pad
    double pad[8];               // 3776 B: consecutive segments start 64 B apart modulo 128 B,
                                 // so the two segments of a half warp use disjoint banks
};
static_assert(sizeof(SegWin) % 128 == 64, "segment windows must alternate between bank halves");

__device__ __forceinline__ void cp_async16_att(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8_att(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_att() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_att() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ double& win(SegWin& sm, int row, int col) {
    return sm.Wf[row * 16 + ((col + row) & 15)];
}

__global__ void __launch_bounds__(32 * kSolveSegWarps) k_att_solve(int n_seg, const int64_t* __restrict__ seg_row,
                                                  const double* __restrict__ bandc, const double* __restrict__ rhs,
                                                  double* __restrict__ urow, double* __restrict__ yv,
                                                  double* __restrict__ x, double tol, int* __restrict__ seg_rd) {
    __shared__ SegWin win_all[kSolveSegWarps][kSegsPerWarp];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int grp = lane / kSegLanes;
    const int sub = lane % kSegLanes;
    const unsigned gmask = ((1u << kSegLanes) - 1u) << (grp * kSegLanes);
    SegWin& sm = win_all[wib][grp];
    const int sg = (blockIdx.x * kSolveSegWarps + wib) * kSegsPerWarp + grp;
    const bool seg_ok = sg < n_seg;
    const int64_t base = seg_ok ? seg_row[sg] : 0;
    const int64_t n = seg_ok ? seg_row[sg + 1] - base : 0;
    int64_t n_max = n;
#pragma unroll
    for (int o = kSegLanes; o < kWarp; o <<= 1) {
        const int64_t v = __shfl_xor_sync(0xffffffffu, n_max, o);
        n_max = v > n_max ? v : n_max;
    }
    if (n_max == 0) return;
    // this lane's 15 window entries per row, (a, b) with 1 <= a <= b <= 15 in row-major
    // order: pair p = 8 t + sub (the a = 1 row, which the next pivot needs, comes first)
    int pa[15], pb[15];
#pragma unroll
    for (int t = 0; t < 15; t++) {
        int p = kSegLanes * t + sub, a = 1;
        while (p >= 16 - a) { p -= 16 - a; a++; }
        pa[t] = a;
        pb[t] = a + p;
    }
    // initial window: rows and columns 0..15 (lane sub loads columns 2 sub and 2 sub + 1)
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int b = 2 * sub + h;
        for (int a = 0; a < 16; a++)
            win(sm, a, b) = (a <= b && b < n) ? bandc[(base + b) * 16 + (b - a)] : 0.0;
        sm.dg[b] = b < n ? bandc[(base + b) * 16] : 0.0;
        sm.z[b] = b < n ? rhs[base + b] : 0.0;
    }
    // the columns 16 .. 16 + kColAhead - 1 into the ring (lane sub: band entries 2 sub, 2 sub + 1;
    // lane 0 also the right-hand side)
#pragma unroll
    for (int q = 0; q < kColAhead; q++) {
        const int64_t c = 16 + q;
        if (c < n) {
            cp_async16_att(&sm.ring[q][2 * sub], bandc + (base + c) * 16 + 2 * sub);
            if (sub == 0) cp_async8_att(&sm.ring[q][16], rhs + base + c);
        }
        cp_async_commit_att();
    }
    __syncwarp();
    int rd = 0;
    for (int64_t r = 0; r < n_max; r++) {
        const bool live = r < n;
        const int s0 = (int)(r & 15);
        const double piv = win(sm, s0, s0);
        const double dg0 = sm.dg[s0];
        // the pivot test of Algorithm C.1; a failing pivot zeroes the row (rank defect)
        const bool pos = piv > tol * dg0;
        const double invd = (pos && piv > 0.0) ? rcp_pos(piv) : 0.0;
        if (live) rd += !pos;
        const double wr = sm.z[s0];
        const double yr = wr * invd;
        // V_{r, r+b} = W[0][b] / D_r and the forward substitution z_b -= V_b w_r, b = sub + 1, sub + 9
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int b = sub + 1 + kSegLanes * h;
            if (b <= 15) {
                const int sb = (int)((r + b) & 15);
                double v = win(sm, s0, sb) * invd;
                if (r + b >= n) v = 0.0;
                sm.U[b] = v;
                sm.z[sb] -= v * wr;
            }
        }
        __syncwarp(gmask);
        if (live) {
            const double v0 = sub == 0 ? invd : sm.U[2 * sub];
            *reinterpret_cast<double2*>(urow + (base + r) * 16 + 2 * sub) = make_double2(v0, sm.U[2 * sub + 1]);
            if (sub == 0) yv[base + r] = yr;
        }
        // the window below the pivot row: W[a][b] -= V_a W[0][b] (= W[0][a] W[0][b] / D_r);
        // row r's slot is not written in this step.  All 45 operands are loaded before the
        // first product and the 15 results stored after the last, so that the loads of one
        // entry do not wait for the store of another.
        {
            int adr[15];
            double wv[15], uv[15], pv[15];
#pragma unroll
            for (int t = 0; t < 15; t++) {
                const int ra = (int)((r + pa[t]) & 15), sb = (int)((r + pb[t]) & 15);
                adr[t] = ra * 16 + ((sb + ra) & 15);
                wv[t] = sm.Wf[adr[t]];
                pv[t] = sm.Wf[s0 * 16 + ((sb + s0) & 15)];
                uv[t] = sm.U[pa[t]];
            }
#pragma unroll
            for (int t = 0; t < 15; t++) wv[t] -= uv[t] * pv[t];
#pragma unroll
            for (int t = 0; t < 15; t++) sm.Wf[adr[t]] = wv[t];
        }
        // the column r + 16 enters in the slot of column r (row r's entries are no longer read)
        cp_async_wait_att<kColAhead - 1>();
        const int64_t c = r + 16;
        const int q = (int)(r % kColAhead);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int k = 2 * sub + h;   // band entry N[c - k][c]: window row a = 15 - k
            const int a = 15 - k;
            win(sm, (int)((r + 1 + a) & 15), s0) = c < n ? sm.ring[q][k] : 0.0;
        }
        if (sub == 0) {
            sm.dg[s0] = c < n ? sm.ring[q][0] : 0.0;
            sm.z[s0] = c < n ? sm.ring[q][16] : 0.0;
        }
        __syncwarp(gmask);
        // refill the ring slot (read above by this lane only) with the column kColAhead on
        const int64_t cn = c + kColAhead;
        if (cn < n) {
            cp_async16_att(&sm.ring[q][2 * sub], bandc + (base + cn) * 16 + 2 * sub);
            if (sub == 0) cp_async8_att(&sm.ring[q][16], rhs + base + cn);
        }
        cp_async_commit_att();
    }
    cp_async_wait_att<0>();
    // back substitution: x_r = y_r - sum_k V_{r,r+k} x_{r+k}, k = 1..15, y_r = w_r / D_r; lane
    // sub forms the products k = sub and sub + 8 and the group adds them in a fixed tree
    for (int k = 0; k < 16; k++)
        if (sub == 0) sm.xs[k] = 0.0;
    __syncwarp();
    // the row's V entries and y are loaded one row ahead (they do not depend on the x chain)
    double u_lo = 0.0, u_hi = 0.0, y_r = 0.0;
    if (n - 1 >= 0) {
        const double* ur = urow + (base + n - 1) * 16;
        u_lo = ur[sub];
        u_hi = ur[sub + 8];
        y_r = yv[base + n - 1];
    }
    for (int64_t kk = 0; kk < n_max; kk++) {
        const int64_t r = n - 1 - kk;
        const bool live = r >= 0;
        const double c_lo = u_lo, c_hi = u_hi, c_y = y_r;
        if (r - 1 >= 0) {
            const double* un = urow + (base + r - 1) * 16;
            u_lo = un[sub];
            u_hi = un[sub + 8];
            y_r = yv[base + r - 1];
        }
        const double p_lo = (live && sub >= 1) ? c_lo * sm.xs[(r + sub) & 15] : 0.0;
        const double p_hi = live ? c_hi * sm.xs[(r + sub + 8) & 15] : 0.0;
        double part = p_lo + p_hi;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o, kSegLanes);
        const double xr = live ? c_y - part : 0.0;
        __syncwarp(gmask);
        if (live && sub == 0) {
            x[base + r] = xr;
            sm.xs[r & 15] = xr;
        }
        __syncwarp(gmask);
    }
    if (sub == 0 && seg_ok) seg_rd[sg] = rd;
}

// a_n += x for the coefficients each segment owns (n in [u_lo, u_hi]); one thread per
// coefficient.  The mixed form also accumulates the update in d_att (FP32); dx, if given,
// receives the update itself (FP64).
__global__ void k_att_apply(int n_coef, int n_seg, const int32_t* __restrict__ seg_u, const int32_t* __restrict__ seg_n,
                            const int64_t* __restrict__ seg_row, const double* __restrict__ x,
                            double* __restrict__ att, float* __restrict__ d_att, double* __restrict__ dx) {
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
            if (dx) dx[4 * (int64_t)n + c] = x[r0 + c];
        }
    }
}

void launch_att_accum(const DevGeo& G, double lambda2, int rhs_norm, const uint32_t* perm_t, const int64_t* ivl_off,
                      int n_iv, const ObsRec* rec, const double* w_att, const double* att, double* blk,
                      const Shapes& sh, cudaStream_t s) {
    int warps = n_iv;
    int blocks = (warps + 3) / 4;
    const int bps = sh.att_bps > 0 ? sh.att_bps : 32;
    if (blocks > 152 * bps) blocks = 152 * bps;
    if (blocks < 1) blocks = 1;
    k_att_accum<<<blocks, 128, 0, s>>>(G, lambda2, rhs_norm, perm_t, ivl_off, n_iv, rec, w_att, att, blk);
}

// d_att (mixed form only, else null) accumulates the applied update in FP32
void launch_att_solve(int n_seg, int max_seg_knots, int n_coef, int64_t n_rows, const int64_t* seg_row, const int32_t* seg_l,
                      const int32_t* seg_n, const int32_t* seg_u, const double* blk, double* bandc, double* rhs,
                      double* urow, double* yv, double* x, double tol, int* seg_rd, double* att, float* d_att,
                      double* dx, cudaStream_t s) {
    // knot runs per segment, enough for the largest segment
    const int runs_per_seg = (max_seg_knots + kAsmKnots - 1) / kAsmKnots;
    int64_t units = (int64_t)n_seg * runs_per_seg;
    int blocks = (int)((units + kAsmWarps - 1) / kAsmWarps);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_att_assemble<<<blocks, 32 * kAsmWarps, 0, s>>>(n_seg, runs_per_seg, seg_row, seg_l, seg_n, blk, bandc, rhs);
    const int seg_warps = (n_seg + kSegsPerWarp - 1) / kSegsPerWarp;
    k_att_solve<<<(seg_warps + kSolveSegWarps - 1) / kSolveSegWarps, 32 * kSolveSegWarps, 0, s>>>(
        n_seg, seg_row, bandc, rhs, urow, yv, x, tol, seg_rd);
    k_att_apply<<<(n_coef + 255) / 256, 256, 0, s>>>(n_coef, n_seg, seg_u, seg_n, seg_row, x, att, d_att, dx);
}

// Block Gauss-Seidel (Sect. 4.6, Eq. precond): before the C block the hand-over residuals
// take the attitude update to first order, R += sum_j B_j g . dx[l-3+j] (dR/da_n = g B_n,
// Eq. dfadq); one thread per observation, FP64.
__global__ void k_rec_att_correct(DevGeo G, int64_t n_obs, ObsRec* __restrict__ rec, const double* __restrict__ dx) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_obs; o += (int64_t)gridDim.x * blockDim.x) {
        ObsRec& r = rec[o];
        const int l = left_index(G, r.t_ns);
        double B[4];
        bspline4(G, r.t_ns, l, B);
        const double* d = dx + 4 * (int64_t)(l - 3);
        double corr = 0.0;
#pragma unroll
        for (int j = 0; j < 4; j++)
            corr += B[j] * (r.g[0] * d[4 * j] + r.g[1] * d[4 * j + 1] + r.g[2] * d[4 * j + 2] + r.g[3] * d[4 * j + 3]);
        r.R += corr;
    }
}
void launch_rec_att_correct(const DevGeo& G, int64_t n_obs, ObsRec* rec, const double* dx, cudaStream_t s) {
    int64_t b = (n_obs + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    k_rec_att_correct<<<(int)b, 256, 0, s>>>(G, n_obs, rec, dx);
}

}  // namespace agis
