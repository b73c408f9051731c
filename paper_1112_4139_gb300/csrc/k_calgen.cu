// k_calgen.cu -- the C block of the full geometric calibration (Sect. 3.4, Eq. etazeta;
// Sect. 5.3, Eqs. normC, calCon, cc1-cc3).
//
// Normals.  An AL observation of field f, CCD n, gate g in short interval j (long interval k)
// touches the three large-scale terms Deta_{r f n g j} (factors L*_r(x), r = 0..2) and one
// small-scale term deta_{n g k b} (factor 1); an AC observation the three Dzeta_{r f n g k}.
// Within an AL group (n, g, k) the normals are
//     [ D_1          B_1 ]        D_j  6x6 (two 3x3 blocks, one per field)
//     [      ...     ... ]        B_j  6 x n_bin
//     [ B_1' ...     E   ]        E    diagonal (each observation has one small-scale term)
// and b = -sum W Phi R.  The update is the least-squares solution under Eq. cc2, which acts on
// the small-scale terms alone: each D_j is eliminated by Algorithm C.1 (D_j = U_j' U_j,
// V_j = U_j'^-1 B_j, w_j = U_j'^-1 b_j), leaving S = E - sum_j V_j' V_j and
// r = b_small - sum_j V_j' w_j; cc2 is imposed on (S, r) by the null-space method (Householder
// reflections of the cc2 columns over the observed bins: Z = the columns beyond the rank), the
// reduced system Z'SZ y = Z'r is solved by Algorithms C.1-C.3, v = Z y, and the large-scale
// terms follow from U_j u_j = w_j - V_j v.  AC groups: 6x6 (two 3x3 blocks) by C.1-C.3.
// Parameters without observations are held (zero update) and counted as rank defects.
// Then Eqs. cc1 (per j: the 124 r = 0 AL terms of gate 0) and cc3 (per k and f: the 62 r = 0
// AC terms of gate 0) by the projection of Eq. calCon (disjoint supports: subtract the mean).
//
// Every sum runs in a fixed order (sorted observations, segmented warp scans, fixed tiles), so
// the update is the same bit for bit from run to run.
#include "agis_internal.cuh"

namespace agis {


constexpr int kTile = 16;

// upper 3x3 index
__device__ __forceinline__ int up3(int a, int b) { return a * 3 - a * (a - 1) / 2 + (b - a); }

// Algorithm C.1 on a 3x3 block (upper entries N[6]); zero rows for failing pivots
__device__ __forceinline__ int chol3(const double* N, double* U, double tol) {
    int d = 0;
    for (int j = 0; j < 3; j++) {
        for (int i = 0; i <= j; i++) {
            double s = 0.0;
            for (int k = 0; k < i; k++) s += U[up3(k, i)] * U[up3(k, j)];
            if (i < j) {
                const double uii = U[up3(i, i)];
                U[up3(i, j)] = uii > 0.0 ? (N[up3(i, j)] - s) / uii : 0.0;
            } else {
                const double x = N[up3(j, j)] - s;
                if (x > tol * N[up3(j, j)]) {
                    U[up3(j, j)] = sqrt(x);
                } else {
                    U[up3(j, j)] = 0.0;
                    d++;
                }
            }
        }
    }
    return d;
}
// Algorithm C.2 (U' y = b) and C.3 (U x = y) on a 3x3 factor; zero where U_ii = 0
__device__ __forceinline__ void fwd3(const double* U, const double* b, double* y) {
    for (int i = 0; i < 3; i++) {
        double s = b[i];
        for (int k = 0; k < i; k++) s -= U[up3(k, i)] * y[k];
        y[i] = U[up3(i, i)] > 0.0 ? s / U[up3(i, i)] : 0.0;
    }
}
__device__ __forceinline__ void back3(const double* U, const double* y, double* x) {
    for (int i = 2; i >= 0; i--) {
        double s = y[i];
        for (int k = i + 1; k < 3; k++) s -= U[up3(i, k)] * x[k];
        x[i] = U[up3(i, i)] > 0.0 ? s / U[up3(i, i)] : 0.0;
    }
}

// ---------------------------------------------------------------------------------------
// AL cells (n, g, j): one warp per cell.  Sums of D_j, b_j in registers; B_j, E, b_small per
// bin in the warp's shared-memory slice by a segmented scan over each chunk of 32 sorted
// observations (the last lane of each bin's run adds the run's sums).  Then D_j = U'U (C.1),
// w = U'^-1 b_j, V = U'^-1 B_j.
// ---------------------------------------------------------------------------------------
__global__ void k_cg_cells(DevGeo G, int64_t n_cells, const ObsRec* __restrict__ rec, const double* __restrict__ mu,
                           CalGenWork w, double tol) {
    extern __shared__ double sm_cg[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int nb = G.cg.n_bin;
    double* Bs = sm_cg + (size_t)wib * 8 * nb;   // rows 0..5 B, 6 E, 7 b_small
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; c < n_cells; c += nw) {
        for (int i = lane; i < 8 * nb; i += kWarp) Bs[i] = 0.0;
        __syncwarp();
        double Dn[2][6], bj[2][3];
        for (int f = 0; f < 2; f++) {
            for (int i = 0; i < 6; i++) Dn[f][i] = 0.0;
            for (int i = 0; i < 3; i++) bj[f][i] = 0.0;
        }
        const int64_t lo = w.off[c], hi = w.off[c + 1];
        for (int64_t base = lo; base < hi; base += kWarp) {
            const int64_t o = base + lane;
            const bool valid = o < hi;
            int bin = -1 - lane;   // distinct for invalid lanes
            double val[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (valid) {
                const uint32_t ob = w.perm[o];
                const ObsRec& e = rec[ob];
                const CalPos p = cal_position(G.cg, e.t_ns, e.meta, mu[ob]);
                const int f = (int)meta_fov(e.meta);
                const double phi[3] = {1.0, p.L1, p.L2};
                const double W = e.W, WR = e.W * e.R;
#pragma unroll
                for (int a = 0; a < 3; a++) {
#pragma unroll
                    for (int b = a; b < 3; b++) Dn[f][up3(a, b)] += W * phi[a] * phi[b];
                    bj[f][a] -= WR * phi[a];
                    val[3 * f + a] = W * phi[a];
                }
                val[6] = W;
                val[7] = -WR;
                bin = p.bin;
            }
            // head of this lane's run of equal bins
            const int prev = __shfl_up_sync(0xffffffffu, bin, 1);
            const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != bin);
            const int head = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const double u = __shfl_up_sync(0xffffffffu, val[q], off);
                    if (lane - off >= head) val[q] += u;
                }
            }
            const int next = __shfl_down_sync(0xffffffffu, bin, 1);
            const bool tail = valid && (lane == 31 || next != bin);
            if (tail)
                for (int q = 0; q < 8; q++) Bs[(size_t)q * nb + bin] += val[q];
            __syncwarp();
        }
        for (int f = 0; f < 2; f++) {
            for (int i = 0; i < 6; i++) Dn[f][i] = warp_sum(Dn[f][i]);
            for (int i = 0; i < 3; i++) bj[f][i] = warp_sum(bj[f][i]);
        }
        // factors (identical in every lane)
        double U[2][6], wv[2][3];
        int rdc = 0;
        for (int f = 0; f < 2; f++) {
            rdc += chol3(Dn[f], U[f], tol);
            fwd3(U[f], bj[f], wv[f]);
        }
        double* V = w.V + (size_t)c * 6 * nb;
        for (int b = lane; b < nb; b += kWarp) {
            for (int f = 0; f < 2; f++) {
                const double Bc[3] = {Bs[(size_t)(3 * f) * nb + b], Bs[(size_t)(3 * f + 1) * nb + b],
                                      Bs[(size_t)(3 * f + 2) * nb + b]};
                double y[3];
                fwd3(U[f], Bc, y);
                for (int a = 0; a < 3; a++) V[(size_t)(3 * f + a) * nb + b] = y[a];
            }
            w.E[(size_t)c * nb + b] = Bs[(size_t)6 * nb + b];
            w.bs[(size_t)c * nb + b] = Bs[(size_t)7 * nb + b];
        }
        if (lane == 0) {
            double* cw = w.cw + (size_t)c * 18;
            for (int f = 0; f < 2; f++) {
                for (int a = 0; a < 3; a++) cw[3 * f + a] = wv[f][a];
                for (int i = 0; i < 6; i++) cw[6 + 6 * f + i] = U[f][i];
            }
            w.rd[c] = rdc;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------------
// AL groups: S = diag(sum_j E_j) - sum_j V_j' V_j in 16x16 tiles (grid: tiles x tiles x groups)
// ---------------------------------------------------------------------------------------
__global__ void k_cg_reduce(int nb, int jpk, CalGenWork w) {
    __shared__ double Va[6][kTile], Vb[6][kTile];
    const int g = blockIdx.z;
    const int a = blockIdx.y * kTile + threadIdx.y;
    const int b = blockIdx.x * kTile + threadIdx.x;
    const int t = threadIdx.y * kTile + threadIdx.x;
    double s = 0.0;
    for (int jj = 0; jj < jpk; jj++) {
        const double* V = w.V + ((size_t)g * jpk + jj) * 6 * nb;
        if (t < 6 * kTile) {
            const int row = t / kTile, col = t % kTile;
            const int ia = blockIdx.y * kTile + col, ib = blockIdx.x * kTile + col;
            Va[row][col] = ia < nb ? V[(size_t)row * nb + ia] : 0.0;
            Vb[row][col] = ib < nb ? V[(size_t)row * nb + ib] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 6; q++) s += Va[q][threadIdx.y] * Vb[q][threadIdx.x];
        __syncthreads();
    }
    if (a < nb && b < nb) {
        double e = 0.0;
        if (a == b)
            for (int jj = 0; jj < jpk; jj++) e += w.E[((size_t)g * jpk + jj) * nb + a];
        w.S[((size_t)g * nb + a) * nb + b] = e - s;
    }
}

// reduced right-hand side and the group's weight per bin (one thread per bin)
__global__ void k_cg_rhs(int64_t n_groups, int nb, int jpk, CalGenWork w) {
    const int64_t total = n_groups * nb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = i / nb;
        const int a = (int)(i - g * nb);
        double rr = 0.0, e = 0.0;
        for (int jj = 0; jj < jpk; jj++) {
            const int64_t c = g * jpk + jj;
            const double* V = w.V + (size_t)c * 6 * nb;
            const double* cw = w.cw + (size_t)c * 18;
            double vw = 0.0;
            for (int q = 0; q < 6; q++) vw += V[(size_t)q * nb + a] * cw[q];
            rr += w.bs[(size_t)c * nb + a] - vw;
            e += w.E[(size_t)c * nb + a];
        }
        w.r[i] = rr;
        w.Et[i] = e;
    }
}

// ---------------------------------------------------------------------------------------
// AL groups: Eq. cc2 on the reduced system by the null-space method, robust Cholesky of
// Z'SZ (Algorithm C.1, right-looking), C.2, C.3, v = Z y.  One block per group; the observed
// bins are compacted (unobserved ones are held at zero and counted).
// ---------------------------------------------------------------------------------------
constexpr int kSolveThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wib] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

__global__ void __launch_bounds__(kSolveThreads) k_cg_solve(int nb, double tol, CalGenWork w, int64_t rd_base) {
    __shared__ double red[33];
    __shared__ double beta_s[3];
    __shared__ int m_s, rank_s;
    const int64_t g = blockIdx.x;
    double* S = w.S + (size_t)g * nb * nb;
    double* r = w.r + (size_t)g * nb;
    const double* Et = w.Et + (size_t)g * nb;
    int* idx = w.idx + (size_t)g * nb;
    double* H = w.H + (size_t)g * 3 * nb;
    double* v = w.v + (size_t)g * nb;
    if (threadIdx.x == 0) {
        int m = 0;
        for (int b = 0; b < nb; b++)
            if (Et[b] > 0.0) idx[m++] = b;
        m_s = m;
    }
    __syncthreads();
    const int m = m_s;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v[b] = 0.0;
    // Householder reflections of the cc2 columns C (m x 3) restricted to the observed bins:
    // H_q = I - beta_q h_q h_q' with h_q zero above row q; the columns of Q = H_0 H_1 H_2 beyond
    // the rank span {x : C' x = 0}.  The columns are reflected in H (3 x m), and h_q replaces
    // column q once it has been used.
    double* Cw = H;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        for (int q = 0; q < 3; q++) Cw[(size_t)q * nb + i] = w.cc2w[(size_t)q * nb + idx[i]];
    __syncthreads();
    // |R_qq| for the rank test of numpy's QR (|R_qq| > 1e-12 max(1, max |R|))
    double Rdiag[3] = {0, 0, 0};
    int rank = 0;
    for (int q = 0; q < 3 && q < m; q++) {
        // x = column q from row q
        double ss = 0.0;
        for (int i = q + threadIdx.x; i < m; i += blockDim.x) ss += Cw[(size_t)q * nb + i] * Cw[(size_t)q * nb + i];
        ss = block_sum(ss, red);
        const double x0 = Cw[(size_t)q * nb + q];
        const double nrm = sqrt(ss);
        const double alpha = x0 > 0.0 ? -nrm : nrm;
        Rdiag[q] = fabs(alpha);
        // h = x - alpha e_q, beta = 2 / h'h (beta = 0 for a zero column)
        const double hh = ss - x0 * x0 + (x0 - alpha) * (x0 - alpha);
        const double beta = hh > 0.0 ? 2.0 / hh : 0.0;
        __syncthreads();
        if (threadIdx.x == 0) beta_s[q] = beta;
        // apply to the later columns: c_p -= beta h (h' c_p)
        for (int p = q + 1; p < 3; p++) {
            double dp = 0.0;
            for (int i = q + threadIdx.x; i < m; i += blockDim.x) {
                const double h = i == q ? x0 - alpha : Cw[(size_t)q * nb + i];
                dp += h * Cw[(size_t)p * nb + i];
            }
            dp = block_sum(dp, red);
            for (int i = q + threadIdx.x; i < m; i += blockDim.x) {
                const double h = i == q ? x0 - alpha : Cw[(size_t)q * nb + i];
                Cw[(size_t)p * nb + i] -= beta * h * dp;
            }
            __syncthreads();
        }
        // the vector h replaces column q (zero above q)
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            if (i < q) Cw[(size_t)q * nb + i] = 0.0;
            else if (i == q) Cw[(size_t)q * nb + i] = x0 - alpha;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mx = fmax(1.0, fmax(Rdiag[0], fmax(Rdiag[1], Rdiag[2])));
        int rk = 0;
        for (int q = 0; q < 3 && q < m; q++) rk += Rdiag[q] > 1e-12 * mx;
        rank_s = rk;
    }
    __syncthreads();
    rank = rank_s;
    // S <- H S H and r <- H r for every reflection of the basis (all three: Q is their product
    // whatever the rank; the columns beyond the rank are taken)
    for (int q = 0; q < 3 && q < m; q++) {
        const double beta = beta_s[q];
        const double* h = Cw + (size_t)q * nb;
        // p = beta S h (over the compacted indices)
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            double s = 0.0;
            const double* Si = S + (size_t)idx[i] * nb;
            for (int k = q; k < m; k++) s += Si[idx[k]] * h[k];
            v[idx[i]] = beta * s;   // v as scratch for p (indexed by bin)
        }
        __syncthreads();
        double hp = 0.0;
        for (int i = q + threadIdx.x; i < m; i += blockDim.x) hp += h[i] * v[idx[i]];
        hp = block_sum(hp, red);
        const double K = 0.5 * beta * hp;
        // q_vec = p - K h; S -= h q' + q h'
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = e / m, k = e % m;
            const double qi = v[idx[i]] - K * (i >= q ? h[i] : 0.0);
            const double qk = v[idx[k]] - K * (k >= q ? h[k] : 0.0);
            const double hi = i >= q ? h[i] : 0.0, hk = k >= q ? h[k] : 0.0;
            S[(size_t)idx[i] * nb + idx[k]] -= hi * qk + qi * hk;
        }
        __syncthreads();
        double hr = 0.0;
        for (int i = q + threadIdx.x; i < m; i += blockDim.x) hr += h[i] * r[idx[i]];
        hr = block_sum(hr, red);
        for (int i = q + threadIdx.x; i < m; i += blockDim.x) r[idx[i]] -= beta * hr * h[i];
        __syncthreads();
    }
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v[b] = 0.0;
    __syncthreads();
    // robust Cholesky of the trailing (m - rank) block, right-looking; each pivot is tested
    // against the block's diagonal before the factorisation (a copy kept in v)
    const int n0 = rank;
    for (int i = n0 + threadIdx.x; i < m; i += blockDim.x) v[idx[i]] = S[(size_t)idx[i] * nb + idx[i]];
    __syncthreads();
    __shared__ int rd_s;
    if (threadIdx.x == 0) rd_s = 0;
    __syncthreads();
    for (int j = n0; j < m; j++) {
        const size_t jj = (size_t)idx[j] * nb;
        __shared__ double piv_s;
        if (threadIdx.x == 0) {
            const double x = S[jj + idx[j]];
            if (x > tol * v[idx[j]]) {
                piv_s = sqrt(x);
            } else {
                piv_s = 0.0;
                rd_s++;
            }
            S[jj + idx[j]] = piv_s;
        }
        __syncthreads();
        const double pv = piv_s;
        // row j of U: U_jk = S_jk / pivot (zero row for a failing pivot)
        for (int k = j + 1 + threadIdx.x; k < m; k += blockDim.x)
            S[jj + idx[k]] = pv > 0.0 ? S[jj + idx[k]] / pv : 0.0;
        __syncthreads();
        // trailing update S_ik -= U_ji U_jk for j < i <= k
        const int t = m - j - 1;
        for (int e = threadIdx.x; e < t * t; e += blockDim.x) {
            const int i = j + 1 + e / t, k = j + 1 + e % t;
            if (k >= i) S[(size_t)idx[i] * nb + idx[k]] -= S[jj + idx[i]] * S[jj + idx[k]];
        }
        __syncthreads();
    }
    // C.2: U' y = r (forward, column-oriented), then C.3: U x = y (backward)
    for (int j = n0; j < m; j++) {
        __shared__ double yj_s;
        if (threadIdx.x == 0) {
            const double u = S[(size_t)idx[j] * nb + idx[j]];
            yj_s = u > 0.0 ? r[idx[j]] / u : 0.0;
            r[idx[j]] = yj_s;
        }
        __syncthreads();
        const double yj = yj_s;
        for (int k = j + 1 + threadIdx.x; k < m; k += blockDim.x) r[idx[k]] -= S[(size_t)idx[j] * nb + idx[k]] * yj;
        __syncthreads();
    }
    for (int j = m - 1; j >= n0; j--) {
        __shared__ double xj_s;
        if (threadIdx.x == 0) {
            const double u = S[(size_t)idx[j] * nb + idx[j]];
            xj_s = u > 0.0 ? r[idx[j]] / u : 0.0;
            r[idx[j]] = xj_s;
        }
        __syncthreads();
        const double xj = xj_s;
        for (int i = n0 + threadIdx.x; i < j; i += blockDim.x) r[idx[i]] -= S[(size_t)idx[i] * nb + idx[j]] * xj;
        __syncthreads();
    }
    // z = [0 (rank); y], v = Q z = H_0 (H_1 (H_2 z))
    for (int i = threadIdx.x; i < m; i += blockDim.x) v[idx[i]] = i < n0 ? 0.0 : r[idx[i]];
    __syncthreads();
    for (int q = (m < 3 ? m : 3) - 1; q >= 0; q--) {
        const double* h = Cw + (size_t)q * nb;
        double hz = 0.0;
        for (int i = q + threadIdx.x; i < m; i += blockDim.x) hz += h[i] * v[idx[i]];
        hz = block_sum(hz, red);
        for (int i = q + threadIdx.x; i < m; i += blockDim.x) v[idx[i]] -= beta_s[q] * hz * h[i];
        __syncthreads();
    }
    if (threadIdx.x == 0) w.rd[rd_base + g] = rd_s + (nb - m);
}

// AL cells: u_j = U_j^-1 (w_j - V_j v) per field block; the group's update into d
__global__ void k_cg_back(DevGeo G, int64_t n_cells, CalGenWork w) {
    const int nb = G.cg.n_bin, jpk = G.cg.j_per_k;
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n_cells; c += nw) {
        const int64_t g = c / jpk;
        const int jj = (int)(c - g * jpk);
        const double* V = w.V + (size_t)c * 6 * nb;
        const double* v = w.v + (size_t)g * nb;
        double t[6] = {0, 0, 0, 0, 0, 0};
        for (int b = lane; b < nb; b += kWarp) {
            const double vb = v[b];
            for (int q = 0; q < 6; q++) t[q] += V[(size_t)q * nb + b] * vb;
        }
        for (int q = 0; q < 6; q++) t[q] = warp_sum(t[q]);
        const double* cw = w.cw + (size_t)c * 18;
        double* d = w.d + (size_t)g * G.cg.al_size;
        if (lane < 2) {
            const int f = lane;
            const double y[3] = {cw[3 * f] - t[3 * f], cw[3 * f + 1] - t[3 * f + 1], cw[3 * f + 2] - t[3 * f + 2]};
            double x[3];
            back3(cw + 6 + 6 * f, y, x);
            for (int a = 0; a < 3; a++) d[jj * 6 + 3 * f + a] = x[a];
        }
        if (jj == 0)
            for (int b = lane; b < nb; b += kWarp) d[6 * jpk + b] = v[b];
    }
}

// AC groups (n, g, k): one warp per group, two 3x3 blocks by C.1-C.3
__global__ void k_cg_ac(DevGeo G, int64_t n_cells, int64_t n_groups, const ObsRec* __restrict__ rec,
                        const double* __restrict__ mu, CalGenWork w, double tol, int64_t rd_base) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < n_groups; g += nw) {
        double Dn[2][6], bj[2][3];
        for (int f = 0; f < 2; f++) {
            for (int i = 0; i < 6; i++) Dn[f][i] = 0.0;
            for (int i = 0; i < 3; i++) bj[f][i] = 0.0;
        }
        const int64_t lo = w.off[n_cells + g], hi = w.off[n_cells + g + 1];
        for (int64_t o = lo + lane; o < hi; o += kWarp) {
            const uint32_t ob = w.perm[o];
            const ObsRec& e = rec[ob];
            const CalPos p = cal_position(G.cg, e.t_ns, e.meta, mu[ob]);
            const int f = (int)meta_fov(e.meta);
            const double phi[3] = {1.0, p.L1, p.L2};
            const double W = e.W, WR = e.W * e.R;
            for (int a = 0; a < 3; a++) {
                for (int b = a; b < 3; b++) Dn[f][up3(a, b)] += W * phi[a] * phi[b];
                bj[f][a] -= WR * phi[a];
            }
        }
        for (int f = 0; f < 2; f++) {
            for (int i = 0; i < 6; i++) Dn[f][i] = warp_sum(Dn[f][i]);
            for (int i = 0; i < 3; i++) bj[f][i] = warp_sum(bj[f][i]);
        }
        if (lane == 0) {
            int rdg = 0;
            double* d = w.d + G.cg.n_al + (size_t)g * 6;
            for (int f = 0; f < 2; f++) {
                double U[6], y[3], x[3];
                rdg += chol3(Dn[f], U, tol);
                fwd3(U, bj[f], y);
                back3(U, y, x);
                for (int a = 0; a < 3; a++) d[3 * f + a] = x[a];
            }
            w.rd[rd_base + g] = rdg;
        }
    }
}

// Eqs. cc1 (per short interval j: the r = 0 AL terms of gate 0, both fields, all CCDs) and
// cc3 (per long interval k and field: the r = 0 AC terms of gate 0) by the projection of
// Eq. calCon: subtract the mean within each constraint's support.  One thread per constraint.
__global__ void k_cg_project(DevGeo G, double* __restrict__ d) {
    const CalGen& C = G.cg;
    const int nc1 = C.n_j, nc3 = 2 * C.n_k;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nc1 + nc3) return;
    double s = 0.0;
    if (q < nc1) {
        const int j = q, k = j / C.j_per_k, jj = j - k * C.j_per_k;
        for (int n = 0; n < kNccd; n++)
            for (int f = 0; f < 2; f++) s += d[(((int64_t)n * C.n_gate) * C.n_k + k) * C.al_size + jj * 6 + f * 3];
        const double m = s / (2.0 * kNccd);
        for (int n = 0; n < kNccd; n++)
            for (int f = 0; f < 2; f++) d[(((int64_t)n * C.n_gate) * C.n_k + k) * C.al_size + jj * 6 + f * 3] -= m;
    } else {
        const int h = q - nc1, k = h >> 1, f = h & 1;
        for (int n = 0; n < kNccd; n++) s += d[C.n_al + (((int64_t)n * C.n_gate) * C.n_k + k) * 6 + f * 3];
        const double m = s / (double)kNccd;
        for (int n = 0; n < kNccd; n++) d[C.n_al + (((int64_t)n * C.n_gate) * C.n_k + k) * 6 + f * 3] -= m;
    }
}

__global__ void k_cg_apply(int64_t n, const double* __restrict__ d, double* __restrict__ cal) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cal[i] += d[i];
}

int cg_cell_warps(int n_bin) {
    // 8 n_bin doubles of shared memory per warp, within 200 KB per block
    int wpb = (int)(200 * 1024 / (8 * 8 * (size_t)n_bin));
    if (wpb > 8) wpb = 8;
    return wpb < 1 ? 1 : wpb;
}

// the cell kernel's shared memory beyond the default 48 KB (set once, outside any capture)
int calgen_prepare() {
    return cudaFuncSetAttribute(k_cg_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) == cudaSuccess
               ? 0 : -1;
}

void launch_calgen(const DevGeo& G, int64_t n_groups, const ObsRec* rec, const double* mu, const CalGenWork& w,
                   double tol, double* cal, cudaStream_t s) {
    const CalGen& C = G.cg;
    const int nb = C.n_bin;
    const int64_t n_cells = n_groups * C.j_per_k;
    const int wpb = cg_cell_warps(nb);
    int64_t blocks = (n_cells + wpb - 1) / wpb;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const size_t smem = (size_t)wpb * 8 * nb * sizeof(double);
    if (n_cells > 0) k_cg_cells<<<(int)blocks, 32 * wpb, smem, s>>>(G, n_cells, rec, mu, w, tol);
    if (n_groups > 0) {
        const int tiles = (nb + kTile - 1) / kTile;
        // one launch per at most 65535 groups (grid z limit)
        for (int64_t g0 = 0; g0 < n_groups; g0 += 65535) {
            const int gz = (int)std::min<int64_t>(65535, n_groups - g0);
            CalGenWork ws = w;
            ws.V = w.V + (size_t)g0 * C.j_per_k * 6 * nb;
            ws.E = w.E + (size_t)g0 * C.j_per_k * nb;
            ws.S = w.S + (size_t)g0 * nb * nb;
            k_cg_reduce<<<dim3(tiles, tiles, gz), dim3(kTile, kTile), 0, s>>>(nb, C.j_per_k, ws);
        }
        const int64_t tot = n_groups * nb;
        int64_t rb = (tot + 255) / 256;
        if (rb > 152 * 16) rb = 152 * 16;
        k_cg_rhs<<<(int)rb, 256, 0, s>>>(n_groups, nb, C.j_per_k, w);
        k_cg_solve<<<(int)n_groups, kSolveThreads, 0, s>>>(nb, tol, w, n_cells);
        k_cg_back<<<(int)blocks, 32 * 4, 0, s>>>(G, n_cells, w);
        int64_t ab = (n_groups + 3) / 4;
        if (ab > 152 * 16) ab = 152 * 16;
        k_cg_ac<<<(int)ab, 128, 0, s>>>(G, n_cells, n_groups, rec, mu, w, tol, n_cells + n_groups);
    }
    k_cg_project<<<(C.n_j + 2 * C.n_k + 127) / 128, 128, 0, s>>>(G, w.d);
    const int64_t n_cal = C.n_al + 6 * n_groups;
    int64_t ab = (n_cal + 255) / 256;
    if (ab > 152 * 16) ab = 152 * 16;
    k_cg_apply<<<(int)ab, 256, 0, s>>>(n_cal, w.d, cal);
}

}  // namespace agis
