// Test harness for the tabulated orbital longitude of the observation model: evaluates
// orbit_sincos with the table (built by fill_orbit_table) and without it (sincospi of the
// linear longitude) at the same times (host arrays in and out).
#include <cstring>
#include <vector>

#include "agis_internal.cuh"

__global__ void k_orbit(agis::DevGeo G, agis::DevGeo G0, const int64_t* __restrict__ t, double* __restrict__ out,
                        int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s, c, s0, c0;
        agis::orbit_sincos(G, t[i], s, c);
        agis::orbit_sincos(G0, t[i], s0, c0);
        out[4 * i] = s;
        out[4 * i + 1] = c;
        out[4 * i + 2] = s0;
        out[4 * i + 3] = c0;
    }
}

// out[4 i .. 4 i + 3] = (sin, cos) from the table, then from sincospi, at t[i]
extern "C" int orbit_eval(double orb_L0, double year_s, int64_t t0, int32_t n_tab, const int64_t* t_host,
                          double* out_host, int64_t n) {
    const double pi = 3.141592653589793;
    agis::DevGeo G;
    std::memset(&G, 0, sizeof(G));
    G.orb_L0_pi = orb_L0 / pi;
    G.inv_year_s = 1.0 / year_s;
    G.orb_rate = 2.0 * pi / year_s;
    G.orb_rad_per_ns = G.orb_rate * 1e-9;
    agis::DevGeo G0 = G;
    std::vector<double> tab(2 * (size_t)n_tab);
    agis::fill_orbit_table(G, t0, n_tab, tab.data());
    double* dtab = nullptr;
    int64_t* dt = nullptr;
    double* dout = nullptr;
    if (cudaMalloc(&dtab, tab.size() * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dt, (size_t)n * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&dout, 4 * (size_t)n * sizeof(double)) != cudaSuccess)
        return 1;
    int rc = 0;
    if (cudaMemcpy(dtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dt, t_host, (size_t)n * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = 2;
    if (!rc) {
        G.orb_tab = dtab;
        G.orb_t0 = t0;
        G.orb_n = n_tab;
        k_orbit<<<152 * 4, 256>>>(G, G0, dt, dout, n);
        if (cudaDeviceSynchronize() != cudaSuccess) rc = 3;
    }
    if (!rc && cudaMemcpy(out_host, dout, 4 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = 4;
    cudaFree(dtab);
    cudaFree(dt);
    cudaFree(dout);
    return rc;
}
