// Test harness for the device reciprocal rcp_pos of the banded attitude solve: evaluates it
// and the correctly rounded division 1.0 / d on the same inputs (host arrays in and out).
#include "agis_internal.cuh"

__global__ void k_rcp(const double* __restrict__ d, double* __restrict__ y, double* __restrict__ q, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        y[i] = agis::rcp_pos(d[i]);
        q[i] = 1.0 / d[i];
    }
}

extern "C" int rcp_pos_eval(const double* d_host, double* y_host, double* q_host, int64_t n) {
    double *d = nullptr, *y = nullptr, *q = nullptr;
    const size_t b = (size_t)n * sizeof(double);
    if (cudaMalloc(&d, b) != cudaSuccess || cudaMalloc(&y, b) != cudaSuccess || cudaMalloc(&q, b) != cudaSuccess) return 1;
    int rc = 0;
    if (cudaMemcpy(d, d_host, b, cudaMemcpyHostToDevice) != cudaSuccess) rc = 2;
    if (!rc) {
        k_rcp<<<152 * 4, 256>>>(d, y, q, n);
        if (cudaDeviceSynchronize() != cudaSuccess) rc = 3;
    }
    if (!rc && (cudaMemcpy(y_host, y, b, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(q_host, q, b, cudaMemcpyDeviceToHost) != cudaSuccess))
        rc = 4;
    cudaFree(d);
    cudaFree(y);
    cudaFree(q);
    return rc;
}
