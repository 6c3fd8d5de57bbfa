// Microbenchmark of 64-bit modular multiplication issue rate: eight
// independent dependency chains per thread, enough warps to fill every SM.
#include "internal.h"

namespace hespmv {

__global__ void k_rate_shoup(uint64_t *out, uint64_t q, uint64_t w, uint64_t ws, int iters) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (t * 8 + k + 12345) % q;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = mul_shoup(x[k], w, ws, q);
    }
    uint64_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= x[k];
    out[t] = r;
}

__global__ void k_rate_barrett(uint64_t *out, ModConst m, int iters) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t x[8], y[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        x[k] = (t * 8 + k + 777) % m.q;
        y[k] = (t * 131 + k * 7 + 99) % m.q;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = mul_mod(x[k], y[k], m);
    }
    uint64_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= x[k];
    out[t] = r;
}

// Returns modular multiplications per second (kind 0: Shoup, 1: two variable
// operands, the Barrett-style mul_mod).
cudaError_t mulmod_rate(const HostTables &h, int kind, double *rate) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256, blocks = sms * 8, iters = 4096;
    uint64_t *out = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)threads * blocks * 8);
    if (e != cudaSuccess) return e;
    const ModConst m = h.mc[0];
    const uint64_t w = h.tw[5] % m.q, ws = (uint64_t)(((unsigned __int128)w << 64) / m.q);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a);
        if (kind == 0)
            k_rate_shoup<<<blocks, threads>>>(out, m.q, w, ws, iters);
        else
            k_rate_barrett<<<blocks, threads>>>(out, m, iters);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;  // first launch is a warm-up
    }
    e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    *rate = (double)threads * blocks * 8.0 * iters / (best * 1e-3);
    return e;
}

}  // namespace hespmv
