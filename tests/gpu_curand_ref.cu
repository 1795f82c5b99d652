// Test helper: cuRAND's Philox4_32_10 (an independent implementation of the
// published generator), built at test time only.  curand_init(seed, q, 4c)
// puts the counter at (c_lo, c_hi, q_lo, q_hi) with key (seed_lo, seed_hi);
// curand4 then returns that block.
#include <curand_kernel.h>

#include <cstdint>

__global__ void k_ref(int n, const unsigned long long* seed, const unsigned long long* sub,
                      const unsigned long long* ctr, uint4* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed[i], sub[i], 4ull * ctr[i], &st);
    out[i] = curand4(&st);
}

extern "C" int curand_philox_ref(int n, const unsigned long long* seed, const unsigned long long* sub,
                                 const unsigned long long* ctr, unsigned int* out)
{
    unsigned long long *ds = nullptr, *dq = nullptr, *dc = nullptr;
    uint4* dout = nullptr;
    if (cudaMalloc(&ds, 8 * n) || cudaMalloc(&dq, 8 * n) || cudaMalloc(&dc, 8 * n) ||
        cudaMalloc(&dout, 16 * n))
        return 1;
    cudaMemcpy(ds, seed, 8 * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dq, sub, 8 * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dc, ctr, 8 * n, cudaMemcpyHostToDevice);
    k_ref<<<(n + 127) / 128, 128>>>(n, ds, dq, dc, dout);
    const int rc = cudaMemcpy(out, dout, 16 * n, cudaMemcpyDeviceToHost) != cudaSuccess;
    cudaFree(ds); cudaFree(dq); cudaFree(dc); cudaFree(dout);
    return rc;
}
