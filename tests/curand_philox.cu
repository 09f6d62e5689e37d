// Test helper (compiled by tests/test_gpu_philox_curand.py): cuRAND's Philox4x32-10 generator, an implementation
// independent of this repository's, evaluated at given keys and counters.  curand_init(seed, subsequence, offset)
// puts the seed's two 32-bit words in the key, adds the subsequence to the counter's high 64 bits and offset / 4
// to its low 64 bits; the first curand4 then returns the block of that counter.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

__global__ void k_curand_blocks(const unsigned long long *seed, const unsigned long long *subseq,
                                const unsigned long long *offset, uint4 *out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed[i], subseq[i], offset[i], &st);
    out[i] = curand4(&st);
}

extern "C" int curand_philox_blocks(const unsigned long long *seed, const unsigned long long *subseq,
                                    const unsigned long long *offset, uint32_t *out, int n) {
    unsigned long long *d = nullptr;
    uint4 *o = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long) * 3 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&o, sizeof(uint4) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(d, seed, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + n, subseq, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + 2 * n, offset, sizeof(unsigned long long) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_curand_blocks<<<(n + 255) / 256, 256>>>(d, d + n, d + 2 * n, o, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, o, sizeof(uint4) * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    cudaFree(o);
    return (int)e;
}
