// Test-only: Philox4x32-10 blocks from NVIDIA's cuRAND (its device API,
// curand_kernel.h), an implementation of the generator of Salmon et al.
// (SC'11) written independently of this repository's oracle and library.
// Built by tests/test_gpu_philox_curand.py into a temporary directory.
//
// cuRAND's Philox state is a 128-bit counter and a 64-bit key (= seed):
// curand_init(seed, subsequence, 0) sets the counter's upper 64 bits to
// `subsequence` and its lower 64 bits to 0; skipahead(m) advances by m
// 32-bit outputs, i.e. m / 4 counters; curand4 then returns the four words
// of the block at the current counter.  So the block of counter
// (c0, c1, c2, c3) is reached with subsequence = c3:c2 and m = 4 * (c1:c0).
#include <curand_kernel.h>
#include <stdint.h>

__global__ void k_curand_blocks(unsigned long long seed, const uint4* ctr, int n, uint4* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = ctr[i];
    curandStatePhilox4_32_10_t st;
    curand_init(seed, ((unsigned long long)c.w << 32) | c.z, 0ull, &st);
    const unsigned long long lo = ((unsigned long long)c.y << 32) | c.x;
    // 4 * lo outputs, in parts that fit 64 bits: the low 62 bits of lo at
    // once, each unit of the top two bits as two skips of 2^63 outputs
    skipahead(4ull * (lo & 0x3fffffffffffffffull), &st);
    for (unsigned long long q = 0; q < 2 * (lo >> 62); ++q) skipahead(1ull << 63, &st);
    out[i] = curand4(&st);
}

extern "C" int curand_philox_blocks(unsigned long long seed, const void* ctr_dev, int n, void* out_dev,
                                    void* stream)
{
    if (n < 1 || !ctr_dev || !out_dev) return 1;
    k_curand_blocks<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(seed, (const uint4*)ctr_dev, n,
                                                                      (uint4*)out_dev);
    if (cudaGetLastError() != cudaSuccess) return 2;
    return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? 0 : 3;
}
