// Ceiling probe for the sparse H|psi> scatter: throughput of float atomic
// adds to pseudo-random addresses drawn from F distinct targets spread over
// an array of N floats (the sigma of the 16-orbital, 8+8-electron space),
// with and without the scatter's membership-bit test.  Every address is in
// bounds: (F - 1) * (N / F) < N.  Standalone: nvcc -gencode
// arch=compute_103a,code=sm_103a -O3 l2_atomics.cu -o l2_atomics
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint32_t mix64(uint64_t x)
{
    // splitmix64 finaliser
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ULL;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebULL;
    x ^= x >> 31;
    return uint32_t(x);
}

__global__ void k_adds(float *s, int64_t n_ops, uint32_t F, int64_t stride, uint32_t *bits,
                       int with_bits)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_ops;
         i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t o = int64_t(mix64(uint64_t(i)) % F) * stride;
        atomicAdd(s + o, 1.0f);
        if (with_bits) {
            const uint32_t bit = 1u << (o & 31);
            if (__ldcg(bits + (o >> 5)) & bit) continue;
            atomicOr(bits + (o >> 5), bit);
        }
    }
}

}  // namespace

int main()
{
    const int64_t N = 165636900, n_ops = 13600000;   // ~ 2,304 amplitudes x 5,900 targets
    float *s = nullptr;
    uint32_t *bits = nullptr;
    if (cudaMalloc(&s, N * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&bits, (N / 32 + 1) * sizeof(uint32_t)) != cudaSuccess) {
        std::printf("allocation failed\n");
        return 1;
    }
    cudaMemset(s, 0, N * sizeof(float));
    cudaMemset(bits, 0, (N / 32 + 1) * sizeof(uint32_t));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const uint32_t footprints[3] = {200000u, 2000000u, 20000000u};
    for (int with_bits = 0; with_bits < 2; ++with_bits)
        for (uint32_t F : footprints) {
            const int64_t stride = N / F;
            for (int g : {sms * 8, sms * 32}) {
                k_adds<<<g, 256>>>(s, n_ops, F, stride, bits, with_bits);
                cudaEventRecord(a);
                for (int r = 0; r < 10; ++r) k_adds<<<g, 256>>>(s, n_ops, F, stride, bits, with_bits);
                cudaEventRecord(b);
                cudaEventSynchronize(b);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, a, b);
                ms /= 10.0f;
                std::printf("{\"bit_test\": %d, \"footprint\": %u, \"grid\": %d, \"ms\": %.4f, "
                            "\"adds_per_s\": %.3e}\n",
                            with_bits, F, g, ms, double(n_ops) / (double(ms) * 1e-3));
            }
        }
    const cudaError_t e = cudaDeviceSynchronize();
    std::printf("status %s\n", cudaGetErrorString(e));
    cudaFree(s);
    cudaFree(bits);
    return e == cudaSuccess ? 0 : 1;
}
