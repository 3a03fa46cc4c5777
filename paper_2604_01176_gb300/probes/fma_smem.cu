// Peak probe: FP64 and FP32 FMA throughput (8 independent FMA chains per
// thread) and the rate of random 4- and 8-byte gathers from a 12,870-entry
// row in shared memory (the coupling kernels' access pattern).  Every thread
// writes exactly one output element, out[blockIdx.x * blockDim.x +
// threadIdx.x].  Standalone: nvcc -gencode arch=compute_103a,code=sm_103a
// -O3 fma_smem.cu -o fma_smem
#include <cstdio>
#include <cuda_runtime.h>

template <typename T>
__global__ void fma_loop(T *out, int iters, T a, T b)
{
    T x0 = T(threadIdx.x), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
    T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
    for (int i = 0; i < iters; ++i) {
        x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
        x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// random gather from a 12870-entry shared row, index from a per-thread LCG
template <typename T>
__global__ void smem_gather(T *out, int iters, int nrow)
{
    extern __shared__ unsigned char raw[];
    T *row = reinterpret_cast<T *>(raw);
    for (int i = threadIdx.x; i < nrow; i += blockDim.x) row[i] = T(i);
    __syncthreads();
    unsigned s = threadIdx.x * 2654435761u + blockIdx.x;
    T acc = T(0);
    for (int i = 0; i < iters; ++i) {
        s = s * 1664525u + 1013904223u;
        acc += row[(s >> 8) % nrow];
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

int main()
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int blocks = sms * 8, threads = 256;
    void *buf;
    cudaMalloc(&buf, size_t(blocks) * threads * 8);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms;
    {
        int it = 4096;
        fma_loop<double><<<blocks, threads>>>((double *)buf, 16, 1.0000001, 1e-9);
        cudaEventRecord(e0);
        fma_loop<double><<<blocks, threads>>>((double *)buf, it, 1.0000001, 1e-9);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        double fma = double(blocks) * threads * it * 8;
        printf("fp64 FMA: %.3f TFMA/s (%.2f ms)\n", fma / ms / 1e9, ms);
    }
    {
        int it = 65536;
        fma_loop<float><<<blocks, threads>>>((float *)buf, 16, 1.0000001f, 1e-9f);
        cudaEventRecord(e0);
        fma_loop<float><<<blocks, threads>>>((float *)buf, it, 1.0000001f, 1e-9f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        double fma = double(blocks) * threads * it * 8;
        printf("fp32 FMA: %.3f TFMA/s (%.2f ms)\n", fma / ms / 1e9, ms);
    }
    for (int sz = 4; sz <= 8; sz += 4) {
        int nrow = 12870, it = 8192;
        size_t smem = size_t(nrow) * sz;
        int gb = sms * 2;
        if (sz == 8) {
            cudaFuncSetAttribute(smem_gather<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            smem_gather<double><<<gb, 512, smem>>>((double *)buf, 16, nrow);
            cudaEventRecord(e0);
            smem_gather<double><<<gb, 512, smem>>>((double *)buf, it, nrow);
        } else {
            cudaFuncSetAttribute(smem_gather<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            smem_gather<float><<<gb, 512, smem>>>((float *)buf, 16, nrow);
            cudaEventRecord(e0);
            smem_gather<float><<<gb, 512, smem>>>((float *)buf, it, nrow);
        }
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        double g = double(gb) * 512 * it;
        printf("smem random gather %dB: %.3f Tgathers/s (%.2f ms)\n", sz, g / ms / 1e9, ms);
    }
    cudaError_t err = cudaDeviceSynchronize();
    printf("status: %s\n", cudaGetErrorString(err));
    return err == cudaSuccess ? 0 : 1;
}
