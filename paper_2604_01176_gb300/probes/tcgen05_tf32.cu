// Peak probe: tcgen05.mma kind::tf32 issue rate for M = 64 / 128 and N = 128 /
// 256 (K = 8 per instruction, no-swizzle K-major operands of zeros in shared
// memory).  One CTA per SM issues `iters` MMAs back to back, commits them to
// an mbarrier and waits for it with a bounded poll; clock64 gives cycles per
// MMA and so tensor MACs per clock per SM.  A wait that runs out sets a flag
// and waits once more (bounded) before the tensor memory is released.
// Standalone: nvcc -gencode arch=compute_103a,code=sm_103a -O3
// tcgen05_tf32.cu -o tcgen05_tf32
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t saddr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo)
{
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t(128u >> 4) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

__global__ void bench(int M, int N, int iters, long long *cycles, int *flag)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 131072);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + 131072 + 64);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < 131072 / 4; i += blockDim.x) reinterpret_cast<float *>(sm)[i] = 0.0f;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(saddr(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
    long long t0 = clock64();
    if (tid == 0) {
        const uint32_t a = saddr(sm), b = saddr(sm + 65536);
        for (int it = 0; it < iters; ++it) {
            const uint32_t ko = uint32_t(it & 3) * 256u;
            asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                         "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                         ::"r"(tmem), "l"(sdesc(a + ko, 1024)), "l"(sdesc(b + ko, 1024)), "r"(idesc), "r"(it > 0 ? 1 : 0));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar)) : "memory");
    }
    uint32_t done = 0;
    for (long long it = 0; it < (1ll << 26) && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\nselp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(saddr(bar)) : "memory");
    long long t1 = clock64();
    if (!done && tid == 0) atomicExch(flag, 1);
    for (long long it = 0; it < (1ll << 26) && !done; ++it)   // drain before the release
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\nselp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(saddr(bar)) : "memory");
    if (tid == 0) cycles[blockIdx.x] = t1 - t0;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

int main()
{
    long long *dc; int *df;
    cudaMalloc(&dc, 152 * 8); cudaMalloc(&df, 4); cudaMemset(df, 0, 4);
    cudaFuncSetAttribute(bench, cudaFuncAttributeMaxDynamicSharedMemorySize, 131072 + 128);
    int shapes[][2] = {{64, 128}, {128, 128}, {128, 256}, {64, 256}};
    for (auto &sh : shapes) {
        const int M = sh[0], N = sh[1], iters = 4096;
        bench<<<152, 128, 131072 + 128>>>(M, N, iters, dc, df);
        cudaError_t e = cudaDeviceSynchronize();
        long long c[152]; int f = 0;
        cudaMemcpy(c, dc, sizeof c, cudaMemcpyDeviceToHost);
        cudaMemcpy(&f, df, 4, cudaMemcpyDeviceToHost);
        double avg = 0; for (int i = 0; i < 152; ++i) avg += c[i]; avg /= 152;
        const double mac = double(M) * N * 8;
        printf("M=%d N=%d err=%s timeout=%d cycles/MMA=%.1f MAC/clk/SM=%.0f\n", M, N, cudaGetErrorString(e), f,
               avg / iters, mac / (avg / iters));
        if (e != cudaSuccess) return 1;
    }
    return 0;
}
