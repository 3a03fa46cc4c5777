// hy_cpl_tc.cu -- phase A of the float alpha-beta coupling on the fifth-
// generation tensor cores (tcgen05, accumulators in tensor memory).
//
// Per alpha string J (one persistent CTA per SM, grid-stride over J) and
// column tile of 128 beta strings b':
//   T[J][m][b'] = sum_t W_J[m][t] G_J[t][b']        m < nexa (tensor cores)
//   T[J][nexa][b'] = sum_t Wd_J[t] G_J[t][b']         (diagonal slot, FP32 SIMT)
// with the beta excitation types t = r*16 + s (r created in b', s its
// partner's orbital; s = r the diagonal pair), G_J[t][b'] = sign * psi[J][b'
// with r -> s] (zero where b' has no such excitation), W_J[m][t] the coupling
// coefficient of the m-th single-excitation partner of J and Wd_J[t] the
// diagonal coefficient sum_{p in J} V[p][p][t] (the same quantities as the
// SIMT kernel k_cpl_gemm, hy_sigma.cu).  Phase B (k_cpl_gather) is shared.
//
// FP32 accuracy from TF32 inputs: every operand is split x = hi + lo with hi
// the top 19 bits (exact in TF32) and lo = x - hi, and the tensor cores add
// hi*hi + hi*lo + lo*hi (the lo*lo term is below 2^-22 relative).
//
// Shared memory per CTA: psi's row J (every gather of G_J reads it), W_J in
// FP32, and two stages of MMA operands -- W hi/lo for 32 types (64 x 32) and
// G hi/lo for 32 types x 128 columns -- in the no-swizzle K-major layout
// (8-row x 16-byte core matrices; consecutive cores along K 128 bytes apart,
// along M/N `sbo` bytes apart).  All threads build one stage while the
// tensor cores multiply the other; the beta excitation entries of the next
// chunk are loaded while the current one is built.  A warp of its own issues
// the MMAs (M = 64, N = 128, K = 8), so its wait for the tensor cores to
// accept them never stalls a builder, and commits each stage to its mbarrier.
// Every wait is bounded (spin_limit polls of the mbarrier): on a timeout the
// kernel records it in *status, waits (bounded) for its own MMAs, frees its
// tensor memory and returns.
#include "hy_kernels.cuh"

namespace hy {
namespace k {

namespace {

// warps 0-7 build G, warps 8-11 build W chunks, warp 12 issues the MMAs
constexpr int kTcThreads = 416;
constexpr int kGThreadsTc = 256;
constexpr int kAWarps = 4;
constexpr int kIssueWarp = 12;
constexpr int kTcN = 128;          // columns per tile (MMA N)
constexpr int kTcM = 64;           // MMA M (single-excitation slots, zero padded)
constexpr int kTcKc = 32;          // types per chunk (two values of r)
constexpr int kTcK = 256;          // padded types (16 r x 16 s)
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kSbo = (kTcKc / 4) * 128;    // 8 rows (A) / columns (B) of a chunk
constexpr int kWRow = kTcK + 4;                           // padded row: 8 rows hit 32 banks
constexpr size_t kWBytes = size_t(kTcM) * kWRow * 4;       // W_J in FP32, 65 KB
constexpr size_t kABytes = size_t(kTcM) * kTcKc * 4;       // one A chunk, 8 KB
constexpr size_t kBBytes = size_t(kTcN) * kTcKc * 4;       // one G chunk, 16 KB
constexpr size_t kStage = 2 * kABytes + 2 * kBBytes;       // hi, lo of both

__device__ __forceinline__ uint32_t saddr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) in a K-major no-swizzle operand
__device__ __forceinline__ uint32_t kmaj(int row, int k, uint32_t sbo)
{
    return uint32_t(row >> 3) * sbo + uint32_t(k >> 2) * 128u + uint32_t(row & 7) * 16u +
           uint32_t(k & 3) * 4u;
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo)
{
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t(128u >> 4) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// kind::tf32, FP32 accumulate, K-major A and B, M = 64, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(kTcN >> 3) << 17) |
                            (uint32_t(kTcM >> 4) << 24);

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 ::"r"(tmem), "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(saddr(bar)) : "memory");
}

// bounded wait for the phase with parity `par` of an mbarrier: at most
// `limit` polls
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t par, long long limit)
{
    uint32_t done = 0;
    for (long long it = 0; it < limit; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(saddr(bar)), "r"(par) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void split(float x, float &hi, float &lo)
{
    hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    lo = x - hi;
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, float *v)
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
                   "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]),
                   "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

size_t cpl_tc_smem(int64_t Nb)
{
    // W_J | 2 stages | Wd [256] | diag partials [2][128] | 2 mbarriers +
    // tensor-memory slot | psi row J
    return kWBytes + 2 * kStage + kTcK * 4 + 2 * kTcN * 4 + 64 + size_t((Nb + 3) / 4 * 16);
}

// issue = 0 is a test mode: nothing is multiplied or committed, so every
// stage barrier stays pending and the builders' bounded waits run out (the
// kernel then reports a timeout in *status and returns; no MMA is in flight)
__global__ void __launch_bounds__(kTcThreads, 1)
k_cpl_tc(CplDenseArgs a, int *status, long long spin_limit, int issue)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    float *Wf = reinterpret_cast<float *>(sm);                  // [64][kWRow]
    unsigned char *stg = sm + kWBytes;                          // stage s at s * kStage
    float *Wd = reinterpret_cast<float *>(stg + 2 * kStage);
    float *dpart = Wd + kTcK;                                   // [2][kTcN]
    uint64_t *bar = reinterpret_cast<uint64_t *>(dpart + 2 * kTcN);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    float *prow = reinterpret_cast<float *>(bar + 8);           // psi[J][0 .. Nb)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n, nn = n * n, nexa = a.nexa;
    const int free_b = n - __popc(a.bstr[0]);                 // empty orbitals of a beta string
    const int nch = (n + 1) / 2;                              // chunks of two r values
    const int64_t Nb = a.Nb;
    const int slots = nexa + 1;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(saddr(tslot)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    uint32_t issued0 = 0, issued1 = 0;   // commits made to each stage's barrier
    uint32_t waited0 = 0, waited1 = 0;   // commits already waited for
    bool ok = true;
    // wait until every commit made to a stage so far has completed
    auto drain = [&](uint64_t *b, uint32_t &waited, uint32_t issued) {
        while (ok && waited < issued) {
            if (!wait_bar(b, waited & 1u, spin_limit)) {
                ok = false;
                atomicExch(status, 1);
            }
            ++waited;
        }
    };
    const bool gb = tid < kGThreadsTc;                        // a G builder
    const int col = tid & (kTcN - 1), half = (tid >> 7) & 1;  // 2 G builders per column

    for (int64_t jj = blockIdx.x; jj < a.nJ && ok; jj += gridDim.x) {
        const int64_t J = a.jlist ? int64_t(a.jlist[jj]) : jj;
        // W_J in FP32 for the 64 MMA rows, Wd_J for the diagonal slot and
        // psi's row J.  The previous J's MMAs have all been waited for.
        const uint32_t jm = a.astr[J];
        for (int idx = tid; idx < kTcM * kTcK; idx += blockDim.x) {
            const int m = idx / kTcK, tp = idx % kTcK;
            const int r = tp >> 4, s = tp & 15;
            float v = 0.0f;
            if (m < nexa && r < n && s < n) {
                const uint32_t u = a.aex[J * nexa + m];
                const int pj = (u >> 16) & 15, qj = (u >> 20) & 15;
                v = a.V[size_t(qj * n + pj) * nn + r * n + s];
                if (u >> 31) v = -v;
            }
            Wf[m * kWRow + tp] = v;
        }
        for (int tp = tid; tp < kTcK; tp += blockDim.x) {
            const int r = tp >> 4, s = tp & 15;
            float v = 0.0f;
            if (r < n && s < n)
                for (uint32_t mm = jm; mm; mm &= mm - 1) {
                    const int p = __ffs(mm) - 1;
                    v += a.V[size_t(p * n + p) * nn + r * n + s];
                }
            Wd[tp] = v;
        }
        const float *src = a.psi + J * Nb;
        for (int64_t i = tid; i < Nb; i += blockDim.x) prow[i] = __ldg(src + i);
        __syncthreads();
        for (int64_t b0 = 0; b0 < Nb && ok; b0 += kTcN) {
            const int64_t b = b0 + col;
            const bool live = gb && b < Nb;
            const uint32_t bm = live ? a.bstr[b] : 0u;
            float dsum = 0.0f;
            bool first = true;
            // beta excitation entries of this thread's r for chunk c, loaded
            // one chunk ahead: u[s] is the entry of (r created in b', s empty
            // in b') -- entry f0 + (empty orbitals below s) of b', since a
            // string lists its excitations by created orbital, then by empty
            // orbital, ascending -- or 0 (a packed entry is never 0: p != q)
            uint32_t un[16];
            auto load_entries = [&](int c, uint32_t *u) {
                const int r = 2 * c + half;
                const bool has = live && r < n && ((bm >> r) & 1u);
                const int f0 = has ? __popc(bm & ((1u << r) - 1u)) * free_b : 0;
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const bool emp = has && s < n && !((bm >> s) & 1u);
                    const int q = s - __popc(bm & ((1u << s) - 1u));
                    u[s] = emp ? __ldg(a.bexT + size_t(f0 + q) * Nb + b) : 0u;
                }
            };
            load_entries(0, un);
            for (int c = 0; c < nch && ok; ++c) {
                const int st = c & 1;
                if (st == 0) drain(&bar[0], waited0, issued0);   // the MMAs that last read
                else drain(&bar[1], waited1, issued1);           // this stage
                uint32_t u[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) u[q] = un[q];
                if (c + 1 < nch) load_entries(c + 1, un);
                // this thread's 16 types: r = 2c + half, s = 0..15
                const int r = 2 * c + half;
                float g[16];
#pragma unroll
                for (int s = 0; s < 16; ++s) g[s] = 0.0f;
                if (live && r < n && ((bm >> r) & 1u)) {
                    const float diag = prow[b];           // the diagonal pair (r, r)
#pragma unroll
                    for (int s = 0; s < 16; ++s) {
                        float v = 0.0f;
                        if (u[s]) {
                            const float pv = prow[u[s] & 0xFFFFu];
                            v = (u[s] >> 31) ? -pv : pv;
                        } else if (s == r) {
                            v = diag;
                        }
                        g[s] = v;
                        dsum = fmaf(Wd[r * 16 + s], v, dsum);
                    }
                }
                unsigned char *Ah = stg + st * kStage, *Al = Ah + kABytes;
                unsigned char *Bh = Al + kABytes, *Bl = Bh + kBBytes;
                if (gb) {
#pragma unroll
                    for (int s4 = 0; s4 < 4; ++s4) {
                        float4 h, l;
                        split(g[4 * s4 + 0], h.x, l.x);
                        split(g[4 * s4 + 1], h.y, l.y);
                        split(g[4 * s4 + 2], h.z, l.z);
                        split(g[4 * s4 + 3], h.w, l.w);
                        const uint32_t off = kmaj(col, half * 16 + 4 * s4, kSbo);
                        *reinterpret_cast<float4 *>(Bh + off) = h;
                        *reinterpret_cast<float4 *>(Bl + off) = l;
                    }
                } else if (warp < kIssueWarp) {
                    // this chunk's 64 x 32 block of W_J, split: a warp writes
                    // one whole 8 x 4 core matrix (128 contiguous bytes) per step
                    const int w4 = warp - kGThreadsTc / 32;
#pragma unroll
                    for (int e = 0; e < (kTcM * kTcKc) / (32 * kAWarps); ++e) {
                        const int core = w4 + e * kAWarps;                 // 0 .. 63
                        const int m = (core >> 3) * 8 + (lane >> 2);       // 8 cores along K per row group
                        const int k = (core & 7) * 4 + (lane & 3);
                        float hi, lo;
                        split(Wf[m * kWRow + c * kTcKc + k], hi, lo);
                        const uint32_t off = uint32_t(core) * 128u + uint32_t(lane) * 4u;
                        *reinterpret_cast<float *>(Ah + off) = hi;
                        *reinterpret_cast<float *>(Al + off) = lo;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                ok = __syncthreads_and(ok) != 0;      // block-uniform from here
                if (!ok) break;
                // the issuing warp builds nothing: its wait for the tensor
                // cores to accept the MMAs stays off the builders' path
                if (warp == kIssueWarp && lane == 0 && issue) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t ah = saddr(Ah), al = saddr(Al), bh = saddr(Bh), bl = saddr(Bl);
#pragma unroll
                    for (int ks = 0; ks < kTcKc / 8; ++ks) {
                        const uint32_t ko = uint32_t(ks) * 256u;
                        mma(tmem, sdesc(ah + ko, kSbo), sdesc(bh + ko, kSbo), first ? 0u : 1u);
                        mma(tmem, sdesc(ah + ko, kSbo), sdesc(bl + ko, kSbo), 1u);
                        mma(tmem, sdesc(al + ko, kSbo), sdesc(bh + ko, kSbo), 1u);
                        first = false;
                    }
                    commit(&bar[st]);
                }
                first = false;
                if (st == 0) ++issued0; else ++issued1;
            }
            if (gb) dpart[half * kTcN + col] = dsum;
            drain(&bar[0], waited0, issued0);
            drain(&bar[1], waited1, issued1);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            ok = __syncthreads_and(ok) != 0;
            if (!ok) break;
            // epilogue: rows 16w .. 16w + 15 sit in lanes 0..15 of sub-partition w
            if (warp < 4) {
                const int m = warp * 16 + lane;
                const uint32_t rowaddr = tmem + (uint32_t(warp * 32) << 16);
#pragma unroll
                for (int cb = 0; cb < kTcN / 32; ++cb) {
                    float v[32];
                    tmem_ld32(rowaddr + uint32_t(cb * 32), v);
                    if (lane < 16 && m < nexa) {
                        float *dst = a.T + (J * slots + m) * a.Nbp + b0 + cb * 32;
#pragma unroll
                        for (int i = 0; i < 32; i += 4)
                            if (b0 + cb * 32 + i + 3 < Nb)
                                *reinterpret_cast<float4 *>(dst + i) =
                                    make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                            else
                                for (int q = 0; q < 4; ++q)
                                    if (b0 + cb * 32 + i + q < Nb) dst[i + q] = v[i + q];
                    }
                }
            } else if (tid < 128 + kTcN) {
                const int cc = tid - 128;
                if (b0 + cc < Nb)
                    a.T[(J * slots + nexa) * a.Nbp + b0 + cc] = dpart[cc] + dpart[kTcN + cc];
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }
    // on a timeout, give the MMAs still in flight a bounded chance to finish
    if (!ok) {
        while (waited0 < issued0) wait_bar(&bar[0], (waited0++) & 1u, spin_limit);
        while (waited1 < issued1) wait_bar(&bar[1], (waited1++) & 1u, spin_limit);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     ::"r"(tmem), "r"(kTmemCols));
}

cudaError_t coupling_tc(const CplDenseArgs &a, int *status, long long spin_limit, int issue,
                        int num_sms, cudaStream_t st)
{
    if (a.Na == 0 || a.Nb == 0) return cudaSuccess;
    if (a.nexa > kTcM || a.n > 16) return cudaErrorInvalidValue;
    const size_t smem = cpl_tc_smem(a.Nb);
    cudaError_t err = cudaFuncSetAttribute(k_cpl_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(smem));
    if (err != cudaSuccess) return err;
    if (a.nJ == 0) return cudaSuccess;
    int64_t grid = num_sms;
    if (grid > a.nJ) grid = a.nJ;
    k_cpl_tc<<<unsigned(grid), kTcThreads, smem, st>>>(a, status, spin_limit, issue);
    hy::count_launch();
    return cudaGetLastError();
}

}  // namespace k
}  // namespace hy
