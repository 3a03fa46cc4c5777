// hy_fold.cu -- the same-spin kernel tables built on the GPU from the
// Jordan-Wigner Pauli table (paper: Sparse State-Vector Emulation section --
// the Hamiltonian is the sum of the mapped fermionic terms, here grouped by
// X-mask).  For one spin, row r of M is the string K = str[r]; its candidate
// columns are K itself, every single excitation and every double excitation
// of K within the spin; the element <K|H|J> of the Pauli table is
//   sum over the terms of the group with X-mask K ^ J of c (-1)^|J & z|
// (J placed on the spin's qubits), summed in the table's term order -- the
// same quantity, in the same order, as the host's PauliTable::element, so
// the device tables equal a host evaluation bit for bit.  Zero elements are
// dropped and each row is sorted by column.
//
//   k_fold_rows: a CTA per row -- every candidate evaluated by one thread,
//     kept entries sorted (bitonic, in shared memory) into a fixed-stride
//     scratch row;
//   k_fold_scan: row pointers (one block);
//   k_fold_compact: the CSR in double and in float.
#include <climits>

#include "hy_kernels.cuh"

namespace hy {
namespace k {

namespace {

constexpr int kFoldThreads = 256;
constexpr int kFoldSlots = 1024;    // >= 1 + 64 + 28 * 28 candidates for n <= 16

__device__ __forceinline__ uint32_t fold_rank(uint32_t m, const uint32_t (*C)[33])
{
    uint32_t r = 0;
    int i = 0;
    for (; m; m &= m - 1, ++i) r += C[__ffs(m) - 1][i + 1];
    return r;
}

__global__ void __launch_bounds__(kFoldThreads)
k_fold_rows(FoldArgs a)
{
    __shared__ uint32_t C[33][33];
    __shared__ int32_t kcol[kFoldSlots];
    __shared__ double kval[kFoldSlots];
    __shared__ uint8_t opi[128], opj[128], vpa[128], vpb[128];   // pair index -> list positions
    __shared__ int occ[16], vir[16];
    __shared__ int kept;
    for (int i = threadIdx.x; i < 33 * 33; i += blockDim.x) C[i / 33][i % 33] = a.binom33[i];
    const int n = a.n, no = a.k, nv = a.n - a.k;
    const int po = no * (no - 1) / 2, pv = nv * (nv - 1) / 2;
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < no; ++i)
            for (int j = i + 1; j < no; ++j, ++t) { opi[t] = uint8_t(i); opj[t] = uint8_t(j); }
        t = 0;
        for (int x = 0; x < nv; ++x)
            for (int y = x + 1; y < nv; ++y, ++t) { vpa[t] = uint8_t(x); vpb[t] = uint8_t(y); }
    }
    const int ns = no * nv, cap = 1 + ns + po * pv;
    __syncthreads();
    for (int64_t r = blockIdx.x; r < a.N; r += gridDim.x) {
        const uint32_t K = a.str[r];
        if (threadIdx.x == 0) {
            int io = 0, iv = 0;
            for (int p = 0; p < n; ++p) {
                if ((K >> p) & 1) occ[io++] = p; else vir[iv++] = p;
            }
            kept = 0;
        }
        __syncthreads();
        const uint64_t ketshift = uint64_t(a.shift);
        for (int s = threadIdx.x; s < kFoldSlots; s += blockDim.x) {
            int32_t col = INT_MAX;
            double v = 0.0;
            if (s < cap) {
                uint32_t J = K;
                if (s > 0 && s <= ns) {
                    const int i = (s - 1) / nv, x = (s - 1) % nv;
                    J = K ^ (1u << occ[i]) ^ (1u << vir[x]);
                } else if (s > ns) {
                    const int d = s - 1 - ns, ij = d / pv, ab = d % pv;
                    J = K ^ (1u << occ[opi[ij]]) ^ (1u << occ[opj[ij]]) ^ (1u << vir[vpa[ab]]) ^
                        (1u << vir[vpb[ab]]);
                }
                const int32_t g = a.grp[K ^ J];
                if (g >= 0) {
                    const uint64_t ket = uint64_t(J) << ketshift;
                    for (int64_t t = a.goff[g]; t < a.goff[g + 1]; ++t)
                        v += (__popcll(ket & a.z[t]) & 1) ? -a.c[t] : a.c[t];
                }
                if (s == 0) v -= a.sub_diag;
                if (v != 0.0) {
                    col = int32_t(fold_rank(J, C));
                    atomicAdd(&kept, 1);
                }
            }
            kcol[s] = col;
            kval[s] = v;
        }
        __syncthreads();
        // bitonic sort of the slots by column (dropped candidates carry
        // INT_MAX and end up behind the kept entries; columns are distinct)
        for (int size = 2; size <= kFoldSlots; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = threadIdx.x; i < kFoldSlots / 2; i += blockDim.x) {
                    const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                    const bool up = (lo & size) == 0;
                    const int32_t cl = kcol[lo], ch = kcol[hi];
                    if ((cl > ch) == up) {
                        kcol[lo] = ch;
                        kcol[hi] = cl;
                        const double vl = kval[lo];
                        kval[lo] = kval[hi];
                        kval[hi] = vl;
                    }
                }
                __syncthreads();
            }
        const int cnt = kept;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            a.tcol[r * a.stride + e] = kcol[e];
            a.tval[r * a.stride + e] = kval[e];
        }
        if (threadIdx.x == 0) a.len[r] = cnt;
        __syncthreads();
    }
}

// ptr[0] = 0, ptr[r + 1] = ptr[r] + len[r]: one block, chunks of its size
__global__ void __launch_bounds__(1024)
k_fold_scan(const int32_t *__restrict__ len, int64_t N, int32_t *__restrict__ ptr)
{
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) {
        carry = 0;
        ptr[0] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t base = 0; base < N; base += blockDim.x) {
        const int64_t r = base + threadIdx.x;
        int32_t x = r < N ? len[r] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t acc = 0;
            for (int i = 0; i < int(blockDim.x >> 5); ++i) {
                const int32_t t = wsum[i];
                wsum[i] = acc;
                acc += t;
            }
        }
        __syncthreads();
        if (r < N) ptr[r + 1] = carry + wsum[w] + x;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += wsum[w] + x;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
k_fold_compact(FoldArgs a, const int32_t *__restrict__ ptr, int32_t *__restrict__ col,
               double *__restrict__ val64, float *__restrict__ val32)
{
    for (int64_t r = blockIdx.x; r < a.N; r += gridDim.x) {
        const int32_t base = ptr[r], cnt = a.len[r];
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const double v = a.tval[r * a.stride + e];
            col[base + e] = a.tcol[r * a.stride + e];
            val64[base + e] = v;
            val32[base + e] = float(v);
        }
    }
}

}  // namespace

int fold_candidates(int n, int k)
{
    const int no = k, nv = n - k;
    return 1 + no * nv + (no * (no - 1) / 2) * (nv * (nv - 1) / 2);
}

cudaError_t fold_rows(const FoldArgs &a, int num_sms, cudaStream_t st)
{
    if (a.n > 16 || fold_candidates(a.n, a.k) > kFoldSlots || a.stride < fold_candidates(a.n, a.k))
        return cudaErrorInvalidValue;
    if (a.N == 0) return cudaSuccess;
    int64_t g = a.N < int64_t(num_sms) * 8 ? a.N : int64_t(num_sms) * 8;
    k_fold_rows<<<unsigned(g), kFoldThreads, 0, st>>>(a); hy::count_launch();
    return cudaGetLastError();
}

cudaError_t fold_compact(const FoldArgs &a, int32_t *ptr, int32_t *col, double *val64,
                         float *val32, int num_sms, cudaStream_t st)
{
    k_fold_scan<<<1, 1024, 0, st>>>(a.len, a.N, ptr); hy::count_launch();
    if (a.N == 0) return cudaGetLastError();
    int64_t g = a.N < int64_t(num_sms) * 8 ? a.N : int64_t(num_sms) * 8;
    k_fold_compact<<<unsigned(g), 256, 0, st>>>(a, ptr, col, val64, val32); hy::count_launch();
    return cudaGetLastError();
}

}  // namespace k
}  // namespace hy
