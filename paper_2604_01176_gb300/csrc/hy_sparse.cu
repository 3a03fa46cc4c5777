// hy_sparse.cu -- the sparse-state path (paper: Sparse State-Vector
// Emulation section -- the state is stored sparse, starts from the single
// Hartree-Fock determinant, and H is applied as a sparse matrix to a sparse
// vector).  Early in ADAPT-VQE psi = prod exp(theta A) |HF> has few nonzero
// amplitudes (exact zeros stay exactly zero under the pair rotations), so:
//   * k_support lists the nonzero amplitudes (warp-aggregated compaction);
//   * k_hpsi_scatter computes sigma = H psi by scattering every nonzero
//     amplitude to all determinants H connects it to (same folded tables
//     and coefficients as the dense sweep, read column-wise; H is real
//     symmetric), with atomic adds into a zeroed sigma;
//   * k_grad_sparse evaluates g_k = 2 <sigma|A_k psi> over the pairs with an
//     endpoint in the support only, applying each constituent's operator
//     string to the determinant's bits (Jordan-Wigner signs) and ranking the
//     partner with the binomial table.
#include "hy_kernels.cuh"

namespace hy {
namespace k {

template <typename T>
__global__ void __launch_bounds__(256)
k_support(const T *__restrict__ psi, int64_t N, int64_t *__restrict__ list, int64_t cap,
          unsigned long long *__restrict__ count)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t Nr = (N + 31) / 32 * 32;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < Nr; i += stride) {
        const bool nz = i < N && psi[i] != T(0);
        const unsigned m = __ballot_sync(0xffffffffu, nz);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (nz) {
            const unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
            if (int64_t(pos) < cap) list[pos] = i;
        }
    }
}

template <typename T>
__device__ __forceinline__ T sum_diag(const T *V, int n, int nn, uint32_t mask, int rs)
{
    T v = T(0);
    for (uint32_t m = mask; m; m &= m - 1) {
        const int p = __ffs(m) - 1;
        v += V[size_t(p * n + p) * nn + rs];
    }
    return v;
}

// one CTA per support entry (grid-stride)
template <typename T>
__global__ void __launch_bounds__(256)
k_hpsi_scatter(SparseArgs<T> a)
{
    const int n = a.n, nn = n * n;
    const int64_t Nb = a.Nb;
    const int ne = a.nexa + 1, nf = a.nexb + 1;
    for (int64_t t = blockIdx.x; t < a.m; t += gridDim.x) {
        const int64_t d = a.list[t];
        const T x = a.psi[d];
        const int64_t A = d / Nb, B = d % Nb;
        for (int k = a.Ma_ptr[A] + threadIdx.x; k < a.Ma_ptr[A + 1]; k += blockDim.x)
            atomicAdd(a.sigma + int64_t(a.Ma_col[k]) * Nb + B, a.Ma_val[k] * x);
        for (int k = a.Mb_ptr[B] + threadIdx.x; k < a.Mb_ptr[B + 1]; k += blockDim.x)
            atomicAdd(a.sigma + A * Nb + a.Mb_col[k], a.Mb_val[k] * x);
        const uint32_t am = a.astr[A], bm = a.bstr[B];
        for (int idx = threadIdx.x; idx < ne * nf; idx += blockDim.x) {
            const int e = idx / nf - 1, f = idx % nf - 1;
            int64_t Ao = A, Bo = B;
            int p = 0, q = 0, r = 0, s = 0;
            bool neg = false;
            if (e >= 0) {   // output alpha string: A with its entry e applied
                const uint32_t u = a.aex[A * a.nexa + e];
                Ao = u & 0xFFFFu;
                p = (u >> 20) & 15;   // created on the output (held by Ao)
                q = (u >> 16) & 15;   // held by A
                neg ^= (u >> 31) != 0;
            }
            if (f >= 0) {
                const uint32_t w = a.bexT[size_t(f) * Nb + B];
                Bo = w & 0xFFFFu;
                r = (w >> 20) & 15;
                s = (w >> 16) & 15;
                neg ^= (w >> 31) != 0;
            }
            T c;
            if (e >= 0 && f >= 0) {
                c = a.V[size_t(p * n + q) * nn + r * n + s];
            } else if (e >= 0) {
                c = T(0);
                for (uint32_t m = bm; m; m &= m - 1) {
                    const int rr = __ffs(m) - 1;
                    c += a.V[size_t(p * n + q) * nn + rr * n + rr];
                }
            } else if (f >= 0) {
                c = sum_diag<T>(a.V, n, nn, am, r * n + s);
            } else {
                c = T(0);
                for (uint32_t m = bm; m; m &= m - 1) {
                    const int rr = __ffs(m) - 1;
                    c += sum_diag<T>(a.V, n, nn, am, rr * n + rr);
                }
            }
            if (neg) c = -c;
            atomicAdd(a.sigma + Ao * Nb + Bo, c * x);
        }
    }
}

__device__ __forceinline__ uint32_t rank_bits(uint32_t m, const uint32_t (*C)[33])
{
    uint32_t r = 0;
    int i = 0;
    for (; m; m &= m - 1, ++i) r += C[__ffs(m) - 1][i + 1];
    return r;
}

// Apply an operator string (application order; codes 2*mode + dagger) to a
// determinant mask; false if it annihilates it.  Sign: (-1)^(occupied modes
// below) per operator (Jordan-Wigner, blocked order).
__device__ __forceinline__ bool apply_string(const int *code, int len, uint64_t &mask, int &sg)
{
    for (int t = 0; t < len; ++t) {
        const int mode = code[t] >> 1, dag = code[t] & 1;
        const uint64_t bit = 1ull << mode;
        if (((mask & bit) != 0) == (dag != 0)) return false;
        if (__popcll(mask & (bit - 1)) & 1) sg = -sg;
        mask ^= bit;
    }
    return true;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_grad_sparse(SparseGradArgs<T> a)
{
    __shared__ uint32_t C[33][33];
    __shared__ double red[256];
    for (int i = threadIdx.x; i < 33 * 33; i += blockDim.x) C[i / 33][i % 33] = a.binom33[i];
    __syncthreads();
    const int n = a.n;
    const uint64_t lowm = (1ull << n) - 1;
    for (int64_t i = blockIdx.x; i < a.n_ops; i += gridDim.x) {
        const int k = a.ops ? a.ops[i] : int(i);
        const int32_t *dsc = a.desc + 11 * k;
        double tot = 0.0;
        for (int c = 0; c < dsc[0]; ++c) {
            const int32_t *q = dsc + 1 + 5 * c;
            int fw[4], bw[4], len;
            if (q[0] == 1) {            // a+_{c0} a_{a0}
                fw[0] = 2 * q[4]; fw[1] = 2 * q[1] + 1;
                bw[0] = 2 * q[1]; bw[1] = 2 * q[4] + 1;
                len = 2;
            } else {                    // a+_{c0} a+_{c1} a_{a1} a_{a0}
                fw[0] = 2 * q[4]; fw[1] = 2 * q[3]; fw[2] = 2 * q[2] + 1; fw[3] = 2 * q[1] + 1;
                bw[0] = 2 * q[1]; bw[1] = 2 * q[2]; bw[2] = 2 * q[3] + 1; bw[3] = 2 * q[4] + 1;
                len = 4;
            }
            for (int64_t t = threadIdx.x; t < a.m; t += blockDim.x) {
                const int64_t d = a.list[t];
                const double x = double(a.psi[d]);
                const uint64_t mask = uint64_t(a.astr[d / a.Nb]) | (uint64_t(a.bstr[d % a.Nb]) << n);
                uint64_t o = mask;
                int sg = 1;
                if (apply_string(fw, len, o, sg)) {       // d is the domain end
                    const int64_t d2 = int64_t(rank_bits(uint32_t(o & lowm), C)) * a.Nb +
                                       rank_bits(uint32_t(o >> n), C);
                    tot += sg * (double(a.sigma[d2]) * x - double(a.sigma[d]) * double(a.psi[d2]));
                    continue;
                }
                o = mask;
                sg = 1;
                if (apply_string(bw, len, o, sg)) {       // d is the image end
                    const int64_t d0 = int64_t(rank_bits(uint32_t(o & lowm), C)) * a.Nb +
                                       rank_bits(uint32_t(o >> n), C);
                    if (a.psi[d0] == T(0)) tot -= sg * double(a.sigma[d0]) * x;
                }
            }
        }
        red[threadIdx.x] = tot;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
            __syncthreads();
        }
        if (threadIdx.x == 0) a.g[i] = 2.0 * red[0];
        __syncthreads();
    }
}

template <typename T>
cudaError_t support(const T *psi, int64_t N, int64_t *list, int64_t cap,
                    unsigned long long *count, int num_sms, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    int64_t g = (N + 255) / 256;
    if (g > int64_t(num_sms) * 16) g = int64_t(num_sms) * 16;
    if (g < 1) g = 1;
    k_support<T><<<unsigned(g), 256, 0, st>>>(psi, N, list, cap, count); hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t hpsi_scatter(const SparseArgs<T> &a, int num_sms, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(a.sigma, 0, size_t(a.Na) * a.Nb * sizeof(T), st);
    if (e != cudaSuccess || a.m == 0) return e;
    int64_t g = a.m;
    if (g > int64_t(num_sms) * 32) g = int64_t(num_sms) * 32;
    k_hpsi_scatter<T><<<unsigned(g), 256, 0, st>>>(a); hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t grad_sparse(const SparseGradArgs<T> &a, int num_sms, cudaStream_t st)
{
    if (a.n_ops == 0) return cudaSuccess;
    int64_t g = a.n_ops;
    if (g > int64_t(num_sms) * 16) g = int64_t(num_sms) * 16;
    k_grad_sparse<T><<<unsigned(g), 256, 0, st>>>(a); hy::count_launch();
    return cudaGetLastError();
}

template cudaError_t support<double>(const double *, int64_t, int64_t *, int64_t,
                                     unsigned long long *, int, cudaStream_t);
template cudaError_t support<float>(const float *, int64_t, int64_t *, int64_t,
                                    unsigned long long *, int, cudaStream_t);
template cudaError_t hpsi_scatter<double>(const SparseArgs<double> &, int, cudaStream_t);
template cudaError_t hpsi_scatter<float>(const SparseArgs<float> &, int, cudaStream_t);
template cudaError_t grad_sparse<double>(const SparseGradArgs<double> &, int, cudaStream_t);
template cudaError_t grad_sparse<float>(const SparseGradArgs<float> &, int, cudaStream_t);

}  // namespace k
}  // namespace hy
