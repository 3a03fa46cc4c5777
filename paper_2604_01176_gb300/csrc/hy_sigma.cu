// hy_sigma.cu -- sigma = H psi on Omega_CIk (paper: the sparse Hamiltonian
// times sparse state-vector product of the Sparse State-Vector Emulation
// section), computed matrix-free from the kernel tables folded out of the
// Jordan-Wigner X-mask groups:
//
//   sigma[a'][b'] = sum_J Ma[a'][J] psi[J][b']                 (alpha part)
//                 + sum_J Mb[b'][J] psi[a'][J]                 (beta part)
//                 + sum_{(p,q) in X(a')} sum_{(r,s) in X(b')}
//                       sa * sb * V[p][q][r][s] * psi[a'^pq][b'^rs]
//
// psi is row-major [N_alpha][N_beta].  The alpha part is a sparse-times-dense
// product whose rows of psi are read contiguously; the beta part is the same
// product on the transposed state; the alpha-beta coupling stages one
// partner row of psi in shared memory per alpha excitation of the output
// row and gathers the beta partners from it.
#include "hy_kernels.cuh"

namespace hy {
namespace k {

// ---------------------------------------------------------------------------
// Y = M X (or Y += M X) with M in CSR over strings and X, Y row-major
// [rows][ncols].  Grid: x = output row (so all rows of one column tile run
// together and the tile of X stays in L2), y = column tile.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_spmm(const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
       const T *__restrict__ val, const T *__restrict__ X, T *__restrict__ Y,
       int64_t ncols, int accumulate)
{
    const int64_t r = blockIdx.x;
    const int64_t c = int64_t(blockIdx.y) * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    const int beg = ptr[r], end = ptr[r + 1];
    T s0 = T(0), s1 = T(0);
    int kk = beg;
    for (; kk + 1 < end; kk += 2) {
        s0 += val[kk] * X[int64_t(col[kk]) * ncols + c];
        s1 += val[kk + 1] * X[int64_t(col[kk + 1]) * ncols + c];
    }
    if (kk < end) s0 += val[kk] * X[int64_t(col[kk]) * ncols + c];
    const T s = s0 + s1;
    T *y = Y + r * ncols + c;
    if (accumulate) *y += s; else *y = s;
}

template <typename T>
cudaError_t spmm(const int32_t *ptr, const int32_t *col, const T *val,
                 int64_t rows, const T *X, T *Y, int64_t ncols, bool accumulate,
                 cudaStream_t st)
{
    if (rows == 0 || ncols == 0) return cudaSuccess;
    dim3 grid(unsigned(rows), unsigned((ncols + 255) / 256));
    k_spmm<T><<<grid, 256, 0, st>>>(ptr, col, val, X, Y, ncols, accumulate ? 1 : 0); hy::count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// out[c][r] = in[r][c]   and   sigma[r][c] += tau[c][r]
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_transpose(const T *__restrict__ in, T *__restrict__ out, int64_t R, int64_t C)
{
    __shared__ T tile[32][33];
    const int64_t c0 = int64_t(blockIdx.x) * 32, r0 = int64_t(blockIdx.y) * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int j = ty; j < 32; j += 8) {
        int64_t r = r0 + j, c = c0 + tx;
        if (r < R && c < C) tile[j][tx] = in[r * C + c];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        int64_t c = c0 + j, r = r0 + tx;
        if (r < R && c < C) out[c * R + r] = tile[tx][j];
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_add_transposed(const T *__restrict__ tau, T *__restrict__ sigma, int64_t R,
                 int64_t C)
{
    __shared__ T tile[32][33];
    const int64_t r0 = int64_t(blockIdx.x) * 32, c0 = int64_t(blockIdx.y) * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int j = ty; j < 32; j += 8) {         // tau is [C][R]
        int64_t c = c0 + j, r = r0 + tx;
        if (r < R && c < C) tile[j][tx] = tau[c * R + r];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        int64_t r = r0 + j, c = c0 + tx;
        if (r < R && c < C) sigma[r * C + c] += tile[tx][j];
    }
}

template <typename T>
cudaError_t transpose(const T *in, T *out, int64_t R, int64_t C, cudaStream_t st)
{
    if (R == 0 || C == 0) return cudaSuccess;
    dim3 grid(unsigned((C + 31) / 32), unsigned((R + 31) / 32)), block(32, 8);
    k_transpose<T><<<grid, block, 0, st>>>(in, out, R, C); hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t add_transposed(const T *tau, T *sigma, int64_t R, int64_t C,
                           cudaStream_t st)
{
    if (R == 0 || C == 0) return cudaSuccess;
    dim3 grid(unsigned((R + 31) / 32), unsigned((C + 31) / 32)), block(32, 8);
    k_add_transposed<T><<<grid, block, 0, st>>>(tau, sigma, R, C); hy::count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// alpha-beta coupling.  One CTA per output alpha row a' (grid-stride).  For
// each partner entry e of a' -- the diagonal (partner a' itself, coefficient
// sum_{p in a'} V[p][p][.][.]) and each single excitation (p, q) (partner
// a'^pq, coefficient sa V[p][q][.][.]) -- the partner row of psi is staged
// in shared memory, the n*n coefficient slice likewise, and every output
// column b' accumulates its diagonal beta term plus its nexb beta
// excitations gathered from the staged row.
//
// Shared-memory staging is done in 32-bit planes: a double is kept as two
// separate arrays of low and high words, so each random gather is two
// 4-byte loads (one bank each) instead of one 8-byte load spanning two
// banks, which conflicts about twice as often.
// ---------------------------------------------------------------------------
template <typename T>
struct Planes;

template <>
struct Planes<float> {
    static constexpr int kWords = 1;
    __device__ static void put(uint32_t *base, int64_t stride, int64_t i, float v)
    {
        base[i] = __float_as_uint(v);
    }
    __device__ static float get(const uint32_t *base, int64_t stride, int64_t i)
    {
        return __uint_as_float(base[i]);
    }
};

template <>
struct Planes<double> {
    static constexpr int kWords = 2;
    __device__ static void put(uint32_t *base, int64_t stride, int64_t i, double v)
    {
        base[i] = uint32_t(__double2loint(v));
        base[stride + i] = uint32_t(__double2hiint(v));
    }
    __device__ static double get(const uint32_t *base, int64_t stride, int64_t i)
    {
        return __hiloint2double(int(base[stride + i]), int(base[i]));
    }
};

// Sign of a staged coefficient flipped by the excitation's sign bit (bit
// 31 of the packed entry) with an integer XOR on the high word, so no
// floating-point instruction is spent on it.
template <typename T>
__device__ __forceinline__ T coef_signed(const uint32_t *C, int nn, int rt, uint32_t sbit);
template <>
__device__ __forceinline__ float coef_signed<float>(const uint32_t *C, int, int rt, uint32_t sbit)
{
    return __uint_as_float(C[rt] ^ sbit);
}
template <>
__device__ __forceinline__ double coef_signed<double>(const uint32_t *C, int nn, int rt,
                                                      uint32_t sbit)
{
    return __hiloint2double(int(C[nn + rt] ^ sbit), int(C[rt]));
}

// Shared memory of the coupling kernel: row planes [W*Nb] | coefficient
// planes [W*n*n] | Cdiag [16] T | diagonal half-mask tables TL, TH [256] T.
// TL[m] (TH[m]) = sum of Cdiag[r] over the set bits r of m (of m shifted by
// 8), so the diagonal beta term of a column is TL[b & 255] + TH[b >> 8].
template <typename T>
size_t coupling_smem(int64_t Nb, int n)
{
    constexpr int W = sizeof(T) / 4;
    size_t words = size_t(W) * Nb + size_t(W) * n * n;
    words = (words + 3) / 4 * 4;
    return words * 4 + (16 + 512) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(1024, 1)
k_coupling(CouplingArgs<T> a, int cpt)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using PL = Planes<T>;
    constexpr int W = sizeof(T) / 4;
    const int64_t Nb = a.Nb;
    const int n = a.n, nn = n * n;
    uint32_t *row = reinterpret_cast<uint32_t *>(smem_raw);     // planes [Nb]
    uint32_t *C = row + W * Nb;                                 // planes [nn]
    size_t words = size_t(W) * Nb + size_t(W) * nn;
    words = (words + 3) / 4 * 4;
    T *Cdiag = reinterpret_cast<T *>(smem_raw + words * 4);     // [16]
    T *TL = Cdiag + 16, *TH = TL + 256;                         // [256] each
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t ar = blockIdx.x; ar < a.Na; ar += gridDim.x) {
        T acc[kCouplingMaxCpt];
#pragma unroll
        for (int j = 0; j < kCouplingMaxCpt; ++j) acc[j] = T(0);
        const uint32_t amask = a.astr[ar];
        for (int e = -1; e < a.nexa; ++e) {
            __syncthreads();
            int64_t Ja;
            if (e < 0) {
                Ja = ar;
                for (int rs = tid; rs < nn; rs += nt) {
                    T v = T(0);
                    for (uint32_t m = amask; m; m &= m - 1) {
                        const int p = __ffs(m) - 1;
                        v += a.V[size_t(p * n + p) * nn + rs];
                    }
                    PL::put(C, nn, rs, v);
                    if (rs / n == rs % n) Cdiag[rs / n] = v;
                }
            } else {
                const uint32_t u = a.aex[ar * a.nexa + e];
                Ja = u & 0xFFFFu;
                const int p = (u >> 16) & 15, q = (u >> 20) & 15;
                const bool neg = (u >> 31) != 0;
                for (int rs = tid; rs < nn; rs += nt) {
                    T v = a.V[size_t(p * n + q) * nn + rs];
                    v = neg ? -v : v;
                    PL::put(C, nn, rs, v);
                    if (rs / n == rs % n) Cdiag[rs / n] = v;
                }
            }
            for (int i = tid; i < 16 - n; i += nt) Cdiag[n + i] = T(0);
            const T *src = a.psi + Ja * Nb;
            for (int64_t b = tid; b < Nb; b += nt) PL::put(row, Nb, b, src[b]);
            __syncthreads();
            for (int i = tid; i < 512; i += nt) {
                const int m = i & 255, base = i < 256 ? 0 : 8;
                T v = T(0);
                for (int r = 0; r < 8; ++r)
                    if ((m >> r) & 1) v += Cdiag[base + r];
                (i < 256 ? TL : TH)[m] = v;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kCouplingMaxCpt; ++j) {
                const int64_t b = tid + int64_t(j) * nt;
                if (j < cpt && b < Nb) {
                    const uint32_t m = a.bstr[b];
                    const T d = TL[m & 255u] + TH[m >> 8];
                    T s = d * PL::get(row, Nb, b) + acc[j];
                    const uint32_t *bx = a.bexT + b;
#pragma unroll 4
                    for (int f = 0; f < a.nexb; ++f) {
                        const uint32_t u = bx[size_t(f) * Nb];
                        const int rt = ((u >> 16) & 15) * n + ((u >> 20) & 15);
                        const T cv = coef_signed<T>(C, nn, rt, u & 0x80000000u);
                        s += cv * PL::get(row, Nb, u & 0xFFFFu);
                    }
                    acc[j] = s;
                }
            }
        }
        T *dst = a.sigma + ar * Nb;
#pragma unroll
        for (int j = 0; j < kCouplingMaxCpt; ++j) {
            const int64_t b = tid + int64_t(j) * nt;
            if (j < cpt && b < Nb) dst[b] += acc[j];
        }
    }
}

template <typename T>
cudaError_t coupling(const CouplingArgs<T> &a, int num_sms, cudaStream_t st)
{
    if (a.Na == 0 || a.Nb == 0) return cudaSuccess;
    int threads = int(a.Nb < 1024 ? (a.Nb + 31) / 32 * 32 : 1024);
    const int cpt = int((a.Nb + threads - 1) / threads);
    if (cpt > kCouplingMaxCpt) return cudaErrorInvalidValue;
    const size_t smem = coupling_smem<T>(a.Nb, a.n);
    cudaError_t err = cudaFuncSetAttribute(
        k_coupling<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coupling<T>, threads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = int64_t(num_sms) * per_sm;
    if (grid > a.Na) grid = a.Na;
    k_coupling<T><<<unsigned(grid), threads, smem, st>>>(a, cpt); hy::count_launch();
    return cudaGetLastError();
}

template cudaError_t spmm<double>(const int32_t *, const int32_t *, const double *,
                                  int64_t, const double *, double *, int64_t, bool,
                                  cudaStream_t);
template cudaError_t spmm<float>(const int32_t *, const int32_t *, const float *,
                                 int64_t, const float *, float *, int64_t, bool,
                                 cudaStream_t);
template cudaError_t transpose<double>(const double *, double *, int64_t, int64_t,
                                       cudaStream_t);
template cudaError_t transpose<float>(const float *, float *, int64_t, int64_t,
                                      cudaStream_t);
template cudaError_t add_transposed<double>(const double *, double *, int64_t,
                                            int64_t, cudaStream_t);
template cudaError_t add_transposed<float>(const float *, float *, int64_t,
                                           int64_t, cudaStream_t);
template cudaError_t coupling<double>(const CouplingArgs<double> &, int,
                                      cudaStream_t);
template cudaError_t coupling<float>(const CouplingArgs<float> &, int,
                                     cudaStream_t);

}  // namespace k
}  // namespace hy
