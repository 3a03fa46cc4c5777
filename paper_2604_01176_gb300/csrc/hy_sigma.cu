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
template <typename T, int VEC>
struct VecOf;
template <> struct VecOf<float, 1> { using type = float; };
template <> struct VecOf<float, 2> { using type = float2; };
template <> struct VecOf<double, 1> { using type = double; };
template <> struct VecOf<double, 2> { using type = double2; };

template <typename T>
__device__ __forceinline__ void vfma(T &acc, T w, T x) { acc += w * x; }
__device__ __forceinline__ void vfma(float2 &acc, float w, float2 x)
{
    acc.x += w * x.x;
    acc.y += w * x.y;
}
__device__ __forceinline__ void vfma(double2 &acc, double w, double2 x)
{
    acc.x += w * x.x;
    acc.y += w * x.y;
}
template <typename V> __device__ __forceinline__ V vzero() { return V{}; }

// Each thread owns VEC consecutive columns (one vector load per partner row
// and nonzero), so the broadcast loads of the CSR value and column index
// are shared by VEC multiply-adds.
template <typename T, int VEC>
__global__ void __launch_bounds__(256)
k_spmm(const int32_t *__restrict__ ptr, const int32_t *__restrict__ col,
       const T *__restrict__ val, const T *__restrict__ X, T *__restrict__ Y,
       int64_t ncols, int accumulate)
{
    using V = typename VecOf<T, VEC>::type;
    const int64_t r = blockIdx.x;
    const int64_t c = (int64_t(blockIdx.y) * blockDim.x + threadIdx.x) * VEC;
    if (c >= ncols) return;
    const int beg = ptr[r], end = ptr[r + 1];
    V s0 = vzero<V>(), s1 = vzero<V>();
    int kk = beg;
    for (; kk + 1 < end; kk += 2) {
        vfma(s0, val[kk], *reinterpret_cast<const V *>(X + int64_t(col[kk]) * ncols + c));
        vfma(s1, val[kk + 1], *reinterpret_cast<const V *>(X + int64_t(col[kk + 1]) * ncols + c));
    }
    if (kk < end) vfma(s0, val[kk], *reinterpret_cast<const V *>(X + int64_t(col[kk]) * ncols + c));
    const T *a0 = reinterpret_cast<const T *>(&s0), *a1 = reinterpret_cast<const T *>(&s1);
    T *y = Y + r * ncols + c;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
        const T sv = a0[v] + a1[v];
        if (accumulate) y[v] += sv; else y[v] = sv;
    }
}

template <typename T>
cudaError_t spmm(const int32_t *ptr, const int32_t *col, const T *val,
                 int64_t rows, const T *X, T *Y, int64_t ncols, bool accumulate,
                 cudaStream_t st)
{
    if (rows == 0 || ncols == 0) return cudaSuccess;
    // two columns per thread when every row starts on a vector boundary
    const bool v2 = (ncols % 2 == 0) &&
                    (reinterpret_cast<uintptr_t>(X) % (2 * sizeof(T)) == 0) &&
                    (reinterpret_cast<uintptr_t>(Y) % (2 * sizeof(T)) == 0);
    if (v2) {
        dim3 grid(unsigned(rows), unsigned((ncols / 2 + 255) / 256));
        k_spmm<T, 2><<<grid, 256, 0, st>>>(ptr, col, val, X, Y, ncols, accumulate ? 1 : 0); hy::count_launch();
    } else {
        dim3 grid(unsigned(rows), unsigned((ncols + 255) / 256));
        k_spmm<T, 1><<<grid, 256, 0, st>>>(ptr, col, val, X, Y, ncols, accumulate ? 1 : 0); hy::count_launch();
    }
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
    for (int64_t ar = a.row0 + blockIdx.x; ar < a.row1; ar += gridDim.x) {
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
        T *dst = a.sigma + (ar - a.row0) * Nb;
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
    if (a.row1 <= a.row0 || a.Nb == 0) return cudaSuccess;
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
    if (grid > a.row1 - a.row0) grid = a.row1 - a.row0;
    k_coupling<T><<<unsigned(grid), threads, smem, st>>>(a, cpt); hy::count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// alpha-beta coupling in float as two dense phases.
//
// Phase A, per alpha string J (one CTA, grid-stride):
//   T[J][m][b'] = sum_t W_J[t][m] G_J[t][b']
// with t = r*n + s running over every beta excitation type (s = r: the
// diagonal pair), G_J[t][b'] = sign * psi[J][b' with r -> s] where that
// excitation exists for b' (else 0), and W_J[t][m] the coupling coefficient
// of output alpha row a_m = the m-th single-excitation partner of J
// (V[q][p][t] with J's entry (p, q), times its sign), or for m = nexa the
// diagonal coefficient sum_{p in J} V[p][p][t].  This is a dense product of
// a (nexa+1) x n^2 by an n^2 x N_beta matrix, tiled 72 x 128 with 8 x 4
// outputs per thread; each gathered amplitude is reused by all 65 output
// rows and each coefficient by every column.  Type rows that are zero for
// every column of a tile (no string of the tile holds r, or every string
// holds s) are skipped: the active set is taken from the OR / AND of the
// tile's beta strings.
//
// Phase B, per output alpha row a' (one CTA, grid-stride):
//   sigma[a'][b'] += T[a'][nexa][b'] + sum_e T[J_e][inv_e][b']
// where inv_e is the position of a' in the partner list of J_e; 65 coalesced
// row reads per output row, no atomics, fixed summation order.
// ---------------------------------------------------------------------------
constexpr int kGM = 72, kGN = 128, kGThreads = 288;

__global__ void __launch_bounds__(kGThreads, 1)
k_cpl_gemm(CplDenseArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t Nb = a.Nb;
    const int n = a.n, nn = n * n, nexa = a.nexa, nexb = a.nexb;
    const int slots = nexa + 1;
    float *W = reinterpret_cast<float *>(smem_raw);             // [nn][kGM]
    float *G = W + size_t(nn) * kGM;                            // [active][kGN]
    int16_t *act = reinterpret_cast<int16_t *>(G + size_t(nn) * kGN);   // [nn]
    int16_t *pos = act + 256;                                   // [nn] type -> row of G
    int *misc = reinterpret_cast<int *>(pos + 256);             // or, and, n_active, warp counts[9]
    const int tid = threadIdx.x, mg = tid >> 5, ng = tid & 31;
    for (int64_t jj = blockIdx.x; jj < a.nJ; jj += gridDim.x) {
        const int64_t J = a.jlist ? int64_t(a.jlist[jj]) : jj;
        __syncthreads();
        const float *src = a.psi + J * Nb;
        const uint32_t jm = a.astr[J];
        for (int idx = tid; idx < nn * kGM; idx += blockDim.x) {
            const int t = idx / kGM, m = idx % kGM;
            float v = 0.0f;
            if (m < nexa) {
                const uint32_t u = a.aex[J * nexa + m];
                const int pj = (u >> 16) & 15, qj = (u >> 20) & 15;
                v = a.V[size_t(qj * n + pj) * nn + t];
                if (u >> 31) v = -v;
            } else if (m == nexa) {
                for (uint32_t mm = jm; mm; mm &= mm - 1) {
                    const int p = __ffs(mm) - 1;
                    v += a.V[size_t(p * n + p) * nn + t];
                }
            }
            W[idx] = v;
        }
        for (int64_t b0 = 0; b0 < Nb; b0 += kGN) {
            __syncthreads();   // W ready; previous tile's G and lists consumed
            if (tid == 0) {
                misc[0] = 0;
                misc[1] = int(0xFFFFFFFFu >> (32 - n));
            }
            __syncthreads();
            if (tid < kGN && b0 + tid < Nb) {
                const int m = int(a.bstr[b0 + tid]);
                atomicOr(&misc[0], m);
                atomicAnd(&misc[1], m);
            }
            __syncthreads();
            // active superset: (r, r) with r in OR; (r, s) with r in OR, s not in AND
            const uint32_t om = uint32_t(misc[0]), am = uint32_t(misc[1]);
            int flag = 0, t = tid;
            if (t < nn) {
                const int r = t / n, s2 = t % n;
                flag = ((om >> r) & 1u) && (r == s2 || !((am >> s2) & 1u));
            }
            const unsigned bal = __ballot_sync(0xffffffffu, flag);
            if ((tid & 31) == 0) misc[3 + mg] = __popc(bal);
            __syncthreads();
            if (t < nn) {
                int base = 0;
                for (int w = 0; w < mg; ++w) base += misc[3 + w];
                const int p = base + __popc(bal & ((1u << (tid & 31)) - 1u));
                pos[t] = flag ? int16_t(p) : int16_t(-1);
                if (flag) act[p] = int16_t(t);
                if (tid == nn - 1) misc[2] = p + flag;
            }
            __syncthreads();
            const int na = misc[2];
            for (int idx = tid; idx < na * kGN; idx += blockDim.x) G[idx] = 0.0f;
            __syncthreads();
            // single-excitation entries: four per thread in flight (entry
            // loads first, then the amplitude loads), so the L2 latency of
            // the two dependent loads overlaps across entries
            constexpr int kU = 4;
            const int nsing = kGN * nexb;
            for (int base = tid; base < nsing; base += kU * blockDim.x) {
                uint32_t u[kU];
                bool ok[kU];
#pragma unroll
                for (int q = 0; q < kU; ++q) {
                    const int idx = base + q * blockDim.x;
                    const int nl = idx % kGN, f = idx / kGN;
                    ok[q] = idx < nsing && b0 + nl < Nb;
                    u[q] = ok[q] ? __ldg(a.bexT + size_t(f) * Nb + b0 + nl) : 0u;
                }
                float v[kU];
#pragma unroll
                for (int q = 0; q < kU; ++q) v[q] = ok[q] ? __ldg(src + (u[q] & 0xFFFFu)) : 0.0f;
#pragma unroll
                for (int q = 0; q < kU; ++q) {
                    if (!ok[q]) continue;
                    const int nl = (base + q * blockDim.x) % kGN;
                    const int r = (u[q] >> 16) & 15, sv = (u[q] >> 20) & 15;
                    G[pos[r * n + sv] * kGN + nl] = (u[q] >> 31) ? -v[q] : v[q];
                }
            }
            // diagonal types: one thread per column writes psi[J][b'] into the
            // (r, r) row of every occupied r
            if (tid < kGN && b0 + tid < Nb) {
                const int64_t b = b0 + tid;
                const float v = __ldg(src + b);
                for (uint32_t mm = __ldg(a.bstr + b); mm; mm &= mm - 1) {
                    const int r = __ffs(mm) - 1;
                    G[pos[r * n + r] * kGN + tid] = v;
                }
            }
            __syncthreads();
            float acc[8][4];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
            const float *wp = W + mg * 8;
            const float *gp = G + ng * 4;
            // operands of the next active type are loaded while the current
            // one is multiplied (register double buffering)
            float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), w1 = w0, g = w0;
            if (na > 0) {
                const int tt = act[0];
                w0 = *reinterpret_cast<const float4 *>(wp + tt * kGM);
                w1 = *reinterpret_cast<const float4 *>(wp + tt * kGM + 4);
                g = *reinterpret_cast<const float4 *>(gp);
            }
            for (int ai = 0; ai < na; ++ai) {
                float4 nw0 = w0, nw1 = w1, ngv = g;
                if (ai + 1 < na) {
                    const int tn = act[ai + 1];
                    nw0 = *reinterpret_cast<const float4 *>(wp + tn * kGM);
                    nw1 = *reinterpret_cast<const float4 *>(wp + tn * kGM + 4);
                    ngv = *reinterpret_cast<const float4 *>(gp + (ai + 1) * kGN);
                }
                const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    acc[i][0] += w[i] * g.x;
                    acc[i][1] += w[i] * g.y;
                    acc[i][2] += w[i] * g.z;
                    acc[i][3] += w[i] * g.w;
                }
                w0 = nw0;
                w1 = nw1;
                g = ngv;
            }
            const int64_t b = b0 + ng * 4;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int m = mg * 8 + i;
                if (m < slots && b + 3 < a.Nbp)
                    *reinterpret_cast<float4 *>(a.T + (J * slots + m) * a.Nbp + b) =
                        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            }
        }
    }
}

__global__ void __launch_bounds__(256)
k_cpl_gather(CplDenseArgs a)
{
    const int64_t Nb = a.Nb;
    const int nexa = a.nexa, slots = nexa + 1;
    for (int64_t ar = a.row0 + blockIdx.x; ar < a.row1; ar += gridDim.x) {
        for (int64_t b = threadIdx.x; b < Nb; b += blockDim.x) {
            float s = a.T[(ar * slots + nexa) * a.Nbp + b];
            for (int e = 0; e < nexa; ++e) {
                const int64_t J = a.aex[ar * nexa + e] & 0xFFFFu;
                const int m = a.inv[ar * nexa + e];
                s += a.T[(J * slots + m) * a.Nbp + b];
            }
            a.sigma[(ar - a.row0) * Nb + b] += s;
        }
    }
}

size_t cpl_dense_smem(int64_t Nb, int n)
{
    (void)Nb;
    // W [n^2][72] + G [n^2][128] floats, type lists 2 x 256 int16, 16 ints
    return size_t(n) * n * (kGM + kGN) * sizeof(float) + 2 * 256 * sizeof(int16_t) +
           16 * sizeof(int);
}

cudaError_t coupling_dense(const CplDenseArgs &a, int num_sms, cudaStream_t st)
{
    if (a.Na == 0 || a.Nb == 0) return cudaSuccess;
    if (a.nexa + 1 > kGM) return cudaErrorInvalidValue;
    const size_t smem = cpl_dense_smem(a.Nb, a.n);
    cudaError_t err = cudaFuncSetAttribute(k_cpl_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(smem));
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cpl_gemm, kGThreads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = int64_t(num_sms) * per_sm;
    if (grid > a.nJ) grid = a.nJ;
    if (grid > 0) {
        k_cpl_gemm<<<unsigned(grid), kGThreads, smem, st>>>(a);
        hy::count_launch();
    }
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return coupling_gather(a, num_sms, st);
}

cudaError_t coupling_gather(const CplDenseArgs &a, int num_sms, cudaStream_t st)
{
    if (a.row1 <= a.row0 || a.Nb == 0) return cudaSuccess;
    int64_t g2 = int64_t(num_sms) * 8;
    if (g2 > a.row1 - a.row0) g2 = a.row1 - a.row0;
    k_cpl_gather<<<unsigned(g2), 256, 0, st>>>(a); hy::count_launch();
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
