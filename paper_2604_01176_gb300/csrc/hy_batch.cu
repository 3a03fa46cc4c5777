// hy_batch.cu -- batched sigma = H psi (and energies) over many molecules of
// uneven size in ONE persistent launch.  The CTA is split into groups of
// `gsize` threads (a tile shape the autotuner picks); each group repeatedly
// takes the next task -- one output alpha row of one molecule -- from a
// device work-list (largest molecules first) through an atomic counter, and
// computes that row completely:
//   sigma[a'][b'] = sum_J Ma[a'][J] psi[J][b']                (alpha part)
//                 + sum_K Mb[b'][K] psi[a'][K]                (beta part)
//                 + sum_{e in X(a'), f in X(b')} C_e[f] psi[J_e][K_f]
// (the same exact decomposition as the single-molecule sweep in
// hy_sigma.cu, without the transposed beta pass, so no task depends on
// another and no workspace is needed).  Each task also writes the row's
// <psi|sigma> partial; a second tiny kernel sums them per molecule in a
// fixed order.  Meant for molecules up to 12 orbitals (N_beta <= 924),
// whose tables stay in L2.
#include "hy_kernels.cuh"

namespace hy {
namespace k {

__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    // named barrier per group (ids 1..15; 0 is __syncthreads)
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <typename T>
__device__ __forceinline__ T plane_get(const uint32_t *base, int stride, int i);
template <>
__device__ __forceinline__ float plane_get<float>(const uint32_t *base, int, int i)
{
    return __uint_as_float(base[i]);
}
template <>
__device__ __forceinline__ double plane_get<double>(const uint32_t *base, int stride, int i)
{
    return __hiloint2double(int(base[stride + i]), int(base[i]));
}
template <typename T>
__device__ __forceinline__ void plane_put(uint32_t *base, int stride, int i, T v);
template <>
__device__ __forceinline__ void plane_put<float>(uint32_t *base, int, int i, float v)
{
    base[i] = __float_as_uint(v);
}
template <>
__device__ __forceinline__ void plane_put<double>(uint32_t *base, int stride, int i, double v)
{
    base[i] = uint32_t(__double2loint(v));
    base[stride + i] = uint32_t(__double2hiint(v));
}

// staged coefficient with its sign flipped by an integer XOR of the sign bit
template <typename T>
__device__ __forceinline__ T sign_xor(const uint32_t *C, int stride, int i, uint32_t sbit);
template <>
__device__ __forceinline__ float sign_xor<float>(const uint32_t *C, int, int i, uint32_t sbit)
{
    return __uint_as_float(C[i] ^ sbit);
}
template <>
__device__ __forceinline__ double sign_xor<double>(const uint32_t *C, int stride, int i,
                                                   uint32_t sbit)
{
    return __hiloint2double(int(C[stride + i] ^ sbit), int(C[i]));
}

template <typename T>
__global__ void __launch_bounds__(1024)
k_batch_rows(BatchArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int W = sizeof(T) / 4;
    const int gsize = a.gsize;
    const int gid = threadIdx.x / gsize, lt = threadIdx.x % gsize;
    const int NB = a.nb_max, NN = a.nn_max;
    // per-group shared memory: acc [NB] T | row planes [W*NB] | C planes
    // [W*NN] | Cdiag [16] T | TL, TH [256] T each | task slot.  TL[m] (TH[m])
    // sums Cdiag over the set bits of m (of m shifted by 8), so a column's
    // diagonal beta term is TL[b & 255] + TH[b >> 8].
    const size_t gbytes = a.group_smem;
    unsigned char *gs = smem_raw + size_t(gid) * gbytes;
    T *acc = reinterpret_cast<T *>(gs);
    uint32_t *row = reinterpret_cast<uint32_t *>(acc + NB);
    uint32_t *C = row + W * NB;
    T *Cdiag = reinterpret_cast<T *>(C + W * NN);
    T *TL = Cdiag + 16, *TH = TL + 256;
    int *slot = reinterpret_cast<int *>(TH + 256);
    const int bar = gid + 1;
    for (;;) {
        if (lt == 0) *slot = atomicAdd(a.counter, 1);
        group_sync(bar, gsize);
        const int task = *slot;
        group_sync(bar, gsize);
        if (task >= a.n_tasks) break;
        const int2 tk = a.tasks[task];
        const BatchMol<T> m = a.mols[tk.x];
        const int64_t ar = tk.y;
        const int Nb = int(m.Nb), n = m.n, nn = n * n;
        const T *psi = a.psi + m.offset;
        T *sigma = a.sigma + m.offset;
        // alpha part (partner rows read from global, coalesced)
        for (int b = lt; b < Nb; b += gsize) {
            T s = T(0);
            for (int kk = m.Ma_ptr[ar]; kk < m.Ma_ptr[ar + 1]; ++kk)
                s += m.Ma_val[kk] * psi[int64_t(m.Ma_col[kk]) * Nb + b];
            acc[b] = s;
        }
        // stage row a' (the diagonal partner), diagonal coefficients
        const uint32_t amask = m.astr[ar];
        for (int b = lt; b < Nb; b += gsize) plane_put<T>(row, NB, b, psi[ar * Nb + b]);
        for (int rs = lt; rs < nn; rs += gsize) {
            T v = T(0);
            for (uint32_t mm = amask; mm; mm &= mm - 1) {
                const int p = __ffs(mm) - 1;
                v += m.V[size_t(p * n + p) * nn + rs];
            }
            plane_put<T>(C, NN, rs, v);
            if (rs / n == rs % n) Cdiag[rs / n] = v;
        }
        group_sync(bar, gsize);
        // beta part from the staged row
        for (int b = lt; b < Nb; b += gsize) {
            T s = T(0);
            for (int kk = m.Mb_ptr[b]; kk < m.Mb_ptr[b + 1]; ++kk)
                s += m.Mb_val[kk] * plane_get<T>(row, NB, m.Mb_col[kk]);
            acc[b] += s;
        }
        for (int e = -1; e < m.nexa; ++e) {
            if (e >= 0) {
                group_sync(bar, gsize);
                const uint32_t u = m.aex[ar * m.nexa + e];
                const int64_t Ja = u & 0xFFFFu;
                const int p = (u >> 16) & 15, q = (u >> 20) & 15;
                const bool neg = (u >> 31) != 0;
                for (int rs = lt; rs < nn; rs += gsize) {
                    T v = m.V[size_t(p * n + q) * nn + rs];
                    v = neg ? -v : v;
                    plane_put<T>(C, NN, rs, v);
                    if (rs / n == rs % n) Cdiag[rs / n] = v;
                }
                for (int b = lt; b < Nb; b += gsize)
                    plane_put<T>(row, NB, b, psi[Ja * Nb + b]);
                group_sync(bar, gsize);
            }
            for (int i = lt; i < 16 - n; i += gsize) Cdiag[n + i] = T(0);
            group_sync(bar, gsize);
            for (int i = lt; i < 512; i += gsize) {
                const int mm = i & 255, base = i < 256 ? 0 : 8;
                T v = T(0);
                for (int r = 0; r < 8; ++r)
                    if ((mm >> r) & 1) v += Cdiag[base + r];
                (i < 256 ? TL : TH)[mm] = v;
            }
            group_sync(bar, gsize);
            for (int b = lt; b < Nb; b += gsize) {
                const uint32_t mb = m.bstr[b];
                const T d = TL[mb & 255u] + TH[mb >> 8];
                T s = d * plane_get<T>(row, NB, b) + acc[b];
                for (int f = 0; f < m.nexb; ++f) {
                    const uint32_t u = m.bexT[int64_t(f) * Nb + b];
                    const int rt = ((u >> 16) & 15) * n + ((u >> 20) & 15);
                    s += sign_xor<T>(C, NN, rt, u & 0x80000000u) * plane_get<T>(row, NB, u & 0xFFFFu);
                }
                acc[b] = s;
            }
        }
        // write the row and its <psi|sigma> partial
        double part = 0.0;
        for (int b = lt; b < Nb; b += gsize) {
            const T v = acc[b];
            sigma[ar * Nb + b] = v;
            part += double(psi[ar * Nb + b]) * double(v);
        }
        if (a.row_energy) {
            // group reduction through the (now free) acc array, fixed order
            group_sync(bar, gsize);
            double *red = reinterpret_cast<double *>(acc);
            red[lt] = part;
            group_sync(bar, gsize);
            if (lt == 0) {
                double s = 0.0;
                for (int i = 0; i < gsize; ++i) s += red[i];
                a.row_energy[m.task_base + ar] = s;
            }
        }
        group_sync(bar, gsize);
    }
}

// energies[m] = sum of molecule m's row partials, in row order
__global__ void k_batch_energy(const double *__restrict__ row_energy,
                               const int64_t *__restrict__ base, const int64_t *__restrict__ rows,
                               int count, double *__restrict__ energies)
{
    const int mol = blockIdx.x * blockDim.x + threadIdx.x;
    if (mol >= count) return;
    double s = 0.0;
    for (int64_t r = 0; r < rows[mol]; ++r) s += row_energy[base[mol] + r];
    energies[mol] = s;
}

// ---------------------------------------------------------------------------
// Batched pool-gradient screen: g_k = 2 <sigma|A_k psi> for listed operators
// of many molecules in one persistent launch.  A task is one row chunk of one
// (molecule, operator) entry; CTAs take tasks through an atomic counter, and
// a task sums, over the chunk's rows of every constituent pattern pair of the
// operator, sb * sa * (sigma[d'] psi[d] - sigma[d] psi[d']) (the pairs of
// C - C^dagger), as the single-molecule screen does; a second kernel adds an
// entry's chunks in a fixed order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double batch_block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_batch_grad(BatchGradArgs<T> a)
{
    __shared__ double red[8];
    __shared__ long long sh_task;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sh_task = (long long)atomicAdd(a.counter, 1ull);
        __syncthreads();
        const int64_t task = sh_task;
        if (task >= a.n_tasks) break;
        const int64_t e = task / a.CH;
        const int chunk = int(task - e * a.CH);
        int lo = 0, hi = a.count;                 // molecule: base[m] <= e < base[m + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) / 2;
            if (a.base[mid] <= e) lo = mid; else hi = mid;
        }
        const BatchPool mp = a.mols[lo];
        const int64_t i = e - a.base[lo];
        const int k = a.ops ? a.ops[e] : int(i);
        if (refuse_op(e, k, mp.K, chunk == 0 ? a.bad : nullptr)) {
            if (threadIdx.x == 0) a.partials[task] = __longlong_as_double(0x7ff8000000000000ll);
            continue;
        }
        const T *psi = a.psi + mp.off, *sigma = a.sigma + mp.off;
        const OpDev od = mp.opd[k];
        double tot = 0.0;
        for (int c = 0; c < od.nc; ++c) {
            const ConsDev cd = mp.cons[c == 0 ? od.c0 : od.c1];
            const int64_t nrows = cd.ap < 0 ? mp.Na : mp.acnt[cd.ap];
            const int64_t ncols = cd.bp < 0 ? mp.Nb : mp.bcnt[cd.bp];
            const uint32_t *ae = cd.ap < 0 ? nullptr : mp.aent + mp.aoff[cd.ap];
            const uint32_t *be = cd.bp < 0 ? nullptr : mp.bent + mp.boff[cd.bp];
            T part = T(0);
            for (int64_t rr = chunk; rr < nrows; rr += a.CH) {
                int64_t A = rr, A2 = rr;
                T sa = T(1);
                if (ae) {
                    const uint32_t u = ae[rr];
                    A = u & 0x7FFFu;
                    A2 = (u >> 15) & 0x7FFFu;
                    if (u >> 31) sa = T(-1);
                }
                const T *pA = psi + A * mp.Nb, *pA2 = psi + A2 * mp.Nb;
                const T *sA = sigma + A * mp.Nb, *sA2 = sigma + A2 * mp.Nb;
                T rowpart = T(0);
                for (int64_t t = threadIdx.x; t < ncols; t += blockDim.x) {
                    int64_t B = t, B2 = t;
                    T sb = T(1);
                    if (be) {
                        const uint32_t u = be[t];
                        B = u & 0x7FFFu;
                        B2 = (u >> 15) & 0x7FFFu;
                        if (u >> 31) sb = T(-1);
                    }
                    rowpart += sb * (sA2[B2] * pA[B] - sA[B] * pA2[B2]);
                }
                part += sa * rowpart;
            }
            tot += double(cd.eps) * double(part);
        }
        tot = batch_block_sum(tot, red);
        if (threadIdx.x == 0) a.partials[task] = tot;
    }
}

__global__ void __launch_bounds__(256)
k_batch_grad_final(const double *__restrict__ partials, int CH, int64_t n, double *__restrict__ g)
{
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s = 0.0;
    for (int c = 0; c < CH; ++c) s += partials[e * CH + c];
    g[e] = 2.0 * s;
}

template <typename T>
cudaError_t batch_grad(const BatchGradArgs<T> &a, int grid, cudaStream_t st)
{
    const int64_t n = a.n_tasks / (a.CH > 0 ? a.CH : 1);
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_batch_grad<T><<<unsigned(grid), 256, 0, st>>>(a); hy::count_launch();
    k_batch_grad_final<<<unsigned((n + 255) / 256), 256, 0, st>>>(a.partials, a.CH, n, a.g);
    hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
size_t batch_group_smem(int nb_max, int nn_max, int gsize)
{
    constexpr int W = sizeof(T) / 4;
    size_t b = size_t(nb_max) * sizeof(T) + size_t(W) * nb_max * 4 + size_t(W) * nn_max * 4 +
               (16 + 512) * sizeof(T) + 16;
    // the energy reduction reuses the group's region for gsize doubles
    if (b < size_t(gsize) * 8 + 16) b = size_t(gsize) * 8 + 16;
    return (b + 15) / 16 * 16;
}

template <typename T>
cudaError_t batch_rows(const BatchArgs<T> &a, int grid, cudaStream_t st)
{
    const int groups = a.threads / a.gsize;
    const size_t smem = a.group_smem * groups;
    cudaError_t e = cudaFuncSetAttribute(k_batch_rows<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_batch_rows<T><<<grid, a.threads, smem, st>>>(a); hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t batch_occupancy(const BatchArgs<T> &a, int *per_sm)
{
    const int groups = a.threads / a.gsize;
    const size_t smem = a.group_smem * groups;
    cudaError_t e = cudaFuncSetAttribute(k_batch_rows<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch_rows<T>, a.threads, smem);
}

cudaError_t batch_energy(const double *row_energy, const int64_t *base, const int64_t *rows,
                         int count, double *energies, cudaStream_t st)
{
    k_batch_energy<<<(count + 63) / 64, 64, 0, st>>>(row_energy, base, rows, count, energies); hy::count_launch();
    return cudaGetLastError();
}

template size_t batch_group_smem<double>(int, int, int);
template size_t batch_group_smem<float>(int, int, int);
template cudaError_t batch_rows<double>(const BatchArgs<double> &, int, cudaStream_t);
template cudaError_t batch_rows<float>(const BatchArgs<float> &, int, cudaStream_t);
template cudaError_t batch_occupancy<double>(const BatchArgs<double> &, int *);
template cudaError_t batch_occupancy<float>(const BatchArgs<float> &, int *);
template cudaError_t batch_grad<double>(const BatchGradArgs<double> &, int, cudaStream_t);
template cudaError_t batch_grad<float>(const BatchGradArgs<float> &, int, cudaStream_t);

}  // namespace k
}  // namespace hy
