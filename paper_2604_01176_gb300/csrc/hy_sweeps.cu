// hy_sweeps.cu -- the sweeps built on the state vector besides H psi:
//   * inner products accumulated in double (paper: sparse-sparse inner
//     products; Method: the energy expectation value, Eq. "ev");
//   * the ADAPT-VQE pool-gradient screen g_k = 2 <sigma | A_k psi>;
//   * exp(theta A_k) applied as exact pair rotations (paper: application of
//     exponentiated fermionic operators to the state);
//   * bit-exact determinant ranking (colexicographic combinadic rank).
#include "hy_kernels.cuh"

namespace hy {
namespace k {

// Block-wide sum of one double per thread (any blockDim multiple of 32,
// <= 1024).  Result valid in thread 0.  Fixed reduction order.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double warp_part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) warp_part[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        const int nw = (blockDim.x + 31) >> 5;
        s = threadIdx.x < nw ? warp_part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

// ---------------------------------------------------------------------------
// <x|y> with FP64 accuracy: fixed grid of G blocks writes G partials, one
// block sums them in index order (deterministic for a given G).  Float
// inputs accumulate through Dot2 (error-free FP32 transformations, flushed to
// FP64 every 32 products), double inputs by FMA in double.  16-byte aligned
// inputs are read as float4 / double2.
// ---------------------------------------------------------------------------
template <typename T> struct Vec2;
template <> struct Vec2<float> { using V = float4; static constexpr int W = 4; };
template <> struct Vec2<double> { using V = double2; static constexpr int W = 2; };

template <typename T>
__device__ __forceinline__ void acc_vec(ProdAcc<T> &acc, const float4 &u, const float4 &w)
{
    acc.add(u.x, w.x);
    acc.add(u.y, w.y);
    acc.add(u.z, w.z);
    acc.add(u.w, w.w);
}
template <typename T>
__device__ __forceinline__ void acc_vec(ProdAcc<T> &acc, const double2 &u, const double2 &w)
{
    acc.add(u.x, w.x);
    acc.add(u.y, w.y);
}

template <typename T>
__global__ void __launch_bounds__(256)
k_dot_partial(const T *__restrict__ x, const T *__restrict__ y, int64_t N,
              double *__restrict__ partials)
{
    using V = typename Vec2<T>::V;
    constexpr int W = Vec2<T>::W;
    ProdAcc<T> acc;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t done = 0;
    if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) == 0) {
        const int64_t NV = N / W;
        const V *xv = reinterpret_cast<const V *>(x), *yv = reinterpret_cast<const V *>(y);
        int64_t v = tid;
        for (; v + stride < NV; v += 2 * stride) {     // two vectors in flight
            const V u0 = xv[v], w0 = yv[v], u1 = xv[v + stride], w1 = yv[v + stride];
            acc_vec<T>(acc, u0, w0);
            acc_vec<T>(acc, u1, w1);
        }
        if (v < NV) acc_vec<T>(acc, xv[v], yv[v]);
        done = NV * W;
    }
    for (int64_t i = done + tid; i < N; i += stride) acc.add(x[i], y[i]);
    const double s = block_sum(acc.total());
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out = sum of the G partials in index order (add: out += that sum)
__global__ void __launch_bounds__(256)
k_sum_partials(const double *__restrict__ partials, int G, double *__restrict__ out, int add)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < G; i += blockDim.x) s += partials[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = add ? *out + s : s;
}

template <typename T>
cudaError_t dot(const T *x, const T *y, int64_t N, double *partials, int G,
                double *out, cudaStream_t st)
{
    k_dot_partial<T><<<G, 256, 0, st>>>(x, y, N, partials); hy::count_launch();
    k_sum_partials<<<1, 256, 0, st>>>(partials, G, out, 0); hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256)
k_scale_rsqrt(T *__restrict__ x, int64_t N, const double *__restrict__ norm2)
{
    using V = typename Vec2<T>::V;
    constexpr int W = Vec2<T>::W;
    const T f = T(1.0 / sqrt(*norm2));
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t done = 0;
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        const int64_t NV = N / W;
        V *xv = reinterpret_cast<V *>(x);
        for (int64_t v = tid; v < NV; v += stride) {
            V u = xv[v];
            if constexpr (W == 4) {
                u.x *= f; u.y *= f; u.z *= f; u.w *= f;
            } else {
                u.x *= f; u.y *= f;
            }
            xv[v] = u;
        }
        done = NV * W;
    }
    for (int64_t i = done + tid; i < N; i += stride) x[i] *= f;
}

template <typename T>
cudaError_t scale_rsqrt(T *x, int64_t N, const double *norm2, cudaStream_t st)
{
    int64_t blocks = (N / Vec2<T>::W + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    k_scale_rsqrt<T><<<unsigned(blocks), 256, 0, st>>>(x, N, norm2); hy::count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gradient screen.  For constituent C with sign s on the pair d -> C d:
//   <sigma|(C - C^dagger) psi> = sum_d s [sigma(Cd) psi(d) - sigma(d) psi(Cd)]
// The pairs factor into alpha pairs (A -> A') times beta pairs (B -> B').
// Block (i, chunk) handles op ops[i] and alpha rows chunk, chunk+CH, ...;
// threads stride over the beta pairs.  Per-thread partial sums are kept in
// T; block sums and the per-op total in double.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_grad_partial(GradArgs<T> a)
{
    const int64_t i = blockIdx.x;
    const int chunk = blockIdx.y;
    const int k = a.ops ? a.ops[i] : int(i);
    if (refuse_op(i, k, a.K, chunk == 0 ? a.bad : nullptr)) {
        if (threadIdx.x == 0) a.partials[i * a.CH + chunk] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const OpDev od = a.opd[k];
    double tot = 0.0;
    for (int c = 0; c < od.nc; ++c) {
        const ConsDev cd = a.cons[c == 0 ? od.c0 : od.c1];
        const int64_t nrows = cd.ap < 0 ? a.Na : a.acnt[cd.ap];
        const int64_t ncols = cd.bp < 0 ? a.Nb : a.bcnt[cd.bp];
        const uint32_t *ae = cd.ap < 0 ? nullptr : a.aent + a.aoff[cd.ap];
        const uint32_t *be = cd.bp < 0 ? nullptr : a.bent + a.boff[cd.bp];
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
            const T *pA = a.psi + A * a.Nb, *pA2 = a.psi + A2 * a.Nb;
            const T *sA = a.sigma + A * a.Nb, *sA2 = a.sigma + A2 * a.Nb;
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
    tot = block_sum(tot);
    if (threadIdx.x == 0) a.partials[i * a.CH + chunk] = tot;
}

__global__ void __launch_bounds__(256)
k_grad_final(const double *__restrict__ partials, int CH, int64_t n_ops,
             double *__restrict__ g)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_ops) return;
    double s = 0.0;
    for (int c = 0; c < CH; ++c) s += partials[i * CH + c];
    g[i] = 2.0 * s;
}

template <typename T>
cudaError_t grad(const GradArgs<T> &a, cudaStream_t st)
{
    if (a.n_ops == 0) return cudaSuccess;
    dim3 grid(unsigned(a.n_ops), unsigned(a.CH));
    k_grad_partial<T><<<grid, 256, 0, st>>>(a); hy::count_launch();
    k_grad_final<<<unsigned((a.n_ops + 255) / 256), 256, 0, st>>>(a.partials, a.CH,
                                                                 a.n_ops, a.g); hy::count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// exp(theta (C - C^dagger)) on every connected pair (d, d' = C d), sign s:
//   psi(d) <- c psi(d) - s sn psi(d'),  psi(d') <- c psi(d') + s sn psi(d).
// Distinct pairs never share an amplitude, so the update is race-free.
// Grid: x = beta pair tile, y = alpha pair.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_excite(T *__restrict__ psi, const uint32_t *__restrict__ ae,
         const uint32_t *__restrict__ be, int64_t ncols, int64_t Nb, T c, T s_eps)
{
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= ncols) return;
    const int64_t rr = blockIdx.y;
    int64_t A = rr, A2 = rr, B = t, B2 = t;
    T sg = s_eps;
    if (ae) {
        const uint32_t u = ae[rr];
        A = u & 0x7FFFu;
        A2 = (u >> 15) & 0x7FFFu;
        if (u >> 31) sg = -sg;
    }
    if (be) {
        const uint32_t u = be[t];
        B = u & 0x7FFFu;
        B2 = (u >> 15) & 0x7FFFu;
        if (u >> 31) sg = -sg;
    }
    T *x = psi + A * Nb + B, *y = psi + A2 * Nb + B2;
    const T xv = *x, yv = *y;
    *x = c * xv - sg * yv;
    *y = c * yv + sg * xv;
}

template <typename T>
cudaError_t excite(T *psi, const uint32_t *ae, int64_t nrows, const uint32_t *be,
                   int64_t ncols, int64_t Nb, double c, double s_eps,
                   cudaStream_t st)
{
    if (nrows == 0 || ncols == 0) return cudaSuccess;
    dim3 grid(unsigned((ncols + 255) / 256), unsigned(nrows));
    k_excite<T><<<grid, 256, 0, st>>>(psi, ae, be, ncols, Nb, T(c), T(s_eps)); hy::count_launch();
    return cudaGetLastError();
}

// exp(theta A) as k_excite on a grid of fixed height (rows strided by
// gridDim.y), each block also writing the FP64-accurate change of the squared
// norm over its pairs: x'^2 + y'^2 - x^2 - y^2.
template <typename T>
__global__ void __launch_bounds__(256)
k_excite_n(T *__restrict__ psi, const uint32_t *__restrict__ ae,
           const uint32_t *__restrict__ be, int64_t nrows, int64_t ncols, int64_t Nb, T c,
           T s_eps, double *__restrict__ partials)
{
    ProdAcc<T> acc;
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t < ncols) {
        int64_t B = t, B2 = t;
        T sb = s_eps;
        if (be) {
            const uint32_t u = be[t];
            B = u & 0x7FFFu;
            B2 = (u >> 15) & 0x7FFFu;
            if (u >> 31) sb = -sb;
        }
        for (int64_t rr = blockIdx.y; rr < nrows; rr += gridDim.y) {
            int64_t A = rr, A2 = rr;
            T sg = sb;
            if (ae) {
                const uint32_t u = ae[rr];
                A = u & 0x7FFFu;
                A2 = (u >> 15) & 0x7FFFu;
                if (u >> 31) sg = -sg;
            }
            T *x = psi + A * Nb + B, *y = psi + A2 * Nb + B2;
            const T xv = *x, yv = *y;
            const T nx = c * xv - sg * yv, ny = c * yv + sg * xv;
            *x = nx;
            *y = ny;
            acc.add(nx, nx);
            acc.add(ny, ny);
            acc.add(-xv, xv);
            acc.add(-yv, yv);
        }
    }
    const double s = block_sum(acc.total());
    if (threadIdx.x == 0) partials[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = s;
}

namespace {
dim3 excite_n_grid(int64_t nrows, int64_t ncols, int num_sms)
{
    const int64_t gx = (ncols + 255) / 256;
    int64_t gy = (int64_t(16) * num_sms + gx - 1) / gx;
    if (gy > nrows) gy = nrows;
    if (gy < 1) gy = 1;
    return dim3(unsigned(gx), unsigned(gy));
}
}  // namespace

int excite_n_partials(int64_t nrows, int64_t ncols, int num_sms)
{
    const dim3 g = excite_n_grid(nrows, ncols, num_sms);
    return int(g.x * g.y);
}

template <typename T>
cudaError_t excite_n(T *psi, const uint32_t *ae, int64_t nrows, const uint32_t *be,
                     int64_t ncols, int64_t Nb, double c, double s_eps, double *partials,
                     double *norm2, int num_sms, cudaStream_t st)
{
    if (nrows == 0 || ncols == 0) return cudaSuccess;
    const dim3 grid = excite_n_grid(nrows, ncols, num_sms);
    k_excite_n<T><<<grid, 256, 0, st>>>(psi, ae, be, nrows, ncols, Nb, T(c), T(s_eps), partials);
    hy::count_launch();
    k_sum_partials<<<1, 256, 0, st>>>(partials, int(grid.x * grid.y), norm2, 1);
    hy::count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Determinant rank / unrank with the binomial table in shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t dev_rank(uint32_t m, const uint32_t (*C)[33])
{
    uint32_t r = 0;
    int i = 0;
    while (m) {
        const int pos = __ffs(m) - 1;
        r += C[pos][i + 1];
        ++i;
        m &= m - 1;
    }
    return r;
}

__device__ __forceinline__ uint32_t dev_unrank(uint32_t r, int k, const uint32_t (*C)[33])
{
    uint32_t m = 0;
    for (int i = k - 1; i >= 0; --i) {
        int pos = i;
        while (C[pos + 1][i + 1] <= r) ++pos;
        m |= 1u << pos;
        r -= C[pos][i + 1];
    }
    return m;
}

__global__ void __launch_bounds__(256)
k_rank(const uint64_t *__restrict__ dets, int64_t *__restrict__ idx, int64_t m,
       int n, int na, int nb, int64_t Nb, const uint32_t *__restrict__ binom33)
{
    __shared__ uint32_t C[33][33];
    for (int t = threadIdx.x; t < 33 * 33; t += blockDim.x) C[t / 33][t % 33] = binom33[t];
    __syncthreads();
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint64_t d = dets[i];
    const uint32_t mask = (1u << n) - 1u;
    const uint32_t al = uint32_t(d) & mask, be = uint32_t(d >> n) & mask;
    if ((d >> (2 * n)) != 0 || __popc(al) != na || __popc(be) != nb) {
        idx[i] = -1;
        return;
    }
    idx[i] = int64_t(dev_rank(al, C)) * Nb + int64_t(dev_rank(be, C));
}

__global__ void __launch_bounds__(256)
k_unrank(const int64_t *__restrict__ idx, uint64_t *__restrict__ dets, int64_t m,
         int n, int na, int nb, int64_t Na, int64_t Nb,
         const uint32_t *__restrict__ binom33)
{
    __shared__ uint32_t C[33][33];
    for (int t = threadIdx.x; t < 33 * 33; t += blockDim.x) C[t / 33][t % 33] = binom33[t];
    __syncthreads();
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t I = idx[i];
    if (I < 0 || I >= Na * Nb) {
        dets[i] = 0;
        return;
    }
    const uint32_t al = dev_unrank(uint32_t(I / Nb), na, C);
    const uint32_t be = dev_unrank(uint32_t(I % Nb), nb, C);
    dets[i] = uint64_t(al) | (uint64_t(be) << n);
}

cudaError_t rank(const uint64_t *dets, int64_t *idx, int64_t m, int n, int na,
                 int nb, int64_t Nb, const uint32_t *binom33, cudaStream_t st)
{
    if (m == 0) return cudaSuccess;
    k_rank<<<unsigned((m + 255) / 256), 256, 0, st>>>(dets, idx, m, n, na, nb, Nb,
                                                     binom33); hy::count_launch();
    return cudaGetLastError();
}

cudaError_t unrank(const int64_t *idx, uint64_t *dets, int64_t m, int n, int na,
                   int nb, int64_t Na, int64_t Nb, const uint32_t *binom33,
                   cudaStream_t st)
{
    if (m == 0) return cudaSuccess;
    k_unrank<<<unsigned((m + 255) / 256), 256, 0, st>>>(idx, dets, m, n, na, nb, Na,
                                                       Nb, binom33); hy::count_launch();
    return cudaGetLastError();
}

template cudaError_t dot<double>(const double *, const double *, int64_t, double *,
                                 int, double *, cudaStream_t);
template cudaError_t dot<float>(const float *, const float *, int64_t, double *, int,
                                double *, cudaStream_t);
template cudaError_t scale_rsqrt<double>(double *, int64_t, const double *,
                                         cudaStream_t);
template cudaError_t scale_rsqrt<float>(float *, int64_t, const double *,
                                        cudaStream_t);
template cudaError_t grad<double>(const GradArgs<double> &, cudaStream_t);
template cudaError_t grad<float>(const GradArgs<float> &, cudaStream_t);
template cudaError_t excite<double>(double *, const uint32_t *, int64_t,
                                   const uint32_t *, int64_t, int64_t, double,
                                   double, cudaStream_t);
template cudaError_t excite<float>(float *, const uint32_t *, int64_t,
                                  const uint32_t *, int64_t, int64_t, double, double,
                                  cudaStream_t);
template cudaError_t excite_n<double>(double *, const uint32_t *, int64_t, const uint32_t *,
                                     int64_t, int64_t, double, double, double *, double *,
                                     int, cudaStream_t);
template cudaError_t excite_n<float>(float *, const uint32_t *, int64_t, const uint32_t *,
                                    int64_t, int64_t, double, double, double *, double *, int,
                                    cudaStream_t);

}  // namespace k
}  // namespace hy
