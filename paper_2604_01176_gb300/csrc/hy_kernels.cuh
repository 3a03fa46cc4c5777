// hy_kernels.cuh -- launch interface of the library's CUDA kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hy {
namespace k {

// Pool metadata on the device.  A constituent C = eps * Ca * Cb with Ca / Cb
// a pattern id into the alpha / beta pattern lists (-1 = identity).
struct ConsDev {
    int32_t ap, bp, eps, pad;
};
struct OpDev {
    int32_t nc, c0, c1, pad;
};

template <typename T>
struct CouplingArgs {
    const T *psi;
    T *sigma;
    const uint32_t *aex;    // [Na][nexa] single excitations of output alpha rows
    const uint32_t *bexT;   // [nexb][Nb] single excitations of output beta columns
    const uint32_t *astr;   // alpha masks
    const uint32_t *bstr;   // beta masks
    const T *V;             // n^4 alpha-beta coupling
    int n, nexa, nexb;
    int64_t Na, Nb;
};

template <typename T>
struct GradArgs {
    const T *psi, *sigma;
    const int32_t *ops;     // device op list or nullptr (all ops in order)
    int64_t n_ops;
    const OpDev *opd;
    const ConsDev *cons;
    const uint32_t *aent;
    const int64_t *aoff, *acnt;
    const uint32_t *bent;
    const int64_t *boff, *bcnt;
    int64_t Na, Nb;
    int CH;                 // row chunks per op (grid.y)
    double *partials;       // [n_ops][CH]
    double *g;              // [n_ops]
};

template <typename T>
cudaError_t spmm(const int32_t *ptr, const int32_t *col, const T *val,
                 int64_t rows, const T *X, T *Y, int64_t ncols, bool accumulate,
                 cudaStream_t st);
template <typename T>
cudaError_t transpose(const T *in, T *out, int64_t R, int64_t C, cudaStream_t st);
template <typename T>
cudaError_t add_transposed(const T *tau, T *sigma, int64_t R, int64_t C,
                           cudaStream_t st);
template <typename T>
cudaError_t coupling(const CouplingArgs<T> &a, int num_sms, cudaStream_t st);
template <typename T>
cudaError_t dot(const T *x, const T *y, int64_t N, double *partials, int G,
                double *out, cudaStream_t st);
template <typename T>
cudaError_t scale_rsqrt(T *x, int64_t N, const double *norm2, cudaStream_t st);
template <typename T>
cudaError_t grad(const GradArgs<T> &a, cudaStream_t st);
template <typename T>
cudaError_t excite(T *psi, const uint32_t *ae, int64_t nrows, const uint32_t *be,
                   int64_t ncols, int64_t Nb, double c, double s_eps,
                   cudaStream_t st);

cudaError_t rank(const uint64_t *dets, int64_t *idx, int64_t m, int n, int na,
                 int nb, int64_t Nb, const uint32_t *binom33, cudaStream_t st);
cudaError_t unrank(const int64_t *idx, uint64_t *dets, int64_t m, int n, int na,
                   int nb, int64_t Na, int64_t Nb, const uint32_t *binom33,
                   cudaStream_t st);

}  // namespace k
}  // namespace hy
