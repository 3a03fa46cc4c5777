// hy_kernels.cuh -- launch interface of the library's CUDA kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hy {
// counts every kernel launch the library makes (hy_launch_count)
void count_launch();
namespace k {

// Pool metadata on the device.  A constituent C = eps * Ca * Cb with Ca / Cb
// a pattern id into the alpha / beta pattern lists (-1 = identity).
struct ConsDev {
    int32_t ap, bp, eps, pad;
};
struct OpDev {
    int32_t nc, c0, c1, pad;
};

// columns of the output row each coupling thread keeps in registers
// (1024 threads x 13 columns covers N_beta = 12,870 at 16 orbitals)
constexpr int kCouplingMaxCpt = 13;

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

// float alpha-beta coupling through the dense intermediate T (hy_sigma.cu)
struct CplDenseArgs {
    const float *psi;
    float *sigma;
    float *T;               // [Na][nexa+1][Nbp]
    const uint32_t *aex;    // [Na][nexa]
    const uint8_t *inv;     // [Na][nexa] position of the row in its partner's list
    const uint32_t *bexT;   // [nexb][Nb]
    const uint32_t *astr, *bstr;
    const float *V;         // n^4
    int n, nexa, nexb;
    int64_t Na, Nb, Nbp;    // Nbp: row stride of T (multiple of 64)
};
size_t cpl_dense_smem(int64_t Nb, int n);
cudaError_t coupling_dense(const CplDenseArgs &a, int num_sms, cudaStream_t st);

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

// learned ranker (hy_ranker.cu)
constexpr int kRankerFeatures = 16;
constexpr int kTopKMax = 8192;
template <typename T>
cudaError_t occupations(const T *psi, int64_t Na, int64_t Nb, const uint32_t *astr,
                        const uint32_t *bstr, int n, double *partial, int G, float *out,
                        cudaStream_t st);
cudaError_t features(const int32_t *desc, int64_t K, int n, const double *h1,
                     const double *eri, const float *occ, const float *extra, const float *Dpsi,
                     const float *Dsig, float *feat, cudaStream_t st);
template <typename T>
cudaError_t touched_weights(const T *psi, int64_t Na, int64_t Nb, const uint32_t *astr,
                            const uint32_t *bstr, int n, float *Bw, float *rs, float *D,
                            int num_sms, cudaStream_t st);

// sparse-state path (hy_sparse.cu)
template <typename T>
struct SparseArgs {
    const T *psi;
    T *sigma;
    const int64_t *list;     // nonzero amplitudes of psi
    int64_t m;
    const int32_t *Ma_ptr, *Ma_col, *Mb_ptr, *Mb_col;
    const T *Ma_val, *Mb_val, *V;
    const uint32_t *aex, *bexT, *astr, *bstr;
    int n, nexa, nexb;
    int64_t Na, Nb;
};
template <typename T>
struct SparseGradArgs {
    const T *psi, *sigma;
    const int64_t *list;
    int64_t m;
    const int32_t *desc;     // [K][11] operator descriptors
    const int32_t *ops;      // operator list or nullptr (all)
    int64_t n_ops;
    const uint32_t *astr, *bstr, *binom33;
    int n;
    int64_t Nb;
    double *g;
};
template <typename T>
cudaError_t support(const T *psi, int64_t N, int64_t *list, int64_t cap,
                    unsigned long long *count, int num_sms, cudaStream_t st);
template <typename T>
cudaError_t hpsi_scatter(const SparseArgs<T> &a, int num_sms, cudaStream_t st);
template <typename T>
cudaError_t grad_sparse(const SparseGradArgs<T> &a, int num_sms, cudaStream_t st);

// batched rows over many molecules (hy_batch.cu)
template <typename T>
struct BatchMol {
    int64_t offset;          // first amplitude of this molecule in the packed state
    int64_t Na, Nb, task_base;
    int n, nexa, nexb, pad;
    const int32_t *Ma_ptr, *Ma_col, *Mb_ptr, *Mb_col;
    const T *Ma_val, *Mb_val, *V;
    const uint32_t *aex, *bexT, *astr, *bstr;
};
template <typename T>
struct BatchArgs {
    const T *psi;
    T *sigma;
    const BatchMol<T> *mols;
    const int2 *tasks;       // (molecule, alpha row)
    int n_tasks;
    int *counter;            // zeroed before each launch
    double *row_energy;      // per-row <psi|sigma> partials or nullptr
    int gsize, threads;      // group size and CTA size (tile shape)
    int nb_max, nn_max;
    size_t group_smem;
};
template <typename T>
size_t batch_group_smem(int nb_max, int nn_max, int gsize);
template <typename T>
cudaError_t batch_rows(const BatchArgs<T> &a, int grid, cudaStream_t st);
template <typename T>
cudaError_t batch_occupancy(const BatchArgs<T> &a, int *per_sm);
cudaError_t batch_energy(const double *row_energy, const int64_t *base, const int64_t *rows,
                         int count, double *energies, cudaStream_t st);

cudaError_t rank(const uint64_t *dets, int64_t *idx, int64_t m, int n, int na,
                 int nb, int64_t Nb, const uint32_t *binom33, cudaStream_t st);
cudaError_t unrank(const int64_t *idx, uint64_t *dets, int64_t m, int n, int na,
                   int nb, int64_t Na, int64_t Nb, const uint32_t *binom33,
                   cudaStream_t st);

}  // namespace k
}  // namespace hy
