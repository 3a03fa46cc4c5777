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
    int64_t row0, row1;     // output alpha rows [row0, row1); sigma holds row row0 first
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
    int64_t K;              // pool size: listed indices outside [0, K) are refused
    unsigned long long *bad;   // (position << 32 | index) of the first refused entry
};

// A listed pool index outside [0, K): the entry's partial becomes NaN (so its
// gradient reads NaN) and the smallest (position, index) key is kept in *bad
// for the host to report; nothing out of range is read.
__device__ __forceinline__ bool refuse_op(int64_t i, int k, int64_t K, unsigned long long *bad)
{
    if (k >= 0 && k < K) return false;
    if (bad && threadIdx.x == 0)
        atomicMin(bad, (static_cast<unsigned long long>(i) << 32) |
                           static_cast<unsigned long long>(static_cast<uint32_t>(k)));
    return true;
}

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
    // phase A: the alpha strings J whose T rows are formed -- jlist[0 .. nJ)
    // (device), or every J when jlist is null (nJ = Na)
    const int32_t *jlist;
    int64_t nJ;
    int64_t row0, row1;     // phase B: output alpha rows; sigma holds row row0 first
};
size_t cpl_dense_smem(int64_t Nb, int n);
// phase A (SIMT) + phase B
cudaError_t coupling_dense(const CplDenseArgs &a, int num_sms, cudaStream_t st);
// phase B alone: sigma[a'][b'] += the 65 rows of T that reach a'
cudaError_t coupling_gather(const CplDenseArgs &a, int num_sms, cudaStream_t st);
// phase A on the tensor cores (hy_cpl_tc.cu); *status (device) is set to 1
// if a bounded wait ran out
size_t cpl_tc_smem(int64_t Nb);
cudaError_t coupling_tc(const CplDenseArgs &a, int *status, long long spin_limit, int issue,
                        int num_sms, cudaStream_t st);

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
// exp(theta A) as excite(), also adding the change of ||psi||^2 over the
// rotated pairs to *norm2 (partials: >= excite_n_partials(...) doubles)
int excite_n_partials(int64_t nrows, int64_t ncols, int num_sms);
template <typename T>
cudaError_t excite_n(T *psi, const uint32_t *ae, int64_t nrows, const uint32_t *be,
                     int64_t ncols, int64_t Nb, double c, double s_eps, double *partials,
                     double *norm2, int num_sms, cudaStream_t st);

// ---------------------------------------------------------------------------
// FP32 products summed with FP64 accuracy at FP32 speed (GB300 issues FP64 at
// 1/64 of the FP32 rate, and a float -> double conversion costs an FP64 slot).
// Dot2 of Ogita, Rump & Oishi ("Accurate sum and dot product", SIAM J. Sci.
// Comput. 26, 2005): TwoProduct writes x*y = h + r exactly with one FMA,
// TwoSum writes p + h = p' + q exactly; p carries the sum, s the exact
// rounding errors.  Every kDot2Run terms (p, s) is added to an FP64 total, so
// a run's error is below gamma_31^2 * sum|x_i y_i| (~3.5e-12 relative, typ.
// ~1e-14) and the FP64 total is as in a plain double accumulation.  Products
// near the FP32 overflow threshold take the exact FP64 product instead.
// ---------------------------------------------------------------------------
constexpr int kDot2Run = 32;
struct Dot2 {
    float p, s;
    double d;
    int n;
};
__device__ __forceinline__ void dot2_init(Dot2 &a)
{
    a.p = 0.f;
    a.s = 0.f;
    a.d = 0.0;
    a.n = 0;
}
__device__ __forceinline__ void dot2_flush(Dot2 &a)
{
    a.d += double(a.p);
    a.d += double(a.s);
    a.p = 0.f;
    a.s = 0.f;
    a.n = 0;
}
__device__ __forceinline__ void dot2_add(Dot2 &a, float x, float y)
{
    const float h = __fmul_rn(x, y);
    if (fabsf(h) > 1e36f) {          // also inf; NaN falls through and propagates
        a.d += double(x) * double(y);
        return;
    }
    const float r = __fmaf_rn(x, y, -h);
    const float p = __fadd_rn(a.p, h);
    const float z = __fsub_rn(p, a.p);
    const float q = __fadd_rn(__fsub_rn(a.p, __fsub_rn(p, z)), __fsub_rn(h, z));
    a.p = p;
    a.s = __fadd_rn(a.s, __fadd_rn(q, r));
    if (++a.n == kDot2Run) dot2_flush(a);
}
__device__ __forceinline__ double dot2_total(Dot2 &a)
{
    dot2_flush(a);
    return a.d;
}
// sum of products accumulated with FP64 accuracy: Dot2 for float, FMA in double
template <typename T>
struct ProdAcc;
template <>
struct ProdAcc<float> {
    Dot2 a;
    __device__ __forceinline__ ProdAcc() { dot2_init(a); }
    __device__ __forceinline__ void add(float x, float y) { dot2_add(a, x, y); }
    __device__ __forceinline__ double total() { return dot2_total(a); }
};
template <>
struct ProdAcc<double> {
    double d;
    __device__ __forceinline__ ProdAcc() : d(0.0) {}
    __device__ __forceinline__ void add(double x, double y) { d = fma(x, y, d); }
    __device__ __forceinline__ double total() { return d; }
};

// learned ranker (hy_ranker.cu)
constexpr int kRankerFeatures = 16;
constexpr int kTopKMax = 8192;
template <typename T>
cudaError_t occupations(const T *psi, int64_t Na, int64_t Nb, const uint32_t *astr,
                        const uint32_t *bstr, int n, double *partial, int G, float *out,
                        cudaStream_t st);
// the same occupations from psi's touched-weight partials (no pass over psi)
// scratch: 34 doubles, the last one zero on first use (left zero after each call)
cudaError_t occupations_from_weights(const float *Bw, const float *rs, const uint32_t *astr,
                                     int64_t Na, int n, double *scratch, float *out,
                                     cudaStream_t st);
cudaError_t features(const int32_t *desc, int64_t K, int n, const double *h1,
                     const double *eri, const float *occ, const float *extra, const float *Dpsi,
                     const float *Dsig, float *feat, cudaStream_t st);
// part: pair_splits() x n^4 floats of scratch; rows: Na + 1 ints of scratch
int pair_splits();
template <typename T>
cudaError_t touched_weights(const T *psi, int64_t Na, int64_t Nb, const uint32_t *astr,
                            const uint32_t *bstr, int n, float *Bw, float *rs, int32_t *rows,
                            float *part, float *D, int num_sms, cudaStream_t st);
// scratch that groups a listed state's entries by alpha row: counts and
// starts [Na + 1], cursors [Na], each entry's beta string and weight [cap]
struct TwGroups {
    int32_t *cnt, *ptr, *cur;
    uint32_t *mask;
    float *w;
    int64_t cap;
};
// the same for a state given by its support list (v dense-backed; the device
// count is clamped to cap; hint ~ the count, for the grid).  With groups
// (g.mask not null, g.cap >= cap) the entries are grouped by alpha row and
// each row summed by one block; else every entry adds to Bw atomically.
template <typename T>
cudaError_t touched_weights_list(const T *v, const int64_t *list, const unsigned long long *count,
                                 int64_t cap, int64_t hint, int64_t Na, int64_t Nb,
                                 const uint32_t *astr, const uint32_t *bstr, int n, float *Bw,
                                 float *rs, int32_t *rows, float *part, float *D,
                                 const TwGroups &g, int num_sms, cudaStream_t st);

// sparse-state path (hy_sparse.cu)
template <typename T>
struct SparseArgs {
    const T *psi;
    T *sigma;
    const int64_t *list;     // nonzero amplitudes of psi
    int64_t m;
    const unsigned long long *d_m;   // device count (overrides m, clamped to cap) or nullptr
    int64_t cap;
    // sigma's support as a sparse vector (list, bitmap, count, capacity), or
    // obits = nullptr: then sigma is zeroed whole and nothing is listed
    uint32_t *obits;
    int64_t *olist;
    unsigned long long *ocount;
    int64_t ocap;
    const int32_t *Ma_ptr, *Ma_col, *Mb_ptr, *Mb_col;
    const T *Ma_val, *Mb_val, *V;
    const uint32_t *aex, *bexT, *astr, *bstr;
    const uint32_t *bex;            // beta excitations, string-major [Nb][nexb]
    int n, nexa, nexb;
    int64_t Na, Nb;
};
template <typename T>
struct SparseGradArgs {
    const T *psi, *sigma;
    const int64_t *list;
    int64_t m;
    const unsigned long long *d_m;   // device count (overrides m, clamped to cap) or nullptr
    int64_t cap;
    const uint32_t *bits;    // membership bitmap of the list, or nullptr: then
                             // the list holds exactly the nonzero amplitudes
    int chunks;              // support chunks per operator (grid.y)
    double *partials;        // [n_ops][chunks]
    const int32_t *desc;     // [K][11] operator descriptors
    const int32_t *ops;      // operator list or nullptr (all)
    int64_t n_ops;
    const uint32_t *astr, *bstr, *binom33;
    const uint16_t *rank16;  // [1 << n] colex rank of every n-bit string
    int n;
    int64_t Nb;
    double *g;
    int64_t K;               // pool size: listed indices outside [0, K) are refused
    unsigned long long *bad; // (position << 32 | index) of the first refused entry, or nullptr
    int qubit;               // 1: qubit excitations (no Jordan-Wigner sign)
};
template <typename T>
cudaError_t support(const T *psi, int64_t N, int64_t *list, int64_t cap,
                    unsigned long long *count, int num_sms, cudaStream_t st);
template <typename T>
cudaError_t hpsi_scatter(const SparseArgs<T> &a, int num_sms, cudaStream_t st);
// the set bits of a membership bitmap of `words` words as a list in
// increasing order (at most cap written; cnt[0] = cnt[1] = the number of set
// bits, cnt[2] = 0); blk: scratch of bits_compact_blocks(words) int64
inline int64_t bits_compact_blocks(int64_t words) { return (words + 2047) / 2048; }
cudaError_t bits_compact(const uint32_t *bits, int64_t words, int64_t *list, int64_t cap,
                         unsigned long long *cnt, int64_t *blk, cudaStream_t st);
// sigma = H psi on the rows of psi's support only (k_sup_alpha, k_sup_beta):
// s holds psi's dense array (zero off the support), sigma and the tables;
// list / cnt / cap the support sorted by determinant, bits its bitmap; the
// rest is scratch (runs, ralpha: Na entries; flagA: Na, flagB, blist: Nb;
// ctr: 4 counters).  sigma is written on the support only.
template <typename T>
struct SupRowsArgs {
    SparseArgs<T> s;
    const int64_t *list;
    const unsigned long long *cnt;
    int64_t cap;
    const uint32_t *bits;
    int64_t *runs;
    int32_t *ralpha;
    uint8_t *flagA, *flagB;
    int32_t *blist;
    unsigned long long *ctr;
};
template <typename T>
cudaError_t hpsi_support(const SupRowsArgs<T> &a, int num_sms, cudaStream_t st);
template <typename T>
cudaError_t grad_sparse(const SparseGradArgs<T> &a, int num_sms, cudaStream_t st);

// Sparse vectors backed by a dense array: v (N amplitudes, zero off the
// support), list[0..count) the support (each index once, values may be 0),
// bits the membership bitmap of the list (bit i of bits[i >> 5]).
template <typename T>
struct SVec {
    T *v;
    int64_t *list;
    uint32_t *bits;
    unsigned long long *count;   // device: live count
    unsigned long long *snap;    // device: count at the start of a rotation
    unsigned long long *done;    // device: blocks of the current rotation finished
    int64_t cap;
    int64_t hint;                // host estimate of the count (grid size only)
};
// a constituent's operator strings and the tables to rank determinants
struct SvOpArgs {
    const int32_t *desc;         // [K][11]
    const uint32_t *astr, *bstr, *binom33;
    const uint16_t *rank16;      // [1 << n] colex rank of every n-bit string
    int n;
    int64_t Nb;
    int qubit;                   // 1: the pool's operators are qubit excitations (no sign)
};
// v <- 0 on the support, bits cleared, count <- 0; then (hf) v[0] = 1 listed
template <typename T>
cudaError_t sv_reset(const SVec<T> &x, bool hf, int num_sms, cudaStream_t st);
// dst <- src (dst must be reset)
template <typename T>
cudaError_t sv_copy(const SVec<T> &dst, const SVec<T> &src, int num_sms, cudaStream_t st);
// exp(theta (C - C^dagger)) for every constituent C of operator k; closed:
// keep the list fixed (a pair with an unlisted end only scales its listed end)
template <typename T>
cudaError_t sv_excite(const SVec<T> &x, const SvOpArgs &o, int k, int nc, double theta,
                      int num_sms, cudaStream_t st, bool closed = false);
// one CTA: clear x's support, |HF>, every constituent rotation of ops[0..L)
// with cs[2l], cs[2l+1] = cos, sin theta_l, then (renorm) divide by the FP64
// norm over the support (written to *norm2 if not null); for small supports.
// step_len (device, or null): the list's length after each constituent
// rotation, in order
template <typename T>
cudaError_t sv_prepare(const SVec<T> &x, const SvOpArgs &o, const int32_t *ops, const double *cs,
                       int L, bool renorm, double *norm2, int64_t *step_len, cudaStream_t st);

// Support programs (hy_sparse.cu).  The support of U_L .. U_1|HF> is fixed by
// the ansatz (a rotation lists its partners whatever its angle), so once it
// is known each constituent rotation is a fixed pairing of its elements:
//   key[t]  = (determinant << 8) | (step that listed it + 1) for the m
//             support elements (t = local index; ascending for m <=
//             kProgMax, listing order beyond);
//   the pairs of step s: (t, p, sign) for every t that step s's forward
//             string takes to a support element p with sign +-1, packed in
//             one word (t's index within its part, p, the sign).  They are
//             kept as compact lists, one per step and part of the support:
//             with `ranks` parts of `chunk` = ceil(m / ranks) elements (one
//             part for one CTA, kClusterCtas for a cluster), the pairs of
//             step s whose domain end t lies in part r are
//             pairs[(s * ranks + r) * chunk + i], i < npairs[s * ranks + r],
//             those with an end listed before step s (the only ones that can
//             be nonzero when the preparation reaches step s), and
//             pairs[(s * ranks + r + 1) * chunk - 1 - i], i < nrest[s * ranks
//             + r], the others; in no fixed order: the pairs of one step are
//             disjoint (an image end has no forward image), so no result
//             depends on it;
//   step_l[s] = the operator (position in the ansatz) of step s;
//   *flag   = 1 when some generator A_l = sum (C - C^dagger) of op l would
//             leave the support from an element that op l's own later
//             constituents listed (then the forward gradient cannot use the
//             tables and must take the general path).
constexpr int kProgMax = 12288;   // shared-memory vectors: 2 x 12288 doubles per CTA
constexpr int kProgSteps = 254;   // steps of one program (8-bit birth tags)
struct ProgTabs {
    const int64_t *key;
    const uint32_t *pairs;
    const int *npairs, *nrest;
    const int *step_l;
    int m, steps, ranks, chunk;
    int optin;                 // the device's opt-in shared memory per block
};
// raises the program kernels' dynamic shared-memory limit on the current
// device to what an opt-in limit of `optin` bytes per block leaves them
cudaError_t prog_attrs(int optin);
// list: the m support elements in the order a structural sv_prepare listed
// them, step_len its lengths after each of the `steps` rotations; pairs holds
// steps * m entries, npairs 2 * steps counts (nrest = npairs + steps), step_l
// `steps` entries
cudaError_t prog_compile(const int64_t *list, int64_t m, const int64_t *step_len, int steps,
                         const SvOpArgs &o, const int32_t *ops, int L, int64_t *key,
                         uint32_t *pairs, int *npairs, int *step_l, int *flag, cudaStream_t st);
// one CTA: the m-vector U_L .. U_1|HF> by the pair lists in shared memory,
// with cs[2l], cs[2l+1] = cos, sin theta_l, then (renorm) divided by its FP64
// norm (*norm2, if not null), written to v[key[t] >> 8]; v outside the
// support is left as is
template <typename T>
cudaError_t prog_prepare(const ProgTabs &g, const double *cs, bool renorm, double *norm2, T *v,
                         cudaStream_t st);
// L CTAs: g[l] = dE/dtheta_l in forward mode by the pair lists, CTA l forming
// U_L .. U_{l+1} A_l U_l .. U_1|HF> in shared memory and reading sigma (dense)
// on the support; norm2 as for sv_grad_fwd
template <typename T>
cudaError_t prog_grad(const ProgTabs &g, const double *cs, int L, const T *sigma,
                      const double *norm2, double *gout, cudaStream_t st);
// Support programs beyond one CTA's shared memory, kProgMax < m <= kProgBig:
// the support in listing order (key unsorted), local indices through idx_map
// (N int32 over Omega_CIk, read where `bits`, the listing's membership
// bitmap, has the determinant), each vector split over the distributed shared
// memory of a cluster of 8 CTAs (prepare: one cluster; gradient: one cluster
// per angle); the pair lists per step and CTA (ranks = kClusterCtas), pairs
// holding steps * kClusterCtas * ceil(m / kClusterCtas) entries and npairs
// 2 * steps * kClusterCtas counts (nrest = npairs + steps * kClusterCtas)
constexpr int64_t kProgBig = 65536;
constexpr int kClusterCtas = 8;
cudaError_t prog_compile_big(const int64_t *list, int64_t m, const int64_t *step_len, int steps,
                             const SvOpArgs &o, const int32_t *ops, int L, const uint32_t *bits,
                             int64_t *key, uint32_t *pairs, int *npairs, int *step_l,
                             int32_t *idx_map, int *flag, cudaStream_t st);
template <typename T>
cudaError_t prog_prepare_big(const ProgTabs &g, const double *cs, bool renorm, double *norm2,
                             T *v, cudaStream_t st);
template <typename T>
cudaError_t prog_grad_big(const ProgTabs &g, const double *cs, int L, const T *sigma,
                          const double *norm2, double *gout, cudaStream_t st);
// The Hamiltonian restricted to a support S (both rows and columns in S):
// row t is the determinant key[t] >> 8 of a support program, its entries
// the couplings to determinants of S (membership bitmap `bits`), columns
// stored as determinant indices.  The energy of a state on S and the
// forward gradients read sigma only on S, so within one ansatz H_SS psi
// serves every evaluation.  hss_fill: the entries of every row (the
// candidates filtered by the support's alpha and beta string sets first,
// then by its bitmap; fixed order); hss_apply: sigma[key[t] >> 8] = sum_e
// val[e] psi[col[e]] for t < m, accumulated in T (sigma untouched elsewhere),
// and with dot not null also *dot = <psi|sigma> over the support in FP64
// (partials: one double per block, at most 16 per SM; done: a counter that
// is zero between launches, the last block to finish adds the partials).
struct HssArgs {
    const int64_t *key;
    int64_t m;
    const uint32_t *bits;
    const int32_t *Ma_ptr, *Ma_col, *Mb_ptr, *Mb_col;
    const double *Ma_val, *Mb_val, *V;
    const uint32_t *aex, *bexT, *astr, *bstr;
    int n, nexa, nexb;
    int64_t Na, Nb;
    uint32_t *sa, *sb;       // scratch: bitmaps over the alpha / beta strings
    int64_t stride;          // entries reserved per row (>= any row's couplings)
    int32_t *cnt;            // [m] entries of each row
    uint32_t *col;           // [m * stride]
    double *val;             // [m * stride]
};
// one pass: row t's entries at [t * stride, t * stride + cnt[t]), fixed
// order; then *nnz (device) = their total
cudaError_t hss_fill(const HssArgs &a, int64_t *nnz, int num_sms, cudaStream_t st);
template <typename T>
cudaError_t hss_apply(const int64_t *key, int64_t m, const int32_t *cnt, int64_t stride,
                      const uint32_t *col, const double *val, const T *psi, T *sigma, int num_sms,
                      double *partials, unsigned *done, double *dot, cudaStream_t st);

// one CTA: g[l] = dE/dtheta_l of psi = U_L .. U_1|HF> in forward mode, f and
// w scratch sparse vectors (clean), sigma = H psi dense; norm2 (device, or
// null): psi was divided by sqrt(*norm2), so the gradient is too
template <typename T>
cudaError_t sv_grad_fwd(const SVec<T> &f, const SVec<T> &w, const SvOpArgs &o, const int32_t *ops,
                        const double *cs, int L, const T *sigma, const double *norm2, double *g,
                        cudaStream_t st);
// sum over the support of x.v * y (y dense), in FP64, into *out (partials:
// 4 * num_sms doubles); scale: x.v <- x.v / sqrt(*norm2) on the support
template <typename T>
cudaError_t sv_dot(const SVec<T> &x, const T *y, double *partials, double *out, int num_sms,
                   cudaStream_t st);
template <typename T>
cudaError_t sv_scale_rsqrt(const SVec<T> &x, const double *norm2, int num_sms,
                           cudaStream_t st);

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
// Same-spin kernel table of one spin folded on the device from the Pauli
// table (hy_fold.cu): candidates of row r = the diagonal, the singles and the
// doubles of str[r]; element = the Pauli group with X-mask K ^ J evaluated on J
// (placed at qubit `shift`), minus sub_diag on the diagonal
struct FoldArgs {
    const uint32_t *str;
    int64_t N;
    int n, k, shift;
    double sub_diag;
    const int32_t *grp;        // [1 << n] group of an X-mask within the spin, or -1
    const int64_t *goff;       // [groups + 1]
    const uint64_t *z;         // [terms]
    const double *c;           // [terms]
    const uint32_t *binom33;
    int64_t stride;            // scratch entries per row (>= fold_candidates)
    int32_t *tcol;             // [N * stride] scratch
    double *tval;              // [N * stride] scratch
    int32_t *len;              // [N]
};
int fold_candidates(int n, int k);
cudaError_t fold_rows(const FoldArgs &a, int num_sms, cudaStream_t st);
// row pointers [N + 1] and the CSR columns and values (double and float)
cudaError_t fold_compact(const FoldArgs &a, int32_t *ptr, int32_t *col, double *val64,
                         float *val32, int num_sms, cudaStream_t st);

// Batched pool-gradient screen: per molecule its pool's pair tables (as in
// GradArgs) and its place in the packed state buffers
struct BatchPool {
    const OpDev *opd;
    const ConsDev *cons;
    const uint32_t *aent, *bent;
    const int64_t *aoff, *acnt, *boff, *bcnt;
    int64_t Na, Nb, off, K;
};
template <typename T>
struct BatchGradArgs {
    const BatchPool *mols;
    int count;
    const T *psi, *sigma;             // packed states
    const int32_t *ops;               // packed per-molecule operator lists, or nullptr
    const int64_t *base;              // [count + 1] entries of each molecule in ops / g
    int CH;                           // row chunks per entry
    int64_t n_tasks;                  // base[count] * CH
    double *partials;                 // [n_tasks]
    double *g;                        // [base[count]]
    unsigned long long *counter;      // work counter, zeroed before the launch
    unsigned long long *bad;          // first refused entry: (position << 32) | index
};
// one persistent launch over the (molecule, entry, row chunk) tasks, then the
// per-entry sums g = 2 * sum of its chunks
template <typename T>
cudaError_t batch_grad(const BatchGradArgs<T> &a, int grid, cudaStream_t st);
cudaError_t batch_energy(const double *row_energy, const int64_t *base, const int64_t *rows,
                         int count, double *energies, cudaStream_t st);

cudaError_t rank(const uint64_t *dets, int64_t *idx, int64_t m, int n, int na,
                 int nb, int64_t Nb, const uint32_t *binom33, cudaStream_t st);
cudaError_t unrank(const int64_t *idx, uint64_t *dets, int64_t m, int n, int na,
                   int nb, int64_t Na, int64_t Nb, const uint32_t *binom33,
                   cudaStream_t st);

}  // namespace k
}  // namespace hy
