// hy_api.cu -- the library's C ABI (include/hyperion.h): argument checks,
// device tables, the per-handle workspace and the launch sequence of each
// call.  Everything numerical runs in the kernels of hy_sigma.cu and
// hy_sweeps.cu; this file only marshals.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "hy_internal.h"
#include "hy_kernels.cuh"

namespace {

thread_local std::string g_err;

hy_status fail(hy_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

hy_status cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? HY_ERR_OOM : HY_ERR_CUDA;
}

#define HY_CUDA(call, what)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);    \
    } while (0)

// Device allocations owned by a handle, released together.
struct DevArena {
    std::vector<void *> ptrs;
    int64_t uploaded = 0;        // bytes copied host -> device
    template <typename T>
    cudaError_t upload(T **dst, const T *src, size_t count)
    {
        *dst = nullptr;
        if (count == 0) return cudaSuccess;
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) return e;
        ptrs.push_back(p);
        e = cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice);
        uploaded += int64_t(count * sizeof(T));
        *dst = static_cast<T *>(p);
        return e;
    }
    // device memory owned by the arena, not copied from the host
    template <typename T>
    cudaError_t alloc(T **dst, size_t count, bool zero = false)
    {
        *dst = nullptr;
        if (count == 0) return cudaSuccess;
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) return e;
        ptrs.push_back(p);
        if (zero) e = cudaMemset(p, 0, count * sizeof(T));
        *dst = static_cast<T *>(p);
        return e;
    }
    void release()
    {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

template <typename T>
struct DevCsr {
    int32_t *ptr = nullptr, *col = nullptr;
    T *val = nullptr;
};

}  // namespace

std::atomic<long long> g_launches{0};

namespace hy {
void set_last_error(const std::string &msg) { g_err = msg; }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace hy

struct hy_ham {
    int n = 0, na = 0, nb = 0;
    int64_t Na = 0, Nb = 0, N = 0;
    int device = 0, num_sms = 0;
    hy::StringSpace A, B;
    hy::PauliTable pauli;
    hy::KernelTables kt;            // E0 and V; Ma / Mb copied from the device on demand
    int64_t nnz_a = 0, nnz_b = 0;   // entries of the same-spin tables
    std::vector<double> h1h, h2h;   // the integrals (host copies)
    DevArena arena;
    uint32_t *d_astr = nullptr, *d_bstr = nullptr;
    uint32_t *d_aex = nullptr, *d_bexT = nullptr;
    uint32_t *d_bex = nullptr;   // beta excitations string-major [Nb][nexb]
    uint8_t *d_ainv = nullptr;   // inverse alpha excitation positions
    uint32_t *d_binom = nullptr;
    uint16_t *d_rank16 = nullptr;   // [1 << n] colex rank of every n-bit string
    DevCsr<double> Ma64, Mb64;
    DevCsr<float> Ma32, Mb32;
    double *d_V64 = nullptr;
    float *d_V32 = nullptr;
    double *d_h1 = nullptr, *d_eri = nullptr;   // integrals (ranker features)
    double *d_occ_partial = nullptr;            // [occ_blocks][33]
    float *d_occ = nullptr;                     // [2n]
    float *d_pairB = nullptr;                   // [2][Na][n^2] touched-weight partials
    float *d_pairRs = nullptr;                  // [2][Na]
    float *d_pairD = nullptr;                   // [2][n^4] touched weights (psi, sigma)
    float *d_pairP = nullptr;                   // [splits][n^4] contraction partials
    int32_t *d_pairRows = nullptr;              // [Na + 1] nonzero alpha rows
    double *d_occw = nullptr;                   // [34] occupations-from-weights scratch
    int occ_blocks = 0;
    // workspace (grown on demand; growth synchronises the device)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    // row groups of a listed state for its touched weights (grown on demand,
    // with a device synchronisation)
    hy::k::TwGroups tw{nullptr, nullptr, nullptr, nullptr, nullptr, 0};
    int dot_blocks = 0;
    // optional CUDA events around the alpha-beta coupling launch(es)
    bool prof = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // float coupling phase A: 0 tensor cores (tcgen05), 1 FP32 SIMT, 2 the
    // tensor-core kernel with its MMAs withheld (a test of the bounded waits)
    int cpl_impl = 0;
    long long tc_spin_limit = 1ll << 26;   // polls of a stage barrier before giving up
    int *d_status = nullptr;        // device: a bounded wait of k_cpl_tc ran out
    int *h_status = nullptr;        // pinned host mirror, copied after each launch
    // alpha strings whose coupling rows a row range needs (hy_apply_h_rows)
    int32_t *d_jlist = nullptr;
    int64_t jl_r0 = -1, jl_r1 = -1, jl_n = 0;
};

struct hy_pool {
    const hy_ham *h = nullptr;
    std::vector<hy::PoolOpHost> ops;
    std::vector<hy::k::ConsDev> cons;
    std::vector<hy::k::OpDev> opd;
    hy::PatternLists pa, pb;
    DevArena arena;
    hy::k::OpDev *d_op = nullptr;
    hy::k::ConsDev *d_cons = nullptr;
    uint32_t *d_aent = nullptr, *d_bent = nullptr;
    int64_t *d_aoff = nullptr, *d_acnt = nullptr, *d_boff = nullptr, *d_bcnt = nullptr;
    int32_t *d_desc = nullptr;   // [K][11] operator descriptors (ranker features)
    // first refused entry of a device operator list (position << 32 | index),
    // ~0 when none; the pinned mirror is copied after each screen that read
    // a device list and reported by the next screen call on this pool
    unsigned long long *d_bad = nullptr;
    unsigned long long *h_bad = nullptr;
    int qubit = 0;                  // HY_POOL_QEB: qubit excitations, no sign
};

struct hy_batch {
    std::vector<const hy_ham *> hams;
    std::vector<int64_t> offsets;   // count + 1
    std::vector<int> order;         // molecules by decreasing row cost
    int64_t total = 0, n_tasks = 0;
    int nb_max = 0, nn_max = 0, num_sms = 0;
    hy_batch_tile tile{64, 4, 0};
    hy::k::BatchMol<double> *d_mols64 = nullptr;
    hy::k::BatchMol<float> *d_mols32 = nullptr;
    int2 *d_tasks = nullptr;
    int *d_counter = nullptr;
    double *d_row_energy = nullptr;
    int64_t *d_base = nullptr, *d_rows = nullptr;
    // captured graph and what it was captured for
    cudaGraphExec_t gexec = nullptr;
    const void *g_psi = nullptr;
    void *g_sigma = nullptr;
    double *g_energies = nullptr;
    int g_dt = -1;
    hy_batch_tile g_tile{0, 0, 0};
    // pool screen (hy_batch_set_pools / hy_batch_gradients)
    std::vector<const hy_pool *> pools;
    std::vector<int64_t> pool_base;            // count + 1: full-screen entries
    hy::k::BatchPool *d_pools = nullptr;
    int64_t *d_pool_base = nullptr;
    double *d_gpart = nullptr;
    int64_t n_gpart = 0;
    unsigned long long *d_gctr = nullptr, *d_gbad = nullptr, *h_gbad = nullptr;
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Workspace layout: [partials: P doubles][scalar: 8 doubles][3 state buffers]
struct WsLayout {
    size_t partials, scalar, buf0, buf1, buf2, total;
};

WsLayout ws_layout(const hy_ham *h, size_t n_partials, size_t elem)
{
    WsLayout L;
    L.partials = 0;
    L.scalar = align_up(n_partials * sizeof(double));
    L.buf0 = L.scalar + align_up(8 * sizeof(double));
    size_t sb = align_up(size_t(h->N) * elem);
    L.buf1 = L.buf0 + sb;
    L.buf2 = L.buf1 + sb;
    L.total = L.buf2 + sb;
    return L;
}

hy_status ensure_ws(hy_ham *h, size_t bytes)
{
    if (bytes <= h->ws_bytes) return HY_OK;
    if (h->ws) {
        cudaError_t e = cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree(workspace)");
    }
    cudaError_t e = cudaMalloc(&h->ws, bytes);
    if (e != cudaSuccess) {
        h->ws = nullptr;
        return cuda_fail(e, "cudaMalloc(workspace)");
    }
    h->ws_bytes = bytes;
    return HY_OK;
}

size_t n_partials_needed(const hy_ham *h, int64_t n_ops)
{
    // dot partials, or the tracked rotation's (<= 16 blocks per SM + 128)
    size_t p = std::max(size_t(h->dot_blocks), size_t(16) * h->num_sms + 128) + 64;
    size_t g = size_t(n_ops) + size_t(4) * h->num_sms + 1024;
    return p > g ? p : g;
}

int grad_chunks(const hy_ham *h, int64_t n_ops)
{
    int64_t ch = (int64_t(4) * h->num_sms + n_ops - 1) / (n_ops > 0 ? n_ops : 1);
    if (ch < 1) ch = 1;
    if (ch > 1024) ch = 1024;
    return int(ch);
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

bool check_symmetric(const double *h1, const double *h2, int n, std::string &why)
{
    double scale = 1.0;
    for (int i = 0; i < n * n; ++i) {
        if (!std::isfinite(h1[i])) { why = "h1 has a non-finite entry"; return false; }
        scale = std::fmax(scale, std::fabs(h1[i]));
    }
    size_t n4 = size_t(n) * n * n * n;
    for (size_t i = 0; i < n4; ++i) {
        if (!std::isfinite(h2[i])) { why = "h2 has a non-finite entry"; return false; }
        scale = std::fmax(scale, std::fabs(h2[i]));
    }
    const double tol = 1e-12 * scale;
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
            if (std::fabs(h1[p * n + q] - h1[q * n + p]) > tol) {
                why = "h1 is not symmetric";
                return false;
            }
    auto at = [&](int p, int q, int r, int s) {
        return h2[((size_t(p) * n + q) * n + r) * n + s];
    };
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
            for (int r = 0; r < n; ++r)
                for (int s = 0; s < n; ++s) {
                    double v = at(p, q, r, s);
                    if (std::fabs(v - at(q, p, s, r)) > tol ||
                        std::fabs(v - at(r, s, p, q)) > tol) {
                        why = "h2 lacks the (pq|rs) = (qp|sr) = (rs|pq) symmetry";
                        return false;
                    }
                }
    return true;
}

// Phase A of the float coupling forms T rows per alpha string J; the output
// rows [r0, r1) need the strings themselves and their single-excitation
// partners.  Every J for the whole range; else a list (sorted, uploaded once
// per distinct range and kept on the handle).
hy_status coupling_jlist(hy_ham *h, int64_t r0, int64_t r1, const int32_t **list, int64_t *nJ)
{
    if (r0 == 0 && r1 == h->Na) {
        *list = nullptr;
        *nJ = h->Na;
        return HY_OK;
    }
    if (h->jl_r0 != r0 || h->jl_r1 != r1) {
        std::vector<uint8_t> need(size_t(h->Na), 0);
        const int nex = h->A.nex;
        for (int64_t a = r0; a < r1; ++a) {
            need[size_t(a)] = 1;
            for (int e = 0; e < nex; ++e) need[h->A.ex[size_t(a) * nex + e] & 0xFFFFu] = 1;
        }
        std::vector<int32_t> js;
        for (int64_t j = 0; j < h->Na; ++j)
            if (need[size_t(j)]) js.push_back(int32_t(j));
        if (!h->d_jlist) {
            cudaError_t e = cudaMalloc(&h->d_jlist, size_t(h->Na) * sizeof(int32_t));
            if (e != cudaSuccess) {
                h->d_jlist = nullptr;
                return cuda_fail(e, "cudaMalloc(coupling row list)");
            }
        }
        HY_CUDA(cudaMemcpy(h->d_jlist, js.data(), js.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice), "upload coupling row list");
        h->jl_r0 = r0;
        h->jl_r1 = r1;
        h->jl_n = int64_t(js.size());
    }
    *list = h->d_jlist;
    *nJ = h->jl_n;
    return HY_OK;
}

// sigma rows [r0, r1) (alpha strings) of H psi; sigma holds those rows only.
// Every output element is formed by the same arithmetic in the same order
// whatever the range, so shards concatenate to the full sigma bit for bit.
template <typename T>
hy_status apply_h_t(hy_ham *h, const T *psi, T *sigma, cudaStream_t st, int64_t r0, int64_t r1)
{
    const int64_t nr = r1 - r0;
    if (nr <= 0) return HY_OK;
    const WsLayout L = ws_layout(h, n_partials_needed(h, 0), sizeof(T));
    // float: room for the dense coupling's intermediate T after the state
    // buffers, sized before any launch; without it the direct kernel runs
    const int64_t Nbp = (h->Nb + 63) / 64 * 64;
    const size_t tbytes = sizeof(T) == sizeof(float)
        ? size_t(h->Na) * size_t(h->A.nex + 1) * size_t(Nbp) * sizeof(float) : 0;
    bool dense = false;
    if (tbytes && ensure_ws(h, L.total + tbytes) == HY_OK) {
        dense = true;
    } else {
        cudaGetLastError();   // clear a failed allocation
        hy_status s = ensure_ws(h, L.total);
        if (s != HY_OK) return s;
    }
    char *ws = static_cast<char *>(h->ws);
    T *psiT = reinterpret_cast<T *>(ws + L.buf1);
    T *tau = reinterpret_cast<T *>(ws + L.buf2);
    const bool f64 = sizeof(T) == sizeof(double);
    const DevCsr<T> *Ma, *Mb;
    const T *V;
    if constexpr (sizeof(T) == sizeof(double)) {
        Ma = &h->Ma64; Mb = &h->Mb64; V = h->d_V64;
    } else {
        Ma = &h->Ma32; Mb = &h->Mb32; V = h->d_V32;
    }
    (void)f64;
    const double rows_det = double(nr) * double(h->Nb);
    hy::ProfScope prof(HY_PROF_HPSI, st, 2.0 * rows_det * sizeof(T),
                       2.0 * double(hy::ham_connections(h)) * rows_det);
    HY_CUDA(hy::k::spmm<T>(Ma->ptr + r0, Ma->col, Ma->val, nr, psi, sigma, h->Nb,
                           false, st), "alpha part");
    HY_CUDA(hy::k::transpose<T>(psi + r0 * h->Nb, psiT, nr, h->Nb, st), "transpose");
    HY_CUDA(hy::k::spmm<T>(Mb->ptr, Mb->col, Mb->val, h->Nb, psiT, tau, nr,
                           false, st), "beta part");
    HY_CUDA(hy::k::add_transposed<T>(tau, sigma, nr, h->Nb, st), "beta add");
    if constexpr (sizeof(T) == sizeof(float)) {
        if (dense) {
            hy::k::CplDenseArgs d;
            d.psi = psi;
            d.sigma = sigma;
            d.T = reinterpret_cast<float *>(static_cast<char *>(h->ws) + L.total);
            d.aex = h->d_aex;
            d.inv = h->d_ainv;
            d.bexT = h->d_bexT;
            d.astr = h->d_astr;
            d.bstr = h->d_bstr;
            d.V = h->d_V32;
            d.n = h->n;
            d.nexa = h->A.nex;
            d.nexb = h->B.nex;
            d.Na = h->Na;
            d.Nb = h->Nb;
            d.Nbp = Nbp;
            d.row0 = r0;
            d.row1 = r1;
            hy_status sj = coupling_jlist(h, r0, r1, &d.jlist, &d.nJ);
            if (sj != HY_OK) return sj;
            if (h->prof) cudaEventRecord(h->ev0, st);
            bool done = false;
            if ((h->cpl_impl == 0 || h->cpl_impl == 2) && h->d_status) {
                const cudaError_t e = hy::k::coupling_tc(d, h->d_status, h->tc_spin_limit,
                                                         h->cpl_impl == 0 ? 1 : 0, h->num_sms, st);
                if (e == cudaSuccess) {
                    HY_CUDA(hy::k::coupling_gather(d, h->num_sms, st), "alpha-beta gather");
                    HY_CUDA(cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int),
                                            cudaMemcpyDeviceToHost, st), "status copy");
                    done = true;
                } else if (e != cudaErrorInvalidValue) {
                    return cuda_fail(e, "alpha-beta coupling (tensor cores)");
                }
            }
            if (!done)
                HY_CUDA(hy::k::coupling_dense(d, h->num_sms, st), "alpha-beta coupling (dense)");
            if (h->prof) cudaEventRecord(h->ev1, st);
            return HY_OK;
        }
    }
    hy::k::CouplingArgs<T> a;
    a.psi = psi;
    a.sigma = sigma;
    a.aex = h->d_aex;
    a.bexT = h->d_bexT;
    a.astr = h->d_astr;
    a.bstr = h->d_bstr;
    a.V = V;
    a.n = h->n;
    a.nexa = h->A.nex;
    a.nexb = h->B.nex;
    a.Na = h->Na;
    a.Nb = h->Nb;
    a.row0 = r0;
    a.row1 = r1;
    if (h->prof) cudaEventRecord(h->ev0, st);
    HY_CUDA(hy::k::coupling<T>(a, h->num_sms, st), "alpha-beta coupling");
    if (h->prof) cudaEventRecord(h->ev1, st);
    return HY_OK;
}

template <typename T>
hy_status dot_t(hy_ham *h, const T *x, const T *y, double *out, cudaStream_t st,
                int64_t len = -1)
{
    if (len < 0) len = h->N;
    const WsLayout L = ws_layout(h, n_partials_needed(h, 0), sizeof(T));
    hy_status s = ensure_ws(h, L.total);
    if (s != HY_OK) return s;
    double *partials = reinterpret_cast<double *>(static_cast<char *>(h->ws) + L.partials);
    hy::ProfScope prof(HY_PROF_REDUCE, st, 2.0 * double(len) * sizeof(T));
    HY_CUDA(hy::k::dot<T>(x, y, len, partials, h->dot_blocks, out, st), "dot");
    return HY_OK;
}

template <typename T>
hy_status normalize_t(hy_ham *h, T *psi, cudaStream_t st)
{
    const WsLayout L = ws_layout(h, n_partials_needed(h, 0), sizeof(T));
    hy_status s = ensure_ws(h, L.total);
    if (s != HY_OK) return s;
    double *n2 = reinterpret_cast<double *>(static_cast<char *>(h->ws) + L.scalar);
    s = dot_t<T>(h, psi, psi, n2, st);
    if (s != HY_OK) return s;
    hy::ProfScope prof(HY_PROF_REDUCE, st, 2.0 * double(h->N) * sizeof(T));
    HY_CUDA(hy::k::scale_rsqrt<T>(psi, h->N, n2, st), "normalize");
    return HY_OK;
}

template <typename T>
hy_status energy_t(hy_ham *h, const T *psi, const T *sigma, double *e, cudaStream_t st)
{
    const WsLayout L = ws_layout(h, n_partials_needed(h, 0), sizeof(T));
    hy_status s = ensure_ws(h, L.total);
    if (s != HY_OK) return s;
    if (!sigma) {
        T *tmp = reinterpret_cast<T *>(static_cast<char *>(h->ws) + L.buf0);
        s = apply_h_t<T>(h, psi, tmp, st, 0, h->Na);
        if (s != HY_OK) return s;
        sigma = tmp;
    }
    return dot_t<T>(h, psi, sigma, e, st);
}

template <typename T>
hy_status grad_t(hy_ham *h, const hy_pool *p, const T *psi, const T *sigma,
                 const int32_t *ops, int64_t n_ops, double *g, cudaStream_t st)
{
    const WsLayout L = ws_layout(h, n_partials_needed(h, n_ops), sizeof(T));
    hy_status s = ensure_ws(h, L.total);
    if (s != HY_OK) return s;
    hy::k::GradArgs<T> a;
    a.psi = psi;
    a.sigma = sigma;
    a.ops = ops;
    a.n_ops = n_ops;
    a.opd = p->d_op;
    a.cons = p->d_cons;
    a.aent = p->d_aent;
    a.aoff = p->d_aoff;
    a.acnt = p->d_acnt;
    a.bent = p->d_bent;
    a.boff = p->d_boff;
    a.bcnt = p->d_bcnt;
    a.Na = h->Na;
    a.Nb = h->Nb;
    a.CH = grad_chunks(h, n_ops);
    a.partials = reinterpret_cast<double *>(static_cast<char *>(h->ws) + L.partials);
    a.g = g;
    a.K = int64_t(p->ops.size());
    a.bad = p->d_bad;
    double bytes = 0.0;     // pairs of the listed operators (known for the whole pool)
    if (!ops)
        for (const auto &od : p->opd)
            for (int q = 0; q < od.nc; ++q) {
                const hy::k::ConsDev &cd = p->cons[q == 0 ? od.c0 : od.c1];
                const double nr = cd.ap < 0 ? double(h->Na) : double(p->pa.cnt[cd.ap]);
                const double nc = cd.bp < 0 ? double(h->Nb) : double(p->pb.cnt[cd.bp]);
                bytes += 4.0 * nr * nc * sizeof(T);
            }
    hy::ProfScope prof(HY_PROF_SCREEN, st, bytes);
    HY_CUDA(hy::k::grad<T>(a, st), "pool gradients");
    return HY_OK;
}

template <typename T>
hy_status excite_t(hy_ham *h, const hy_pool *p, int64_t k, double theta, T *psi,
                   cudaStream_t st)
{
    const hy::k::OpDev &od = p->opd[k];
    const double c = std::cos(theta), sn = std::sin(theta);
    for (int q = 0; q < od.nc; ++q) {
        const hy::k::ConsDev &cd = p->cons[q == 0 ? od.c0 : od.c1];
        const uint32_t *ae = nullptr, *be = nullptr;
        int64_t nr = h->Na, nc = h->Nb;
        if (cd.ap >= 0) { ae = p->d_aent + p->pa.off[cd.ap]; nr = p->pa.cnt[cd.ap]; }
        if (cd.bp >= 0) { be = p->d_bent + p->pb.off[cd.bp]; nc = p->pb.cnt[cd.bp]; }
        hy::ProfScope prof(HY_PROF_EXCITE, st, 4.0 * double(nr) * double(nc) * sizeof(T));
        HY_CUDA(hy::k::excite<T>(psi, ae, nr, be, nc, h->Nb, c, cd.eps * sn, st),
                "excitation");
    }
    return HY_OK;
}

// exp(theta A_k) adding the FP64-accurate change of ||psi||^2 to *norm2
template <typename T>
hy_status excite_tracked_t(hy_ham *h, const hy_pool *p, int64_t k, double theta, T *psi,
                           double *norm2, cudaStream_t st)
{
    const WsLayout L = ws_layout(h, n_partials_needed(h, 0), sizeof(T));
    hy_status s = ensure_ws(h, L.total);
    if (s != HY_OK) return s;
    double *partials = reinterpret_cast<double *>(static_cast<char *>(h->ws) + L.partials);
    const hy::k::OpDev &od = p->opd[k];
    const double c = std::cos(theta), sn = std::sin(theta);
    for (int q = 0; q < od.nc; ++q) {
        const hy::k::ConsDev &cd = p->cons[q == 0 ? od.c0 : od.c1];
        const uint32_t *ae = nullptr, *be = nullptr;
        int64_t nr = h->Na, nc = h->Nb;
        if (cd.ap >= 0) { ae = p->d_aent + p->pa.off[cd.ap]; nr = p->pa.cnt[cd.ap]; }
        if (cd.bp >= 0) { be = p->d_bent + p->pb.off[cd.bp]; nc = p->pb.cnt[cd.bp]; }
        hy::ProfScope prof(HY_PROF_EXCITE, st, 4.0 * double(nr) * double(nc) * sizeof(T));
        HY_CUDA(hy::k::excite_n<T>(psi, ae, nr, be, nc, h->Nb, c, cd.eps * sn, partials, norm2,
                                   h->num_sms, st),
                "tracked excitation");
    }
    return HY_OK;
}

bool valid_dtype(hy_dtype dt) { return dt == HY_F64 || dt == HY_F32; }

// Export a Pauli table in the Hermitian-Pauli convention: since
// X^x Z^z = (-i)^#Y P, the coefficient of P is c_xz (-1)^(#Y/2) (#Y even).
void copy_pauli(const hy::PauliTable &t, uint64_t *x, uint64_t *z, double *coeff,
                int64_t *group_offsets)
{
    for (size_t i = 0; i < t.x.size(); ++i) {
        x[i] = t.x[i];
        z[i] = t.z[i];
        int ny = __builtin_popcountll(t.x[i] & t.z[i]);
        coeff[i] = ((ny / 2) & 1) ? -t.cxz[i] : t.cxz[i];
    }
    for (size_t g = 0; g < t.group_off.size(); ++g) group_offsets[g] = t.group_off[g];
}

}  // namespace

namespace {
hy_status finish_ham(hy_ham *h, hy_ham **out);
}  // namespace

extern "C" {

const char *hy_last_error(void) { return g_err.c_str(); }

const char *hy_version(void) { return "hyperion-gb300 0.1 (sm_103a)"; }

int64_t hy_launch_count(void) { return int64_t(g_launches.load(std::memory_order_relaxed)); }

hy_status hy_build_hamiltonian(const double *h1, const double *h2, double e_core,
                               int n_orb, int n_alpha, int n_beta,
                               double prune_tol, hy_ham **out)
{
    if (!out) return fail(HY_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!h1 || !h2) return fail(HY_ERR_ARG, "h1 / h2 is NULL");
    if (n_orb < 1 || n_orb > hy::kMaxOrb)
        return fail(HY_ERR_ARG, "n_orb must be in [1, 16]");
    if (n_alpha < 0 || n_beta < 0 || n_alpha > n_orb || n_beta > n_orb)
        return fail(HY_ERR_ARG, "electron counts must be in [0, n_orb]");
    if (!(prune_tol >= 0.0) || !std::isfinite(e_core))
        return fail(HY_ERR_ARG, "prune_tol must be >= 0 and e_core finite");
    std::string why;
    if (!check_symmetric(h1, h2, n_orb, why)) return fail(HY_ERR_ARG, why);

    hy_ham *h = new (std::nothrow) hy_ham;
    if (!h) return fail(HY_ERR_OOM, "host allocation failed");
    h->n = n_orb;
    h->na = n_alpha;
    h->nb = n_beta;
    hy::build_string_space(n_orb, n_alpha, h->A);
    hy::build_string_space(n_orb, n_beta, h->B);
    h->Na = h->A.N;
    h->Nb = h->B.N;
    h->N = h->Na * h->Nb;
    if (!hy::build_pauli_table(h1, h2, e_core, n_orb, prune_tol, h->pauli, why) ||
        !hy::check_two_body_structure(h->pauli, n_orb, why)) {
        delete h;
        return fail(HY_ERR_UNSUPPORTED, why);
    }
    h->h1h.assign(h1, h1 + size_t(n_orb) * n_orb);
    h->h2h.assign(h2, h2 + size_t(n_orb) * n_orb * n_orb * n_orb);
    return finish_ham(h, out);
}

}  // extern "C"

namespace {

// The rest of a build from h's Pauli table (set, with the string spaces and
// the host integrals): fold the kernel tables, query the device and upload.
// Takes ownership of h (released on failure).
// The same-spin tables Ma (alpha strings) and Mb (beta strings, minus E0 on
// the diagonal) folded on the device from the Pauli table (hy_fold.cu): the
// table's groups and terms and, per spin, a direct map from an X-mask within
// the spin to its group are uploaded; rows go through a fixed-stride scratch
// and are compacted into CSR arrays shared by the double and float views.
hy_status fold_same_spin(hy_ham *h)
{
    const int n = h->n;
    const hy::PauliTable &t = h->pauli;
    std::vector<int32_t> grpA(size_t(1) << n, -1), grpB(size_t(1) << n, -1);
    const uint64_t low = (uint64_t(1) << n) - 1;
    for (const auto &kv : t.group_of_x) {
        if ((kv.first & ~low) == 0) grpA[kv.first] = int32_t(kv.second);
        if ((kv.first & low) == 0 && (kv.first >> n) <= low) grpB[kv.first >> n] = int32_t(kv.second);
    }
    DevArena &ar = h->arena;
    int32_t *d_grpA = nullptr, *d_grpB = nullptr;
    int64_t *d_goff = nullptr;
    uint64_t *d_z = nullptr;
    double *d_c = nullptr;
    HY_CUDA(ar.upload(&d_grpA, grpA.data(), grpA.size()), "upload Pauli groups");
    HY_CUDA(ar.upload(&d_grpB, grpB.data(), grpB.size()), "upload Pauli groups");
    HY_CUDA(ar.upload(&d_goff, t.group_off.data(), t.group_off.size()), "upload Pauli groups");
    HY_CUDA(ar.upload(&d_z, t.z.data(), t.z.size()), "upload Pauli terms");
    HY_CUDA(ar.upload(&d_c, t.cxz.data(), t.cxz.size()), "upload Pauli terms");
    const int64_t stride = std::max(hy::k::fold_candidates(n, h->na), hy::k::fold_candidates(n, h->nb));
    const int64_t rows = std::max(h->Na, h->Nb);
    int32_t *tcol = nullptr, *len = nullptr;
    double *tval = nullptr;
    cudaError_t e = cudaMalloc(&tcol, size_t(rows * stride) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&tval, size_t(rows * stride) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&len, size_t(rows) * sizeof(int32_t));
    auto done = [&]() {
        cudaFree(tcol);
        cudaFree(tval);
        cudaFree(len);
    };
    for (int spin = 0; spin < 2 && e == cudaSuccess; ++spin) {
        const int64_t N = spin == 0 ? h->Na : h->Nb;
        hy::k::FoldArgs a;
        a.str = spin == 0 ? h->d_astr : h->d_bstr;
        a.N = N;
        a.n = n;
        a.k = spin == 0 ? h->na : h->nb;
        a.shift = spin == 0 ? 0 : n;
        a.sub_diag = spin == 0 ? 0.0 : h->kt.E0;
        a.grp = spin == 0 ? d_grpA : d_grpB;
        a.goff = d_goff;
        a.z = d_z;
        a.c = d_c;
        a.binom33 = h->d_binom;
        a.stride = stride;
        a.tcol = tcol;
        a.tval = tval;
        a.len = len;
        DevCsr<double> &M64 = spin == 0 ? h->Ma64 : h->Mb64;
        DevCsr<float> &M32 = spin == 0 ? h->Ma32 : h->Mb32;
        const int64_t cap = N * hy::k::fold_candidates(n, a.k);
        e = ar.alloc(&M64.ptr, size_t(N + 1));
        if (e == cudaSuccess) e = ar.alloc(&M64.col, size_t(cap > 0 ? cap : 1));
        if (e == cudaSuccess) e = ar.alloc(&M64.val, size_t(cap > 0 ? cap : 1));
        if (e == cudaSuccess) e = ar.alloc(&M32.val, size_t(cap > 0 ? cap : 1));
        if (e != cudaSuccess) break;
        M32.ptr = M64.ptr;
        M32.col = M64.col;
        e = hy::k::fold_rows(a, h->num_sms, nullptr);
        if (e == cudaSuccess)
            e = hy::k::fold_compact(a, M64.ptr, M64.col, M64.val, M32.val, h->num_sms, nullptr);
        int32_t nnz = 0;
        if (e == cudaSuccess)
            e = cudaMemcpy(&nnz, M64.ptr + N, sizeof(int32_t), cudaMemcpyDeviceToHost);
        (spin == 0 ? h->nnz_a : h->nnz_b) = nnz;
    }
    done();
    if (e != cudaSuccess) return cuda_fail(e, "same-spin tables");
    return HY_OK;
}

// host copies of the same-spin tables, for host consumers (the explicit-H
// builder); copied once from the device
hy_status ensure_host_csr(hy_ham *h)
{
    if (!h->kt.Ma.ptr.empty()) return HY_OK;
    for (int spin = 0; spin < 2; ++spin) {
        hy::CsrHost &M = spin == 0 ? h->kt.Ma : h->kt.Mb;
        const DevCsr<double> &D = spin == 0 ? h->Ma64 : h->Mb64;
        const int64_t N = spin == 0 ? h->Na : h->Nb, nnz = spin == 0 ? h->nnz_a : h->nnz_b;
        M.rows = N;
        M.ptr.resize(size_t(N + 1));
        M.col.resize(size_t(nnz));
        M.val.resize(size_t(nnz));
        HY_CUDA(cudaMemcpy(M.ptr.data(), D.ptr, size_t(N + 1) * sizeof(int32_t),
                           cudaMemcpyDeviceToHost), "copy same-spin table");
        if (nnz) {
            HY_CUDA(cudaMemcpy(M.col.data(), D.col, size_t(nnz) * sizeof(int32_t),
                               cudaMemcpyDeviceToHost), "copy same-spin table");
            HY_CUDA(cudaMemcpy(M.val.data(), D.val, size_t(nnz) * sizeof(double),
                               cudaMemcpyDeviceToHost), "copy same-spin table");
        }
    }
    return HY_OK;
}

hy_status finish_ham(hy_ham *h, hy_ham **out)
{
    const int n_orb = h->n;
    const double *h1 = h->h1h.data(), *h2 = h->h2h.data();
    hy::fold_coupling(h->pauli, n_orb, h->kt);

    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "device query");
    }
    h->dot_blocks = 8 * h->num_sms;
    e = cudaMalloc(&h->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_status, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(h->d_status);
        delete h;
        return cuda_fail(e, "status flag");
    }
    *h->h_status = 0;

    // bexT: beta excitations transposed to [nexb][Nb] for coalesced reads
    std::vector<uint32_t> bexT(size_t(h->B.nex) * h->Nb);
    for (int64_t b = 0; b < h->Nb; ++b)
        for (int f = 0; f < h->B.nex; ++f)
            bexT[size_t(f) * h->Nb + b] = h->B.ex[size_t(b) * h->B.nex + f];
    std::vector<uint32_t> binom(33 * 33);
    for (int i = 0; i < 33; ++i)
        for (int j = 0; j < 33; ++j) binom[i * 33 + j] = hy::binom(i, j);
    // colex rank of every n-bit string (sum over its set bits, the i-th from
    // the bottom at position p, of C(p, i + 1)), one string at a time from
    // the string without its top bit
    std::vector<uint16_t> rank16(size_t(1) << n_orb, 0);
    for (uint32_t msk = 1; msk < (1u << n_orb); ++msk) {
        const int top = 31 - __builtin_clz(msk);
        rank16[msk] = uint16_t(rank16[msk & ~(1u << top)] +
                               hy::binom(top, __builtin_popcount(msk)));
    }
    std::vector<float> V32(h->kt.V.begin(), h->kt.V.end());

    hy_status s = HY_OK;
    DevArena &ar = h->arena;
    auto up = [&](cudaError_t err, const char *what) {
        if (s == HY_OK && err != cudaSuccess) s = cuda_fail(err, what);
    };
    up(ar.upload(&h->d_astr, h->A.str.data(), h->A.str.size()), "upload alpha strings");
    up(ar.upload(&h->d_bstr, h->B.str.data(), h->B.str.size()), "upload beta strings");
    up(ar.upload(&h->d_aex, h->A.ex.data(), h->A.ex.size()), "upload alpha excitations");
    up(ar.upload(&h->d_ainv, h->A.inv.data(), h->A.inv.size()), "upload inverse excitations");
    up(ar.upload(&h->d_bexT, bexT.data(), bexT.size()), "upload beta excitations");
    up(ar.upload(&h->d_bex, h->B.ex.data(), h->B.ex.size()), "upload beta excitations");
    up(ar.upload(&h->d_binom, binom.data(), binom.size()), "upload binomials");
    up(ar.upload(&h->d_rank16, rank16.data(), rank16.size()), "upload string ranks");
    up(ar.upload(&h->d_V64, h->kt.V.data(), h->kt.V.size()), "upload V");
    up(ar.upload(&h->d_V32, V32.data(), V32.size()), "upload V32");
    up(ar.upload(&h->d_h1, h1, size_t(n_orb) * n_orb), "upload h1");
    up(ar.upload(&h->d_eri, h2, size_t(n_orb) * n_orb * n_orb * n_orb), "upload h2");
    h->occ_blocks = 2 * h->num_sms;
    {
        const size_t nn = size_t(n_orb) * n_orb;
        up(ar.alloc(&h->d_occ_partial, size_t(h->occ_blocks) * 33, true), "occupation partials");
        up(ar.alloc(&h->d_occ, size_t(2 * n_orb), true), "occupations");
        up(ar.alloc(&h->d_pairB, 2 * size_t(h->Na) * nn, true), "touched-weight partials");
        up(ar.alloc(&h->d_pairRs, 2 * size_t(h->Na), true), "touched-weight partials");
        up(ar.alloc(&h->d_pairD, 2 * nn * nn, true), "touched weights");
        up(ar.alloc(&h->d_pairP, size_t(hy::k::pair_splits()) * nn * nn, true),
           "touched-weight partials");
        up(ar.alloc(&h->d_pairRows, size_t(h->Na) + 1, true), "touched-weight rows");
        up(ar.alloc(&h->d_occw, size_t(34), true), "occupation scratch");
    }
    if (s == HY_OK) s = fold_same_spin(h);
    if (s != HY_OK) {
        std::string msg = g_err;
        hy_ham_destroy(h);
        g_err = msg;
        return s;
    }
    *out = h;
    return HY_OK;
}

// position of spin orbital j (blocked order) along the qubit chain the
// partition cuts: blocked keeps it, interleaved puts orbital p's alpha and
// beta spin orbitals next to each other (2p, 2p + 1)
int chain_position(int j, int n, int interleaved)
{
    if (!interleaved) return j;
    return j < n ? 2 * j : 2 * (j - n) + 1;
}

}  // namespace

extern "C" {

hy_status hy_ham_partition(const hy_ham *src, int eta, int interleaved, int part, hy_ham **out)
{
    if (!out) return fail(HY_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!src) return fail(HY_ERR_ARG, "handle is NULL");
    const int n = src->n, nq = 2 * n;
    if (eta < 0 || eta > 5 || (nq % (1 << eta)) != 0)
        return fail(HY_ERR_ARG, "2^eta must divide the qubit count");
    if (part != 0 && part != 1) return fail(HY_ERR_ARG, "part must be 0 (H_eta) or 1 (the rest)");
    const int width = nq >> eta;                      // qubits per block
    hy_ham *h = new (std::nothrow) hy_ham;
    if (!h) return fail(HY_ERR_OOM, "host allocation failed");
    h->n = n;
    h->na = src->na;
    h->nb = src->nb;
    h->A = src->A;
    h->B = src->B;
    h->Na = src->Na;
    h->Nb = src->Nb;
    h->N = src->N;
    h->h1h = src->h1h;
    h->h2h = src->h2h;
    // the terms whose support (x | z) lies inside one block (the identity
    // included), or the others
    const hy::PauliTable &t = src->pauli;
    hy::PauliTable &f = h->pauli;
    f.n_qubits = t.n_qubits;
    const size_t G = t.group_off.size() - 1;
    f.group_off.push_back(0);
    for (size_t g = 0; g < G; ++g) {
        for (int64_t i = t.group_off[g]; i < t.group_off[g + 1]; ++i) {
            const uint64_t sup = t.x[size_t(i)] | t.z[size_t(i)];
            int blk = -1;
            bool inside = true;
            for (uint64_t m = sup; m; m &= m - 1) {
                const int b = chain_position(__builtin_ctzll(m), n, interleaved) / width;
                if (blk < 0) blk = b;
                else if (b != blk) { inside = false; break; }
            }
            if (inside != (part == 0)) continue;
            f.x.push_back(t.x[size_t(i)]);
            f.z.push_back(t.z[size_t(i)]);
            f.cxz.push_back(t.cxz[size_t(i)]);
        }
        if (int64_t(f.x.size()) > f.group_off.back()) {
            f.group_of_x[f.x.back()] = int64_t(f.group_off.size()) - 1;
            f.group_off.push_back(int64_t(f.x.size()));
        }
    }
    std::string why;
    if (!hy::check_two_body_structure(f, n, why)) {
        delete h;
        return fail(HY_ERR_UNSUPPORTED, why);
    }
    return finish_ham(h, out);
}

hy_status hy_ham_destroy(hy_ham *h)
{
    if (!h) return HY_OK;
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    cudaFree(h->d_status);
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->d_jlist) cudaFree(h->d_jlist);
    h->arena.release();
    if (h->ws) cudaFree(h->ws);
    cudaFree(h->tw.cnt);
    cudaFree(h->tw.ptr);
    cudaFree(h->tw.cur);
    cudaFree(h->tw.mask);
    cudaFree(h->tw.w);
    delete h;
    return HY_OK;
}

hy_status hy_ham_set_coupling(hy_ham *h, int impl)
{
    if (!h) return fail(HY_ERR_ARG, "handle is NULL");
    if (impl < 0 || impl > 2)
        return fail(HY_ERR_ARG, "impl must be 0 (tensor cores), 1 (SIMT) or 2 (test mode)");
    h->cpl_impl = impl;
    return HY_OK;
}

hy_status hy_ham_set_wait_limit(hy_ham *h, int64_t polls)
{
    if (!h) return fail(HY_ERR_ARG, "handle is NULL");
    if (polls < 1) return fail(HY_ERR_ARG, "the wait limit must be at least one poll");
    h->tc_spin_limit = polls;
    return HY_OK;
}

hy_status hy_ham_profile(hy_ham *h, int enable)
{
    if (!h) return fail(HY_ERR_ARG, "handle is NULL");
    if (enable && !h->ev0) {
        HY_CUDA(cudaEventCreate(&h->ev0), "event");
        HY_CUDA(cudaEventCreate(&h->ev1), "event");
    }
    h->prof = enable != 0;
    return HY_OK;
}

hy_status hy_ham_coupling_ms(const hy_ham *h, float *ms)
{
    if (!h || !ms) return fail(HY_ERR_ARG, "NULL argument");
    if (!h->ev0) return fail(HY_ERR_ARG, "profiling was never enabled");
    HY_CUDA(cudaEventSynchronize(h->ev1), "event synchronize");
    HY_CUDA(cudaEventElapsedTime(ms, h->ev0, h->ev1), "event elapsed");
    return HY_OK;
}

hy_status hy_ham_info(const hy_ham *h, int64_t *n_det, int64_t *n_alpha_str,
                      int64_t *n_beta_str, int64_t *n_groups, int64_t *n_terms)
{
    if (!h) return fail(HY_ERR_ARG, "handle is NULL");
    if (n_det) *n_det = h->N;
    if (n_alpha_str) *n_alpha_str = h->Na;
    if (n_beta_str) *n_beta_str = h->Nb;
    if (n_groups) *n_groups = int64_t(h->pauli.group_off.size()) - 1;
    if (n_terms) *n_terms = int64_t(h->pauli.x.size());
    return HY_OK;
}

hy_status hy_ham_upload_bytes(const hy_ham *h, const hy_pool *p, int64_t *bytes)
{
    if (!h || !bytes) return fail(HY_ERR_ARG, "bad arguments");
    if (p && p->h != h) return fail(HY_ERR_ARG, "pool belongs to another Hamiltonian");
    *bytes = h->arena.uploaded + (p ? p->arena.uploaded : 0);
    return HY_OK;
}

hy_status hy_ham_pauli_table(const hy_ham *h, uint64_t *x, uint64_t *z,
                             double *coeff, int64_t *group_offsets)
{
    if (!h || !x || !z || !coeff || !group_offsets)
        return fail(HY_ERR_ARG, "NULL argument");
    copy_pauli(h->pauli, x, z, coeff, group_offsets);
    return HY_OK;
}

hy_status hy_pauli_table_build(const double *h1, const double *h2, double e_core,
                               int n_orb, double prune_tol, int64_t capacity,
                               uint64_t *x, uint64_t *z, double *coeff,
                               int64_t *group_offsets, int64_t *n_terms,
                               int64_t *n_groups)
{
    if (!h1 || !h2 || !n_terms || !n_groups) return fail(HY_ERR_ARG, "NULL argument");
    if (n_orb < 1 || n_orb > hy::kMaxOrb) return fail(HY_ERR_ARG, "n_orb must be in [1, 16]");
    if (!(prune_tol >= 0.0) || !std::isfinite(e_core))
        return fail(HY_ERR_ARG, "prune_tol must be >= 0 and e_core finite");
    std::string why;
    if (!check_symmetric(h1, h2, n_orb, why)) return fail(HY_ERR_ARG, why);
    hy::PauliTable t;
    if (!hy::build_pauli_table(h1, h2, e_core, n_orb, prune_tol, t, why))
        return fail(HY_ERR_UNSUPPORTED, why);
    *n_terms = int64_t(t.x.size());
    *n_groups = int64_t(t.group_off.size()) - 1;
    if (capacity == 0 || !x || !z || !coeff || !group_offsets) return HY_OK;
    if (capacity < *n_terms) return fail(HY_ERR_ARG, "capacity below n_terms");
    copy_pauli(t, x, z, coeff, group_offsets);
    return HY_OK;
}

hy_status hy_rank(const hy_ham *h, const uint64_t *dets, int64_t *idx, int64_t m,
                  void *stream)
{
    if (!h || m < 0 || (m > 0 && (!dets || !idx))) return fail(HY_ERR_ARG, "bad arguments");
    HY_CUDA(hy::k::rank(dets, idx, m, h->n, h->na, h->nb, h->Nb, h->d_binom,
                        as_stream(stream)), "rank");
    return HY_OK;
}

hy_status hy_unrank(const hy_ham *h, const int64_t *idx, uint64_t *dets, int64_t m,
                    void *stream)
{
    if (!h || m < 0 || (m > 0 && (!dets || !idx))) return fail(HY_ERR_ARG, "bad arguments");
    HY_CUDA(hy::k::unrank(idx, dets, m, h->n, h->na, h->nb, h->Na, h->Nb, h->d_binom,
                          as_stream(stream)), "unrank");
    return HY_OK;
}

hy_status hy_apply_h(const hy_ham *hc, const void *psi, void *sigma, hy_dtype dt,
                     void *stream)
{
    hy_ham *h = const_cast<hy_ham *>(hc);
    if (!h || !psi || !sigma || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    if (psi == sigma) return fail(HY_ERR_ARG, "psi and sigma must not alias");
    if (h->h_status && *h->h_status) {
        // an earlier tensor-core coupling gave up waiting: report it once
        *h->h_status = 0;
        HY_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(int), as_stream(stream)), "status reset");
        return fail(HY_ERR_TIMEOUT, "an earlier H psi's tensor-core coupling timed out");
    }
    if (dt == HY_F64)
        return apply_h_t<double>(h, static_cast<const double *>(psi),
                                 static_cast<double *>(sigma), as_stream(stream), 0, h->Na);
    return apply_h_t<float>(h, static_cast<const float *>(psi),
                            static_cast<float *>(sigma), as_stream(stream), 0, h->Na);
}

hy_status hy_dot_rows(const hy_ham *hc, const void *x_rows, const void *y_rows, hy_dtype dt,
                      int64_t row_begin, int64_t row_end, double *out, void *stream)
{
    hy_ham *h = const_cast<hy_ham *>(hc);
    if (!h || !out || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    if (row_begin < 0 || row_end < row_begin || row_end > h->Na)
        return fail(HY_ERR_ARG, "row range outside [0, N_alpha]");
    const int64_t len = (row_end - row_begin) * h->Nb;
    if (len > 0 && (!x_rows || !y_rows)) return fail(HY_ERR_ARG, "bad arguments");
    if (len == 0) {
        HY_CUDA(cudaMemsetAsync(out, 0, sizeof(double), as_stream(stream)), "zero dot");
        return HY_OK;
    }
    if (dt == HY_F64)
        return dot_t<double>(h, static_cast<const double *>(x_rows),
                             static_cast<const double *>(y_rows), out, as_stream(stream), len);
    return dot_t<float>(h, static_cast<const float *>(x_rows), static_cast<const float *>(y_rows),
                        out, as_stream(stream), len);
}

hy_status hy_apply_h_rows(const hy_ham *hc, const void *psi, void *sigma_rows, hy_dtype dt,
                          int64_t row_begin, int64_t row_end, void *stream)
{
    hy_ham *h = const_cast<hy_ham *>(hc);
    if (!h || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    if (row_begin < 0 || row_end < row_begin || row_end > h->Na)
        return fail(HY_ERR_ARG, "row range [" + std::to_string(row_begin) + ", " +
                                    std::to_string(row_end) + ") outside [0, " +
                                    std::to_string(h->Na) + ")");
    if (row_end == row_begin) return HY_OK;       // an empty block: nothing written
    if (!psi || !sigma_rows) return fail(HY_ERR_ARG, "bad arguments");
    const size_t es = dt == HY_F64 ? 8 : 4;
    const char *pb = static_cast<const char *>(psi), *sb = static_cast<const char *>(sigma_rows);
    const size_t psi_bytes = size_t(h->N) * es;
    const size_t sig_bytes = size_t(row_end - row_begin) * size_t(h->Nb) * es;
    if (sb < pb + psi_bytes && pb < sb + sig_bytes)
        return fail(HY_ERR_ARG, "psi and sigma_rows must not overlap");
    if (h->h_status && *h->h_status) {
        *h->h_status = 0;
        HY_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(int), as_stream(stream)), "status reset");
        return fail(HY_ERR_TIMEOUT, "an earlier H psi's tensor-core coupling timed out");
    }
    if (dt == HY_F64)
        return apply_h_t<double>(h, static_cast<const double *>(psi),
                                 static_cast<double *>(sigma_rows), as_stream(stream), row_begin,
                                 row_end);
    return apply_h_t<float>(h, static_cast<const float *>(psi), static_cast<float *>(sigma_rows),
                            as_stream(stream), row_begin, row_end);
}

hy_status hy_energy(const hy_ham *hc, const void *psi, const void *sigma_or_null,
                    hy_dtype dt, double *e_out, void *stream)
{
    hy_ham *h = const_cast<hy_ham *>(hc);
    if (!h || !psi || !e_out || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    if (dt == HY_F64)
        return energy_t<double>(h, static_cast<const double *>(psi),
                                static_cast<const double *>(sigma_or_null), e_out,
                                as_stream(stream));
    return energy_t<float>(h, static_cast<const float *>(psi),
                           static_cast<const float *>(sigma_or_null), e_out,
                           as_stream(stream));
}

hy_status hy_dot(const hy_ham *hc, const void *x, const void *y, hy_dtype dt,
                 double *out, void *stream)
{
    hy_ham *h = const_cast<hy_ham *>(hc);
    if (!h || !x || !y || !out || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    if (dt == HY_F64)
        return dot_t<double>(h, static_cast<const double *>(x),
                             static_cast<const double *>(y), out, as_stream(stream));
    return dot_t<float>(h, static_cast<const float *>(x), static_cast<const float *>(y),
                        out, as_stream(stream));
}

hy_status hy_normalize(const hy_ham *hc, void *psi, hy_dtype dt, void *stream)
{
    hy_ham *h = const_cast<hy_ham *>(hc);
    if (!h || !psi || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    if (dt == HY_F64) return normalize_t<double>(h, static_cast<double *>(psi), as_stream(stream));
    return normalize_t<float>(h, static_cast<float *>(psi), as_stream(stream));
}

hy_status hy_pool_create(const hy_ham *h, hy_pool_kind kind, hy_pool **out)
{
    if (!out) return fail(HY_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!h) return fail(HY_ERR_ARG, "handle is NULL");
    if (kind != HY_POOL_SPIN_ADAPTED_SD && kind != HY_POOL_QEB)
        return fail(HY_ERR_UNSUPPORTED, "unknown pool kind");
    hy_pool *p = new (std::nothrow) hy_pool;
    if (!p) return fail(HY_ERR_OOM, "host allocation failed");
    p->h = h;
    p->qubit = kind == HY_POOL_QEB ? 1 : 0;
    if (p->qubit)
        hy::build_pool_qeb(h->n, h->na, h->nb, p->ops);
    else
        hy::build_pool_spin_adapted(h->n, h->na, h->nb, p->ops);
    const int n = h->n;
    for (const auto &op : p->ops) {
        hy::k::OpDev od{op.desc[0], -1, -1, 0};
        for (int q = 0; q < op.desc[0]; ++q) {
            const int32_t *t = op.desc + 1 + 5 * q;
            int modes[4], dags[4], no = 0;
            if (t[0] == 1) {
                modes[0] = t[1]; dags[0] = 1;
                modes[1] = t[4]; dags[1] = 0;
                no = 2;
            } else {
                modes[0] = t[1]; dags[0] = 1;
                modes[1] = t[2]; dags[1] = 1;
                modes[2] = t[3]; dags[2] = 0;
                modes[3] = t[4]; dags[3] = 0;
                no = 4;
            }
            // C = eps * (alpha ops in order) * (beta ops in order); eps counts
            // the transpositions that move alpha operators left of beta ones.
            hy::PatternKey ka{0, {0, 0, 0, 0}, p->qubit}, kb{0, {0, 0, 0, 0}, p->qubit};
            int inv = 0, nbeta_seen = 0;
            for (int u = 0; u < no; ++u) {
                bool beta = modes[u] >= n;
                int code = 2 * (modes[u] % n) + dags[u];
                if (beta) {
                    kb.ops[kb.nops++] = code;
                    ++nbeta_seen;
                } else {
                    ka.ops[ka.nops++] = code;
                    inv += nbeta_seen;
                }
            }
            if ((ka.nops & 1) || (kb.nops & 1)) {
                delete p;
                return fail(HY_ERR_UNSUPPORTED, "constituent changes a spin's particle number");
            }
            hy::k::ConsDev cd;
            cd.ap = ka.nops ? p->pa.get(ka) : -1;
            cd.bp = kb.nops ? p->pb.get(kb) : -1;
            // qubit operators on different qubits commute: no reordering sign
            cd.eps = (!p->qubit && (inv & 1)) ? -1 : 1;
            cd.pad = 0;
            int ci = int(p->cons.size());
            p->cons.push_back(cd);
            if (q == 0) od.c0 = ci; else od.c1 = ci;
        }
        p->opd.push_back(od);
    }
    p->pa.finalize(h->A);
    p->pb.finalize(h->B);
    hy_status s = HY_OK;
    auto up = [&](cudaError_t err, const char *what) {
        if (s == HY_OK && err != cudaSuccess) s = cuda_fail(err, what);
    };
    DevArena &ar = p->arena;
    up(ar.upload(&p->d_op, p->opd.data(), p->opd.size()), "upload ops");
    up(ar.upload(&p->d_cons, p->cons.data(), p->cons.size()), "upload constituents");
    up(ar.upload(&p->d_aent, p->pa.entry.data(), p->pa.entry.size()), "upload alpha pairs");
    up(ar.upload(&p->d_bent, p->pb.entry.data(), p->pb.entry.size()), "upload beta pairs");
    up(ar.upload(&p->d_aoff, p->pa.off.data(), p->pa.off.size()), "upload offsets");
    up(ar.upload(&p->d_acnt, p->pa.cnt.data(), p->pa.cnt.size()), "upload counts");
    up(ar.upload(&p->d_boff, p->pb.off.data(), p->pb.off.size()), "upload offsets");
    up(ar.upload(&p->d_bcnt, p->pb.cnt.data(), p->pb.cnt.size()), "upload counts");
    {
        std::vector<int32_t> desc;
        desc.reserve(p->ops.size() * 11);
        for (const auto &op : p->ops) desc.insert(desc.end(), op.desc, op.desc + 11);
        up(ar.upload(&p->d_desc, desc.data(), desc.size()), "upload descriptors");
        const unsigned long long none = ~0ull;
        up(ar.upload(&p->d_bad, &none, 1), "upload list-check flag");
        up(cudaMallocHost(&p->h_bad, sizeof(unsigned long long)), "list-check mirror");
        if (p->h_bad) *p->h_bad = none;
    }
    if (s != HY_OK) {
        std::string msg = g_err;
        hy_pool_destroy(p);
        g_err = msg;
        return s;
    }
    *out = p;
    return HY_OK;
}

hy_status hy_pool_destroy(hy_pool *p)
{
    if (!p) return HY_OK;
    if (p->h_bad) cudaFreeHost(p->h_bad);
    p->arena.release();
    delete p;
    return HY_OK;
}

hy_status hy_pool_size(const hy_pool *p, int64_t *k)
{
    if (!p || !k) return fail(HY_ERR_ARG, "NULL argument");
    *k = int64_t(p->ops.size());
    return HY_OK;
}

hy_status hy_pool_qubit(const hy_pool *p, int *qubit)
{
    if (!p || !qubit) return fail(HY_ERR_ARG, "bad arguments");
    *qubit = p->qubit;
    return HY_OK;
}

hy_status hy_pool_describe(const hy_pool *p, int64_t k, int32_t *desc)
{
    if (!p || !desc) return fail(HY_ERR_ARG, "NULL argument");
    if (k < 0 || k >= int64_t(p->ops.size())) return fail(HY_ERR_ARG, "op index out of range");
    std::memcpy(desc, p->ops[k].desc, sizeof(int32_t) * 11);
    return HY_OK;
}

hy_status hy_pool_gradients(const hy_ham *hc, const hy_pool *p, const void *psi,
                            const void *sigma, const int32_t *ops_or_null,
                            int64_t n_ops, double *g_out, hy_dtype dt, void *stream)
{
    hy_ham *h = const_cast<hy_ham *>(hc);
    if (!h || !p || !psi || !sigma || !g_out || !valid_dtype(dt))
        return fail(HY_ERR_ARG, "bad arguments");
    if (p->h != h) return fail(HY_ERR_ARG, "pool belongs to another Hamiltonian");
    if (!ops_or_null) n_ops = int64_t(p->ops.size());
    if (n_ops < 0 || n_ops > (int64_t(1) << 24)) return fail(HY_ERR_ARG, "n_ops out of range");
    bool device_list = false;
    hy_status s = hy::check_op_list(p, ops_or_null, n_ops, &device_list, stream);
    if (s != HY_OK) return s;
    s = hy::pool_gradients_unchecked(h, p, psi, sigma, ops_or_null, n_ops, g_out, dt, stream);
    if (s == HY_OK && device_list) s = hy::fetch_op_list_flag(p, stream);
    return s;
}

}  // extern "C"

namespace hy {

HamView ham_view(const hy_ham *h, bool host_tables)
{
    // the same-spin tables live on the device; host consumers get a copy
    // (made once per handle)
    if (host_tables && h->kt.Ma.ptr.empty()) ensure_host_csr(const_cast<hy_ham *>(h));
    HamView v;
    v.n = h->n; v.na = h->na; v.nb = h->nb; v.device = h->device; v.num_sms = h->num_sms;
    v.Na = h->Na; v.Nb = h->Nb; v.N = h->N;
    v.A = &h->A; v.B = &h->B; v.kt = &h->kt;
    return v;
}

hy_status pool_gradients_unchecked(const hy_ham *hc, const hy_pool *p, const void *psi,
                                   const void *sigma, const int32_t *ops, int64_t n_ops,
                                   double *g_out, hy_dtype dt, void *stream)
{
    hy_ham *h = const_cast<hy_ham *>(hc);
    if (dt == HY_F64)
        return grad_t<double>(h, p, static_cast<const double *>(psi),
                              static_cast<const double *>(sigma), ops, n_ops, g_out,
                              as_stream(stream));
    return grad_t<float>(h, p, static_cast<const float *>(psi),
                         static_cast<const float *>(sigma), ops, n_ops, g_out,
                         as_stream(stream));
}

// Operator lists of the public screens.  A list in pageable host memory (the
// caller wrote it on the host) is range-checked here, before any launch; a
// device, pinned or managed list may still be written by work queued on the
// stream, so the kernels check it (refuse_op: the entry's gradient becomes
// NaN) and the first refused entry is reported by the next screen call on the
// pool.  Indices are compared with the pool size.
hy_status check_op_list(const hy_pool *p, const int32_t *ops, int64_t n_ops,
                        bool *device_list, void *stream)
{
    *device_list = false;
    const int64_t K = int64_t(p->ops.size());
    if (p->h_bad && *p->h_bad != ~0ull) {
        const unsigned long long v = *p->h_bad;
        *p->h_bad = ~0ull;
        HY_CUDA(cudaMemsetAsync(p->d_bad, 0xFF, sizeof(unsigned long long), as_stream(stream)),
                "list-check reset");
        return fail(HY_ERR_ARG, "an earlier screen's operator list held " +
                                    std::to_string(int32_t(uint32_t(v & 0xFFFFFFFFull))) +
                                    " at position " + std::to_string(v >> 32) +
                                    ", not a pool index (pool size " + std::to_string(K) +
                                    "); that gradient was returned as NaN");
    }
    if (!ops || n_ops == 0) return HY_OK;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ops) != cudaSuccess) {
        cudaGetLastError();
        return fail(HY_ERR_ARG, "ops_or_null is not a pointer the CUDA runtime can classify");
    }
    if (at.type != cudaMemoryTypeUnregistered) {
        *device_list = true;
        return HY_OK;
    }
    int dev = 0, pageable = 0;
    HY_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    HY_CUDA(cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev),
            "device attribute");
    if (!pageable)
        return fail(HY_ERR_ARG, "ops_or_null is pageable host memory the device cannot read; "
                                "pass a device, pinned or managed list");
    for (int64_t i = 0; i < n_ops; ++i)
        if (ops[i] < 0 || int64_t(ops[i]) >= K)
            return fail(HY_ERR_ARG, "ops_or_null[" + std::to_string(i) + "] = " +
                                        std::to_string(ops[i]) +
                                        " is not a pool index (pool size " + std::to_string(K) +
                                        ")");
    return HY_OK;
}

// after a screen that read a device list: bring the kernels' refusal flag to
// the host (stream-ordered; read by the next screen call)
hy_status fetch_op_list_flag(const hy_pool *p, void *stream)
{
    HY_CUDA(cudaMemcpyAsync(p->h_bad, p->d_bad, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, as_stream(stream)),
            "list-check flag copy");
    return HY_OK;
}

}  // namespace hy

// ---------------------------------------------------------------------------
// Allocation-free gradient screen.  Some callers cannot let a library call
// cudaMalloc / cudaFree: a serving loop whose device memory is entirely
// reserved by another allocator, or one that must never hit the implicit
// device-wide synchronisation of cudaFree or the latency of a first-use
// allocation.  hy_pool_gradients_noalloc gives them the screen with its
// per-(operator, row-chunk) partial sums in a fixed, file-scope device array
// instead of the handle's cudaMalloc'd workspace.  The array is
// kNoAllocPartials doubles (2 MiB) and stays resident on every device that
// loads the library until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocPartials = int64_t(1) << 18;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_partials on the current device (the host-side
// name is only a stand-in, not a device address).  Resolved once per device.
hy_status noalloc_scratch(double **out)
{
    int dev = 0;
    HY_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(HY_ERR_UNSUPPORTED, "device ordinal beyond the no-alloc table");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_ptr[dev] = static_cast<double *>(ptr);
    }
    *out = g_noalloc_ptr[dev];
    return HY_OK;
}

template <typename T>
hy_status grad_noalloc_t(hy_ham *h, const hy_pool *p, const T *psi, const T *sigma,
                         const int32_t *ops, int64_t n_ops, double *g, double *scratch,
                         cudaStream_t st)
{
    hy::k::GradArgs<T> a;
    a.psi = psi;
    a.sigma = sigma;
    a.ops = ops;
    a.n_ops = n_ops;
    a.opd = p->d_op;
    a.cons = p->d_cons;
    a.aent = p->d_aent;
    a.aoff = p->d_aoff;
    a.acnt = p->d_acnt;
    a.bent = p->d_bent;
    a.boff = p->d_boff;
    a.bcnt = p->d_bcnt;
    a.Na = h->Na;
    a.Nb = h->Nb;
    a.CH = grad_chunks(h, n_ops);
    a.partials = scratch;
    a.g = g;
    a.K = int64_t(p->ops.size());
    a.bad = p->d_bad;
    HY_CUDA(hy::k::grad<T>(a, st), "pool gradients (no-alloc)");
    return HY_OK;
}

}  // namespace

extern "C" {

hy_status hy_pool_gradients_noalloc(const hy_ham *hc, const hy_pool *p, const void *psi,
                                    const void *sigma, const int32_t *ops_or_null,
                                    int64_t n_ops, double *g_out, hy_dtype dt, void *stream)
{
    hy_ham *h = const_cast<hy_ham *>(hc);
    if (!h || !p || !psi || !sigma || !g_out || !valid_dtype(dt))
        return fail(HY_ERR_ARG, "bad arguments");
    if (p->h != h) return fail(HY_ERR_ARG, "pool belongs to another Hamiltonian");
    if (!ops_or_null) n_ops = int64_t(p->ops.size());
    if (n_ops < 0) return fail(HY_ERR_ARG, "n_ops out of range");
    // every launch uses n_ops * chunks <= n_ops + 4 * SMs partial sums
    const int64_t need = n_ops * int64_t(grad_chunks(h, n_ops));
    if (need > kNoAllocPartials)
        return fail(HY_ERR_ARG, "n_ops = " + std::to_string(n_ops) +
                                    " needs more partial sums than the no-alloc scratch holds (" +
                                    std::to_string(kNoAllocPartials) + "); use hy_pool_gradients");
    bool device_list = false;
    hy_status s = hy::check_op_list(p, ops_or_null, n_ops, &device_list, stream);
    if (s != HY_OK) return s;
    double *scratch = nullptr;
    s = noalloc_scratch(&scratch);
    if (s != HY_OK) return s;
    if (dt == HY_F64)
        s = grad_noalloc_t<double>(h, p, static_cast<const double *>(psi),
                                   static_cast<const double *>(sigma), ops_or_null, n_ops,
                                   g_out, scratch, as_stream(stream));
    else
        s = grad_noalloc_t<float>(h, p, static_cast<const float *>(psi),
                                  static_cast<const float *>(sigma), ops_or_null, n_ops, g_out,
                                  scratch, as_stream(stream));
    if (s == HY_OK && device_list) s = hy::fetch_op_list_flag(p, stream);
    return s;
}

hy_status hy_apply_excitation(const hy_ham *hc, const hy_pool *p, int64_t k,
                              double theta, void *psi, hy_dtype dt, int renormalize,
                              void *stream)
{
    hy_ham *h = const_cast<hy_ham *>(hc);
    if (!h || !p || !psi || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    if (p->h != h) return fail(HY_ERR_ARG, "pool belongs to another Hamiltonian");
    if (k < 0 || k >= int64_t(p->ops.size())) return fail(HY_ERR_ARG, "op index out of range");
    if (!std::isfinite(theta)) return fail(HY_ERR_ARG, "theta is not finite");
    hy_status s;
    if (dt == HY_F64) {
        s = excite_t<double>(h, p, k, theta, static_cast<double *>(psi), as_stream(stream));
        if (s == HY_OK && renormalize)
            s = normalize_t<double>(h, static_cast<double *>(psi), as_stream(stream));
    } else {
        s = excite_t<float>(h, p, k, theta, static_cast<float *>(psi), as_stream(stream));
        if (s == HY_OK && renormalize)
            s = normalize_t<float>(h, static_cast<float *>(psi), as_stream(stream));
    }
    return s;
}

hy_status hy_apply_excitation_tracked(const hy_ham *hc, const hy_pool *p, int64_t k, double theta,
                                      void *psi, hy_dtype dt, double *norm2, void *stream)
{
    hy_ham *h = const_cast<hy_ham *>(hc);
    if (!h || !p || !psi || !norm2 || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    if (p->h != h) return fail(HY_ERR_ARG, "pool belongs to another Hamiltonian");
    if (k < 0 || k >= int64_t(p->ops.size())) return fail(HY_ERR_ARG, "op index out of range");
    if (!std::isfinite(theta)) return fail(HY_ERR_ARG, "theta is not finite");
    if (dt == HY_F64)
        return excite_tracked_t<double>(h, p, k, theta, static_cast<double *>(psi), norm2,
                                        as_stream(stream));
    return excite_tracked_t<float>(h, p, k, theta, static_cast<float *>(psi), norm2,
                                   as_stream(stream));
}

hy_status hy_renormalize(const hy_ham *h, void *psi, hy_dtype dt, const double *norm2,
                         void *stream)
{
    if (!h || !psi || !norm2 || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    hy::ProfScope prof(HY_PROF_REDUCE, stream, 2.0 * double(h->N) * (dt == HY_F64 ? 8 : 4));
    if (dt == HY_F64)
        HY_CUDA(hy::k::scale_rsqrt<double>(static_cast<double *>(psi), h->N, norm2,
                                           as_stream(stream)), "renormalize");
    else
        HY_CUDA(hy::k::scale_rsqrt<float>(static_cast<float *>(psi), h->N, norm2,
                                          as_stream(stream)), "renormalize");
    return HY_OK;
}

hy_status hy_support(const hy_ham *h, const void *psi, hy_dtype dt, int64_t *list, int64_t cap,
                     int64_t *count, void *stream)
{
    if (!h || !psi || !count || !valid_dtype(dt) || cap < 0 || (cap > 0 && !list))
        return fail(HY_ERR_ARG, "bad arguments");
    auto *cnt = reinterpret_cast<unsigned long long *>(count);
    if (dt == HY_F64)
        HY_CUDA(hy::k::support<double>(static_cast<const double *>(psi), h->N, list, cap, cnt,
                                       h->num_sms, as_stream(stream)), "support");
    else
        HY_CUDA(hy::k::support<float>(static_cast<const float *>(psi), h->N, list, cap, cnt,
                                      h->num_sms, as_stream(stream)), "support");
    return HY_OK;
}

}  // extern "C"

namespace {
// support chunks per operator of the sparse screen: about 4 blocks per SM
// in all, at most one chunk per 256 listed entries
int sparse_chunks(const hy_ham *h, int64_t n_ops, int64_t m)
{
    int64_t ch = int64_t(4) * h->num_sms / (n_ops > 0 ? n_ops : 1);
    const int64_t by_m = (m + 255) / 256;
    if (ch > by_m) ch = by_m;
    if (ch > 1024) ch = 1024;
    return int(ch < 1 ? 1 : ch);
}

template <typename T>
hy::k::SparseArgs<T> sparse_args(const hy_ham *h, const void *psi, void *sigma,
                                 const int64_t *list, int64_t m)
{
    hy::k::SparseArgs<T> a;
    a.psi = static_cast<const T *>(psi);
    a.sigma = static_cast<T *>(sigma);
    a.list = list;
    a.m = m;
    a.d_m = nullptr;
    a.cap = m;
    a.obits = nullptr;
    a.olist = nullptr;
    a.ocount = nullptr;
    a.ocap = 0;
    const DevCsr<T> *Ma, *Mb;
    if constexpr (sizeof(T) == 8) {
        Ma = &h->Ma64; Mb = &h->Mb64; a.V = h->d_V64;
    } else {
        Ma = &h->Ma32; Mb = &h->Mb32; a.V = h->d_V32;
    }
    a.Ma_ptr = Ma->ptr; a.Ma_col = Ma->col; a.Ma_val = Ma->val;
    a.Mb_ptr = Mb->ptr; a.Mb_col = Mb->col; a.Mb_val = Mb->val;
    a.aex = h->d_aex; a.bexT = h->d_bexT; a.astr = h->d_astr; a.bstr = h->d_bstr;
    a.bex = h->d_bex;
    a.n = h->n; a.nexa = h->A.nex; a.nexb = h->B.nex; a.Na = h->Na; a.Nb = h->Nb;
    return a;
}
}  // namespace

extern "C" {

hy_status hy_apply_h_sparse(const hy_ham *h, const void *psi, void *sigma, hy_dtype dt,
                            const int64_t *list, int64_t m, void *stream)
{
    if (!h || !psi || !sigma || !valid_dtype(dt) || m < 0 || (m > 0 && !list))
        return fail(HY_ERR_ARG, "bad arguments");
    if (psi == sigma) return fail(HY_ERR_ARG, "psi and sigma must not alias");
    // work: the atomic adds, at most one per coupling of a listed amplitude
    hy::ProfScope prof(HY_PROF_HPSI_SPARSE, stream, double(h->N) * (dt == HY_F64 ? 8 : 4),
                       double(m) * double(hy::ham_connections(h)));
    if (dt == HY_F64)
        HY_CUDA(hy::k::hpsi_scatter<double>(sparse_args<double>(h, psi, sigma, list, m), h->num_sms,
                                            as_stream(stream)), "sparse H psi");
    else
        HY_CUDA(hy::k::hpsi_scatter<float>(sparse_args<float>(h, psi, sigma, list, m), h->num_sms,
                                           as_stream(stream)), "sparse H psi");
    return HY_OK;
}

hy_status hy_pool_gradients_sparse(const hy_ham *h, const hy_pool *p, const void *psi,
                                   const void *sigma, const int64_t *list, int64_t m,
                                   const int32_t *ops_or_null, int64_t n_ops, double *g_out,
                                   hy_dtype dt, void *stream)
{
    if (!h || !p || !psi || !sigma || !g_out || !valid_dtype(dt) || m < 0 || (m > 0 && !list))
        return fail(HY_ERR_ARG, "bad arguments");
    if (p->h != h) return fail(HY_ERR_ARG, "pool belongs to another Hamiltonian");
    if (!ops_or_null) n_ops = int64_t(p->ops.size());
    if (n_ops < 0) return fail(HY_ERR_ARG, "n_ops out of range");
    bool device_list = false;
    hy_status st = hy::check_op_list(p, ops_or_null, n_ops, &device_list, stream);
    if (st != HY_OK) return st;
    hy_ham *hm = const_cast<hy_ham *>(h);
    const WsLayout L = ws_layout(hm, n_partials_needed(hm, n_ops), dt == HY_F64 ? 8 : 4);
    st = ensure_ws(hm, L.total);
    if (st != HY_OK) return st;
    auto fill = [&](auto &a) {
        a.list = list; a.m = m; a.d_m = nullptr; a.cap = m; a.bits = nullptr;
        a.chunks = sparse_chunks(h, n_ops, m);
        a.partials = reinterpret_cast<double *>(static_cast<char *>(hm->ws) + L.partials);
        a.desc = p->d_desc; a.ops = ops_or_null; a.n_ops = n_ops;
        a.astr = h->d_astr; a.bstr = h->d_bstr; a.binom33 = h->d_binom; a.n = h->n;
        a.rank16 = h->d_rank16;
        a.Nb = h->Nb; a.g = g_out; a.K = int64_t(p->ops.size()); a.bad = p->d_bad;
        a.qubit = p->qubit;
    };
    hy::ProfScope prof(HY_PROF_SCREEN_SPARSE, stream, 0.0);
    if (dt == HY_F64) {
        hy::k::SparseGradArgs<double> a;
        a.psi = static_cast<const double *>(psi);
        a.sigma = static_cast<const double *>(sigma);
        fill(a);
        HY_CUDA(hy::k::grad_sparse<double>(a, h->num_sms, as_stream(stream)), "sparse screen");
    } else {
        hy::k::SparseGradArgs<float> a;
        a.psi = static_cast<const float *>(psi);
        a.sigma = static_cast<const float *>(sigma);
        fill(a);
        HY_CUDA(hy::k::grad_sparse<float>(a, h->num_sms, as_stream(stream)), "sparse screen");
    }
    return device_list ? hy::fetch_op_list_flag(p, stream) : HY_OK;
}

hy_status hy_ranker_features(const hy_ham *h, const hy_pool *p, const void *psi,
                             const void *sigma_or_null, hy_dtype dt, const float *extra,
                             float *feat, void *stream)
{
    return hy::ranker_features_impl(h, p, psi, nullptr, sigma_or_null, nullptr, dt, extra, feat,
                                    stream);
}

hy_status hy_touched_weights(const hy_ham *h, const void *psi, hy_dtype dt, float *D,
                             void *stream)
{
    if (!h || !psi || !D || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    cudaStream_t st = as_stream(stream);
    if (dt == HY_F64)
        HY_CUDA(hy::k::touched_weights<double>(static_cast<const double *>(psi), h->Na, h->Nb,
                                               h->d_astr, h->d_bstr, h->n, h->d_pairB,
                                               h->d_pairRs, h->d_pairRows, h->d_pairP, D,
                                               h->num_sms, st),
                "touched weights");
    else
        HY_CUDA(hy::k::touched_weights<float>(static_cast<const float *>(psi), h->Na, h->Nb,
                                              h->d_astr, h->d_bstr, h->n, h->d_pairB,
                                              h->d_pairRs, h->d_pairRows, h->d_pairP, D,
                                              h->num_sms, st),
                "touched weights");
    return HY_OK;
}

}  // extern "C"

namespace {
// row groups for a list of up to cap entries (grown with a device
// synchronisation: work in flight may still read the old ones)
hy_status ensure_tw(hy_ham *h, int64_t cap)
{
    if (h->tw.mask && h->tw.cap >= cap) return HY_OK;
    if (cap > int64_t(INT32_MAX)) return HY_OK;      // the atomic fallback serves it
    HY_CUDA(cudaDeviceSynchronize(), "synchronise before growing row groups");
    cudaFree(h->tw.mask);
    cudaFree(h->tw.w);
    h->tw.mask = nullptr;
    h->tw.w = nullptr;
    h->tw.cap = 0;
    cudaError_t e = cudaSuccess;
    if (!h->tw.cnt) {
        e = cudaMalloc(&h->tw.cnt, size_t(h->Na + 1) * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&h->tw.ptr, size_t(h->Na + 1) * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&h->tw.cur, size_t(h->Na) * sizeof(int32_t));
    }
    if (e == cudaSuccess) e = cudaMalloc(&h->tw.mask, size_t(cap) * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&h->tw.w, size_t(cap) * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(row groups)");
    h->tw.cap = cap;
    return HY_OK;
}
}  // namespace

extern "C" {

hy_status hy_touched_weights_sparse(const hy_ham *hc, const void *psi, hy_dtype dt,
                                    const int64_t *list, int64_t m, float *D, void *stream)
{
    hy_ham *h = const_cast<hy_ham *>(hc);
    if (!h || !psi || !D || !valid_dtype(dt) || m < 0 || (m > 0 && !list))
        return fail(HY_ERR_ARG, "bad arguments");
    cudaStream_t st = as_stream(stream);
    // the kernel reads the count from the device: stage m in the workspace
    const WsLayout L = ws_layout(h, n_partials_needed(h, 0), dt == HY_F64 ? 8 : 4);
    hy_status s = ensure_ws(h, L.total);
    if (s != HY_OK) return s;
    auto *cnt = reinterpret_cast<unsigned long long *>(static_cast<char *>(h->ws) + L.scalar);
    s = ensure_tw(h, m);
    if (s != HY_OK) return s;
    const unsigned long long mm = (unsigned long long)m;
    HY_CUDA(cudaMemcpyAsync(cnt, &mm, sizeof(mm), cudaMemcpyHostToDevice, st), "count");
    if (dt == HY_F64)
        HY_CUDA(hy::k::touched_weights_list<double>(static_cast<const double *>(psi), list, cnt, m,
                                                    m, h->Na, h->Nb, h->d_astr, h->d_bstr, h->n,
                                                    h->d_pairB, h->d_pairRs, h->d_pairRows,
                                                    h->d_pairP, D, h->tw, h->num_sms, st),
                "touched weights (list)");
    else
        HY_CUDA(hy::k::touched_weights_list<float>(static_cast<const float *>(psi), list, cnt, m,
                                                   m, h->Na, h->Nb, h->d_astr, h->d_bstr, h->n,
                                                   h->d_pairB, h->d_pairRs, h->d_pairRows,
                                                   h->d_pairP, D, h->tw, h->num_sms, st),
                "touched weights (list)");
    // (a copy from pageable host memory has left `mm` when the call returns)
    return HY_OK;
}

hy_status hy_occupations(const hy_ham *h, const void *psi, hy_dtype dt, float *occ,
                         void *stream)
{
    if (!h || !psi || !occ || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    cudaStream_t st = as_stream(stream);
    if (dt == HY_F64)
        HY_CUDA(hy::k::occupations<double>(static_cast<const double *>(psi), h->Na, h->Nb,
                                           h->d_astr, h->d_bstr, h->n, h->d_occ_partial,
                                           h->occ_blocks, occ, st), "occupations");
    else
        HY_CUDA(hy::k::occupations<float>(static_cast<const float *>(psi), h->Na, h->Nb,
                                          h->d_astr, h->d_bstr, h->n, h->d_occ_partial,
                                          h->occ_blocks, occ, st), "occupations");
    return HY_OK;
}

}  // extern "C"

namespace {

template <typename T>
hy::k::BatchArgs<T> batch_args(const hy_batch *b, const void *psi, void *sigma, double *row_e)
{
    hy::k::BatchArgs<T> a;
    a.psi = static_cast<const T *>(psi);
    a.sigma = static_cast<T *>(sigma);
    if constexpr (sizeof(T) == 8) a.mols = b->d_mols64; else a.mols = b->d_mols32;
    a.tasks = b->d_tasks;
    a.n_tasks = int(b->n_tasks);
    a.counter = b->d_counter;
    a.row_energy = row_e;
    a.gsize = b->tile.gsize;
    a.threads = b->tile.gsize * b->tile.groups;
    a.nb_max = b->nb_max;
    a.nn_max = b->nn_max;
    a.group_smem = hy::k::batch_group_smem<T>(b->nb_max, b->nn_max, b->tile.gsize);
    return a;
}

bool tile_ok(const hy_batch *b, const hy_batch_tile &t, size_t elem)
{
    if (t.gsize < 32 || t.gsize > 1024 || (t.gsize & (t.gsize - 1))) return false;
    if (t.groups < 1 || t.groups > 15 || t.gsize * t.groups > 1024) return false;
    if (t.ctas_per_sm < 0) return false;
    const size_t g = elem == 8 ? hy::k::batch_group_smem<double>(b->nb_max, b->nn_max, t.gsize)
                               : hy::k::batch_group_smem<float>(b->nb_max, b->nn_max, t.gsize);
    return g * t.groups <= 227 * 1024;
}

template <typename T>
hy_status batch_apply_t(hy_batch *b, const void *psi, void *sigma, double *energies,
                        cudaStream_t st)
{
    if (!tile_ok(b, b->tile, sizeof(T))) return fail(HY_ERR_ARG, "tile shape does not fit");
    hy::k::BatchArgs<T> a = batch_args<T>(b, psi, sigma, energies ? b->d_row_energy : nullptr);
    int per_sm = 0;
    HY_CUDA(hy::k::batch_occupancy<T>(a, &per_sm), "batch occupancy");
    if (per_sm < 1) return fail(HY_ERR_ARG, "tile shape does not fit an SM");
    if (b->tile.ctas_per_sm > 0 && b->tile.ctas_per_sm < per_sm) per_sm = b->tile.ctas_per_sm;
    int64_t grid = int64_t(b->num_sms) * per_sm;
    const int64_t need = (b->n_tasks + b->tile.groups - 1) / b->tile.groups;
    if (grid > need) grid = need > 0 ? need : 1;
    HY_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(int), st), "reset task counter");
    HY_CUDA(hy::k::batch_rows<T>(a, int(grid), st), "batch rows");
    if (energies)
        HY_CUDA(hy::k::batch_energy(b->d_row_energy, b->d_base, b->d_rows, int(b->hams.size()),
                                    energies, st), "batch energies");
    return HY_OK;
}

hy_status batch_apply(hy_batch *b, const void *psi, void *sigma, hy_dtype dt, double *energies,
                      cudaStream_t st)
{
    if (dt == HY_F64) return batch_apply_t<double>(b, psi, sigma, energies, st);
    return batch_apply_t<float>(b, psi, sigma, energies, st);
}

}  // namespace

extern "C" {

hy_status hy_batch_create(const hy_ham *const *hams, int count, hy_batch **out)
{
    if (!out) return fail(HY_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!hams || count < 1) return fail(HY_ERR_ARG, "empty batch");
    for (int i = 0; i < count; ++i)
        if (!hams[i]) return fail(HY_ERR_ARG, "NULL Hamiltonian in batch");
    hy_batch *b = new (std::nothrow) hy_batch;
    if (!b) return fail(HY_ERR_OOM, "host allocation failed");
    b->hams.assign(hams, hams + count);
    b->num_sms = hams[0]->num_sms;
    std::vector<double> cost(count);
    for (int i = 0; i < count; ++i) {
        const hy_ham *h = hams[i];
        const double rowc = double(h->Nb) *
            (double(h->nnz_a) / double(h->Na) + double(h->nnz_b) / double(h->Nb) +
             double(h->A.nex + 1) * double(h->B.nex + 1));
        cost[i] = rowc;
        b->order.push_back(i);
        b->nb_max = std::max<int>(b->nb_max, int(h->Nb));
        b->nn_max = std::max(b->nn_max, h->n * h->n);
    }
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int x, int y) { return cost[x] > cost[y]; });
    b->offsets.assign(count + 1, 0);
    int64_t off = 0;
    for (int i = 0; i < count; ++i) {
        b->offsets[i] = off;
        off += (hams[i]->N + 31) / 32 * 32;
    }
    b->offsets[count] = off;
    b->total = off;
    std::vector<hy::k::BatchMol<double>> m64(count);
    std::vector<hy::k::BatchMol<float>> m32(count);
    std::vector<int64_t> base(count), rows(count);
    int64_t tb = 0;
    for (int i = 0; i < count; ++i) {
        const hy_ham *h = hams[i];
        auto fill = [&](auto &m, const auto &Ma, const auto &Mb, const auto *V) {
            m.offset = b->offsets[i];
            m.Na = h->Na;
            m.Nb = h->Nb;
            m.task_base = tb;
            m.n = h->n;
            m.nexa = h->A.nex;
            m.nexb = h->B.nex;
            m.pad = 0;
            m.Ma_ptr = Ma.ptr; m.Ma_col = Ma.col; m.Ma_val = Ma.val;
            m.Mb_ptr = Mb.ptr; m.Mb_col = Mb.col; m.Mb_val = Mb.val;
            m.V = V;
            m.aex = h->d_aex; m.bexT = h->d_bexT; m.astr = h->d_astr; m.bstr = h->d_bstr;
        };
        fill(m64[i], h->Ma64, h->Mb64, h->d_V64);
        fill(m32[i], h->Ma32, h->Mb32, h->d_V32);
        base[i] = tb;
        rows[i] = h->Na;
        tb += h->Na;
    }
    std::vector<int2> tasks;
    for (int i : b->order)
        for (int64_t r = 0; r < hams[i]->Na; ++r) tasks.push_back(make_int2(i, int(r)));
    b->n_tasks = int64_t(tasks.size());
    hy_status s = HY_OK;
    auto up = [&](cudaError_t err, const char *what) {
        if (s == HY_OK && err != cudaSuccess) s = cuda_fail(err, what);
    };
    auto put = [&](auto **dst, const auto *src, size_t cnt, const char *what) {
        if (s != HY_OK) return;
        up(cudaMalloc(reinterpret_cast<void **>(dst), cnt * sizeof(**dst)), what);
        if (s == HY_OK && src)
            up(cudaMemcpy(*dst, src, cnt * sizeof(**dst), cudaMemcpyHostToDevice), what);
    };
    put(&b->d_mols64, m64.data(), m64.size(), "batch tables");
    put(&b->d_mols32, m32.data(), m32.size(), "batch tables");
    put(&b->d_tasks, tasks.data(), tasks.size(), "batch tasks");
    put(&b->d_counter, static_cast<const int *>(nullptr), 1, "batch counter");
    put(&b->d_row_energy, static_cast<const double *>(nullptr), size_t(tb), "batch partials");
    put(&b->d_base, base.data(), base.size(), "batch tables");
    put(&b->d_rows, rows.data(), rows.size(), "batch tables");
    if (s != HY_OK) {
        std::string msg = g_err;
        hy_batch_destroy(b);
        g_err = msg;
        return s;
    }
    *out = b;
    return HY_OK;
}

hy_status hy_batch_destroy(hy_batch *b)
{
    if (!b) return HY_OK;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    cudaFree(b->d_mols64);
    cudaFree(b->d_mols32);
    cudaFree(b->d_tasks);
    cudaFree(b->d_counter);
    cudaFree(b->d_row_energy);
    cudaFree(b->d_base);
    cudaFree(b->d_rows);
    cudaFree(b->d_pools);
    cudaFree(b->d_pool_base);
    cudaFree(b->d_gpart);
    cudaFree(b->d_gctr);
    cudaFree(b->d_gbad);
    cudaFreeHost(b->h_gbad);
    delete b;
    return HY_OK;
}

hy_status hy_batch_set_pools(hy_batch *b, const hy_pool *const *pools)
{
    if (!b || !pools) return fail(HY_ERR_ARG, "NULL argument");
    const int count = int(b->hams.size());
    std::vector<hy::k::BatchPool> mp(count);
    std::vector<int64_t> base(count + 1, 0);
    for (int m = 0; m < count; ++m) {
        const hy_pool *p = pools[m];
        if (!p || p->h != b->hams[m])
            return fail(HY_ERR_ARG, "pool m must be built on the batch's Hamiltonian m");
        const hy_ham *h = b->hams[m];
        hy::k::BatchPool &q = mp[m];
        q.opd = p->d_op; q.cons = p->d_cons;
        q.aent = p->d_aent; q.bent = p->d_bent;
        q.aoff = p->d_aoff; q.acnt = p->d_acnt; q.boff = p->d_boff; q.bcnt = p->d_bcnt;
        q.Na = h->Na; q.Nb = h->Nb; q.off = b->offsets[m]; q.K = int64_t(p->ops.size());
        base[m + 1] = base[m] + q.K;
    }
    cudaError_t e = cudaSuccess;
    if (!b->d_pools) e = cudaMalloc(&b->d_pools, size_t(count) * sizeof(hy::k::BatchPool));
    if (e == cudaSuccess && !b->d_pool_base)
        e = cudaMalloc(&b->d_pool_base, size_t(count + 1) * sizeof(int64_t));
    if (e == cudaSuccess && !b->d_gctr) e = cudaMalloc(&b->d_gctr, sizeof(unsigned long long));
    if (e == cudaSuccess && !b->d_gbad) e = cudaMalloc(&b->d_gbad, sizeof(unsigned long long));
    if (e == cudaSuccess && !b->h_gbad) e = cudaMallocHost(&b->h_gbad, sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_pools, mp.data(), size_t(count) * sizeof(hy::k::BatchPool),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_pool_base, base.data(), size_t(count + 1) * sizeof(int64_t),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_gbad, 0xFF, sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e, "batch pools");
    *b->h_gbad = ~0ull;
    b->pools.assign(pools, pools + count);
    b->pool_base = base;
    return HY_OK;
}

hy_status hy_batch_pool_offsets(const hy_batch *b, int64_t *offsets)
{
    if (!b || !offsets) return fail(HY_ERR_ARG, "NULL argument");
    if (b->pools.empty()) return fail(HY_ERR_ARG, "no pools set (hy_batch_set_pools)");
    std::copy(b->pool_base.begin(), b->pool_base.end(), offsets);
    return HY_OK;
}

hy_status hy_batch_gradients(hy_batch *b, const void *psi, const void *sigma, const int32_t *ops,
                             const int64_t *op_offsets, int64_t n_entries, double *g, hy_dtype dt,
                             void *stream)
{
    if (!b || !psi || !sigma || !g || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    if (b->pools.empty()) return fail(HY_ERR_ARG, "no pools set (hy_batch_set_pools)");
    if (ops && (!op_offsets || n_entries < 0)) return fail(HY_ERR_ARG, "operator lists need offsets");
    // a refused entry of the previous call's lists (read after that call's
    // stream work finished)
    if (*b->h_gbad != ~0ull) {
        const unsigned long long v = *b->h_gbad;
        *b->h_gbad = ~0ull;
        cudaMemset(b->d_gbad, 0xFF, sizeof(unsigned long long));
        return fail(HY_ERR_ARG, "operator index out of range at entry " +
                                    std::to_string(v >> 32) + ": " +
                                    std::to_string(int32_t(uint32_t(v))));
    }
    const int64_t n = ops ? n_entries : b->pool_base.back();
    if (n == 0) return HY_OK;
    cudaStream_t st = as_stream(stream);
    int64_t ch = (int64_t(8) * b->num_sms + n - 1) / n;
    if (ch < 1) ch = 1;
    if (ch > 256) ch = 256;
    if (n * ch > b->n_gpart) {
        // before any graph capture: the first call of a size allocates
        HY_CUDA(cudaStreamSynchronize(st), "sync");
        cudaFree(b->d_gpart);
        b->d_gpart = nullptr;
        b->n_gpart = 0;
        HY_CUDA(cudaMalloc(&b->d_gpart, size_t(n * ch) * sizeof(double)), "cudaMalloc(partials)");
        b->n_gpart = n * ch;
    }
    hy::ProfScope prof(HY_PROF_SCREEN, stream, 0.0);
    auto run = [&](auto *tag) -> cudaError_t {
        using T = std::remove_pointer_t<decltype(tag)>;
        hy::k::BatchGradArgs<T> a;
        a.mols = b->d_pools;
        a.count = int(b->hams.size());
        a.psi = static_cast<const T *>(psi);
        a.sigma = static_cast<const T *>(sigma);
        a.ops = ops;
        a.base = ops ? op_offsets : b->d_pool_base;
        a.CH = int(ch);
        a.n_tasks = n * ch;
        a.partials = b->d_gpart;
        a.g = g;
        a.counter = b->d_gctr;
        a.bad = b->d_gbad;
        cudaError_t e = hy::k::batch_grad<T>(a, 8 * b->num_sms, st);
        if (e == cudaSuccess && ops)
            e = cudaMemcpyAsync(b->h_gbad, b->d_gbad, sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, st);
        return e;
    };
    if (dt == HY_F64)
        HY_CUDA(run(static_cast<double *>(nullptr)), "batched pool gradients");
    else
        HY_CUDA(run(static_cast<float *>(nullptr)), "batched pool gradients");
    return HY_OK;
}

hy_status hy_batch_info(const hy_batch *b, int64_t *total, int64_t *n_tasks)
{
    if (!b) return fail(HY_ERR_ARG, "batch is NULL");
    if (total) *total = b->total;
    if (n_tasks) *n_tasks = b->n_tasks;
    return HY_OK;
}

hy_status hy_batch_offsets(const hy_batch *b, int64_t *offsets)
{
    if (!b || !offsets) return fail(HY_ERR_ARG, "NULL argument");
    std::memcpy(offsets, b->offsets.data(), b->offsets.size() * sizeof(int64_t));
    return HY_OK;
}

hy_status hy_batch_set_tile(hy_batch *b, const hy_batch_tile *tile)
{
    if (!b || !tile) return fail(HY_ERR_ARG, "NULL argument");
    if (!tile_ok(b, *tile, 8) && !tile_ok(b, *tile, 4)) return fail(HY_ERR_ARG, "invalid tile shape");
    b->tile = *tile;
    return HY_OK;
}

hy_status hy_batch_get_tile(const hy_batch *b, hy_batch_tile *tile)
{
    if (!b || !tile) return fail(HY_ERR_ARG, "NULL argument");
    *tile = b->tile;
    return HY_OK;
}

hy_status hy_batch_apply_h(hy_batch *b, const void *psi, void *sigma, hy_dtype dt,
                           double *energies, void *stream)
{
    if (!b || !psi || !sigma || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    if (psi == sigma) return fail(HY_ERR_ARG, "psi and sigma must not alias");
    return batch_apply(b, psi, sigma, dt, energies, as_stream(stream));
}

hy_status hy_batch_graph_launch(hy_batch *b, const void *psi, void *sigma, hy_dtype dt,
                                double *energies, void *stream)
{
    if (!b || !psi || !sigma || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    if (psi == sigma) return fail(HY_ERR_ARG, "psi and sigma must not alias");
    cudaStream_t st = as_stream(stream);
    const bool same = b->gexec && b->g_psi == psi && b->g_sigma == sigma &&
                      b->g_energies == energies && b->g_dt == int(dt) &&
                      b->g_tile.gsize == b->tile.gsize && b->g_tile.groups == b->tile.groups &&
                      b->g_tile.ctas_per_sm == b->tile.ctas_per_sm;
    if (!same) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaStream_t cap = nullptr;
        HY_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        hy_status s = HY_OK;
        if (e == cudaSuccess) {
            s = batch_apply(b, psi, sigma, dt, energies, cap);
            cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
            if (s == HY_OK && e2 != cudaSuccess) s = cuda_fail(e2, "end capture");
        } else {
            s = cuda_fail(e, "begin capture");
        }
        cudaStreamDestroy(cap);
        if (s != HY_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        e = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->gexec = nullptr;
            return cuda_fail(e, "graph instantiate");
        }
        b->g_psi = psi;
        b->g_sigma = sigma;
        b->g_energies = energies;
        b->g_dt = int(dt);
        b->g_tile = b->tile;
    }
    HY_CUDA(cudaGraphLaunch(b->gexec, st), "graph launch");
    hy::count_launch();                       // the persistent rows kernel
    if (energies) hy::count_launch();         // the per-molecule energy sums
    return HY_OK;
}

hy_status hy_batch_tune(hy_batch *b, const void *psi, void *sigma, hy_dtype dt,
                        hy_batch_tile *best, double *ms, void *stream)
{
    if (!b || !psi || !sigma || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    cudaStream_t st = as_stream(stream);
    const size_t elem = dt == HY_F64 ? 8 : 4;
    cudaEvent_t e0, e1;
    HY_CUDA(cudaEventCreate(&e0), "event");
    HY_CUDA(cudaEventCreate(&e1), "event");
    const hy_batch_tile saved = b->tile;
    hy_batch_tile win = saved;
    double win_ms = 1e300;
    hy_status s = HY_OK;
    for (int gsize = 32; gsize <= 512 && s == HY_OK; gsize *= 2)
        for (int groups = 1; groups <= 8 && s == HY_OK; groups *= 2) {
            hy_batch_tile t{gsize, groups, 0};
            if (!tile_ok(b, t, elem)) continue;
            b->tile = t;
            for (int w = 0; w < 2 && s == HY_OK; ++w) s = batch_apply(b, psi, sigma, dt, nullptr, st);
            if (s != HY_OK) break;
            cudaEventRecord(e0, st);
            for (int r = 0; r < 3 && s == HY_OK; ++r) s = batch_apply(b, psi, sigma, dt, nullptr, st);
            cudaEventRecord(e1, st);
            cudaError_t ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) {
                s = cuda_fail(ce, "tuning");
                break;
            }
            float t_ms = 0.0f;
            cudaEventElapsedTime(&t_ms, e0, e1);
            if (t_ms / 3.0 < win_ms) {
                win_ms = t_ms / 3.0;
                win = t;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tile = s == HY_OK ? win : saved;
    if (s != HY_OK) return s;
    if (best) *best = win;
    if (ms) *ms = win_ms;
    return HY_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Sparse state vectors for the ADAPT driver (hy_internal.h).
// ---------------------------------------------------------------------------
struct hy::SparseState {
    const hy_ham *h = nullptr;
    hy_dtype dt = HY_F64;
    void *v = nullptr;
    int64_t cap = 0, words = 0;
    int64_t *list = nullptr;
    uint32_t *bits = nullptr;
    unsigned long long *cnt = nullptr;   // [count, snapshot, finished blocks, pad]
    double *partials = nullptr;
    int64_t n_partials = 0;
    int64_t hint = 0;                    // host estimate of the count (grids)
    int64_t *blk = nullptr;              // scratch of the bitmap compaction
    // scratch of the support-row H psi, allocated on first use: runs and
    // ralpha [Na], flags [Na + Nb], blist [Nb], counters [4]
    int64_t *runs = nullptr;
    int32_t *ralpha = nullptr, *blist = nullptr;
    uint8_t *flags = nullptr;
    unsigned long long *ctr = nullptr;
};

namespace {
template <typename T>
hy::k::SVec<T> svec(const hy::SparseState *s)
{
    hy::k::SVec<T> x;
    x.v = static_cast<T *>(s->v);
    x.list = s->list;
    x.bits = s->bits;
    x.count = s->cnt;
    x.snap = s->cnt + 1;
    x.done = s->cnt + 2;
    x.cap = s->cap;
    x.hint = s->hint;
    return x;
}

hy_status sstate_partials(hy::SparseState *s, int64_t need, cudaStream_t st)
{
    if (need <= s->n_partials) return HY_OK;
    // queued kernels may still read the old buffer
    HY_CUDA(cudaStreamSynchronize(st), "sync");
    cudaFree(s->partials);
    s->partials = nullptr;
    s->n_partials = 0;
    HY_CUDA(cudaMalloc(&s->partials, size_t(need) * sizeof(double)), "cudaMalloc(partials)");
    s->n_partials = need;
    return HY_OK;
}
}  // namespace

namespace hy {

hy_status sstate_create(const hy_ham *h, hy_dtype dt, void *v, int64_t cap, SparseState **out)
{
    if (!h || !v || !out || !valid_dtype(dt) || cap < 1) return fail(HY_ERR_ARG, "bad arguments");
    *out = nullptr;
    SparseState *s = new (std::nothrow) SparseState;
    if (!s) return fail(HY_ERR_OOM, "host allocation failed");
    s->h = h;
    s->dt = dt;
    s->v = v;
    s->cap = cap;
    s->words = (h->N + 31) / 32;
    cudaError_t e = cudaMalloc(&s->list, size_t(cap) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&s->bits, size_t(s->words) * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&s->cnt, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(s->cnt, 0, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(s->bits, 0, size_t(s->words) * sizeof(uint32_t));
    if (e == cudaSuccess) {
        s->n_partials = int64_t(8) * h->num_sms;
        e = cudaMalloc(&s->partials, size_t(s->n_partials) * sizeof(double));
    }
    if (e == cudaSuccess)
        e = cudaMalloc(&s->blk, size_t(hy::k::bits_compact_blocks(s->words)) * sizeof(int64_t));
    if (e != cudaSuccess) {
        sstate_destroy(s);
        return cuda_fail(e, "cudaMalloc(sparse state)");
    }
    *out = s;
    return HY_OK;
}

void sstate_destroy(SparseState *s)
{
    if (!s) return;
    cudaFree(s->list);
    cudaFree(s->bits);
    cudaFree(s->cnt);
    cudaFree(s->partials);
    cudaFree(s->blk);
    cudaFree(s->runs);
    cudaFree(s->ralpha);
    cudaFree(s->blist);
    cudaFree(s->flags);
    cudaFree(s->ctr);
    delete s;
}

hy_status sstate_reset(SparseState *s, bool full, bool hf, void *stream)
{
    cudaStream_t st = as_stream(stream);
    const hy_ham *h = s->h;
    if (full) {
        HY_CUDA(cudaMemsetAsync(s->v, 0, size_t(h->N) * (s->dt == HY_F64 ? 8 : 4), st), "memset");
        HY_CUDA(cudaMemsetAsync(s->bits, 0, size_t(s->words) * sizeof(uint32_t), st), "memset");
        HY_CUDA(cudaMemsetAsync(s->cnt, 0, 4 * sizeof(unsigned long long), st), "memset");
    }
    if (s->dt == HY_F64)
        HY_CUDA(hy::k::sv_reset<double>(svec<double>(s), hf, h->num_sms, st), "sparse reset");
    else
        HY_CUDA(hy::k::sv_reset<float>(svec<float>(s), hf, h->num_sms, st), "sparse reset");
    return HY_OK;
}

hy_status sstate_copy(SparseState *dst, const SparseState *src, void *stream)
{
    if (dst->dt != src->dt || dst->h != src->h || dst->cap < src->cap)
        return fail(HY_ERR_ARG, "sparse states do not match");
    cudaStream_t st = as_stream(stream);
    if (src->dt == HY_F64)
        HY_CUDA(hy::k::sv_copy<double>(svec<double>(dst), svec<double>(src), src->h->num_sms, st),
                "sparse copy");
    else
        HY_CUDA(hy::k::sv_copy<float>(svec<float>(dst), svec<float>(src), src->h->num_sms, st),
                "sparse copy");
    return HY_OK;
}

void sstate_set_hint(SparseState *s, int64_t n) { s->hint = n; }

hy_status sstate_excite(SparseState *s, const hy_pool *p, int64_t k, double theta, void *stream,
                        bool closed)
{
    const hy_ham *h = s->h;
    if (!p || p->h != h || k < 0 || k >= int64_t(p->ops.size()))
        return fail(HY_ERR_ARG, "bad operator");
    hy::k::SvOpArgs o;
    o.desc = p->d_desc;
    o.astr = h->d_astr;
    o.bstr = h->d_bstr;
    o.binom33 = h->d_binom;
    o.rank16 = h->d_rank16;
    o.n = h->n;
    o.Nb = h->Nb;
    o.qubit = p->qubit;
    const int nc = p->ops[k].desc[0];
    cudaStream_t st = as_stream(stream);
    // bytes estimated from the support the host last read back (the count
    // itself lives on the device): per listed entry and constituent, its list
    // slot and bitmap word plus two amplitudes read and written
    const double es = s->dt == HY_F64 ? 8.0 : 4.0;
    hy::ProfScope prof(HY_PROF_SPARSE_EXCITE, stream,
                       double(std::max<int64_t>(s->hint, 0)) * nc * (12.0 + 4.0 * es));
    if (s->dt == HY_F64)
        HY_CUDA(hy::k::sv_excite<double>(svec<double>(s), o, int(k), nc, theta, h->num_sms, st,
                                         closed),
                "sparse excitation");
    else
        HY_CUDA(hy::k::sv_excite<float>(svec<float>(s), o, int(k), nc, theta, h->num_sms, st,
                                        closed),
                "sparse excitation");
    return HY_OK;
}

hy_status sstate_prepare(SparseState *s, const hy_pool *p, const int32_t *ops, const double *cs,
                         int64_t L, bool renorm, double *norm2, void *stream, int64_t *step_len)
{
    const hy_ham *h = s->h;
    if (!p || p->h != h || (L > 0 && (!ops || !cs)) || L < 0 || L > (1 << 20))
        return fail(HY_ERR_ARG, "bad arguments");
    hy::k::SvOpArgs o;
    o.desc = p->d_desc;
    o.astr = h->d_astr;
    o.bstr = h->d_bstr;
    o.binom33 = h->d_binom;
    o.rank16 = h->d_rank16;
    o.n = h->n;
    o.Nb = h->Nb;
    o.qubit = p->qubit;
    cudaStream_t st = as_stream(stream);
    hy::ProfScope prof(HY_PROF_SPARSE_EXCITE, stream, 0.0);
    if (s->dt == HY_F64)
        HY_CUDA(hy::k::sv_prepare<double>(svec<double>(s), o, ops, cs, int(L), renorm, norm2,
                                          step_len, st),
                "sparse preparation");
    else
        HY_CUDA(hy::k::sv_prepare<float>(svec<float>(s), o, ops, cs, int(L), renorm, norm2,
                                         step_len, st),
                "sparse preparation");
    return HY_OK;
}

struct SupportProgram {
    const hy_ham *h = nullptr;
    int max_steps = 0;
    int optin = 0;                // opt-in shared memory per block of its device
    int64_t m = 0, steps = 0;
    int64_t *key = nullptr, *step_len = nullptr;
    // the pair lists of the steps (hy_kernels.cuh, ProgTabs), their counts
    // and the operator of each step
    uint32_t *pairs = nullptr;
    int *npairs = nullptr, *step_l = nullptr;
    int *flag = nullptr;
    // supports beyond one CTA's shared memory (allocated on first use): keys
    // in listing order, pair lists per cluster rank and the index map over
    // Omega_CIk (the vectors live in the shared memory of a cluster of CTAs)
    int64_t *key_big = nullptr;
    uint32_t *pairs_big = nullptr;
    int32_t *idx_map = nullptr;
    // H restricted to the program's support (rows in key order, columns as
    // determinant indices): valid while hss_ok
    // (row t's entries at [t * hss_w, t * hss_w + hss_cnt[t]))
    int32_t *hss_cnt = nullptr;
    uint32_t *hss_strs = nullptr;   // the support's alpha and beta string sets
    double *hss_part = nullptr;     // per-block partial energies of an apply
    unsigned *hss_done = nullptr;   // its blocks' finish counter (zero between applies)
    uint32_t *hss_col = nullptr;
    double *hss_val = nullptr;
    int64_t hss_cap = 0, hss_w = 0;
    bool hss_ok = false;
    int64_t *d_nnz = nullptr;     // the entries' total (device) ...
    int64_t *h_nnz = nullptr;     // ... copied to a pinned slot, valid after the next sync
};

hy_status prog_create(const hy_ham *h, int max_steps, SupportProgram **out)
{
    if (!h || !out || max_steps < 1 || max_steps > hy::k::kProgSteps)
        return fail(HY_ERR_ARG, "bad arguments");
    *out = nullptr;
    SupportProgram *g = new (std::nothrow) SupportProgram;
    if (!g) return fail(HY_ERR_OOM, "host allocation failed");
    g->h = h;
    g->max_steps = max_steps;
    // the kernels' shared-memory limits are raised once, on the device the
    // program is created on (and used on)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&g->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = hy::k::prog_attrs(g->optin);
    if (e == cudaSuccess) e = cudaMalloc(&g->key, size_t(hy::k::kProgMax) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&g->step_len, size_t(max_steps) * sizeof(int64_t));
    if (e == cudaSuccess)
        e = cudaMalloc(&g->pairs, size_t(max_steps) * hy::k::kProgMax * sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMalloc(&g->npairs, 2 * size_t(max_steps) * hy::k::kClusterCtas * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&g->step_l, size_t(max_steps) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&g->flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(g->flag, 0, sizeof(int));
    if (e != cudaSuccess) {
        prog_destroy(g);
        return cuda_fail(e, "cudaMalloc(support program)");
    }
    *out = g;
    return HY_OK;
}

void prog_destroy(SupportProgram *g)
{
    if (!g) return;
    cudaFree(g->key);
    cudaFree(g->step_len);
    cudaFree(g->pairs);
    cudaFree(g->npairs);
    cudaFree(g->step_l);
    cudaFree(g->flag);
    cudaFree(g->key_big);
    cudaFree(g->pairs_big);
    cudaFree(g->idx_map);
    cudaFree(g->d_nnz);
    cudaFree(g->hss_cnt);
    cudaFree(g->hss_strs);
    cudaFree(g->hss_part);
    cudaFree(g->hss_done);
    cudaFree(g->hss_col);
    cudaFree(g->hss_val);
    if (g->h_nnz) cudaFreeHost(g->h_nnz);
    delete g;
}

int64_t prog_capacity() { return hy::k::kProgBig; }

int64_t *prog_step_len(SupportProgram *g) { return g->step_len; }
const int *prog_flag(const SupportProgram *g) { return g->flag; }

int64_t prog_steps(const hy_pool *p, const int32_t *ops_host, int64_t L)
{
    int64_t s = 0;
    for (int64_t l = 0; l < L; ++l) s += p->ops[size_t(ops_host[l])].desc[0];
    return s;
}

namespace {
hy::k::SvOpArgs sv_op_args(const hy_ham *h, const hy_pool *p)
{
    hy::k::SvOpArgs o;
    o.desc = p->d_desc;
    o.astr = h->d_astr;
    o.bstr = h->d_bstr;
    o.binom33 = h->d_binom;
    o.rank16 = h->d_rank16;
    o.n = h->n;
    o.Nb = h->Nb;
    o.qubit = p->qubit;
    return o;
}
}  // namespace

hy_status prog_compile(SupportProgram *g, const SparseState *s, int64_t m, const hy_pool *p,
                       const int32_t *ops, int64_t L, int64_t steps, void *stream)
{
    if (!g || !s || !p || p->h != g->h || s->h != g->h || !ops || L < 1 || m < 1 ||
        m > hy::k::kProgBig || m > s->cap || steps < 1 || steps > g->max_steps)
        return fail(HY_ERR_ARG, "bad arguments");
    cudaStream_t st = as_stream(stream);
    hy::ProfScope prof(HY_PROF_SPARSE_EXCITE, stream, 0.0);
    if (m <= hy::k::kProgMax) {
        HY_CUDA(hy::k::prog_compile(s->list, m, g->step_len, int(steps), sv_op_args(g->h, p), ops,
                                    int(L), g->key, g->pairs, g->npairs, g->step_l, g->flag, st),
                "support program");
    } else {
        const size_t kb = size_t(hy::k::kProgBig);
        cudaError_t e = cudaSuccess;
        if (!g->key_big) e = cudaMalloc(&g->key_big, kb * sizeof(int64_t));
        // kClusterCtas lists of ceil(m / kClusterCtas) <= kb / kClusterCtas
        // pairs per step
        if (e == cudaSuccess && !g->pairs_big)
            e = cudaMalloc(&g->pairs_big, size_t(g->max_steps) * kb * sizeof(uint32_t));
        if (e == cudaSuccess && !g->idx_map)
            e = cudaMalloc(&g->idx_map, size_t(g->h->N) * sizeof(int32_t));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(support program)");
        HY_CUDA(hy::k::prog_compile_big(s->list, m, g->step_len, int(steps), sv_op_args(g->h, p),
                                        ops, int(L), s->bits, g->key_big, g->pairs_big,
                                        g->npairs, g->step_l, g->idx_map, g->flag, st),
                "support program");
    }
    g->m = m;
    g->steps = steps;
    g->hss_ok = false;
    return HY_OK;
}

namespace {
const int64_t *prog_keys(const SupportProgram *g)
{
    return g->m > hy::k::kProgMax ? g->key_big : g->key;
}
}  // namespace

hy_status prog_build_hss(SupportProgram *g, const SparseState *s, int64_t max_nnz, void *stream)
{
    if (!g || !s || s->h != g->h || g->m < 1) return fail(HY_ERR_ARG, "bad arguments");
    const hy_ham *h = g->h;
    cudaStream_t st = as_stream(stream);
    g->hss_ok = false;
    if (!g->hss_w) {
        // a row's couplings: its CSR rows of both spins (at most the
        // diagonal, the singles and the doubles of its string), then the
        // (1 + nexa) x (1 + nexb) grid of alpha-beta terms
        g->hss_w = int64_t(hy::k::fold_candidates(h->n, h->na)) +
                   hy::k::fold_candidates(h->n, h->nb) + int64_t(h->A.nex + 1) * (h->B.nex + 1);
    }
    const int64_t need = g->m * g->hss_w;
    if (need > max_nnz) return HY_OK;              // too large to pay off: not built
    cudaError_t e = cudaSuccess;
    const size_t kb = size_t(hy::k::kProgBig);
    const size_t wa = size_t((h->Na + 31) >> 5), wb = size_t((h->Nb + 31) >> 5);
    if (!g->hss_cnt) e = cudaMalloc(&g->hss_cnt, kb * sizeof(int32_t));
    if (e == cudaSuccess && !g->hss_strs) e = cudaMalloc(&g->hss_strs, (wa + wb) * sizeof(uint32_t));
    if (e == cudaSuccess && !g->hss_part)
        e = cudaMalloc(&g->hss_part, size_t(h->num_sms) * 16 * sizeof(double));
    if (e == cudaSuccess && !g->hss_done) {
        e = cudaMalloc(&g->hss_done, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemsetAsync(g->hss_done, 0, sizeof(unsigned), st);
    }
    if (e == cudaSuccess && !g->d_nnz) e = cudaMalloc(&g->d_nnz, sizeof(int64_t));
    if (e == cudaSuccess && !g->h_nnz) {
        e = cudaMallocHost(&g->h_nnz, sizeof(int64_t));
        if (e == cudaSuccess) *g->h_nnz = 0;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(support Hamiltonian)");
    if (need > g->hss_cap) {
        // queued applies may still read the old arrays
        HY_CUDA(cudaStreamSynchronize(st), "sync");
        cudaFree(g->hss_col);
        cudaFree(g->hss_val);
        g->hss_col = nullptr;
        g->hss_val = nullptr;
        g->hss_cap = 0;
        const int64_t cap = need + need / 4 + 1024;
        e = cudaMalloc(&g->hss_col, size_t(cap) * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&g->hss_val, size_t(cap) * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(g->hss_col);
            g->hss_col = nullptr;
            return HY_OK;                         // no room: the scatter serves
        }
        g->hss_cap = cap;
    }
    hy::k::HssArgs a;
    a.key = prog_keys(g);
    a.m = g->m;
    a.bits = s->bits;
    a.Ma_ptr = h->Ma64.ptr; a.Ma_col = h->Ma64.col; a.Ma_val = h->Ma64.val;
    a.Mb_ptr = h->Mb64.ptr; a.Mb_col = h->Mb64.col; a.Mb_val = h->Mb64.val;
    a.V = h->d_V64;
    a.aex = h->d_aex; a.bexT = h->d_bexT; a.astr = h->d_astr; a.bstr = h->d_bstr;
    a.n = h->n; a.nexa = h->A.nex; a.nexb = h->B.nex; a.Na = h->Na; a.Nb = h->Nb;
    a.sa = g->hss_strs; a.sb = g->hss_strs + wa;
    a.stride = g->hss_w; a.cnt = g->hss_cnt; a.col = g->hss_col; a.val = g->hss_val;
    hy::ProfScope prof(HY_PROF_SPARSE_EXCITE, stream, 0.0);
    HY_CUDA(hy::k::hss_fill(a, g->d_nnz, h->num_sms, st), "support Hamiltonian fill");
    HY_CUDA(cudaMemcpyAsync(g->h_nnz, g->d_nnz, sizeof(int64_t), cudaMemcpyDeviceToHost, st),
            "support Hamiltonian size");
    g->hss_ok = true;
    return HY_OK;
}

bool prog_hss_ready(const SupportProgram *g) { return g && g->hss_ok; }

hy_status prog_hss_apply(const SupportProgram *g, const void *psi, void *sigma, hy_dtype dt,
                         double *dot, void *stream)
{
    if (!g || !g->hss_ok || !psi || !sigma || (dot && (!g->hss_part || !g->hss_done)))
        return fail(HY_ERR_ARG, "bad arguments");
    cudaStream_t st = as_stream(stream);
    const double es = dt == HY_F64 ? 8.0 : 4.0;
    // bytes: the stored entries (12 each) and psi / sigma on the support;
    // the entry count is the pinned copy of the last build's total, read
    // without waiting (an ansatz's first apply, queued right after its build,
    // may count with the previous support's)
    const double nnz = double(*g->h_nnz);
    hy::ProfScope prof(HY_PROF_HPSI_SPARSE, stream, nnz * 12.0 + 2.0 * double(g->m) * es,
                       2.0 * nnz);
    if (dt == HY_F64)
        HY_CUDA(hy::k::hss_apply<double>(prog_keys(g), g->m, g->hss_cnt, g->hss_w, g->hss_col,
                                         g->hss_val, static_cast<const double *>(psi),
                                         static_cast<double *>(sigma), g->h->num_sms,
                                         g->hss_part, g->hss_done, dot, st),
                "support Hamiltonian apply");
    else
        HY_CUDA(hy::k::hss_apply<float>(prog_keys(g), g->m, g->hss_cnt, g->hss_w, g->hss_col,
                                        g->hss_val, static_cast<const float *>(psi),
                                        static_cast<float *>(sigma), g->h->num_sms,
                                        g->hss_part, g->hss_done, dot, st),
                "support Hamiltonian apply");
    return HY_OK;
}

namespace {
// the compiled program's tables as the kernels read them
hy::k::ProgTabs prog_tabs(const SupportProgram *g)
{
    hy::k::ProgTabs t;
    const bool big = g->m > hy::k::kProgMax;
    t.key = big ? g->key_big : g->key;
    t.pairs = big ? g->pairs_big : g->pairs;
    t.npairs = g->npairs;
    t.nrest = g->npairs + g->steps * (big ? hy::k::kClusterCtas : 1);
    t.step_l = g->step_l;
    t.m = int(g->m);
    t.steps = int(g->steps);
    t.ranks = big ? hy::k::kClusterCtas : 1;
    t.chunk = big ? int((g->m + hy::k::kClusterCtas - 1) / hy::k::kClusterCtas) : int(g->m);
    t.optin = g->optin;
    return t;
}
}  // namespace

hy_status prog_prepare(const SupportProgram *g, SparseState *s, const hy_pool *p,
                       const int32_t *ops, const double *cs, int64_t L, bool renorm,
                       double *norm2, void *stream)
{
    if (!g || !s || !p || p->h != g->h || s->h != g->h || !ops || !cs || L < 1 || g->m < 1)
        return fail(HY_ERR_ARG, "bad arguments");
    cudaStream_t st = as_stream(stream);
    hy::ProfScope prof(HY_PROF_SPARSE_EXCITE, stream, 0.0);
    const hy::k::ProgTabs t = prog_tabs(g);
    if (g->m > hy::k::kProgMax) {
        if (s->dt == HY_F64)
            HY_CUDA(hy::k::prog_prepare_big<double>(t, cs, renorm, norm2,
                                                    static_cast<double *>(s->v), st),
                    "support program preparation");
        else
            HY_CUDA(hy::k::prog_prepare_big<float>(t, cs, renorm, norm2,
                                                   static_cast<float *>(s->v), st),
                    "support program preparation");
        return HY_OK;
    }
    if (s->dt == HY_F64)
        HY_CUDA(hy::k::prog_prepare<double>(t, cs, renorm, norm2, static_cast<double *>(s->v), st),
                "support program preparation");
    else
        HY_CUDA(hy::k::prog_prepare<float>(t, cs, renorm, norm2, static_cast<float *>(s->v), st),
                "support program preparation");
    return HY_OK;
}

hy_status prog_grad(const SupportProgram *g, const hy_pool *p, const int32_t *ops,
                    const double *cs, int64_t L, const void *sigma, hy_dtype dt,
                    const double *norm2, double *g_out, void *stream)
{
    if (!g || !p || p->h != g->h || !ops || !cs || L < 1 || !sigma || !g_out || g->m < 1 ||
        !valid_dtype(dt))
        return fail(HY_ERR_ARG, "bad arguments");
    cudaStream_t st = as_stream(stream);
    hy::ProfScope prof(HY_PROF_SPARSE_EXCITE, stream, 0.0);
    const hy::k::ProgTabs t = prog_tabs(g);
    if (g->m > hy::k::kProgMax) {
        if (dt == HY_F64)
            HY_CUDA(hy::k::prog_grad_big<double>(t, cs, int(L), static_cast<const double *>(sigma),
                                                 norm2, g_out, st),
                    "support program gradient");
        else
            HY_CUDA(hy::k::prog_grad_big<float>(t, cs, int(L), static_cast<const float *>(sigma),
                                                norm2, g_out, st),
                    "support program gradient");
        return HY_OK;
    }
    if (dt == HY_F64)
        HY_CUDA(hy::k::prog_grad<double>(t, cs, int(L), static_cast<const double *>(sigma), norm2,
                                         g_out, st),
                "support program gradient");
    else
        HY_CUDA(hy::k::prog_grad<float>(t, cs, int(L), static_cast<const float *>(sigma), norm2,
                                        g_out, st),
                "support program gradient");
    return HY_OK;
}

hy_status sstate_grad_forward(SparseState *f, SparseState *w, const hy_pool *p, const int32_t *ops,
                              const double *cs, int64_t L, const void *sigma, const double *norm2,
                              double *g, void *stream)
{
    const hy_ham *h = f->h;
    if (!p || p->h != h || w->h != h || w->dt != f->dt || !sigma || !g || L < 1 ||
        L > (1 << 20) || !ops || !cs)
        return fail(HY_ERR_ARG, "bad arguments");
    hy::k::SvOpArgs o;
    o.desc = p->d_desc;
    o.astr = h->d_astr;
    o.bstr = h->d_bstr;
    o.binom33 = h->d_binom;
    o.rank16 = h->d_rank16;
    o.n = h->n;
    o.Nb = h->Nb;
    o.qubit = p->qubit;
    cudaStream_t st = as_stream(stream);
    hy::ProfScope prof(HY_PROF_SPARSE_EXCITE, stream, 0.0);
    if (f->dt == HY_F64)
        HY_CUDA(hy::k::sv_grad_fwd<double>(svec<double>(f), svec<double>(w), o, ops, cs, int(L),
                                           static_cast<const double *>(sigma), norm2, g, st),
                "forward gradient");
    else
        HY_CUDA(hy::k::sv_grad_fwd<float>(svec<float>(f), svec<float>(w), o, ops, cs, int(L),
                                          static_cast<const float *>(sigma), norm2, g, st),
                "forward gradient");
    return HY_OK;
}

hy_status sstate_dot(const SparseState *s, const void *y, double *out, void *stream)
{
    cudaStream_t st = as_stream(stream);
    hy::ProfScope prof(HY_PROF_REDUCE, stream, 0.0);
    const int sms = s->h->num_sms;
    if (s->dt == HY_F64)
        HY_CUDA(hy::k::sv_dot<double>(svec<double>(s), static_cast<const double *>(y),
                                      s->partials, out, sms, st), "sparse dot");
    else
        HY_CUDA(hy::k::sv_dot<float>(svec<float>(s), static_cast<const float *>(y), s->partials,
                                     out, sms, st), "sparse dot");
    return HY_OK;
}

hy_status sstate_scale_rsqrt(SparseState *s, const double *norm2, void *stream)
{
    cudaStream_t st = as_stream(stream);
    hy::ProfScope prof(HY_PROF_REDUCE, stream, 0.0);
    if (s->dt == HY_F64)
        HY_CUDA(hy::k::sv_scale_rsqrt<double>(svec<double>(s), norm2, s->h->num_sms, st),
                "sparse scale");
    else
        HY_CUDA(hy::k::sv_scale_rsqrt<float>(svec<float>(s), norm2, s->h->num_sms, st),
                "sparse scale");
    return HY_OK;
}

hy_status sstate_apply_h(const SparseState *s, SparseState *sig, void *sigma, void *stream)
{
    cudaStream_t st = as_stream(stream);
    const hy_ham *h = s->h;
    // bytes: the clearing of sigma when its support is not listed; work: the
    // atomic adds, at most one per coupling of a listed amplitude (from the
    // support the host last read back)
    hy::ProfScope prof(HY_PROF_HPSI_SPARSE, stream, sig ? 0.0 : double(h->N) * (s->dt == HY_F64 ? 8 : 4),
                       double(s->hint) * double(hy::ham_connections(h)));
    if (sig && (sig->dt != s->dt || sig->v != sigma)) return fail(HY_ERR_ARG, "sigma state mismatch");
    auto out = [&](auto &a) {
        a.d_m = s->cnt;
        a.cap = s->cap;
        if (sig) {
            a.obits = sig->bits;
            a.olist = sig->list;
            a.ocount = sig->cnt;
            a.ocap = sig->cap;
        }
    };
    if (s->dt == HY_F64) {
        auto a = sparse_args<double>(h, s->v, sigma, s->list, 0);
        out(a);
        HY_CUDA(hy::k::hpsi_scatter<double>(a, h->num_sms, st), "sparse H psi");
    } else {
        auto a = sparse_args<float>(h, s->v, sigma, s->list, 0);
        out(a);
        HY_CUDA(hy::k::hpsi_scatter<float>(a, h->num_sms, st), "sparse H psi");
    }
    return HY_OK;
}

hy_status sstate_apply_h_support(const SparseState *s, SparseState *sig, void *sigma, void *stream)
{
    cudaStream_t st = as_stream(stream);
    const hy_ham *h = s->h;
    if (!sig || sig->dt != s->dt || sig->v != sigma || sig->cap < s->cap)
        return fail(HY_ERR_ARG, "sigma state mismatch");
    // bytes: psi read once per listed row, sigma written once; work: the
    // bitmap probes, one per coupling of a listed row
    const double es = s->dt == HY_F64 ? 8.0 : 4.0;
    hy::ProfScope prof(HY_PROF_HPSI_SPARSE, stream, double(s->hint) * 2.0 * es,
                       double(s->hint) * double(hy::ham_connections(h)));
    // sigma's bitmap becomes psi's, its list psi's support in determinant
    // order (rows gathered together then share their alpha string, and the
    // alpha rows of psi and of the bitmap that their couplings reach stay in
    // L2), its count psi's; every listed row of sigma is then written
    HY_CUDA(cudaMemcpyAsync(sig->bits, s->bits, size_t(s->words) * sizeof(uint32_t),
                            cudaMemcpyDeviceToDevice, st), "copy bitmap");
    HY_CUDA(hy::k::bits_compact(sig->bits, sig->words, sig->list, sig->cap, sig->cnt, sig->blk, st),
            "support list");
    if (!sig->runs) {
        cudaError_t e = cudaMalloc(&sig->runs, size_t(h->Na) * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc(&sig->ralpha, size_t(h->Na) * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&sig->blist, size_t(h->Nb) * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&sig->flags, size_t(h->Na + h->Nb));
        if (e == cudaSuccess) e = cudaMalloc(&sig->ctr, 4 * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(support rows)");
    }
    auto run = [&](auto &a) {
        a.list = sig->list;
        a.cnt = sig->cnt;
        a.cap = sig->cap;
        a.bits = sig->bits;
        a.runs = sig->runs;
        a.ralpha = sig->ralpha;
        a.flagA = sig->flags;
        a.flagB = sig->flags + h->Na;
        a.blist = sig->blist;
        a.ctr = sig->ctr;
    };
    if (s->dt == HY_F64) {
        hy::k::SupRowsArgs<double> a;
        a.s = sparse_args<double>(h, s->v, sigma, sig->list, 0);
        run(a);
        HY_CUDA(hy::k::hpsi_support<double>(a, h->num_sms, st), "support H psi");
    } else {
        hy::k::SupRowsArgs<float> a;
        a.s = sparse_args<float>(h, s->v, sigma, sig->list, 0);
        run(a);
        HY_CUDA(hy::k::hpsi_support<float>(a, h->num_sms, st), "support H psi");
    }
    return HY_OK;
}

hy_status sstate_gradients(const SparseState *sc, const void *lam, const hy_pool *p,
                           const int32_t *ops, int64_t n_ops, int64_t m_hint, double *g,
                           void *stream)
{
    SparseState *s = const_cast<SparseState *>(sc);
    const hy_ham *h = s->h;
    if (!p || p->h != h || !lam || !g) return fail(HY_ERR_ARG, "bad arguments");
    if (!ops) n_ops = int64_t(p->ops.size());
    if (n_ops <= 0) return HY_OK;
    cudaStream_t st = as_stream(stream);
    const int chunks = sparse_chunks(h, n_ops, m_hint < s->cap ? m_hint : s->cap);
    hy_status r = sstate_partials(s, n_ops * chunks, st);
    if (r != HY_OK) return r;
    hy::ProfScope prof(HY_PROF_SCREEN_SPARSE, stream, 0.0);
    auto fill = [&](auto &a) {
        a.list = s->list; a.m = 0; a.d_m = s->cnt; a.cap = s->cap; a.bits = s->bits;
        a.chunks = chunks; a.partials = s->partials;
        a.desc = p->d_desc; a.ops = ops; a.n_ops = n_ops;
        a.astr = h->d_astr; a.bstr = h->d_bstr; a.binom33 = h->d_binom; a.n = h->n;
        a.rank16 = h->d_rank16;
        a.Nb = h->Nb; a.g = g; a.K = int64_t(p->ops.size()); a.bad = p->d_bad;
        a.qubit = p->qubit;
    };
    if (s->dt == HY_F64) {
        hy::k::SparseGradArgs<double> a;
        a.psi = static_cast<const double *>(s->v);
        a.sigma = static_cast<const double *>(lam);
        fill(a);
        HY_CUDA(hy::k::grad_sparse<double>(a, h->num_sms, st), "sparse gradients");
    } else {
        hy::k::SparseGradArgs<float> a;
        a.psi = static_cast<const float *>(s->v);
        a.sigma = static_cast<const float *>(lam);
        fill(a);
        HY_CUDA(hy::k::grad_sparse<float>(a, h->num_sms, st), "sparse gradients");
    }
    return HY_OK;
}

const int64_t *sstate_count(const SparseState *s)
{
    return reinterpret_cast<const int64_t *>(s->cnt);
}
const int64_t *sstate_list(const SparseState *s) { return s->list; }

int64_t ham_connections(const hy_ham *h)
{
    const int64_t sa = int64_t(h->na) * (h->n - h->na), sb = int64_t(h->nb) * (h->n - h->nb);
    const int64_t da = int64_t(hy::binom(h->na, 2)) * hy::binom(h->n - h->na, 2);
    const int64_t db = int64_t(hy::binom(h->nb, 2)) * hy::binom(h->n - h->nb, 2);
    return 1 + sa + sb + da + db + sa * sb;
}
int64_t sstate_cap(const SparseState *s) { return s->cap; }
int64_t ham_list_weight_adds(const hy_ham *h) { return 1 + int64_t(h->nb) * (h->nb + 1) / 2; }

}  // namespace hy

namespace hy {

// hy_ranker_features, with psi's touched weights taken from its support
// list when psi_state (a clean sparse vector over psi) is given
hy_status ranker_features_impl(const hy_ham *h, const hy_pool *p, const void *psi,
                               const SparseState *psi_state, const void *sigma_or_null,
                               const SparseState *sigma_state, hy_dtype dt, const float *extra,
                               float *feat, void *stream)
{
    if (!h || !p || !psi || !feat || !valid_dtype(dt)) return fail(HY_ERR_ARG, "bad arguments");
    if (p->h != h) return fail(HY_ERR_ARG, "pool belongs to another Hamiltonian");
    if (psi_state && (psi_state->v != psi || psi_state->dt != dt))
        return fail(HY_ERR_ARG, "sparse state does not match psi");
    if (sigma_state && (!sigma_or_null || sigma_state->v != sigma_or_null || sigma_state->dt != dt))
        return fail(HY_ERR_ARG, "sparse state does not match sigma");
    cudaStream_t st = as_stream(stream);
    const size_t nn = size_t(h->n) * h->n;
    // bytes only: the touched-weight product skips all-zero tiles, so its
    // executed arithmetic depends on the state and is not known here.  A
    // dense vector is read once; a listed one costs its index and value per
    // support entry (the host's estimate of the support size)
    const double esz = dt == HY_F64 ? 8.0 : 4.0;
    const SparseState *states[2] = {psi_state, sigma_state};
    const void *vecs[2] = {psi, sigma_or_null};
    double bytes = 0.0;
    for (int v = 0; v < 2 && vecs[v]; ++v)
        bytes += states[v] ? double(states[v]->hint) * (esz + 8.0) : double(h->N) * esz;
    hy::ProfScope prof(HY_PROF_FEATURES, st, bytes);
    for (int v = 0; v < 2 && vecs[v]; ++v) {
        float *B = h->d_pairB + size_t(v) * h->Na * nn, *rs = h->d_pairRs + size_t(v) * h->Na;
        float *D = h->d_pairD + size_t(v) * nn * nn;
        if (const SparseState *S = states[v]) {
            hy_status r = ensure_tw(const_cast<hy_ham *>(h), S->cap);
            if (r != HY_OK) return r;
            if (dt == HY_F64)
                HY_CUDA(hy::k::touched_weights_list<double>(
                            static_cast<const double *>(S->v), S->list, S->cnt, S->cap, S->hint,
                            h->Na, h->Nb, h->d_astr, h->d_bstr, h->n, B, rs, h->d_pairRows,
                            h->d_pairP, D, h->tw, h->num_sms, st),
                        "touched weights (list)");
            else
                HY_CUDA(hy::k::touched_weights_list<float>(
                            static_cast<const float *>(S->v), S->list, S->cnt, S->cap, S->hint,
                            h->Na, h->Nb, h->d_astr, h->d_bstr, h->n, B, rs, h->d_pairRows,
                            h->d_pairP, D, h->tw, h->num_sms, st),
                        "touched weights (list)");
        } else if (dt == HY_F64) {
            HY_CUDA(hy::k::touched_weights<double>(static_cast<const double *>(vecs[v]), h->Na,
                                                   h->Nb, h->d_astr, h->d_bstr, h->n, B, rs,
                                                   h->d_pairRows, h->d_pairP, D, h->num_sms, st),
                    "touched weights");
        } else {
            HY_CUDA(hy::k::touched_weights<float>(static_cast<const float *>(vecs[v]), h->Na,
                                                  h->Nb, h->d_astr, h->d_bstr, h->n, B, rs,
                                                  h->d_pairRows, h->d_pairP, D, h->num_sms, st),
                    "touched weights");
        }
    }
    // occupations from psi's touched-weight partials: no further pass over psi
    HY_CUDA(hy::k::occupations_from_weights(h->d_pairB, h->d_pairRs, h->d_astr, h->Na, h->n,
                                            h->d_occw, h->d_occ, st), "occupations");
    const float *Dp = sigma_or_null ? h->d_pairD : nullptr;
    const float *Ds = sigma_or_null ? h->d_pairD + nn * nn : nullptr;
    HY_CUDA(hy::k::features(p->d_desc, int64_t(p->ops.size()), h->n, h->d_h1, h->d_eri,
                            h->d_occ, extra, Dp, Ds, feat, st), "features");
    return HY_OK;
}

}  // namespace hy
