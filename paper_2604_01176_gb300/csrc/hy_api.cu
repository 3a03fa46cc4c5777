// hy_api.cu -- the library's C ABI (include/hyperion.h): argument checks,
// device tables, the per-handle workspace and the launch sequence of each
// call.  Everything numerical runs in the kernels of hy_sigma.cu and
// hy_sweeps.cu; this file only marshals.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
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

namespace hy {
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace hy

struct hy_ham {
    int n = 0, na = 0, nb = 0;
    int64_t Na = 0, Nb = 0, N = 0;
    int device = 0, num_sms = 0;
    hy::StringSpace A, B;
    hy::PauliTable pauli;
    hy::KernelTables kt;
    DevArena arena;
    uint32_t *d_astr = nullptr, *d_bstr = nullptr;
    uint32_t *d_aex = nullptr, *d_bexT = nullptr;
    uint32_t *d_binom = nullptr;
    DevCsr<double> Ma64, Mb64;
    DevCsr<float> Ma32, Mb32;
    double *d_V64 = nullptr;
    float *d_V32 = nullptr;
    // workspace (grown on demand; growth synchronises the device)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int dot_blocks = 0;
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
    size_t p = size_t(h->dot_blocks) + 64;
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

template <typename T>
hy_status upload_csr(DevArena &ar, const hy::CsrHost &M, DevCsr<T> &D)
{
    std::vector<T> v(M.val.begin(), M.val.end());
    HY_CUDA(ar.upload(&D.ptr, M.ptr.data(), M.ptr.size()), "upload csr ptr");
    HY_CUDA(ar.upload(&D.col, M.col.data(), M.col.size()), "upload csr col");
    HY_CUDA(ar.upload(&D.val, v.data(), v.size()), "upload csr val");
    return HY_OK;
}

template <typename T>
hy_status apply_h_t(hy_ham *h, const T *psi, T *sigma, cudaStream_t st)
{
    const WsLayout L = ws_layout(h, n_partials_needed(h, 0), sizeof(T));
    hy_status s = ensure_ws(h, L.total);
    if (s != HY_OK) return s;
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
    HY_CUDA(hy::k::spmm<T>(Ma->ptr, Ma->col, Ma->val, h->Na, psi, sigma, h->Nb,
                           false, st), "alpha part");
    HY_CUDA(hy::k::transpose<T>(psi, psiT, h->Na, h->Nb, st), "transpose");
    HY_CUDA(hy::k::spmm<T>(Mb->ptr, Mb->col, Mb->val, h->Nb, psiT, tau, h->Na,
                           false, st), "beta part");
    HY_CUDA(hy::k::add_transposed<T>(tau, sigma, h->Na, h->Nb, st), "beta add");
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
    HY_CUDA(hy::k::coupling<T>(a, h->num_sms, st), "alpha-beta coupling");
    return HY_OK;
}

template <typename T>
hy_status dot_t(hy_ham *h, const T *x, const T *y, double *out, cudaStream_t st)
{
    const WsLayout L = ws_layout(h, n_partials_needed(h, 0), sizeof(T));
    hy_status s = ensure_ws(h, L.total);
    if (s != HY_OK) return s;
    double *partials = reinterpret_cast<double *>(static_cast<char *>(h->ws) + L.partials);
    HY_CUDA(hy::k::dot<T>(x, y, h->N, partials, h->dot_blocks, out, st), "dot");
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
        s = apply_h_t<T>(h, psi, tmp, st);
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
        HY_CUDA(hy::k::excite<T>(psi, ae, nr, be, nc, h->Nb, c, cd.eps * sn, st),
                "excitation");
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

extern "C" {

const char *hy_last_error(void) { return g_err.c_str(); }

const char *hy_version(void) { return "hyperion-gb300 0.1 (sm_103a)"; }

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
    hy::fold_tables(h->pauli, n_orb, h->A, h->B, h->kt);

    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "device query");
    }
    h->dot_blocks = 4 * h->num_sms;

    // bexT: beta excitations transposed to [nexb][Nb] for coalesced reads
    std::vector<uint32_t> bexT(size_t(h->B.nex) * h->Nb);
    for (int64_t b = 0; b < h->Nb; ++b)
        for (int f = 0; f < h->B.nex; ++f)
            bexT[size_t(f) * h->Nb + b] = h->B.ex[size_t(b) * h->B.nex + f];
    std::vector<uint32_t> binom(33 * 33);
    for (int i = 0; i < 33; ++i)
        for (int j = 0; j < 33; ++j) binom[i * 33 + j] = hy::binom(i, j);
    std::vector<float> V32(h->kt.V.begin(), h->kt.V.end());

    hy_status s = HY_OK;
    DevArena &ar = h->arena;
    auto up = [&](cudaError_t err, const char *what) {
        if (s == HY_OK && err != cudaSuccess) s = cuda_fail(err, what);
    };
    up(ar.upload(&h->d_astr, h->A.str.data(), h->A.str.size()), "upload alpha strings");
    up(ar.upload(&h->d_bstr, h->B.str.data(), h->B.str.size()), "upload beta strings");
    up(ar.upload(&h->d_aex, h->A.ex.data(), h->A.ex.size()), "upload alpha excitations");
    up(ar.upload(&h->d_bexT, bexT.data(), bexT.size()), "upload beta excitations");
    up(ar.upload(&h->d_binom, binom.data(), binom.size()), "upload binomials");
    up(ar.upload(&h->d_V64, h->kt.V.data(), h->kt.V.size()), "upload V");
    up(ar.upload(&h->d_V32, V32.data(), V32.size()), "upload V32");
    if (s == HY_OK) s = upload_csr<double>(ar, h->kt.Ma, h->Ma64);
    if (s == HY_OK) s = upload_csr<double>(ar, h->kt.Mb, h->Mb64);
    if (s == HY_OK) s = upload_csr<float>(ar, h->kt.Ma, h->Ma32);
    if (s == HY_OK) s = upload_csr<float>(ar, h->kt.Mb, h->Mb32);
    if (s != HY_OK) {
        std::string msg = g_err;
        hy_ham_destroy(h);
        g_err = msg;
        return s;
    }
    *out = h;
    return HY_OK;
}

hy_status hy_ham_destroy(hy_ham *h)
{
    if (!h) return HY_OK;
    h->arena.release();
    if (h->ws) cudaFree(h->ws);
    delete h;
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
    if (dt == HY_F64)
        return apply_h_t<double>(h, static_cast<const double *>(psi),
                                 static_cast<double *>(sigma), as_stream(stream));
    return apply_h_t<float>(h, static_cast<const float *>(psi),
                            static_cast<float *>(sigma), as_stream(stream));
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
    if (kind != HY_POOL_SPIN_ADAPTED_SD) return fail(HY_ERR_UNSUPPORTED, "unknown pool kind");
    hy_pool *p = new (std::nothrow) hy_pool;
    if (!p) return fail(HY_ERR_OOM, "host allocation failed");
    p->h = h;
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
            hy::PatternKey ka{0, {0, 0, 0, 0}}, kb{0, {0, 0, 0, 0}};
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
            cd.ap = ka.nops ? p->pa.get(ka, h->A) : -1;
            cd.bp = kb.nops ? p->pb.get(kb, h->B) : -1;
            cd.eps = (inv & 1) ? -1 : 1;
            cd.pad = 0;
            int ci = int(p->cons.size());
            p->cons.push_back(cd);
            if (q == 0) od.c0 = ci; else od.c1 = ci;
        }
        p->opd.push_back(od);
    }
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
    if (dt == HY_F64)
        return grad_t<double>(h, p, static_cast<const double *>(psi),
                              static_cast<const double *>(sigma), ops_or_null, n_ops,
                              g_out, as_stream(stream));
    return grad_t<float>(h, p, static_cast<const float *>(psi),
                         static_cast<const float *>(sigma), ops_or_null, n_ops, g_out,
                         as_stream(stream));
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

}  // extern "C"
