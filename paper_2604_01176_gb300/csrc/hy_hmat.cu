// hy_hmat.cu -- the Hamiltonian stored explicitly over Omega_CIk and H psi
// streamed from it.
//
// The paper assembles H on the GPUs as a sparse matrix in CSR form over the
// symmetry-restricted determinant space, by summing the mapped fermionic
// terms, and distributes its rows (Sparse State-Vector Emulation section;
// Table 1 lists its size per molecule).  This file builds the same matrix,
// restricted to a range of output rows, from the library's folded tables and
// applies it with one pass over its entries, so H psi becomes an HBM stream.
//
// Storage ("sliced by alpha string").  Rows are grouped by output alpha
// string a' (N_beta rows each).  The columns of such a row block fall into
// segments, one per alpha partner a'' of a' -- a' itself, its s_a single and
// its d_a double excitations -- and within a segment every row has the same
// number of entries: 1 + s_b + d_b for a'' = a' (the beta diagonal, singles
// and doubles), 1 + s_b for a single (the beta diagonal and singles) and 1
// for a double (the beta diagonal).  So every row holds
//     w = (1 + s_b + d_b) + s_a (1 + s_b) + d_a
// entries (5,793 at 32 qubits), and an entry is its beta column b'' (16-bit)
// and its value; the segment's alpha partner is stored once per segment.
// Entry j of the rows of a block is stored for all rows together
// ([j][b'], rows padded to N_bp = N_beta rounded up to 8), so a thread that
// owns four consecutive rows reads its entries with one 8-byte and one 16- or
// 32-byte load, and the row block's reads are one contiguous stream.
//
// H psi over it: one CTA per row block (persistent over blocks), each thread
// four rows.  For the wide segments (a' itself and the singles) the psi row
// of the segment's partner is copied to shared memory ahead of use
// (cp.async, double-buffered), so the random beta gathers hit shared memory;
// the double segments gather psi[a''][b'] from global memory, coalesced.
// The matrix is read once with streaming loads; psi stays in L2.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "hy_internal.h"
#include "hy_kernels.cuh"

struct hy_hmat {
    const hy_ham *h = nullptr;
    hy_dtype dt = HY_F64;
    int n = 0;
    int64_t r0 = 0, r1 = 0, nr = 0, Nb = 0, Nbp = 0;
    int sa = 0, da = 0, sb = 0, db = 0, wD = 0, wS = 0, w = 0, S = 0;
    uint16_t *seg = nullptr;     // [nr][S] alpha partner of each segment
    uint16_t *col = nullptr;     // [nr][w][Nbp] beta column of each entry
    void *val = nullptr;         // [nr][w][Nbp] value (dt)
    size_t bytes = 0;
    int num_sms = 0;
};

namespace hy {
namespace k {
namespace {

struct BuildArgs {
    int n, sa, da, sb, wD, wS, w, S;
    int64_t r0, nr, Nb, Nbp;
    const uint32_t *astr, *bstr;
    const uint32_t *aex;        // [Na][sa] packed singles of every alpha string
    const uint32_t *bex;        // [Nb][sb] packed singles of every beta string
    const double *V;            // n^4
    const double *a_diag;       // [Na]     M_alpha[a][a]
    const double *a_sval;       // [Na][sa] M_alpha[a][single e]
    const uint16_t *a_drank;    // [Na][da] double partners (rank order)
    const double *a_dval;       // [Na][da] M_alpha[a][double d]
    const uint16_t *b_rank;     // [Nb][wD] partners of b: itself, singles, doubles (rank order)
    const int16_t *b_kind;      // [Nb][wD] -1 itself, -2 double, f >= 0 single f of b
    const double *b_val;        // [Nb][wD] M_beta[b][partner]
    const uint16_t *b_sd;       // [Nb][wS] positions in b's list of itself and its singles
};

template <typename T>
__global__ void __launch_bounds__(256)
k_hmat_build(BuildArgs a, uint16_t *seg, uint16_t *col, T *val)
{
    // Cd[r*16+s] = sum_{p in a'} V[p][p][r][s]: the alpha-diagonal coupling
    __shared__ double Cd[256];
    const int n = a.n, nn = n * n;
    for (int64_t blk = blockIdx.x; blk < a.nr; blk += gridDim.x) {
        const int64_t ap = a.r0 + blk;
        const uint32_t am = a.astr[ap];
        __syncthreads();
        for (int t = threadIdx.x; t < 256; t += blockDim.x) {
            const int r = t >> 4, s = t & 15;
            double v = 0.0;
            if (r < n && s < n)
                for (uint32_t m = am; m; m &= m - 1) {
                    const int p = __ffs(m) - 1;
                    v += a.V[size_t(p * n + p) * nn + r * n + s];
                }
            Cd[t] = v;
        }
        for (int k = threadIdx.x; k < a.S; k += blockDim.x) {
            uint16_t al;
            if (k == 0) al = uint16_t(ap);
            else if (k <= a.sa) al = uint16_t(a.aex[ap * a.sa + (k - 1)] & 0xFFFFu);
            else al = a.a_drank[ap * a.da + (k - 1 - a.sa)];
            seg[blk * a.S + k] = al;
        }
        __syncthreads();
        uint16_t *cb = col + size_t(blk) * a.w * a.Nbp;
        T *vb = val + size_t(blk) * a.w * a.Nbp;
        for (int64_t b = threadIdx.x; b < a.Nbp; b += blockDim.x) {
            if (b >= a.Nb) {                      // padding rows: no entries
                for (int j = 0; j < a.w; ++j) {
                    cb[size_t(j) * a.Nbp + b] = 0;
                    vb[size_t(j) * a.Nbp + b] = T(0);
                }
                continue;
            }
            const uint32_t bm = a.bstr[b];
            double cdd = 0.0;
            for (uint32_t m = bm; m; m &= m - 1) {
                const int r = __ffs(m) - 1;
                cdd += Cd[r * 16 + r];
            }
            const uint16_t *br = a.b_rank + b * a.wD;
            const int16_t *bk = a.b_kind + b * a.wD;
            const double *bv = a.b_val + b * a.wD;
            // a'' = a': the beta part, the diagonal, and the alpha-diagonal
            // coupling of the beta singles
            for (int j = 0; j < a.wD; ++j) {
                double v = bv[j];
                const int kind = bk[j];
                if (kind == -1) {
                    v += a.a_diag[ap] + cdd;
                } else if (kind >= 0) {
                    const uint32_t u = a.bex[b * a.sb + kind];
                    const int r = (u >> 16) & 15, s = (u >> 20) & 15;
                    v += (u >> 31) ? -Cd[r * 16 + s] : Cd[r * 16 + s];
                }
                cb[size_t(j) * a.Nbp + b] = br[j];
                vb[size_t(j) * a.Nbp + b] = T(v);
            }
            // a'' = the single e of a': its one-body element on the beta
            // diagonal plus the coupling with every beta single
            for (int e = 0; e < a.sa; ++e) {
                const uint32_t ue = a.aex[ap * a.sa + e];
                const int p = (ue >> 16) & 15, q = (ue >> 20) & 15;
                const double sgn = (ue >> 31) ? -1.0 : 1.0;
                const double *Vpq = a.V + size_t(p * n + q) * nn;
                double dsum = 0.0;
                for (uint32_t m = bm; m; m &= m - 1) {
                    const int r = __ffs(m) - 1;
                    dsum += Vpq[r * n + r];
                }
                const double mav = a.a_sval[ap * a.sa + e];
                for (int jj = 0; jj < a.wS; ++jj) {
                    const int idx = a.b_sd[b * a.wS + jj];
                    const int kind = bk[idx];
                    double v;
                    if (kind == -1) {
                        v = mav + sgn * dsum;
                    } else {
                        const uint32_t u = a.bex[b * a.sb + kind];
                        const int r = (u >> 16) & 15, s = (u >> 20) & 15;
                        v = ((u >> 31) ? -sgn : sgn) * Vpq[r * n + s];
                    }
                    const size_t j = size_t(a.wD) + size_t(e) * a.wS + jj;
                    cb[j * a.Nbp + b] = br[idx];
                    vb[j * a.Nbp + b] = T(v);
                }
            }
            // a'' = a double of a': the beta diagonal only
            for (int d = 0; d < a.da; ++d) {
                const size_t j = size_t(a.wD) + size_t(a.sa) * a.wS + d;
                cb[j * a.Nbp + b] = uint16_t(b);
                vb[j * a.Nbp + b] = T(a.a_dval[ap * a.da + d]);
            }
        }
    }
}

template <typename T>
struct SpmvArgs {
    const uint16_t *seg, *col;
    const T *val;
    const T *psi;
    T *sigma;
    int64_t nr, Nb, Nbp;
    int sa, da, wD, wS, w, S;
};

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    __device__ static void load(const float *p, float v[4])
    {
        const float4 x = __ldcs(reinterpret_cast<const float4 *>(p));
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    }
};
template <> struct Vec4<double> {
    __device__ static void load(const double *p, double v[4])
    {
        const double2 x = __ldcs(reinterpret_cast<const double2 *>(p));
        const double2 y = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
    }
};

__device__ __forceinline__ void cp_async_elem(void *dst, const void *src, int bytes)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Each thread owns MAXG groups of four rows b' (group g = tid + i*blockDim).
// The float one-group form fits 32 registers, so two CTAs share an SM and
// twice the loads are in flight.
template <typename T, int MAXG>
__global__ void __launch_bounds__(1024, (MAXG == 1 && sizeof(T) == 4) ? 2 : 1)
k_hmat_spmv(SpmvArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T *buf = reinterpret_cast<T *>(smraw);              // [2][Nb]
    const int tid = threadIdx.x, nt = blockDim.x;
    const int G = int(a.Nbp >> 2);
    const int64_t Nb = a.Nb, Nbp = a.Nbp;
    const int nst = 1 + a.sa;
    for (int64_t blk = blockIdx.x; blk < a.nr; blk += gridDim.x) {
        const uint16_t *sal = a.seg + blk * a.S;
        const uint16_t *cb = a.col + size_t(blk) * a.w * Nbp;
        const T *vb = a.val + size_t(blk) * a.w * Nbp;
        T acc[MAXG][4];
#pragma unroll
        for (int i = 0; i < MAXG; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][q] = T(0);
        __syncthreads();                                 // the previous block's readers are done
        {
            const T *src = a.psi + size_t(sal[0]) * Nb;
            for (int64_t i = tid; i < Nb; i += nt) cp_async_elem(buf + i, src + i, sizeof(T));
            cp_async_commit();
        }
        for (int k = 0; k < nst; ++k) {
            if (k + 1 < nst) {
                const T *src = a.psi + size_t(sal[k + 1]) * Nb;
                T *dst = buf + ((k + 1) & 1) * Nb;
                for (int64_t i = tid; i < Nb; i += nt) cp_async_elem(dst + i, src + i, sizeof(T));
                cp_async_commit();
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const T *ps = buf + (k & 1) * Nb;
            const int j0 = k == 0 ? 0 : a.wD + (k - 1) * a.wS;
            const int j1 = j0 + (k == 0 ? a.wD : a.wS);
#pragma unroll 2
            for (int j = j0; j < j1; ++j) {
#pragma unroll
                for (int i = 0; i < MAXG; ++i) {
                    const int g = tid + i * nt;
                    if (g < G) {
                        const size_t o = size_t(j) * Nbp + 4 * size_t(g);
                        const ushort4 c = __ldcs(reinterpret_cast<const ushort4 *>(cb + o));
                        T v[4];
                        Vec4<T>::load(vb + o, v);
                        acc[i][0] += v[0] * ps[c.x];
                        acc[i][1] += v[1] * ps[c.y];
                        acc[i][2] += v[2] * ps[c.z];
                        acc[i][3] += v[3] * ps[c.w];
                    }
                }
            }
            __syncthreads();                             // buffer k & 1 is refilled at k + 2
        }
        for (int d = 0; d < a.da; ++d) {
            const int j = a.wD + a.sa * a.wS + d;
            const T *prow = a.psi + size_t(sal[1 + a.sa + d]) * Nb;
#pragma unroll
            for (int i = 0; i < MAXG; ++i) {
                const int g = tid + i * nt;
                if (g < G) {
                    const size_t o = size_t(j) * Nbp + 4 * size_t(g);
                    const ushort4 c = __ldcs(reinterpret_cast<const ushort4 *>(cb + o));
                    T v[4];
                    Vec4<T>::load(vb + o, v);
                    acc[i][0] += v[0] * __ldg(prow + c.x);
                    acc[i][1] += v[1] * __ldg(prow + c.y);
                    acc[i][2] += v[2] * __ldg(prow + c.z);
                    acc[i][3] += v[3] * __ldg(prow + c.w);
                }
            }
        }
        T *out = a.sigma + blk * Nb;
#pragma unroll
        for (int i = 0; i < MAXG; ++i) {
            const int g = tid + i * nt;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t b = 4 * int64_t(g) + q;
                if (g < G && b < Nb) out[b] = acc[i][q];
            }
        }
    }
}

template <typename T, int MAXG>
cudaError_t launch_spmv(const SpmvArgs<T> &a, int threads, int num_sms, cudaStream_t st)
{
    const size_t smem = 2 * size_t(a.Nb) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_hmat_spmv<T, MAXG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hmat_spmv<T, MAXG>, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = int64_t(num_sms) * per_sm;
    if (grid > a.nr) grid = a.nr;
    k_hmat_spmv<T, MAXG><<<unsigned(grid), threads, smem, st>>>(a);
    hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t spmv(const SpmvArgs<T> &a, int num_sms, cudaStream_t st)
{
    if (a.nr == 0) return cudaSuccess;
    const int G = int(a.Nbp / 4);
    const int threads = std::min(1024, (G + 31) / 32 * 32);
    const int groups = (G + threads - 1) / threads;
    if (groups <= 1) return launch_spmv<T, 1>(a, threads, num_sms, st);
    if (groups == 2) return launch_spmv<T, 2>(a, threads, num_sms, st);
    if (groups <= 4) return launch_spmv<T, 4>(a, threads, num_sms, st);
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace k

namespace {

int64_t choose2(int64_t m) { return m * (m - 1) / 2; }

// partners of string r in rank order: itself, its singles and its doubles
void partner_list(const StringSpace &S, int64_t r, std::vector<uint32_t> &out)
{
    const uint32_t K = S.str[size_t(r)];
    const int n = S.n;
    out.clear();
    out.push_back(uint32_t(r));
    int occ[kMaxOrb], vir[kMaxOrb], no = 0, nv = 0;
    for (int p = 0; p < n; ++p) {
        if ((K >> p) & 1) occ[no++] = p; else vir[nv++] = p;
    }
    for (int i = 0; i < no; ++i)
        for (int a = 0; a < nv; ++a)
            out.push_back(string_rank(K ^ (1u << occ[i]) ^ (1u << vir[a])));
    for (int i = 0; i < no; ++i)
        for (int j = i + 1; j < no; ++j)
            for (int a = 0; a < nv; ++a)
                for (int b = a + 1; b < nv; ++b)
                    out.push_back(string_rank(K ^ (1u << occ[i]) ^ (1u << occ[j]) ^
                                              (1u << vir[a]) ^ (1u << vir[b])));
    std::sort(out.begin(), out.end());
}

// the folded same-spin matrix element M[r][c] (0 where the CSR holds none)
double csr_at(const CsrHost &M, int64_t r, uint32_t c)
{
    const int32_t *b = M.col.data() + M.ptr[size_t(r)], *e = M.col.data() + M.ptr[size_t(r) + 1];
    const int32_t *it = std::lower_bound(b, e, int32_t(c));
    return (it != e && *it == int32_t(c)) ? M.val[size_t(it - M.col.data())] : 0.0;
}

struct Geometry {
    int sa, da, sb, db, wD, wS, w, S;
    int64_t Nbp;
};

Geometry geometry(const HamView &v)
{
    Geometry g;
    g.sa = v.na * (v.n - v.na);
    g.da = int(choose2(v.na) * choose2(v.n - v.na));
    g.sb = v.nb * (v.n - v.nb);
    g.db = int(choose2(v.nb) * choose2(v.n - v.nb));
    g.wD = 1 + g.sb + g.db;
    g.wS = 1 + g.sb;
    g.w = g.wD + g.sa * g.wS + g.da;
    g.S = 1 + g.sa + g.da;
    g.Nbp = (v.Nb + 7) / 8 * 8;
    return g;
}

size_t matrix_bytes(const Geometry &g, int64_t nr, hy_dtype dt)
{
    const size_t es = dt == HY_F64 ? 8 : 4;
    return size_t(nr) * (size_t(g.S) * 2 + size_t(g.w) * size_t(g.Nbp) * (2 + es));
}

template <typename T>
cudaError_t dev_upload(std::vector<void *> &tmp, T **dst, const std::vector<T> &src)
{
    *dst = nullptr;
    if (src.empty()) return cudaSuccess;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, src.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    tmp.push_back(p);
    *dst = static_cast<T *>(p);
    return cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

hy_status hfail(hy_status s, const std::string &msg)
{
    set_last_error(msg);
    return s;
}

}  // namespace
}  // namespace hy

extern "C" {

hy_status hy_hmat_bytes(const hy_ham *h, hy_dtype dt, int64_t row_begin, int64_t row_end,
                        int64_t *bytes, int64_t *nnz)
{
    if (!h || (dt != HY_F64 && dt != HY_F32)) return hy::hfail(HY_ERR_ARG, "bad arguments");
    const hy::HamView v = hy::ham_view(h, true);
    if (row_begin < 0 || row_end < row_begin || row_end > v.Na)
        return hy::hfail(HY_ERR_ARG, "row range outside [0, N_alpha]");
    const hy::Geometry g = hy::geometry(v);
    if (bytes) *bytes = int64_t(hy::matrix_bytes(g, row_end - row_begin, dt));
    if (nnz) *nnz = (row_end - row_begin) * v.Nb * int64_t(g.w);
    return HY_OK;
}

hy_status hy_hmat_build(const hy_ham *h, hy_dtype dt, int64_t row_begin, int64_t row_end,
                        hy_hmat **out)
{
    if (!out) return hy::hfail(HY_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!h || (dt != HY_F64 && dt != HY_F32)) return hy::hfail(HY_ERR_ARG, "bad arguments");
    const hy::HamView v = hy::ham_view(h, true);
    if (row_begin < 0 || row_end < row_begin || row_end > v.Na)
        return hy::hfail(HY_ERR_ARG, "row range outside [0, N_alpha]");
    const hy::Geometry g = hy::geometry(v);
    if (v.Na > 65536 || v.Nb > 65536)
        return hy::hfail(HY_ERR_UNSUPPORTED, "string ranks beyond 16 bits");
    const int64_t nr = row_end - row_begin;
    const size_t need = hy::matrix_bytes(g, nr, dt);
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return hy::hfail(HY_ERR_CUDA, std::string("cudaMemGetInfo: ") +
                                                             cudaGetErrorString(e));
    const size_t margin = size_t(1) << 30;       // build tables and the caller's next buffers
    if (need + margin > free_b)
        return hy::hfail(HY_ERR_OOM, "the explicit H of rows [" + std::to_string(row_begin) +
                                         ", " + std::to_string(row_end) + ") needs " +
                                         std::to_string(need) + " bytes; " +
                                         std::to_string(free_b) + " are free");
    hy_hmat *m = new (std::nothrow) hy_hmat;
    if (!m) return hy::hfail(HY_ERR_OOM, "host allocation failed");
    m->h = h;
    m->dt = dt;
    m->n = v.n;
    m->r0 = row_begin;
    m->r1 = row_end;
    m->nr = nr;
    m->Nb = v.Nb;
    m->Nbp = g.Nbp;
    m->sa = g.sa; m->da = g.da; m->sb = g.sb; m->db = g.db;
    m->wD = g.wD; m->wS = g.wS; m->w = g.w; m->S = g.S;
    m->bytes = need;
    m->num_sms = v.num_sms;
    if (nr == 0) {
        *out = m;
        return HY_OK;
    }

    // host tables of the build (rank-ordered partner lists and the folded
    // same-spin matrix elements on them)
    const hy::StringSpace &A = *v.A, &B = *v.B;
    const hy::KernelTables &kt = *v.kt;
    std::vector<double> a_diag(size_t(v.Na)), a_sval(size_t(v.Na) * g.sa), a_dval(size_t(v.Na) * g.da);
    std::vector<uint16_t> a_drank(size_t(v.Na) * g.da);
    std::vector<uint16_t> b_rank(size_t(v.Nb) * g.wD), b_sd(size_t(v.Nb) * g.wS);
    std::vector<int16_t> b_kind(size_t(v.Nb) * g.wD);
    std::vector<double> b_val(size_t(v.Nb) * g.wD);
    int shape_ok = 1;
#pragma omp parallel for schedule(dynamic, 64) reduction(min : shape_ok)
    for (int64_t a = 0; a < v.Na; ++a) {
        std::vector<uint32_t> pl;
        hy::partner_list(A, a, pl);
        a_diag[size_t(a)] = hy::csr_at(kt.Ma, a, uint32_t(a));
        for (int e2 = 0; e2 < g.sa; ++e2)
            a_sval[size_t(a) * g.sa + e2] =
                hy::csr_at(kt.Ma, a, A.ex[size_t(a) * A.nex + e2] & 0xFFFFu);
        // doubles: the partners that are neither a itself nor a single
        std::vector<uint32_t> sing;
        for (int e2 = 0; e2 < g.sa; ++e2) sing.push_back(A.ex[size_t(a) * A.nex + e2] & 0xFFFFu);
        std::sort(sing.begin(), sing.end());
        int d = 0;
        for (uint32_t c : pl) {
            if (c == uint32_t(a) || std::binary_search(sing.begin(), sing.end(), c)) continue;
            if (d < g.da) {
                a_drank[size_t(a) * g.da + d] = uint16_t(c);
                a_dval[size_t(a) * g.da + d] = hy::csr_at(kt.Ma, a, c);
            }
            ++d;
        }
        if (d != g.da || int(pl.size()) != 1 + g.sa + g.da) shape_ok = 0;
    }
#pragma omp parallel for schedule(dynamic, 64) reduction(min : shape_ok)
    for (int64_t b = 0; b < v.Nb; ++b) {
        std::vector<uint32_t> pl;
        hy::partner_list(B, b, pl);
        if (int(pl.size()) != g.wD) {
            shape_ok = 0;
            continue;
        }
        int jj = 0;
        for (int j = 0; j < g.wD; ++j) {
            const uint32_t c = pl[size_t(j)];
            int kind = -2;
            if (c == uint32_t(b)) {
                kind = -1;
            } else {
                for (int f = 0; f < g.sb; ++f)
                    if ((B.ex[size_t(b) * B.nex + f] & 0xFFFFu) == c) { kind = f; break; }
            }
            b_rank[size_t(b) * g.wD + j] = uint16_t(c);
            b_kind[size_t(b) * g.wD + j] = int16_t(kind);
            b_val[size_t(b) * g.wD + j] = hy::csr_at(kt.Mb, b, c);
            if (kind != -2 && jj < g.wS) b_sd[size_t(b) * g.wS + jj++] = uint16_t(j);
        }
        if (jj != g.wS) shape_ok = 0;
    }
    if (!shape_ok) {
        delete m;
        return hy::hfail(HY_ERR_UNSUPPORTED, "string partner lists do not have the expected shape");
    }
    std::vector<uint32_t> bex(B.ex.begin(), B.ex.end());
    std::vector<uint32_t> aex(A.ex.begin(), A.ex.end());
    std::vector<uint32_t> astr(A.str.begin(), A.str.end()), bstr(B.str.begin(), B.str.end());

    std::vector<void *> tmp;
    hy::k::BuildArgs ba{};
    ba.n = v.n; ba.sa = g.sa; ba.da = g.da; ba.sb = g.sb; ba.wD = g.wD; ba.wS = g.wS;
    ba.w = g.w; ba.S = g.S; ba.r0 = row_begin; ba.nr = nr; ba.Nb = v.Nb; ba.Nbp = g.Nbp;
    hy_status s = HY_OK;
    auto up = [&](cudaError_t err, const char *what) {
        if (s == HY_OK && err != cudaSuccess) s = hy::hfail(HY_ERR_CUDA, std::string(what) + ": " +
                                                                           cudaGetErrorString(err));
    };
    up(hy::dev_upload(tmp, const_cast<uint32_t **>(&ba.astr), astr), "upload alpha strings");
    up(hy::dev_upload(tmp, const_cast<uint32_t **>(&ba.bstr), bstr), "upload beta strings");
    up(hy::dev_upload(tmp, const_cast<uint32_t **>(&ba.aex), aex), "upload alpha singles");
    up(hy::dev_upload(tmp, const_cast<uint32_t **>(&ba.bex), bex), "upload beta singles");
    up(hy::dev_upload(tmp, const_cast<double **>(&ba.V), kt.V), "upload V");
    up(hy::dev_upload(tmp, const_cast<double **>(&ba.a_diag), a_diag), "upload tables");
    up(hy::dev_upload(tmp, const_cast<double **>(&ba.a_sval), a_sval), "upload tables");
    up(hy::dev_upload(tmp, const_cast<uint16_t **>(&ba.a_drank), a_drank), "upload tables");
    up(hy::dev_upload(tmp, const_cast<double **>(&ba.a_dval), a_dval), "upload tables");
    up(hy::dev_upload(tmp, const_cast<uint16_t **>(&ba.b_rank), b_rank), "upload tables");
    up(hy::dev_upload(tmp, const_cast<int16_t **>(&ba.b_kind), b_kind), "upload tables");
    up(hy::dev_upload(tmp, const_cast<double **>(&ba.b_val), b_val), "upload tables");
    up(hy::dev_upload(tmp, const_cast<uint16_t **>(&ba.b_sd), b_sd), "upload tables");
    const size_t es = dt == HY_F64 ? 8 : 4;
    const size_t n_ent = size_t(nr) * g.w * size_t(g.Nbp);
    if (s == HY_OK) up(cudaMalloc(&m->seg, size_t(nr) * g.S * sizeof(uint16_t)), "cudaMalloc(segments)");
    if (s == HY_OK) up(cudaMalloc(&m->col, n_ent * sizeof(uint16_t)), "cudaMalloc(columns)");
    if (s == HY_OK) up(cudaMalloc(&m->val, n_ent * es), "cudaMalloc(values)");
    if (s == HY_OK) {
        int64_t grid = int64_t(v.num_sms) * 8;
        if (grid > nr) grid = nr;
        if (dt == HY_F64)
            hy::k::k_hmat_build<double><<<unsigned(grid), 256>>>(ba, m->seg, m->col,
                                                                 static_cast<double *>(m->val));
        else
            hy::k::k_hmat_build<float><<<unsigned(grid), 256>>>(ba, m->seg, m->col,
                                                                static_cast<float *>(m->val));
        hy::count_launch();
        up(cudaGetLastError(), "explicit H build");
        up(cudaDeviceSynchronize(), "explicit H build");
    }
    for (void *p : tmp) cudaFree(p);
    if (s != HY_OK) {
        if (m->val) cudaFree(m->val);
        if (m->col) cudaFree(m->col);
        if (m->seg) cudaFree(m->seg);
        delete m;
        if (s == HY_ERR_CUDA) cudaGetLastError();
        return s;
    }
    *out = m;
    return HY_OK;
}

hy_status hy_hmat_destroy(hy_hmat *m)
{
    if (!m) return HY_OK;
    if (m->val) cudaFree(m->val);
    if (m->col) cudaFree(m->col);
    if (m->seg) cudaFree(m->seg);
    delete m;
    return HY_OK;
}

hy_status hy_hmat_info(const hy_hmat *m, int64_t *row_begin, int64_t *row_end, int64_t *nnz,
                       int64_t *row_len, int64_t *bytes)
{
    if (!m) return hy::hfail(HY_ERR_ARG, "handle is NULL");
    if (row_begin) *row_begin = m->r0;
    if (row_end) *row_end = m->r1;
    if (nnz) *nnz = m->nr * m->Nb * int64_t(m->w);
    if (row_len) *row_len = m->w;
    if (bytes) *bytes = int64_t(m->bytes);
    return HY_OK;
}

hy_status hy_hmat_apply(const hy_hmat *m, const void *psi, void *sigma_rows, void *stream)
{
    if (!m) return hy::hfail(HY_ERR_ARG, "handle is NULL");
    if (m->nr == 0) return HY_OK;                 // nothing stored, nothing written
    if (!psi || !sigma_rows) return hy::hfail(HY_ERR_ARG, "bad arguments");
    if (psi == sigma_rows) return hy::hfail(HY_ERR_ARG, "psi and sigma_rows must not alias");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t es = m->dt == HY_F64 ? 8 : 4;
    const double bytes = double(m->bytes) + double(m->nr * m->Nb) * double(es) * 2.0;
    hy::ProfScope prof(HY_PROF_HMAT, stream, bytes,
                       2.0 * double(m->nr) * double(m->Nb) * double(m->w));
    cudaError_t e;
    if (m->dt == HY_F64) {
        hy::k::SpmvArgs<double> a{m->seg, m->col, static_cast<const double *>(m->val),
                                  static_cast<const double *>(psi), static_cast<double *>(sigma_rows),
                                  m->nr, m->Nb, m->Nbp, m->sa, m->da, m->wD, m->wS, m->w, m->S};
        e = hy::k::spmv<double>(a, m->num_sms, st);
    } else {
        hy::k::SpmvArgs<float> a{m->seg, m->col, static_cast<const float *>(m->val),
                                 static_cast<const float *>(psi), static_cast<float *>(sigma_rows),
                                 m->nr, m->Nb, m->Nbp, m->sa, m->da, m->wD, m->wS, m->w, m->S};
        e = hy::k::spmv<float>(a, m->num_sms, st);
    }
    if (e != cudaSuccess) return hy::hfail(HY_ERR_CUDA, std::string("explicit H psi: ") +
                                                            cudaGetErrorString(e));
    return HY_OK;
}

hy_status hy_hmat_row(const hy_hmat *m, int64_t det, int64_t *cols, double *vals, int64_t cap,
                      int64_t *len)
{
    if (!m || !len) return hy::hfail(HY_ERR_ARG, "bad arguments");
    const int64_t a = m->Nb ? det / m->Nb : 0, b = m->Nb ? det % m->Nb : 0;
    if (det < 0 || a < m->r0 || a >= m->r1)
        return hy::hfail(HY_ERR_ARG, "determinant outside the stored rows");
    *len = m->w;
    if (cap < m->w || !cols || !vals) return HY_OK;
    const int64_t blk = a - m->r0;
    std::vector<uint16_t> seg(size_t(m->S)), col(size_t(m->w));
    const size_t es = m->dt == HY_F64 ? 8 : 4;
    std::vector<unsigned char> raw(size_t(m->w) * es);
    cudaError_t e = cudaMemcpy(seg.data(), m->seg + blk * m->S, size_t(m->S) * 2,
                               cudaMemcpyDeviceToHost);
    const size_t base = size_t(blk) * m->w * size_t(m->Nbp) + size_t(b);
    if (e == cudaSuccess)
        e = cudaMemcpy2D(col.data(), 2, m->col + base, size_t(m->Nbp) * 2, 2, size_t(m->w),
                         cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy2D(raw.data(), es, static_cast<const char *>(m->val) + base * es,
                         size_t(m->Nbp) * es, es, size_t(m->w), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return hy::hfail(HY_ERR_CUDA, std::string("row copy: ") +
                                                            cudaGetErrorString(e));
    for (int j = 0; j < m->w; ++j) {
        int k;
        if (j < m->wD) k = 0;
        else if (j < m->wD + m->sa * m->wS) k = 1 + (j - m->wD) / m->wS;
        else k = 1 + m->sa + (j - m->wD - m->sa * m->wS);
        cols[j] = int64_t(seg[size_t(k)]) * m->Nb + col[size_t(j)];
        if (m->dt == HY_F64) {
            double x;
            std::memcpy(&x, raw.data() + size_t(j) * 8, 8);
            vals[j] = x;
        } else {
            float x;
            std::memcpy(&x, raw.data() + size_t(j) * 4, 4);
            vals[j] = double(x);
        }
    }
    return HY_OK;
}

}  // extern "C"
