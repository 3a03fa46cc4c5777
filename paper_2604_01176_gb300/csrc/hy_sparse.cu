// hy_sparse.cu -- the sparse-state path (paper: Sparse State-Vector
// Emulation section -- the state is stored sparse, starts from the single
// Hartree-Fock determinant, and H is applied as a sparse matrix to a sparse
// vector).  Early in ADAPT-VQE psi = prod exp(theta A) |HF> has few nonzero
// amplitudes (exact zeros stay exactly zero under the pair rotations), so:
//   * k_support lists the nonzero amplitudes (warp-aggregated compaction);
//   * k_hpsi_scatter computes sigma = H psi by scattering every nonzero
//     amplitude to all determinants H connects it to (same folded tables
//     and coefficients as the dense sweep, read column-wise; H is real
//     symmetric), with atomic adds into a zeroed sigma;
//   * k_grad_sparse evaluates g_k = 2 <sigma|A_k psi> over the pairs with an
//     endpoint in the support only, applying each constituent's operator
//     string to the determinant's bits (Jordan-Wigner signs) and ranking the
//     partner with the binomial table.
#include <cmath>

#include <cooperative_groups.h>

#include "hy_kernels.cuh"

namespace cg = cooperative_groups;

namespace hy {
namespace k {

template <typename T>
__global__ void __launch_bounds__(256)
k_support(const T *__restrict__ psi, int64_t N, int64_t *__restrict__ list, int64_t cap,
          unsigned long long *__restrict__ count)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t Nr = (N + 31) / 32 * 32;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < Nr; i += stride) {
        const bool nz = i < N && psi[i] != T(0);
        const unsigned m = __ballot_sync(0xffffffffu, nz);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (nz) {
            const unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
            if (int64_t(pos) < cap) list[pos] = i;
        }
    }
}

// support length: the device count clamped to the list's capacity, or m
__device__ __forceinline__ int64_t list_len(const unsigned long long *d_m, int64_t m, int64_t cap)
{
    if (!d_m) return m;
    const unsigned long long c = *d_m;
    return c < (unsigned long long)cap ? int64_t(c) : cap;
}

__device__ __forceinline__ bool member(const uint32_t *bits, int64_t i)
{
    return (bits[i >> 5] >> (i & 31)) & 1u;
}

// sum over the set bits p of mask (n <= 16 orbitals), in ascending order, of
// base[p * stride]: the loads are independent and issued together, the
// additions keep the ascending order
template <typename T>
__device__ __forceinline__ T sum_mask(const T *base, int stride, uint32_t mask)
{
    T v = T(0);
#pragma unroll
    for (int p = 0; p < 16; ++p)
        if ((mask >> p) & 1u) v += base[size_t(p) * stride];
    return v;
}

// sum over the occupied orbitals p of mask of V[pp][rs]
template <typename T>
__device__ __forceinline__ T sum_diag(const T *V, int n, int nn, uint32_t mask, int rs)
{
    return sum_mask(V + rs, (n + 1) * nn, mask);
}

// sigma[o] += v; with an output list, o is also listed the first time it is
// reached (the bitmap word is read first, so an already listed target costs
// no atomic on the bitmap)
template <typename T>
__device__ __forceinline__ void emit(const SparseArgs<T> &a, int64_t o, T v)
{
    atomicAdd(a.sigma + o, v);
    if (!a.obits) return;
    const uint32_t bit = 1u << (o & 31);
    if (__ldcg(a.obits + (o >> 5)) & bit) return;
    if (atomicOr(a.obits + (o >> 5), bit) & bit) return;
    const unsigned long long pos = atomicAdd(a.ocount, 1ull);
    if (pos < (unsigned long long)a.ocap) a.olist[pos] = o;
}

// One CTA per support entry (grid-stride).  The alpha-beta part's targets
// form a (1 + s_a) x (1 + s_b) grid: a thread keeps one beta excitation f
// (its target column, orbitals and sign in registers) and walks a stride of
// the alpha excitations, staged once per entry in shared memory, so the
// inner loop is one table read, one V load and one atomic add; the
// no-excitation row and column (diagonal sums) are taken apart.
template <typename T>
__global__ void __launch_bounds__(256)
k_hpsi_scatter(SparseArgs<T> a)
{
    __shared__ uint32_t aexs[64];
    const int n = a.n, nn = n * n, nexa = a.nexa, nexb = a.nexb;
    const int64_t Nb = a.Nb;
    const int64_t m = list_len(a.d_m, a.m, a.cap);
    // beta slot and alpha phase of this thread
    const int P = nexb > 0 ? int(blockDim.x) / nexb : 0;
    const bool slot = int(threadIdx.x) < P * nexb;
    const int fs = slot ? int(threadIdx.x) % nexb : 0, ph = slot ? int(threadIdx.x) / nexb : 0;
    for (int64_t t = blockIdx.x; t < m; t += gridDim.x) {
        const int64_t d = a.list[t];
        const T x = a.psi[d];
        const int64_t A = d / Nb, B = d % Nb;
        __syncthreads();                              // the previous entry's readers are done
        if (int(threadIdx.x) < nexa) aexs[threadIdx.x] = a.aex[A * nexa + threadIdx.x];
        for (int k = a.Ma_ptr[A] + threadIdx.x; k < a.Ma_ptr[A + 1]; k += blockDim.x)
            emit(a, int64_t(a.Ma_col[k]) * Nb + B, a.Ma_val[k] * x);
        for (int k = a.Mb_ptr[B] + threadIdx.x; k < a.Mb_ptr[B + 1]; k += blockDim.x)
            emit(a, A * Nb + a.Mb_col[k], a.Mb_val[k] * x);
        __syncthreads();
        const uint32_t am = a.astr[A], bm = a.bstr[B];
        if (slot) {
            const uint32_t w = a.bexT[size_t(fs) * Nb + B];
            const int64_t Bo = w & 0xFFFFu;
            const int rs = int((w >> 20) & 15) * n + int((w >> 16) & 15);
            const bool negb = (w >> 31) != 0;
            if (ph == 0) {                            // no alpha excitation
                const T c = sum_diag<T>(a.V, n, nn, am, rs);
                emit(a, A * Nb + Bo, (negb ? -c : c) * x);
            }
            const T *Vrs = a.V + rs;
            for (int e = ph; e < nexa; e += P) {
                const uint32_t u = aexs[e];
                const int64_t Ao = u & 0xFFFFu;
                const int pq = int((u >> 20) & 15) * n + int((u >> 16) & 15);
                const T c = Vrs[size_t(pq) * nn];
                emit(a, Ao * Nb + Bo, (negb != ((u >> 31) != 0) ? -c : c) * x);
            }
        }
        // no beta excitation: the diagonal beta sum for each alpha excitation
        for (int e = int(threadIdx.x) - 1; e < nexa; e += blockDim.x) {
            T c = T(0);
            if (e < 0) {
                for (uint32_t mm = bm; mm; mm &= mm - 1) {
                    const int rr = __ffs(mm) - 1;
                    c += sum_diag<T>(a.V, n, nn, am, rr * n + rr);
                }
                emit(a, A * Nb + B, c * x);
            } else {
                const uint32_t u = aexs[e];
                const int pq = int((u >> 20) & 15) * n + int((u >> 16) & 15);
                c = sum_mask(a.V + size_t(pq) * nn, n + 1, bm);
                emit(a, int64_t(u & 0xFFFFu) * Nb + B, ((u >> 31) ? -c : c) * x);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// sigma = H psi on psi's support S only, for large supports (rows = S's
// determinants, sorted).  H's couplings of a row d = (A, B) are enumerated as
// k_hpsi_scatter enumerates the targets of d (H is real symmetric, so the
// column of d is its row); psi is zero off S, so each row's sum needs no
// membership test.  Two passes, each reading psi from shared memory:
//   k_sup_alpha, one CTA per alpha string A of S (the run of S's rows with
//     that alpha string): psi's row A is staged, then, one alpha excitation
//     e of A at a time, psi's row A_e; the rows (A, B) of the run collect
//       the same-alpha part (beta-string CSR M_beta, the beta excitations
//       with no alpha excitation, the diagonal) from row A and
//       the alpha-beta part, sum_f sgn V[pq_e][rs_f] psi[A_e][B_f] plus the
//       alpha excitation with a diagonal beta part, from row A_e,
//     a warp per row, lanes over its beta excitations (B-major table);
//     sigma[A, B] is written;
//   k_sup_beta, one CTA per beta string B of S: psi's column B on the alpha
//     strings of S is staged, and each row (A, B) of S adds the same-beta
//     part (alpha-string CSR M_alpha) from it.
// Every sum runs in a fixed order, so the result is deterministic.  Work is
// handed out through an atomic counter (runs differ in length).
// ---------------------------------------------------------------------------

// the runs of the sorted support by alpha string (unordered; the CTA of a run
// counts its length from the bitmap) and the beta strings present
__global__ void __launch_bounds__(256)
k_sup_runs(const int64_t *__restrict__ list, const unsigned long long *__restrict__ cnt,
           int64_t cap, int64_t Nb, int64_t *__restrict__ runs, int32_t *__restrict__ ralpha,
           uint8_t *__restrict__ flagA, uint8_t *__restrict__ flagB,
           unsigned long long *__restrict__ ctr)
{
    const int64_t m = list_len(cnt, 0, cap);
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t d = list[t], A = d / Nb;
        flagB[d - A * Nb] = 1;
        if (t == 0 || list[t - 1] / Nb != A) {
            const unsigned long long pos = atomicAdd(ctr + 0, 1ull);
            runs[pos] = t;
            ralpha[pos] = int32_t(A);
            flagA[A] = 1;
        }
    }
}

__global__ void __launch_bounds__(256)
k_sup_blist(const uint8_t *__restrict__ flagB, int64_t Nb, int32_t *__restrict__ blist,
            unsigned long long *__restrict__ ctr)
{
    for (int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; b < Nb;
         b += int64_t(gridDim.x) * blockDim.x)
        if (flagB[b]) blist[atomicAdd(ctr + 1, 1ull)] = int32_t(b);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kSupThreads = 512;

template <typename T>
size_t sup_alpha_smem(int64_t Nb, int nn)
{
    return (2 * size_t((Nb + 3) / 4 * 4) + 2 * size_t(nn)) * sizeof(T);
}

// stage psi's row R (Nb amplitudes) into shared memory: every thread issues
// its element copies without waiting (cp.async), then waits for its own;
// the caller's barrier makes the row visible to the block
template <typename T>
__device__ __forceinline__ void stage_row(T *row, const T *src, int64_t Nb)
{
    for (int64_t i = threadIdx.x; i < Nb; i += blockDim.x) {
        const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(row + i));
        if (sizeof(T) == 8)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src + i)
                         : "memory");
        else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src + i)
                         : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// The alpha-beta part runs a thread per row (A, B): the row's beta
// excitations stay in registers, and each staged row A_e costs it one fused
// multiply-add per beta excitation (plus one per occupied beta orbital, the
// diagonal beta part) and no cross-lane reduction -- in double precision the
// GB300's FP64 pipe is the bound, so every FP64 instruction is useful work.
// The same-alpha part (CSR rows of ~n^4/4 entries) keeps a warp per row with
// its lanes over the entries, reduced once per row.
template <typename T>
__global__ void __launch_bounds__(kSupThreads)
k_sup_alpha(SupRowsArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char sup_sm[];
    const SparseArgs<T> &h = a.s;
    const int n = h.n, nn = n * n, nexa = h.nexa, nexb = h.nexb;
    const int64_t Nb = h.Nb, Nbp = (Nb + 3) / 4 * 4;
    T *row = reinterpret_cast<T *>(sup_sm);       // a staged row of psi
    T *acc = row + Nbp;                           // the run's same-alpha sums
    T *vrow = acc + Nbp;                          // V[pq_e][.] with e's sign
    T *dA = vrow + nn;                            // sum_{p in A} V[pp][.]
    __shared__ uint32_t aexs[64];
    __shared__ int64_t sh_r, sh_cnt[kSupThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kSupThreads / 32;
    for (;;) {
        __syncthreads();                          // the previous run is written
        if (tid == 0) sh_r = int64_t(atomicAdd(a.ctr + 2, 1ull));
        __syncthreads();
        const int64_t r = sh_r;
        if (r >= int64_t(a.ctr[0])) break;
        const int64_t t0 = a.runs[r], A = a.ralpha[r];
        // the run's length: A's row of the bitmap (bits A Nb .. A Nb + Nb - 1)
        {
            const int64_t b0 = A * Nb, b1 = b0 + Nb, w0 = b0 >> 5, w1 = (b1 - 1) >> 5;
            int64_t c = 0;
            for (int64_t w = w0 + tid; w <= w1; w += kSupThreads) {
                uint32_t x = a.bits[w];
                if (w == w0) x &= ~0u << (b0 & 31);
                if (w == w1 && (b1 & 31)) x &= (1u << (b1 & 31)) - 1u;
                c += __popc(x);
            }
            c = warp_sum(c);
            if (lane == 0) sh_cnt[warp] = c;
        }
        if (tid < nexa) aexs[tid] = h.aex[A * nexa + tid];
        const uint32_t am = h.astr[A];
        for (int i = tid; i < nn; i += kSupThreads) dA[i] = sum_diag<T>(h.V, n, nn, am, i);
        stage_row(row, h.psi + A * Nb, Nb);
        __syncthreads();
        int64_t mA = 0;
        for (int w = 0; w < nwarps; ++w) mA += sh_cnt[w];
        if (t0 + mA > a.cap) mA = a.cap - t0;    // an overflowed (invalid) support
        const int64_t *Brun = a.list + t0;
        // same alpha string: M_beta, beta excitations without an alpha
        // excitation, the diagonal; a warp per row
        for (int64_t i = warp; i < mA; i += nwarps) {
            const int64_t B = Brun[i] - A * Nb;
            T part = T(0);
            for (int k = h.Mb_ptr[B] + lane; k < h.Mb_ptr[B + 1]; k += 32)
                part = fma(h.Mb_val[k], row[h.Mb_col[k]], part);
            for (int f = lane; f < nexb; f += 32) {
                const uint32_t w = h.bex[B * nexb + f];
                const T c = dA[int((w >> 20) & 15) * n + int((w >> 16) & 15)];
                part = fma((w >> 31) ? -c : c, row[w & 0xFFFFu], part);
            }
            if (lane < n && ((h.bstr[B] >> lane) & 1u))      // occupied beta orbital
                part = fma(dA[lane * n + lane], row[B], part);
            part = warp_sum(part);
            if (lane == 0) acc[i] = part;
        }
        // alpha excitations: psi's rows A_e, a thread per row (A, B), chunks
        // of one row per thread
        for (int64_t c0 = 0; c0 < mA; c0 += kSupThreads) {
            const int64_t i = c0 + tid;
            const bool act = i < mA;
            const int64_t B = act ? Brun[i] - A * Nb : 0;
            uint32_t bx[64];
#pragma unroll
            for (int f = 0; f < 64; ++f) bx[f] = act && f < nexb ? h.bex[B * nexb + f] : 0u;
            const uint32_t bm = act ? h.bstr[B] : 0u;
            T s = T(0);
            for (int e = 0; e < nexa; ++e) {
                const uint32_t u = aexs[e];
                const int64_t Ao = u & 0xFFFFu;
                if (!a.flagA[Ao]) continue;       // psi's row A_e is zero
                __syncthreads();                  // the previous row's readers are done
                const int pq = int((u >> 20) & 15) * n + int((u >> 16) & 15);
                for (int q = tid; q < nn; q += kSupThreads) {
                    const T c = h.V[size_t(pq) * nn + q];
                    vrow[q] = (u >> 31) ? -c : c;
                }
                stage_row(row, h.psi + Ao * Nb, Nb);
                __syncthreads();
                if (act) {
#pragma unroll
                    for (int f = 0; f < 64; ++f) {
                        if (f < nexb) {
                            const uint32_t w = bx[f];
                            const T c = vrow[int((w >> 20) & 15) * n + int((w >> 16) & 15)];
                            s = fma((w >> 31) ? -c : c, row[w & 0xFFFFu], s);
                        }
                    }
                    const T xb = row[B];
                    for (uint32_t mm = bm; mm; mm &= mm - 1) {
                        const int rr = __ffs(mm) - 1;
                        s = fma(vrow[rr * n + rr], xb, s);
                    }
                }
            }
            __syncthreads();
            if (act) h.sigma[Brun[i]] = acc[i] + s;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kSupThreads)
k_sup_beta(SupRowsArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char sup_sm[];
    const SparseArgs<T> &h = a.s;
    const int64_t Na = h.Na, Nb = h.Nb;
    T *col = reinterpret_cast<T *>(sup_sm);       // psi's column B over alpha strings
    __shared__ int64_t sh_r;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kSupThreads / 32;
    for (;;) {
        __syncthreads();
        if (tid == 0) sh_r = int64_t(atomicAdd(a.ctr + 3, 1ull));
        __syncthreads();
        const int64_t r = sh_r;
        if (r >= int64_t(a.ctr[1])) break;
        const int64_t B = a.blist[r];
        const int64_t nr = int64_t(a.ctr[0]);
        for (int64_t i = tid; i < Na; i += kSupThreads) col[i] = T(0);
        __syncthreads();
        for (int64_t j = tid; j < nr; j += kSupThreads) {
            const int64_t A = a.ralpha[j];
            col[A] = h.psi[A * Nb + B];
        }
        __syncthreads();
        // the rows (A, B) of S: a warp per row, lanes over A's M_alpha entries
        for (int64_t j0 = int64_t(warp) * 32; j0 < nr; j0 += int64_t(nwarps) * 32) {
            const int64_t j = j0 + lane;
            const int64_t Aj = j < nr ? a.ralpha[j] : 0;
            unsigned msk = __ballot_sync(0xffffffffu, j < nr && member(a.bits, Aj * Nb + B));
            while (msk) {
                const int l = __ffs(msk) - 1;
                msk &= msk - 1;
                const int64_t A = __shfl_sync(0xffffffffu, Aj, l);
                T part = T(0);
                for (int k = h.Ma_ptr[A] + lane; k < h.Ma_ptr[A + 1]; k += 32)
                    part = fma(h.Ma_val[k], col[h.Ma_col[k]], part);
                part = warp_sum(part);
                if (lane == 0) h.sigma[A * Nb + B] += part;
            }
        }
    }
}

__device__ __forceinline__ uint32_t rank_bits(uint32_t m, const uint32_t (*C)[33])
{
    uint32_t r = 0;
    int i = 0;
    for (; m; m &= m - 1, ++i) r += C[__ffs(m) - 1][i + 1];
    return r;
}

// index of the determinant with spin strings u = alpha | beta << n, from the
// table of colex ranks of all n-bit strings (the same rank as rank_bits)
__device__ __forceinline__ int64_t det_index(const uint16_t *__restrict__ r16, uint64_t u, int n,
                                             uint64_t lowm, int64_t Nb)
{
    return int64_t(__ldg(r16 + (u & lowm))) * Nb + __ldg(r16 + (u >> n));
}

// Apply an operator string (application order; codes 2*mode + dagger) to a
// determinant mask; false if it annihilates it.  Sign: (-1)^(occupied modes
// below) per fermionic operator (Jordan-Wigner, blocked order); qubit
// operators carry none.
__device__ __forceinline__ bool apply_string(const int *code, int len, uint64_t &mask, int &sg,
                                             int qubit)
{
    for (int t = 0; t < len; ++t) {
        const int mode = code[t] >> 1, dag = code[t] & 1;
        const uint64_t bit = 1ull << mode;
        if (((mask & bit) != 0) == (dag != 0)) return false;
        if (!qubit && (__popcll(mask & (bit - 1)) & 1)) sg = -sg;
        mask ^= bit;
    }
    return true;
}

// Operator strings of a constituent descriptor (rank, c0, c1, a1, a0) in
// application order: fw applies C = a+_{c0} [a+_{c1} a_{a1}] a_{a0}, bw its
// adjoint.
__device__ __forceinline__ void op_strings(const int32_t *q, int *fw, int *bw, int &len)
{
    if (q[0] == 1) {
        fw[0] = 2 * q[4]; fw[1] = 2 * q[1] + 1;
        bw[0] = 2 * q[1]; bw[1] = 2 * q[4] + 1;
        len = 2;
    } else {
        fw[0] = 2 * q[4]; fw[1] = 2 * q[3]; fw[2] = 2 * q[2] + 1; fw[3] = 2 * q[1] + 1;
        bw[0] = 2 * q[1]; bw[1] = 2 * q[2]; bw[2] = 2 * q[3] + 1; bw[3] = 2 * q[4] + 1;
        len = 4;
    }
}

// sum over a block of 256 threads, fixed order; valid in thread 0
__device__ __forceinline__ double block_sum_d(double v)
{
    __shared__ double wp[8];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) wp[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += wp[w];
    return s;
}

// Block (i, chunk): operator ops[i] over the support entries chunk,
// chunk + chunks, ... (stride chunks * blockDim).  A pair is counted once:
// from its domain end if that is listed, else from its image end.
template <typename T>
__global__ void __launch_bounds__(256)
k_grad_sparse(SparseGradArgs<T> a)
{
    const int n = a.n;
    const uint64_t lowm = (1ull << n) - 1;
    const int64_t m = list_len(a.d_m, a.m, a.cap);
    const int64_t i = blockIdx.x;
    const int k = a.ops ? a.ops[i] : int(i);
    if (refuse_op(i, k, a.K, blockIdx.y == 0 ? a.bad : nullptr)) {
        if (threadIdx.x == 0)
            a.partials[i * gridDim.y + blockIdx.y] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const int32_t *dsc = a.desc + 11 * k;
    double tot = 0.0;
    for (int c = 0; c < dsc[0]; ++c) {
        int fw[4], bw[4], len;
        op_strings(dsc + 1 + 5 * c, fw, bw, len);
        for (int64_t t = int64_t(blockIdx.y) * blockDim.x + threadIdx.x; t < m;
             t += int64_t(gridDim.y) * blockDim.x) {
            const int64_t d = a.list[t];
            const double x = double(a.psi[d]);
            const uint64_t mask = uint64_t(a.astr[d / a.Nb]) | (uint64_t(a.bstr[d % a.Nb]) << n);
            uint64_t o = mask;
            int sg = 1;
            if (apply_string(fw, len, o, sg, a.qubit)) {       // d is the domain end
                const int64_t d2 = det_index(a.rank16, o, n, lowm, a.Nb);
                tot += sg * (double(a.sigma[d2]) * x - double(a.sigma[d]) * double(a.psi[d2]));
                continue;
            }
            o = mask;
            sg = 1;
            if (apply_string(bw, len, o, sg, a.qubit)) {       // d is the image end
                const int64_t d0 = det_index(a.rank16, o, n, lowm, a.Nb);
                const bool listed = a.bits ? member(a.bits, d0) : a.psi[d0] != T(0);
                if (!listed) tot -= sg * double(a.sigma[d0]) * x;
            }
        }
    }
    tot = block_sum_d(tot);
    if (threadIdx.x == 0) a.partials[i * gridDim.y + blockIdx.y] = tot;
}

__global__ void __launch_bounds__(256)
k_grad_sparse_final(const double *__restrict__ partials, int chunks, int64_t n_ops,
                    double *__restrict__ g)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_ops) return;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += partials[i * chunks + c];
    g[i] = 2.0 * s;
}

// ---------------------------------------------------------------------------
// Sparse vectors: amplitudes in a dense array (zero off the support), the
// support as a list plus a membership bitmap, the count on the device.  The
// state preparation prod_l exp(theta_l A_l)|HF> then costs O(support) per
// rotation and needs no host synchronisation: the count stays on the device
// and an overflowing list is detected afterwards (count > cap).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_sv_clear(SVec<T> x)
{
    // every set bit belongs to a listed entry, and all of them are cleared,
    // so whole bitmap words can be zeroed
    const int64_t m = list_len(x.count, 0, x.cap);
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = x.list[t];
        x.v[i] = T(0);
        x.bits[i >> 5] = 0u;
    }
}

template <typename T>
__global__ void k_sv_finish_reset(SVec<T> x, int hf)
{
    if (hf) {
        x.v[0] = T(1);
        x.bits[0] = 1u;
        x.list[0] = 0;
    }
    *x.count = hf ? 1ull : 0ull;
    *x.snap = *x.count;
    *x.done = 0ull;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_sv_copy(SVec<T> dst, SVec<T> src)
{
    const int64_t m = list_len(src.count, 0, src.cap < dst.cap ? src.cap : dst.cap);
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = src.list[t];
        dst.v[i] = src.v[i];
        dst.list[t] = i;
        atomicOr(dst.bits + (i >> 5), 1u << (i & 31));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *dst.count = *src.count;
        *dst.snap = *src.count;
        *dst.done = 0ull;
    }
}

// the rotation loop of k_sv_excite over this block's share of entries < m
template <typename T>
__device__ __forceinline__ void sv_rotate(SVec<T> &x, const SvOpArgs &o, int k, int ci, T c, T s,
                                          int64_t m, const uint32_t (*C)[33], bool closed = false)
{
    int fw[4], bw[4], len;
    op_strings(o.desc + 11 * k + 1 + 5 * ci, fw, bw, len);
    const int n = o.n;
    const uint64_t lowm = (1ull << n) - 1;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t d = x.list[t];
        const uint64_t mask = uint64_t(o.astr[d / o.Nb]) | (uint64_t(o.bstr[d % o.Nb]) << n);
        uint64_t u = mask;
        int sg = 1;
        int64_t dom, img, fresh;
        if (apply_string(fw, len, u, sg, o.qubit)) {
            dom = d;
            img = det_index(o.rank16, u, n, lowm, o.Nb);
            fresh = member(x.bits, img) ? -1 : img;
        } else {
            u = mask;
            sg = 1;
            if (!apply_string(bw, len, u, sg, o.qubit)) continue;    // C and C^dagger annihilate d
            img = d;
            dom = det_index(o.rank16, u, n, lowm, o.Nb);
            if (member(x.bits, dom)) continue;              // the domain end rotates the pair
            fresh = dom;
        }
        const T ss = sg > 0 ? s : -s;
        if (closed && fresh >= 0) {
            // the other end lies off the support: its amplitude is zero and
            // is not kept, only the listed end is scaled
            x.v[d] = c * x.v[d];
            continue;
        }
        const T xv = x.v[dom], yv = x.v[img];
        x.v[dom] = c * xv - ss * yv;
        x.v[img] = c * yv + ss * xv;
        if (fresh >= 0) {
            atomicOr(x.bits + (fresh >> 5), 1u << (fresh & 31));
            const unsigned long long pos = atomicAdd(x.count, 1ull);
            if (pos < (unsigned long long)x.cap) x.list[pos] = fresh;
        }
    }
}

// One constituent C of operator k: every pair (d, C d) with a listed end is
// rotated by its processor -- the domain end if listed, else the image end --
// and the other end is listed if it was not.  Pairs of one constituent are
// disjoint, so the rotation is race-free; entries appended here (positions >=
// the snapshot) are not visited again.  The last block to finish copies the
// final count into the snapshot for the next rotation.
// closed: the list is kept as it is (a pair whose other end is unlisted only
// scales its listed end), for vectors needed on a fixed support only.
template <typename T>
__global__ void __launch_bounds__(256)
k_sv_excite(SVec<T> x, SvOpArgs o, int k, int ci, T c, T s, int closed)
{
    const int64_t m = list_len(x.snap, 0, x.cap);
    const bool idle = int64_t(blockIdx.x) * blockDim.x >= m;     // block-uniform
    __shared__ uint32_t C[33][33];
    if (!idle) {
        for (int i = threadIdx.x; i < 33 * 33; i += blockDim.x) C[i / 33][i % 33] = o.binom33[i];
        __syncthreads();
        sv_rotate(x, o, k, ci, c, s, m, C, closed != 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(x.done, 1ull) == gridDim.x - 1) {
            __threadfence();
            *x.snap = atomicAdd(x.count, 0ull);
            *x.done = 0ull;
        }
    }
}


// ---------------------------------------------------------------------------
// Single-CTA routines for small supports: block barriers take the place of
// launch boundaries and of the count snapshot.
// ---------------------------------------------------------------------------
constexpr int kPrepThreads = 1024;

// zero x on its support (bits included) and empty the list
template <typename T>
__device__ void blk_clear(SVec<T> &x)
{
    const int64_t m = list_len(x.count, 0, x.cap);
    for (int64_t t = threadIdx.x; t < m; t += blockDim.x) {
        const int64_t i = x.list[t];
        x.v[i] = T(0);
        x.bits[i >> 5] = 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0) *x.count = 0ull;
    __syncthreads();
}

// list index i of x (unlisted before) -- the caller owns i's bit
template <typename T>
__device__ __forceinline__ void blk_list(SVec<T> &x, int64_t i)
{
    atomicOr(x.bits + (i >> 5), 1u << (i & 31));
    const unsigned long long pos = atomicAdd(x.count, 1ull);
    if (pos < (unsigned long long)x.cap) x.list[pos] = i;
}

// current length of x's list, the same in every thread
template <typename T>
__device__ int64_t blk_len(const SVec<T> &x, unsigned long long *m_sh)
{
    __syncthreads();
    if (threadIdx.x == 0) *m_sh = *x.count;
    __syncthreads();
    return *m_sh < (unsigned long long)x.cap ? int64_t(*m_sh) : x.cap;
}

// exp(theta (C - C^dagger)) for constituent ci of operator k, as k_sv_excite
template <typename T>
__device__ void blk_rotate(SVec<T> &x, const SvOpArgs &o, int k, int ci, T c, T sn,
                           const uint32_t (*C)[33], unsigned long long *m_sh)
{
    const int64_t m = blk_len(x, m_sh);
    int fw[4], bw[4], len;
    op_strings(o.desc + 11 * k + 1 + 5 * ci, fw, bw, len);
    const int n = o.n;
    const uint64_t lowm = (1ull << n) - 1;
    for (int64_t t = threadIdx.x; t < m; t += blockDim.x) {
        const int64_t d = x.list[t];
        const uint64_t mask = uint64_t(o.astr[d / o.Nb]) | (uint64_t(o.bstr[d % o.Nb]) << n);
        uint64_t u = mask;
        int sg = 1;
        int64_t dom, img, fresh;
        if (apply_string(fw, len, u, sg, o.qubit)) {
            dom = d;
            img = det_index(o.rank16, u, n, lowm, o.Nb);
            fresh = member(x.bits, img) ? -1 : img;
        } else {
            u = mask;
            sg = 1;
            if (!apply_string(bw, len, u, sg, o.qubit)) continue;
            img = d;
            dom = det_index(o.rank16, u, n, lowm, o.Nb);
            if (member(x.bits, dom)) continue;
            fresh = dom;
        }
        const T ss = sg > 0 ? sn : -sn;
        const T xv = x.v[dom], yv = x.v[img];
        x.v[dom] = c * xv - ss * yv;
        x.v[img] = c * yv + ss * xv;
        if (fresh >= 0) blk_list(x, fresh);
    }
}

// w <- w + (C - C^dagger) f for constituent ci of operator k over f's
// entries < m.  The constituent pairs determinants one to one, so a target
// has a single source (its partner) and is written by one thread.
template <typename T>
__device__ void blk_generator(const SVec<T> &f, SVec<T> &w, const SvOpArgs &o, int k, int ci,
                              int64_t m, const uint32_t (*C)[33])
{
    int fw[4], bw[4], len;
    op_strings(o.desc + 11 * k + 1 + 5 * ci, fw, bw, len);
    const int n = o.n;
    const uint64_t lowm = (1ull << n) - 1;
    for (int64_t t = threadIdx.x; t < m; t += blockDim.x) {
        const int64_t d = f.list[t];
        const uint64_t mask = uint64_t(o.astr[d / o.Nb]) | (uint64_t(o.bstr[d % o.Nb]) << n);
        uint64_t u = mask;
        int sg = 1;
        int64_t tgt;
        T val;
        if (apply_string(fw, len, u, sg, o.qubit)) {          // C|d> = sg |tgt>
            tgt = det_index(o.rank16, u, n, lowm, o.Nb);
            val = sg > 0 ? f.v[d] : -f.v[d];
        } else {
            u = mask;
            sg = 1;
            if (!apply_string(bw, len, u, sg, o.qubit)) continue;
            // -C^dagger |d> = -sg |tgt>
            tgt = det_index(o.rank16, u, n, lowm, o.Nb);
            val = sg > 0 ? -f.v[d] : f.v[d];
        }
        if (!member(w.bits, tgt)) blk_list(w, tgt);  // tgt is reached from d alone
        w.v[tgt] += val;
    }
}

// sum over x's support of x * y (y dense), FP64, block-reduced; thread 0
template <typename T>
__device__ double blk_dot(const SVec<T> &x, const T *y, int64_t m, double *red)
{
    double acc = 0.0;
    for (int64_t t = threadIdx.x; t < m; t += blockDim.x) {
        const int64_t i = x.list[t];
        acc = fma(double(x.v[i]), double(y[i]), acc);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// The whole state preparation of a small support in one CTA: clear the
// previous support, set |HF>, apply every constituent rotation of the
// ansatz in order, and for float states divide by the FP64 norm over the
// support.  cs[2l], cs[2l+1] = cos, sin theta_l.  step_len (optional): the
// list's length after each constituent rotation (the list only grows, so
// these date every listed determinant to the rotation that listed it).
template <typename T>
__global__ void __launch_bounds__(kPrepThreads)
k_sv_prepare(SVec<T> x, SvOpArgs o, const int32_t *__restrict__ ops,
             const double *__restrict__ cs, int L, int renorm, double *__restrict__ norm2,
             int64_t *__restrict__ step_len)
{
    __shared__ uint32_t C[33][33];
    __shared__ unsigned long long m_sh;
    __shared__ double red[kPrepThreads / 32];
    __shared__ double fac;
    const int tid = threadIdx.x;
    for (int i = tid; i < 33 * 33; i += blockDim.x) C[i / 33][i % 33] = o.binom33[i];
    blk_clear(x);
    if (tid == 0) {
        x.v[0] = T(1);
        blk_list(x, 0);
    }
    int step = 0;
    for (int l = 0; l < L; ++l) {
        const int k = ops[l];
        const int nc = o.desc[11 * k];
        for (int ci = 0; ci < nc; ++ci, ++step) {
            blk_rotate(x, o, k, ci, T(cs[2 * l]), T(cs[2 * l + 1]), C, &m_sh);
            if (step_len) {
                const int64_t ml = blk_len(x, &m_sh);
                if (tid == 0) step_len[step] = ml;
            }
        }
    }
    const int64_t m = blk_len(x, &m_sh);
    if (tid == 0) {                 // leave the snapshot consistent for later rotations
        *x.snap = *x.count;
        *x.done = 0ull;
    }
    if (!renorm) return;
    const double sum = blk_dot(x, x.v, m, red);
    if (tid == 0) {
        if (norm2) *norm2 = sum;
        fac = 1.0 / sqrt(sum);
    }
    __syncthreads();
    const T f = T(fac);
    for (int64_t t = tid; t < m; t += blockDim.x) x.v[x.list[t]] *= f;
}

// Gradient of E = <psi|H|psi>, psi = U_L .. U_1 |HF> (U_l = exp(theta_l A_l)),
// in forward mode for small supports, in one CTA:
//   dE/dtheta_l = 2 <sigma| U_L .. U_{l+1} A_l phi_l>,  phi_l = U_l .. U_1 |HF>,
// with sigma = H psi (dense array).  phi (f) is advanced one operator at a
// time; w = A_l phi_l is formed in a second sparse vector and carried
// through the later rotations.  Every vector stays within psi's support, so
// each of the O(L^2) rotations costs O(support).  norm2 (float states): psi
// was divided by sqrt(*norm2) while phi here is not, so each g_l is too.
template <typename T>
__global__ void __launch_bounds__(kPrepThreads)
k_sv_grad_fwd(SVec<T> f, SVec<T> w, SvOpArgs o, const int32_t *__restrict__ ops,
              const double *__restrict__ cs, int L, const T *__restrict__ sigma,
              const double *__restrict__ norm2, double *__restrict__ g)
{
    __shared__ uint32_t C[33][33];
    __shared__ unsigned long long m_sh;
    __shared__ double red[kPrepThreads / 32];
    const int tid = threadIdx.x;
    for (int i = tid; i < 33 * 33; i += blockDim.x) C[i / 33][i % 33] = o.binom33[i];
    blk_clear(f);
    if (tid == 0) {
        f.v[0] = T(1);
        blk_list(f, 0);
    }
    const double scale = norm2 ? 2.0 / sqrt(*norm2) : 2.0;
    for (int l = 0; l < L; ++l) {
        const int k = ops[l];
        const int nc = o.desc[11 * k];
        for (int ci = 0; ci < nc; ++ci)
            blk_rotate(f, o, k, ci, T(cs[2 * l]), T(cs[2 * l + 1]), C, &m_sh);
        blk_clear(w);
        const int64_t mf = blk_len(f, &m_sh);
        for (int ci = 0; ci < nc; ++ci) {
            blk_generator(f, w, o, k, ci, mf, C);
            __syncthreads();                         // constituents add in order
        }
        for (int l2 = l + 1; l2 < L; ++l2) {
            const int k2 = ops[l2];
            const int nc2 = o.desc[11 * k2];
            for (int ci = 0; ci < nc2; ++ci)
                blk_rotate(w, o, k2, ci, T(cs[2 * l2]), T(cs[2 * l2 + 1]), C, &m_sh);
        }
        const int64_t mw = blk_len(w, &m_sh);
        const double gl = blk_dot(w, sigma, mw, red);
        if (tid == 0) g[l] = scale * gl;
    }
    __syncthreads();
    if (tid == 0) {
        *f.snap = *f.count;
        *f.done = 0ull;
        *w.snap = *w.count;
        *w.done = 0ull;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_sv_dot_partial(SVec<T> x, const T *__restrict__ y, double *__restrict__ partials)
{
    const int64_t m = list_len(x.count, 0, x.cap);
    double acc = 0.0;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = x.list[t];
        acc = fma(double(x.v[i]), double(y[i]), acc);
    }
    acc = block_sum_d(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256)
k_sv_sum(const double *__restrict__ partials, int G, double *__restrict__ out)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < G; i += blockDim.x) s += partials[i];
    s = block_sum_d(s);
    if (threadIdx.x == 0) *out = s;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_sv_scale(SVec<T> x, const double *__restrict__ norm2)
{
    const T f = T(1.0 / sqrt(*norm2));
    const int64_t m = list_len(x.count, 0, x.cap);
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m;
         t += int64_t(gridDim.x) * blockDim.x)
        x.v[x.list[t]] *= f;
}

// ---------------------------------------------------------------------------
// Support programs: the rotations of a fixed ansatz as pairings of the
// support's elements (local indices), so that every evaluation of one ADAPT
// iteration runs on m-vectors in shared memory, with no string ranking,
// membership tests or list appends.
// ---------------------------------------------------------------------------
constexpr int kProgThreads = 512;

// key[0..m) = (determinant << 8) | birth, ascending, birth = 0 for |HF> and
// s + 1 for an element listed by rotation step s (from the list's lengths
// after each step).  One CTA, bitonic sort over the next power of two (P
// keys of dynamic shared memory).
constexpr int kProgSortMax = 16384;   // the power of two >= kProgMax
static_assert(kProgSortMax >= kProgMax, "sort buffer");

__global__ void __launch_bounds__(1024)
k_prog_sort(const int64_t *__restrict__ list, int64_t m, const int64_t *__restrict__ step_len,
            int steps, int64_t *__restrict__ key)
{
    extern __shared__ __align__(16) int64_t kk[];
    int P = 1;
    while (P < m) P <<= 1;
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
        int64_t v = INT64_MAX;
        if (t < m) {
            int lo = 0, hi = steps;                  // first step whose length exceeds t
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (int64_t(t) < step_len[mid]) hi = mid;
                else lo = mid + 1;
            }
            v = (list[t] << 8) | int64_t(t == 0 ? 0 : lo + 1);
        }
        kk[t] = v;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                const int u = t ^ j;
                if (u > t) {
                    const int64_t a = kk[t], b = kk[u];
                    if ((a > b) == ((t & k) == 0)) {
                        kk[t] = b;
                        kk[u] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int t = threadIdx.x; t < m; t += blockDim.x) key[t] = kk[t];
}

// local index of determinant d in the sorted keys, or -1
__device__ __forceinline__ int prog_find(const int64_t *__restrict__ key, int m, int64_t d)
{
    int lo = 0, hi = m;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((key[mid] >> 8) < d) lo = mid + 1;
        else hi = mid;
    }
    return lo < m && (key[lo] >> 8) == d ? lo : -1;
}

// a pair of a step packed into one word: the domain end's index within its
// part (tl < 2^14), the image end p (< 2^16) and the sign of the forward
// string; kNoPair marks an empty register slot
__device__ __forceinline__ uint32_t pair_word(int tl, int p, bool neg)
{
    return uint32_t(tl) | (uint32_t(p) << 14) | (neg ? 1u << 30 : 0u);
}
constexpr uint32_t kNoPair = 0xFFFFFFFFu;

// warp-aggregated append: every lane with `has` adds v to list `slot`
// (count counts[slot], items from out + slot * stride forwards, or with
// `back` from out + (slot + 1) * stride - 1 backwards); the lanes of one warp
// that share a slot take one atomic.  Every lane of the warp must call it.
__device__ __forceinline__ void warp_append(bool has, int slot, uint32_t v,
                                            uint32_t *__restrict__ out, int64_t stride,
                                            int *__restrict__ counts, bool back = false)
{
    const unsigned act = __ballot_sync(0xffffffffu, has);
    if (!has) return;
    const unsigned grp = __match_any_sync(act, slot);
    const int lane = int(threadIdx.x & 31);
    const int leader = __ffs(int(grp)) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counts + slot, __popc(grp));
    base = __shfl_sync(grp, base, leader);
    const int64_t i = base + __popc(grp & ((1u << lane) - 1u));
    out[back ? (int64_t(slot) + 1) * stride - 1 - i : int64_t(slot) * stride + i] = v;
}

// the op (l), constituent (ci) and last step of op l for step s; l = L when
// s is beyond the ansatz's steps
__device__ __forceinline__ void prog_step_op(const int32_t *__restrict__ desc,
                                             const int32_t *__restrict__ ops, int L, int s, int &l,
                                             int &ci, int &last)
{
    int acc = 0;
    ci = 0;
    last = -1;
    for (l = 0; l < L; ++l) {
        const int nc = desc[11 * ops[l]];
        if (s < acc + nc) {
            ci = s - acc;
            last = acc + nc - 1;
            return;
        }
        acc += nc;
    }
}

// the pairs of step s = blockIdx.y (constituent ci of op l), one list per step
__global__ void __launch_bounds__(256)
k_prog_tables(const int64_t *__restrict__ key, int m, SvOpArgs o, const int32_t *__restrict__ ops,
              int L, uint32_t *__restrict__ pairs, int *__restrict__ npairs,
              int *__restrict__ nrest, int *__restrict__ step_l, int *__restrict__ flag)
{
    __shared__ uint32_t C[33][33];
    for (int i = threadIdx.x; i < 33 * 33; i += blockDim.x) C[i / 33][i % 33] = o.binom33[i];
    __syncthreads();
    const int s = blockIdx.y;
    int l, ci, last;
    prog_step_op(o.desc, ops, L, s, l, ci, last);
    if (l >= L) return;                              // whole block
    if (blockIdx.x == 0 && threadIdx.x == 0) step_l[s] = l;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    int p = -1;
    bool neg = false, active = false;
    if (t < m) {
        int fw[4], bw[4], len;
        op_strings(o.desc + 11 * ops[l] + 1 + 5 * ci, fw, bw, len);
        const int64_t kt = key[t], d = kt >> 8;
        const int birth = int(kt & 255) - 1;         // -1: |HF>, else the listing step
        const int n = o.n;
        const uint64_t lowm = (1ull << n) - 1;
        const uint64_t mask = uint64_t(o.astr[d / o.Nb]) | (uint64_t(o.bstr[d % o.Nb]) << n);
        uint64_t u = mask;
        int sg = 1;
        bool escape = false;
        if (apply_string(fw, len, u, sg, o.qubit)) {
            const int64_t img = det_index(o.rank16, u, n, lowm, o.Nb);
            p = prog_find(key, m, img);
            neg = sg < 0;
            escape = p < 0;
            // a pair can be nonzero before step s only if an end was listed
            // before it (tag = listing step + 1, 0 for |HF>)
            active = p >= 0 && (int(kt & 255) <= s || int(key[p] & 255) <= s);
        } else {
            u = mask;
            sg = 1;
            if (apply_string(bw, len, u, sg, o.qubit)) {
                const int64_t dom = det_index(o.rank16, u, n, lowm, o.Nb);
                escape = prog_find(key, m, dom) < 0;
            }
        }
        // a partner outside the support is harmless to the rotations (both
        // ends are zero when step s runs) but not to op l's generator when t
        // is in phi_l's support without having been seen by step s: listed
        // later by op l's own constituents
        if (escape && birth > s && birth <= last) *flag = 1;
    }
    warp_append(p >= 0 && active, s, pair_word(t, p, neg), pairs, m, npairs);
    warp_append(p >= 0 && !active, s, pair_word(t, p, neg), pairs, m, nrest, true);
}

// pairs a thread takes per round of a step read from global memory (loaded
// together, so that their latencies overlap)
constexpr int kPairU = 4;

__device__ __forceinline__ void pairs_load(uint32_t (&q)[kPairU], const uint32_t *__restrict__ pr,
                                           int n, int i0)
{
#pragma unroll
    for (int k = 0; k < kPairU; ++k) {
        const int i = i0 + k * int(blockDim.x);
        q[k] = i < n ? pr[i] : kNoPair;
    }
}

// a vector in one CTA's shared memory
template <typename T>
struct LocalVec {
    T *x;
    __device__ __forceinline__ T *own(int tl) const { return x + tl; }
    __device__ __forceinline__ T *img(int p) const { return x + p; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// a vector split over the shared memories of a cluster's CTAs, chunk
// elements each: element t lives in CTA t / chunk and is reached through
// distributed shared memory when it is another CTA's.  A CTA's pair lists
// hold the pairs whose domain end is its own (own: by its local index)
template <typename T>
struct ClusterVec {
    T *loc;
    int chunk, rank;
    __device__ __forceinline__ T *own(int tl) const { return loc + tl; }
    __device__ __forceinline__ T *img(int p) const
    {
        const int r = p / chunk;
        return r == rank ? loc + (p - r * chunk)
                         : cg::this_cluster().map_shared_rank(loc, r) + (p - r * chunk);
    }
    __device__ __forceinline__ void sync() const { cg::this_cluster().sync(); }
};

// one pair of a constituent rotation (the pairs of a step are disjoint: each
// has one writer)
template <typename T, class V>
__device__ __forceinline__ void pair_rotate(const V &x, uint32_t w, T c, T sn)
{
    const T ss = (w >> 30) & 1u ? -sn : sn;
    T *xt = x.own(int(w & 0x3FFFu)), *xp = x.img(int((w >> 14) & 0xFFFFu));
    const T xv = *xt, yv = *xp;
    *xt = c * xv - ss * yv;
    *xp = c * yv + ss * xv;
}

// one pair of w <- w + (C - C^dagger) f for one constituent: C|t> = sg|p>
// adds sg f_t to w_p and -sg f_p to w_t
template <class V>
__device__ __forceinline__ void pair_generator(const V &f, const V &w, uint32_t wd)
{
    const int tl = int(wd & 0x3FFFu), p = int((wd >> 14) & 0xFFFFu);
    const auto ft = *f.own(tl), fp = *f.img(p);
    auto *wp = w.img(p), *wt = w.own(tl);
    if ((wd >> 30) & 1u) {
        *wp -= ft;
        *wt += fp;
    } else {
        *wp += ft;
        *wt -= fp;
    }
}

// per-step values of a program in shared memory: this part's pair counts
// (np: pairs with an end listed before the step, at the front of the step's
// list; nr: the others, at its back), the operator of each step and its
// cos / sin, and where the step's pairs were staged in shared memory (np
// words, then nr; -1: read from global memory)
template <typename T>
struct ProgSteps {
    int np[kProgSteps], nr[kProgSteps];
    int sl[kProgSteps];
    int off[kProgSteps];
    T c[kProgSteps], sn[kProgSteps];
};

// fills st.np, sl, c, sn (the caller synchronises); every thread calls it
template <typename T>
__device__ __forceinline__ void prog_load_steps(const ProgTabs &g, int rank,
                                                const double *__restrict__ cs, ProgSteps<T> &st)
{
    for (int s = threadIdx.x; s < g.steps; s += blockDim.x) {
        const int l = g.step_l[s];
        st.sl[s] = l;
        st.np[s] = g.npairs[s * g.ranks + rank];
        st.nr[s] = g.nrest[s * g.ranks + rank];
        st.c[s] = T(cs[2 * l]);
        st.sn[s] = T(cs[2 * l + 1]);
    }
}

__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                 ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))), "l"(src)
                 : "memory");
}

// copies the pair lists of this part into sp (cap words of shared memory),
// steps in order while they fit, and sets st.off (after st.np is loaded and
// synchronised); ends synchronised
template <typename T>
__device__ __forceinline__ void prog_stage(const ProgTabs &g, int rank, ProgSteps<T> &st,
                                           uint32_t *sp, int cap)
{
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int s = 0; s < g.steps; ++s) {
            const int n = st.np[s] + st.nr[s];
            if (n <= cap - acc) {
                st.off[s] = acc;
                acc += n;
            } else {
                st.off[s] = -1;
            }
        }
    }
    __syncthreads();
    for (int s = 0; s < g.steps; ++s) {
        const int o = st.off[s];
        if (o < 0) continue;
        const uint32_t *src = g.pairs + (int64_t(s) * g.ranks + rank) * g.chunk;
        const int np = st.np[s], nr = st.nr[s];
        for (int i = threadIdx.x; i < np; i += blockDim.x) cp_async4(sp + o + i, src + i);
        const uint32_t *rest = src + g.chunk - nr;
        for (int i = threadIdx.x; i < nr; i += blockDim.x) cp_async4(sp + o + np + i, rest + i);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
}

// n pairs from global memory at pr, a round of kPairU per thread at a time
template <typename T, class V>
__device__ __forceinline__ void pairs_rotate_global(const V &x, const uint32_t *__restrict__ pr,
                                                    int n, T c, T sn)
{
    const int R = kPairU * int(blockDim.x);
    for (int i0 = threadIdx.x; i0 < n; i0 += R) {
        uint32_t q[kPairU];
        pairs_load(q, pr, n, i0);
#pragma unroll
        for (int k = 0; k < kPairU; ++k)
            if (q[k] != kNoPair) pair_rotate<T>(x, q[k], c, sn);
    }
}

// steps [s0, s1) on x, one barrier (CTA or cluster) after each: the pairs
// with an end listed before the step only (x is U_s .. U_1|HF>, zero on
// determinants listed later), or with `all` every pair
template <typename T, class V>
__device__ __forceinline__ void prog_run(const V &x, const ProgTabs &g, int rank,
                                         const ProgSteps<T> &st, const uint32_t *sp, int s0,
                                         int s1, bool all)
{
    for (int s = s0; s < s1; ++s) {
        const int np = st.np[s], nr = all ? st.nr[s] : 0, o = st.off[s];
        const T c = st.c[s], sn = st.sn[s];
        if (o >= 0) {
            const uint32_t *pr = sp + o;
            const int n = np + nr;
#pragma unroll 4
            for (int i = threadIdx.x; i < n; i += blockDim.x) pair_rotate<T>(x, pr[i], c, sn);
        } else {
            const uint32_t *pr = g.pairs + (int64_t(s) * g.ranks + rank) * g.chunk;
            pairs_rotate_global<T>(x, pr, np, c, sn);
            if (nr) pairs_rotate_global<T>(x, pr + g.chunk - nr, nr, c, sn);
        }
        x.sync();
    }
}

// the generator of op lg (its constituent steps [b, e), in order, every
// pair) from f into w, one barrier after each constituent
template <typename T, class V>
__device__ __forceinline__ void prog_generate(const V &f, const V &w, const ProgTabs &g, int rank,
                                              const ProgSteps<T> &st, const uint32_t *sp, int b,
                                              int e)
{
    for (int s = b; s < e; ++s) {
        const int np = st.np[s], nr = st.nr[s], o = st.off[s];
        if (o >= 0) {
            for (int i = threadIdx.x; i < np + nr; i += blockDim.x) pair_generator(f, w, sp[o + i]);
        } else {
            const uint32_t *pr = g.pairs + (int64_t(s) * g.ranks + rank) * g.chunk;
            for (int i = threadIdx.x; i < np; i += blockDim.x) pair_generator(f, w, pr[i]);
            const uint32_t *rest = pr + g.chunk - nr;
            for (int i = threadIdx.x; i < nr; i += blockDim.x) pair_generator(f, w, rest[i]);
        }
        f.sync();
    }
}

// the steps of op lg: [*b, *e) (steps are in ansatz order)
__device__ __forceinline__ void prog_op_steps(const int *sl, int steps, int lg, int &b, int &e)
{
    b = 0;
    e = 0;
    for (int s = 0; s < steps; ++s) {
        if (sl[s] < lg) b = s + 1;
        if (sl[s] <= lg) e = s + 1;
    }
}

// FP64 block sum, valid in thread 0
__device__ __forceinline__ double prog_block_sum(double acc, double *red)
{
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// The program kernels take all of a block's opt-in shared memory: the
// vectors first, then (cap words) the staged pair lists
template <typename T>
__global__ void __launch_bounds__(kProgThreads)
k_prog_prepare(ProgTabs g, const double *__restrict__ cs, int renorm, double *__restrict__ norm2,
               T *__restrict__ v, int cap)
{
    extern __shared__ __align__(16) unsigned char prog_sm[];
    const int m = g.m;
    const LocalVec<T> x{reinterpret_cast<T *>(prog_sm)};
    uint32_t *sp = reinterpret_cast<uint32_t *>(x.x + m);
    __shared__ ProgSteps<T> st;
    __shared__ double red[kProgThreads / 32];
    __shared__ double fac;
    for (int t = threadIdx.x; t < m; t += blockDim.x) x.x[t] = t == 0 ? T(1) : T(0);   // |HF>
    prog_load_steps(g, 0, cs, st);
    __syncthreads();
    prog_stage(g, 0, st, sp, cap);
    prog_run<T>(x, g, 0, st, sp, 0, g.steps, false);
    if (renorm) {
        double acc = 0.0;
        for (int t = threadIdx.x; t < m; t += blockDim.x)
            acc = fma(double(x.x[t]), double(x.x[t]), acc);
        const double sum = prog_block_sum(acc, red);
        if (threadIdx.x == 0) {
            if (norm2) *norm2 = sum;
            fac = 1.0 / sqrt(sum);
        }
        __syncthreads();
        const T f = T(fac);
        for (int t = threadIdx.x; t < m; t += blockDim.x) v[g.key[t] >> 8] = x.x[t] * f;
    } else {
        for (int t = threadIdx.x; t < m; t += blockDim.x) v[g.key[t] >> 8] = x.x[t];
    }
}

// CTA l: g[l] = scale <sigma| U_L .. U_{l+1} A_l U_l .. U_1 |HF>
template <typename T>
__global__ void __launch_bounds__(kProgThreads)
k_prog_grad(ProgTabs g, const double *__restrict__ cs, const T *__restrict__ sigma,
            const double *__restrict__ norm2, double *__restrict__ gout, int cap)
{
    extern __shared__ __align__(16) unsigned char prog_sm[];
    const int m = g.m;
    const LocalVec<T> f{reinterpret_cast<T *>(prog_sm)}, w{reinterpret_cast<T *>(prog_sm) + m};
    uint32_t *sp = reinterpret_cast<uint32_t *>(w.x + m);
    __shared__ ProgSteps<T> st;
    __shared__ double red[kProgThreads / 32];
    const int lg = blockIdx.x;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        f.x[t] = t == 0 ? T(1) : T(0);
        w.x[t] = T(0);
    }
    prog_load_steps(g, 0, cs, st);
    __syncthreads();
    prog_stage(g, 0, st, sp, cap);
    int b, e;
    prog_op_steps(st.sl, g.steps, lg, b, e);
    prog_run<T>(f, g, 0, st, sp, 0, e, false);       // phi_lg = U_lg .. U_1 |HF>
    prog_generate<T>(f, w, g, 0, st, sp, b, e);      // constituents add in order
    prog_run<T>(w, g, 0, st, sp, e, g.steps, true);  // w may hold later-listed elements
    double acc = 0.0;
    for (int t = threadIdx.x; t < m; t += blockDim.x)
        acc = fma(double(w.x[t]), double(sigma[g.key[t] >> 8]), acc);
    const double dot = prog_block_sum(acc, red);
    if (threadIdx.x == 0) gout[lg] = (norm2 ? 2.0 / sqrt(*norm2) : 2.0) * dot;
}

// ---------------------------------------------------------------------------
// Support programs beyond shared memory (kProgMax < m <= kProgBig).  The
// support keeps the order in which the structural preparation listed it
// (key[t] = (determinant << 8) | birth, as above, unsorted), an index map
// over Omega_CIk gives each listed determinant its local index (read only
// where the listing's membership bitmap has the determinant), and the
// vectors are split over the shared memories of a thread-block cluster
// (ClusterVec).  Same pairs, same arithmetic, same order of operations per
// element.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_prog_keys_big(const int64_t *__restrict__ list, int64_t m, const int64_t *__restrict__ step_len,
                int steps, int64_t *__restrict__ key, int32_t *__restrict__ idx_map)
{
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m;
         t += int64_t(gridDim.x) * blockDim.x) {
        int lo = 0, hi = steps;                      // first step whose length exceeds t
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (t < step_len[mid]) hi = mid;
            else lo = mid + 1;
        }
        const int64_t d = list[t];
        key[t] = (d << 8) | int64_t(t == 0 ? 0 : lo + 1);
        idx_map[d] = int32_t(t);
    }
}

// as k_prog_tables, with the partner found through the bitmap and index map
// and one list per step and cluster rank (the part holding the domain end)
__global__ void __launch_bounds__(256)
k_prog_tables_big(const int64_t *__restrict__ key, int m, SvOpArgs o,
                  const int32_t *__restrict__ ops, int L, const uint32_t *__restrict__ bits,
                  const int32_t *__restrict__ idx_map, uint32_t *__restrict__ pairs,
                  int *__restrict__ npairs, int *__restrict__ nrest, int *__restrict__ step_l,
                  int *__restrict__ flag)
{
    __shared__ uint32_t C[33][33];
    for (int i = threadIdx.x; i < 33 * 33; i += blockDim.x) C[i / 33][i % 33] = o.binom33[i];
    __syncthreads();
    const int s = blockIdx.y;
    int l, ci, last;
    prog_step_op(o.desc, ops, L, s, l, ci, last);
    if (l >= L) return;                              // whole block
    if (blockIdx.x == 0 && threadIdx.x == 0) step_l[s] = l;
    int fw[4], bw[4], len;
    op_strings(o.desc + 11 * ops[l] + 1 + 5 * ci, fw, bw, len);
    const int n = o.n;
    const uint64_t lowm = (1ull << n) - 1;
    const int chunk = (m + kClusterCtas - 1) / kClusterCtas;
    // block-uniform trip count: every lane reaches the warp-wide append
    for (int t0 = blockIdx.x * blockDim.x; t0 < m; t0 += gridDim.x * blockDim.x) {
        const int t = t0 + int(threadIdx.x);
        int p = -1;
        bool neg = false, active = false;
        if (t < m) {
            const int64_t kt = key[t], d = kt >> 8;
            const int birth = int(kt & 255) - 1;
            const uint64_t mask = uint64_t(o.astr[d / o.Nb]) | (uint64_t(o.bstr[d % o.Nb]) << n);
            uint64_t u = mask;
            int sg = 1;
            bool escape = false;
            if (apply_string(fw, len, u, sg, o.qubit)) {
                const int64_t img = det_index(o.rank16, u, n, lowm, o.Nb);
                if (member(bits, img)) {
                    p = idx_map[img];
                    neg = sg < 0;
                    active = int(kt & 255) <= s || int(key[p] & 255) <= s;
                } else {
                    escape = true;
                }
            } else {
                u = mask;
                sg = 1;
                if (apply_string(bw, len, u, sg, o.qubit)) {
                    const int64_t dom = det_index(o.rank16, u, n, lowm, o.Nb);
                    escape = !member(bits, dom);
                }
            }
            if (escape && birth > s && birth <= last) *flag = 1;
        }
        const int r = (t < m ? t : 0) / chunk;
        const uint32_t wd = pair_word(t - r * chunk, p, neg);
        warp_append(p >= 0 && active, s * kClusterCtas + r, wd, pairs, chunk, npairs);
        warp_append(p >= 0 && !active, s * kClusterCtas + r, wd, pairs, chunk, nrest, true);
    }
}

// FP64 sum over the cluster (each CTA's block sum, then the CTAs' sums in
// rank order); valid in thread 0 of every CTA.  red: 40 doubles of shared
// memory (32 per-warp slots, 8 per-CTA slots used on rank 0)
__device__ __forceinline__ double cl_sum(cg::cluster_group &cl, double acc, double *red, int rank)
{
    const double s = prog_block_sum(acc, red);
    if (threadIdx.x == 0) cl.map_shared_rank(red + 32, 0)[rank] = s;
    cl.sync();
    double tot = 0.0;
    if (threadIdx.x == 0) {
        const double *slot = cl.map_shared_rank(red + 32, 0);
        for (int r = 0; r < kClusterCtas; ++r) tot += slot[r];
    }
    return tot;
}

// one cluster: as k_prog_prepare, the vector over the cluster's CTAs
template <typename T>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(1024, 1)
k_prog_prepare_big(ProgTabs g, const double *__restrict__ cs, int renorm,
                   double *__restrict__ norm2, T *__restrict__ v, int cap)
{
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char clsm[];
    __shared__ ProgSteps<T> st;
    __shared__ double red[40];
    __shared__ double fac;
    const int rank = int(cl.block_rank());
    const int m = g.m, chunk = g.chunk;
    const int t0 = rank * chunk, t1 = min(m, t0 + chunk);
    const ClusterVec<T> x{reinterpret_cast<T *>(clsm), chunk, rank};
    uint32_t *sp = reinterpret_cast<uint32_t *>(x.loc + chunk);
    for (int t = t0 + int(threadIdx.x); t < t1; t += blockDim.x) x.loc[t - t0] = t == 0 ? T(1) : T(0);
    prog_load_steps(g, rank, cs, st);
    __syncthreads();
    prog_stage(g, rank, st, sp, cap);
    cl.sync();                                       // every CTA of the cluster is running
    prog_run<T>(x, g, rank, st, sp, 0, g.steps, false);
    T f = T(1);
    if (renorm) {
        double acc = 0.0;
        for (int t = t0 + int(threadIdx.x); t < t1; t += blockDim.x) {
            const double xv = double(x.loc[t - t0]);
            acc = fma(xv, xv, acc);
        }
        const double tot = cl_sum(cl, acc, red, rank);
        if (threadIdx.x == 0) {
            if (rank == 0 && norm2) *norm2 = tot;
            fac = 1.0 / sqrt(tot);
        }
        __syncthreads();
        f = T(fac);
    }
    for (int t = t0 + int(threadIdx.x); t < t1; t += blockDim.x)
        v[g.key[t] >> 8] = renorm ? x.loc[t - t0] * f : x.loc[t - t0];
    cl.sync();                                       // no CTA leaves while others may read it
}

// cluster lg (of L): as k_prog_grad, f and w over the cluster's CTAs
template <typename T>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(1024, 1)
k_prog_grad_big(ProgTabs g, const double *__restrict__ cs, const T *__restrict__ sigma,
                const double *__restrict__ norm2, double *__restrict__ gout, int cap)
{
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char clsm[];
    __shared__ ProgSteps<T> st;
    __shared__ double red[40];
    const int rank = int(cl.block_rank());
    const int lg = int(blockIdx.x) / kClusterCtas;
    const int m = g.m, chunk = g.chunk;
    const int t0 = rank * chunk, t1 = min(m, t0 + chunk);
    const ClusterVec<T> f{reinterpret_cast<T *>(clsm), chunk, rank};
    const ClusterVec<T> w{reinterpret_cast<T *>(clsm) + chunk, chunk, rank};
    uint32_t *sp = reinterpret_cast<uint32_t *>(w.loc + chunk);
    for (int t = t0 + int(threadIdx.x); t < t1; t += blockDim.x) {
        f.loc[t - t0] = t == 0 ? T(1) : T(0);
        w.loc[t - t0] = T(0);
    }
    prog_load_steps(g, rank, cs, st);
    __syncthreads();
    prog_stage(g, rank, st, sp, cap);
    cl.sync();
    int b, e;
    prog_op_steps(st.sl, g.steps, lg, b, e);
    prog_run<T>(f, g, rank, st, sp, 0, e, false);    // phi_lg = U_lg .. U_1 |HF>
    prog_generate<T>(f, w, g, rank, st, sp, b, e);   // constituents add in order
    prog_run<T>(w, g, rank, st, sp, e, g.steps, true);
    double acc = 0.0;
    for (int t = t0 + int(threadIdx.x); t < t1; t += blockDim.x)
        acc = fma(double(w.loc[t - t0]), double(sigma[g.key[t] >> 8]), acc);
    const double dot = cl_sum(cl, acc, red, rank);
    if (threadIdx.x == 0 && rank == 0) gout[lg] = (norm2 ? 2.0 / sqrt(*norm2) : 2.0) * dot;
    cl.sync();
}

// ---------------------------------------------------------------------------
// H restricted to a support (see HssArgs).  Row t enumerates the couplings of
// its determinant d = (A, B) in the order k_hpsi_scatter enumerates the
// targets of d (H is real symmetric, so the column of d is its row), keeping
// those whose determinant is in the support.  A coupling (A', B') can be in
// the support only if A' is the alpha string and B' the beta string of some
// support element, so the alpha and beta partners of the row are first
// filtered by the support's string sets (sa, sb: bitmaps over the alpha and
// beta strings, in shared memory), and only the surviving candidates are
// tested against the support's bitmap.  Each row has a fixed slot of
// `stride` entries (an upper bound of its couplings), so one launch builds the
// whole matrix with no count pass and no host round trip: per row the block
// counts each thread's entries, a block scan places them, and a second walk of
// the same fixed-order enumeration writes them.
// ---------------------------------------------------------------------------
constexpr int kHssStrWords = (12870 + 31) / 32;   // C(16, 8) strings of one spin

// the row's alpha excitations whose partner string is in the support's alpha
// set (fa, *naf) and its beta excitations likewise (fb, *nbf), in excitation
// order; warp 0 filters alpha, warp 1 beta
__device__ __forceinline__ void hss_filter(const HssArgs &a, int64_t A, int64_t B,
                                           const uint32_t *sa, const uint32_t *sb, uint32_t *fa,
                                           uint32_t *fb, int *naf, int *nbf)
{
    const int w = int(threadIdx.x >> 5), lane = int(threadIdx.x & 31);
    if (w > 1) return;
    const int nex = w == 0 ? a.nexa : a.nexb;
    const uint32_t *bits = w == 0 ? sa : sb;
    uint32_t *out = w == 0 ? fa : fb;
    int cnt = 0;
    for (int e0 = 0; e0 < nex; e0 += 32) {
        const int e = e0 + lane;
        uint32_t u = 0u;
        bool keep = false;
        if (e < nex) {
            u = w == 0 ? a.aex[A * a.nexa + e] : a.bexT[size_t(e) * a.Nb + B];
            const uint32_t o = u & 0xFFFFu;
            keep = (bits[o >> 5] >> (o & 31)) & 1u;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) out[cnt + __popc(bal & ((1u << lane) - 1u))] = u;
        cnt += __popc(bal);
    }
    if (lane == 0) *(w == 0 ? naf : nbf) = cnt;
}

template <typename F>
__device__ __forceinline__ void hss_enumerate(const HssArgs &a, int64_t A, int64_t B,
                                              const uint32_t *sa, const uint32_t *sb,
                                              const uint32_t *fa, int naf, const uint32_t *fb,
                                              int nbf, F &&take)
{
    const int n = a.n, nn = n * n;
    const int64_t Nb = a.Nb;
    const int bd = int(blockDim.x), tid = int(threadIdx.x);
    // same-spin couplings: the CSR rows of both strings
    for (int k = a.Ma_ptr[A] + tid; k < a.Ma_ptr[A + 1]; k += bd) {
        const uint32_t Ao = uint32_t(a.Ma_col[k]);
        if ((sa[Ao >> 5] >> (Ao & 31)) & 1u) take(int64_t(Ao) * Nb + B, a.Ma_val[k]);
    }
    for (int k = a.Mb_ptr[B] + tid; k < a.Mb_ptr[B + 1]; k += bd) {
        const uint32_t Bo = uint32_t(a.Mb_col[k]);
        if ((sb[Bo >> 5] >> (Bo & 31)) & 1u) take(A * Nb + Bo, a.Mb_val[k]);
    }
    const uint32_t am = a.astr[A], bm = a.bstr[B];
    // alpha-beta couplings with a beta excitation: the (alpha diagonal +
    // filtered alpha excitations) x (filtered beta excitations) grid
    const int na1 = naf + 1;
    for (int i = tid; i < nbf * na1; i += bd) {
        const uint32_t wv = fb[i / na1];
        const int e = i % na1 - 1;
        const int64_t Bo = wv & 0xFFFFu;
        const int rs = int((wv >> 20) & 15) * n + int((wv >> 16) & 15);
        const bool negb = (wv >> 31) != 0;
        if (e < 0) {
            const double c = sum_diag<double>(a.V, n, nn, am, rs);
            take(A * Nb + Bo, negb ? -c : c);
        } else {
            const uint32_t u = fa[e];
            const int pq = int((u >> 20) & 15) * n + int((u >> 16) & 15);
            const double c = a.V[size_t(pq) * nn + rs];
            take(int64_t(u & 0xFFFFu) * Nb + Bo, negb != ((u >> 31) != 0) ? -c : c);
        }
    }
    // alpha-beta couplings diagonal in beta: the diagonal and the filtered
    // alpha excitations
    for (int e = tid - 1; e < naf; e += bd) {
        double c = 0.0;
        if (e < 0) {
            for (uint32_t mm = bm; mm; mm &= mm - 1) {
                const int rr = __ffs(mm) - 1;
                c += sum_diag<double>(a.V, n, nn, am, rr * n + rr);
            }
            take(A * Nb + B, c);
        } else {
            const uint32_t u = fa[e];
            const int pq = int((u >> 20) & 15) * n + int((u >> 16) & 15);
            c = sum_mask(a.V + size_t(pq) * nn, n + 1, bm);
            take(int64_t(u & 0xFFFFu) * Nb + B, (u >> 31) ? -c : c);
        }
    }
}

// the support's alpha and beta string sets (sa, sb cleared before)
__global__ void __launch_bounds__(256)
k_hss_strings(const int64_t *__restrict__ key, int64_t m, int64_t Nb, uint32_t *__restrict__ sa,
              uint32_t *__restrict__ sb)
{
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t d = key[t] >> 8, A = d / Nb, B = d % Nb;
        atomicOr(sa + (A >> 5), 1u << (A & 31));
        atomicOr(sb + (B >> 5), 1u << (B & 31));
    }
}

// exclusive prefix of v over the block (256 threads), total in *tot
__device__ __forceinline__ int block_excl_scan(int v, int *warp_tot, int *tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int i = 0; i < int(blockDim.x >> 5); ++i) {
            const int t = warp_tot[i];
            warp_tot[i] = acc;
            acc += t;
        }
        *tot = acc;
    }
    __syncthreads();
    return warp_tot[w] + x - v;
}

// ---------------------------------------------------------------------------
// A support list in determinant order from its membership bitmap (stream
// compaction in three passes): block b owns words [b * 2048, (b + 1) * 2048)
// (8 consecutive words a thread), counts their set bits, the block totals
// are scanned by one block, and every block then writes its determinants in
// order from its offset.  Rows processed together by a later kernel are then
// neighbours in Omega_CIk: they share their alpha string, and with it the
// alpha rows their couplings reach.
// ---------------------------------------------------------------------------
constexpr int kCompactWords = 8;
constexpr int kCompactThreads = 256;

__global__ void __launch_bounds__(kCompactThreads)
k_bits_count(const uint32_t *__restrict__ bits, int64_t words, int64_t *__restrict__ blk)
{
    __shared__ int wsum[kCompactThreads / 32];
    const int64_t w0 = (int64_t(blockIdx.x) * kCompactThreads + threadIdx.x) * kCompactWords;
    int c = 0;
    for (int j = 0; j < kCompactWords; ++j)
        if (w0 + j < words) c += __popc(bits[w0 + j]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kCompactThreads / 32; ++w) t += wsum[w];
        blk[blockIdx.x] = t;
    }
}

// exclusive scan of blk[0..nb) in place by one block of 1024 threads, each
// owning a contiguous run; the total goes to cnt[0] (count) and cnt[1]
// (rotation snapshot), cnt[2] (finished blocks) is cleared
__global__ void __launch_bounds__(1024)
k_blk_scan(int64_t *__restrict__ blk, int64_t nb, unsigned long long *__restrict__ cnt)
{
    __shared__ long long wt[32];
    const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = int64_t(threadIdx.x) * per, b1 = b0 + per < nb ? b0 + per : nb;
    long long run = 0;
    for (int64_t b = b0; b < b1; ++b) run += blk[b];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = run;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int i = 0; i < int(blockDim.x >> 5); ++i) {
            const long long t = wt[i];
            wt[i] = acc;
            acc += t;
        }
        cnt[0] = (unsigned long long)acc;
        cnt[1] = (unsigned long long)acc;
        cnt[2] = 0ull;
    }
    __syncthreads();
    long long off = wt[w] + x - run;
    for (int64_t b = b0; b < b1; ++b) {
        const long long c = blk[b];
        blk[b] = off;
        off += c;
    }
}

__global__ void __launch_bounds__(kCompactThreads)
k_bits_emit(const uint32_t *__restrict__ bits, int64_t words, const int64_t *__restrict__ blk,
            int64_t *__restrict__ list, int64_t cap)
{
    __shared__ int wt[kCompactThreads / 32], tot;
    const int64_t w0 = (int64_t(blockIdx.x) * kCompactThreads + threadIdx.x) * kCompactWords;
    uint32_t wv[kCompactWords];
    int c = 0;
    for (int j = 0; j < kCompactWords; ++j) {
        wv[j] = w0 + j < words ? bits[w0 + j] : 0u;
        c += __popc(wv[j]);
    }
    int64_t pos = blk[blockIdx.x] + block_excl_scan(c, wt, &tot);
    for (int j = 0; j < kCompactWords; ++j)
        for (uint32_t m = wv[j]; m; m &= m - 1, ++pos)
            if (pos < cap) list[pos] = (w0 + j) * 32 + (__ffs(m) - 1);
}

__global__ void __launch_bounds__(256)
k_hss_fill(HssArgs a)
{
    __shared__ uint32_t sa[kHssStrWords], sb[kHssStrWords];
    __shared__ uint32_t fa[64], fb[64];
    __shared__ int naf, nbf;
    __shared__ int wt[8], tot;
    for (int i = threadIdx.x; i < int((a.Na + 31) >> 5); i += blockDim.x) sa[i] = a.sa[i];
    for (int i = threadIdx.x; i < int((a.Nb + 31) >> 5); i += blockDim.x) sb[i] = a.sb[i];
    for (int64_t t = blockIdx.x; t < a.m; t += gridDim.x) {
        const int64_t d = a.key[t] >> 8;
        const int64_t A = d / a.Nb, B = d % a.Nb;
        __syncthreads();
        hss_filter(a, A, B, sa, sb, fa, fb, &naf, &nbf);
        __syncthreads();
        const int na = naf, nb = nbf;
        int c = 0;
        hss_enumerate(a, A, B, sa, sb, fa, na, fb, nb, [&](int64_t o, double) {
            if (member(a.bits, o)) ++c;
        });
        // row t owns entries [t * stride, (t + 1) * stride); stride bounds the
        // enumeration's length, and no write passes the row's end
        const int64_t row0 = t * a.stride, row1 = row0 + a.stride;
        int64_t pos = row0 + block_excl_scan(c, wt, &tot);
        hss_enumerate(a, A, B, sa, sb, fa, na, fb, nb, [&](int64_t o, double v) {
            if (member(a.bits, o)) {
                if (pos < row1) {
                    a.col[pos] = uint32_t(o);
                    a.val[pos] = v;
                }
                ++pos;
            }
        });
        if (threadIdx.x == 0) a.cnt[t] = int32_t(tot < a.stride ? tot : a.stride);
    }
}

// *nnz = sum of cnt[0 .. m), one block, fixed order
__global__ void __launch_bounds__(1024)
k_hss_total(const int32_t *__restrict__ cnt, int64_t m, int64_t *__restrict__ nnz)
{
    __shared__ long long wsum[32];
    long long x = 0;
    for (int64_t t = threadIdx.x; t < m; t += blockDim.x) x += cnt[t];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tot = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) tot += wsum[w];
        *nnz = tot;
    }
}

// one warp per row: sigma[key[t] >> 8] = sum val * psi[col], lanes strided,
// a fixed-order warp sum; with partials, also *dot = <psi|sigma> over the
// rows in FP64 (each warp its rows in order, the block's warps in order, then
// the last block to finish adds the blocks' partials in block order, as
// k_sv_sum would, and re-arms *done for the next launch)
template <typename T>
__global__ void __launch_bounds__(256)
k_hss_apply(const int64_t *__restrict__ key, int64_t m, const int32_t *__restrict__ cnt,
            int64_t stride, const uint32_t *__restrict__ col, const double *__restrict__ val,
            const T *__restrict__ psi, T *__restrict__ sigma, double *__restrict__ partials,
            unsigned *__restrict__ done, double *__restrict__ out)
{
    __shared__ double red[8];
    __shared__ bool last;
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    double dot = 0.0;
    for (int64_t t = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); t < m;
         t += warps) {
        T acc = T(0);
        const int64_t e1 = t * stride + cnt[t];
        for (int64_t e = t * stride + lane; e < e1; e += 32)
            acc += T(val[e]) * psi[col[e]];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const int64_t d = key[t] >> 8;
            sigma[d] = acc;
            dot = fma(double(psi[d]), double(acc), dot);
        }
    }
    if (!partials) return;
    if (lane == 0) red[threadIdx.x >> 5] = dot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w];
        partials[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < int(gridDim.x); b += blockDim.x) s += __ldcg(partials + b);
    s = block_sum_d(s);
    if (threadIdx.x == 0) {
        *out = s;
        *done = 0u;
    }
}

cudaError_t hss_fill(const HssArgs &a, int64_t *nnz, int num_sms, cudaStream_t st)
{
    if (a.m < 1 || a.stride < 1 || a.Na > 12870 || a.Nb > 12870 || a.nexa > 64 || a.nexb > 64)
        return cudaErrorInvalidValue;
    const size_t wa = size_t((a.Na + 31) >> 5), wb = size_t((a.Nb + 31) >> 5);
    cudaError_t e = cudaMemsetAsync(a.sa, 0, wa * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.sb, 0, wb * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    int64_t gs = (a.m + 255) / 256;
    if (gs > int64_t(num_sms) * 8) gs = int64_t(num_sms) * 8;
    k_hss_strings<<<unsigned(gs), 256, 0, st>>>(a.key, a.m, a.Nb, a.sa, a.sb);
    hy::count_launch();
    int64_t g = a.m < int64_t(num_sms) * 16 ? a.m : int64_t(num_sms) * 16;
    k_hss_fill<<<unsigned(g), 256, 0, st>>>(a); hy::count_launch();
    k_hss_total<<<1, 1024, 0, st>>>(a.cnt, a.m, nnz); hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t hss_apply(const int64_t *key, int64_t m, const int32_t *cnt, int64_t stride,
                      const uint32_t *col, const double *val, const T *psi, T *sigma, int num_sms,
                      double *partials, unsigned *done, double *dot, cudaStream_t st)
{
    if (m < 1) return cudaSuccess;
    if (dot && (!partials || !done)) return cudaErrorInvalidValue;
    int64_t g = (m + 7) / 8;
    if (g > int64_t(num_sms) * 16) g = int64_t(num_sms) * 16;
    k_hss_apply<T><<<unsigned(g), 256, 0, st>>>(key, m, cnt, stride, col, val, psi, sigma,
                                                dot ? partials : nullptr, done, dot);
    hy::count_launch();
    return cudaGetLastError();
}

template cudaError_t hss_apply<double>(const int64_t *, int64_t, const int32_t *, int64_t,
                                       const uint32_t *, const double *, const double *,
                                       double *, int, double *, unsigned *, double *,
                                       cudaStream_t);
template cudaError_t hss_apply<float>(const int64_t *, int64_t, const int32_t *, int64_t,
                                      const uint32_t *, const double *, const float *, float *,
                                      int, double *, unsigned *, double *, cudaStream_t);

namespace {
// blocks for a list of about n entries (grid-stride loops cover any count)
unsigned sv_grid(int64_t n, int num_sms)
{
    int64_t g = (n + 255) / 256;
    if (g > int64_t(num_sms) * 8) g = int64_t(num_sms) * 8;
    return unsigned(g < 1 ? 1 : g);
}
}  // namespace

// entries to size a grid for: twice the host's estimate, within the capacity
template <typename T>
int64_t sv_n(const SVec<T> &x)
{
    const int64_t h = x.hint > 0 ? 2 * x.hint : x.cap;
    return h < x.cap ? h : x.cap;
}

template <typename T>
cudaError_t sv_reset(const SVec<T> &x, bool hf, int num_sms, cudaStream_t st)
{
    k_sv_clear<T><<<sv_grid(sv_n(x), num_sms), 256, 0, st>>>(x); hy::count_launch();
    k_sv_finish_reset<T><<<1, 1, 0, st>>>(x, hf ? 1 : 0); hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t sv_copy(const SVec<T> &dst, const SVec<T> &src, int num_sms, cudaStream_t st)
{
    k_sv_copy<T><<<sv_grid(sv_n(src), num_sms), 256, 0, st>>>(dst, src); hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t sv_excite(const SVec<T> &x, const SvOpArgs &o, int k, int nc, double theta,
                      int num_sms, cudaStream_t st, bool closed)
{
    const T c = T(std::cos(theta)), s = T(std::sin(theta));
    for (int ci = 0; ci < nc; ++ci) {
        k_sv_excite<T><<<sv_grid(sv_n(x), num_sms), 256, 0, st>>>(x, o, k, ci, c, s,
                                                                  closed ? 1 : 0);
        hy::count_launch();
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t sv_prepare(const SVec<T> &x, const SvOpArgs &o, const int32_t *ops, const double *cs,
                       int L, bool renorm, double *norm2, int64_t *step_len, cudaStream_t st)
{
    k_sv_prepare<T><<<1, kPrepThreads, 0, st>>>(x, o, ops, cs, L, renorm ? 1 : 0, norm2, step_len);
    hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t sv_grad_fwd(const SVec<T> &f, const SVec<T> &w, const SvOpArgs &o, const int32_t *ops,
                        const double *cs, int L, const T *sigma, const double *norm2, double *g,
                        cudaStream_t st)
{
    k_sv_grad_fwd<T><<<1, kPrepThreads, 0, st>>>(f, w, o, ops, cs, L, sigma, norm2, g);
    hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t sv_dot(const SVec<T> &x, const T *y, double *partials, double *out, int num_sms,
                   cudaStream_t st)
{
    const int G = 4 * num_sms;
    k_sv_dot_partial<T><<<G, 256, 0, st>>>(x, y, partials); hy::count_launch();
    k_sv_sum<<<1, 256, 0, st>>>(partials, G, out); hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t sv_scale_rsqrt(const SVec<T> &x, const double *norm2, int num_sms, cudaStream_t st)
{
    k_sv_scale<T><<<sv_grid(sv_n(x), num_sms), 256, 0, st>>>(x, norm2); hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t support(const T *psi, int64_t N, int64_t *list, int64_t cap,
                    unsigned long long *count, int num_sms, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    int64_t g = (N + 255) / 256;
    if (g > int64_t(num_sms) * 16) g = int64_t(num_sms) * 16;
    if (g < 1) g = 1;
    k_support<T><<<unsigned(g), 256, 0, st>>>(psi, N, list, cap, count); hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t hpsi_scatter(const SparseArgs<T> &a, int num_sms, cudaStream_t st)
{
    // with an output list the caller has cleared sigma's previous support
    cudaError_t e = a.obits ? cudaSuccess
                            : cudaMemsetAsync(a.sigma, 0, size_t(a.Na) * a.Nb * sizeof(T), st);
    if (e != cudaSuccess || (!a.d_m && a.m == 0)) return e;
    int64_t g = a.d_m ? a.cap : a.m;
    if (g > int64_t(num_sms) * 32) g = int64_t(num_sms) * 32;
    if (g < 1) g = 1;
    k_hpsi_scatter<T><<<unsigned(g), 256, 0, st>>>(a); hy::count_launch();
    return cudaGetLastError();
}

cudaError_t bits_compact(const uint32_t *bits, int64_t words, int64_t *list, int64_t cap,
                         unsigned long long *cnt, int64_t *blk, cudaStream_t st)
{
    const int64_t nb = bits_compact_blocks(words);
    k_bits_count<<<unsigned(nb), kCompactThreads, 0, st>>>(bits, words, blk); hy::count_launch();
    k_blk_scan<<<1, 1024, 0, st>>>(blk, nb, cnt); hy::count_launch();
    k_bits_emit<<<unsigned(nb), kCompactThreads, 0, st>>>(bits, words, blk, list, cap);
    hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t hpsi_support(const SupRowsArgs<T> &a, int num_sms, cudaStream_t st)
{
    const SparseArgs<T> &h = a.s;
    if (h.nexa > 64 || h.n > 16) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(a.ctr, 0, 4 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.flagA, 0, size_t(h.Na), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.flagB, 0, size_t(h.Nb), st);
    if (e != cudaSuccess) return e;
    int64_t g = (a.cap + 255) / 256;
    if (g > int64_t(num_sms) * 8) g = int64_t(num_sms) * 8;
    if (g < 1) g = 1;
    k_sup_runs<<<unsigned(g), 256, 0, st>>>(a.list, a.cnt, a.cap, h.Nb, a.runs, a.ralpha,
                                             a.flagA, a.flagB, a.ctr);
    hy::count_launch();
    k_sup_blist<<<unsigned(num_sms), 256, 0, st>>>(a.flagB, h.Nb, a.blist, a.ctr);
    hy::count_launch();
    const size_t sa = sup_alpha_smem<T>(h.Nb, h.n * h.n), sb = size_t(h.Na) * sizeof(T);
    e = cudaFuncSetAttribute(k_sup_alpha<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sa));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sup_beta<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sb));
    if (e != cudaSuccess) return e;
    const unsigned per_sm = sizeof(T) == 8 ? 1u : 2u;
    k_sup_alpha<T><<<unsigned(num_sms) * per_sm, kSupThreads, sa, st>>>(a);
    hy::count_launch();
    k_sup_beta<T><<<unsigned(num_sms) * per_sm, kSupThreads, sb, st>>>(a);
    hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t grad_sparse(const SparseGradArgs<T> &a, int num_sms, cudaStream_t st)
{
    (void)num_sms;
    if (a.n_ops == 0) return cudaSuccess;
    k_grad_sparse<T><<<dim3(unsigned(a.n_ops), unsigned(a.chunks)), 256, 0, st>>>(a);
    hy::count_launch();
    k_grad_sparse_final<<<unsigned((a.n_ops + 255) / 256), 256, 0, st>>>(a.partials, a.chunks,
                                                                       a.n_ops, a.g);
    hy::count_launch();
    return cudaGetLastError();
}

cudaError_t prog_compile(const int64_t *list, int64_t m, const int64_t *step_len, int steps,
                         const SvOpArgs &o, const int32_t *ops, int L, int64_t *key,
                         uint32_t *pairs, int *npairs, int *step_l, int *flag, cudaStream_t st)
{
    if (m < 1 || m > kProgMax || steps < 1 || steps > kProgSteps) return cudaErrorInvalidValue;
    // up to 128 KB of dynamic shared memory (set per call: the attribute
    // belongs to the current device)
    cudaError_t e = cudaFuncSetAttribute(k_prog_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(kProgSortMax * 8));
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    // the counts of the front (npairs[0, steps)) and back (npairs[steps,
    // 2 steps)) lists
    if (e == cudaSuccess) e = cudaMemsetAsync(npairs, 0, 2 * size_t(steps) * sizeof(int), st);
    if (e != cudaSuccess) return e;
    int64_t P = 1;
    while (P < m) P <<= 1;
    k_prog_sort<<<1, 1024, size_t(P) * 8, st>>>(list, m, step_len, steps, key);
    hy::count_launch();
    k_prog_tables<<<dim3(unsigned((m + 255) / 256), unsigned(steps)), 256, 0, st>>>(
        key, int(m), o, ops, L, pairs, npairs, npairs + steps, step_l, flag);
    hy::count_launch();
    return cudaGetLastError();
}

namespace {
// static shared memory of a program kernel: its ProgSteps and reduction
// slots, at most sizeof(ProgSteps<T>) + 512 bytes
template <typename T>
constexpr size_t prog_static() { return sizeof(ProgSteps<T>) + 512; }

// dynamic shared memory of a program launch: the vectors (vec bytes) and as
// many staged pair words (*cap) as the block's opt-in limit leaves beside the
// kernel's static shared memory (prog_attrs has raised the kernels' limit)
template <typename T>
cudaError_t prog_smem(const ProgTabs &g, size_t vec, size_t *smem, int *cap)
{
    const size_t stat = prog_static<T>();
    if (g.optin < 0 || size_t(g.optin) < stat + vec) return cudaErrorInvalidValue;
    const size_t words = (size_t(g.optin) - stat - vec) / 4;
    *cap = int(words);
    *smem = vec + words * 4;
    return cudaSuccess;
}

template <typename T, typename K>
cudaError_t prog_attr(K kernel, int optin)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - int(prog_static<T>()));
}
}  // namespace

cudaError_t prog_attrs(int optin)
{
    if (optin < int(prog_static<double>()) + 1024) return cudaErrorInvalidValue;
    cudaError_t e = prog_attr<double>(k_prog_prepare<double>, optin);
    if (e == cudaSuccess) e = prog_attr<float>(k_prog_prepare<float>, optin);
    if (e == cudaSuccess) e = prog_attr<double>(k_prog_grad<double>, optin);
    if (e == cudaSuccess) e = prog_attr<float>(k_prog_grad<float>, optin);
    if (e == cudaSuccess) e = prog_attr<double>(k_prog_prepare_big<double>, optin);
    if (e == cudaSuccess) e = prog_attr<float>(k_prog_prepare_big<float>, optin);
    if (e == cudaSuccess) e = prog_attr<double>(k_prog_grad_big<double>, optin);
    if (e == cudaSuccess) e = prog_attr<float>(k_prog_grad_big<float>, optin);
    return e;
}

template <typename T>
cudaError_t prog_prepare(const ProgTabs &g, const double *cs, bool renorm, double *norm2, T *v,
                         cudaStream_t st)
{
    if (g.m < 1 || g.m > kProgMax || g.steps < 1 || g.steps > kProgSteps || g.ranks != 1 ||
        g.chunk != g.m)
        return cudaErrorInvalidValue;
    size_t smem = 0;
    int cap = 0;
    const cudaError_t e = prog_smem<T>(g, size_t(g.m) * sizeof(T), &smem, &cap);
    if (e != cudaSuccess) return e;
    k_prog_prepare<T><<<1, kProgThreads, smem, st>>>(g, cs, renorm ? 1 : 0, norm2, v, cap);
    hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t prog_grad(const ProgTabs &g, const double *cs, int L, const T *sigma,
                      const double *norm2, double *gout, cudaStream_t st)
{
    if (g.m < 1 || g.m > kProgMax || g.steps < 1 || g.steps > kProgSteps || g.ranks != 1 ||
        g.chunk != g.m || L < 1)
        return cudaErrorInvalidValue;
    size_t smem = 0;
    int cap = 0;
    const cudaError_t e = prog_smem<T>(g, 2 * size_t(g.m) * sizeof(T), &smem, &cap);
    if (e != cudaSuccess) return e;
    k_prog_grad<T><<<unsigned(L), kProgThreads, smem, st>>>(g, cs, sigma, norm2, gout, cap);
    hy::count_launch();
    return cudaGetLastError();
}

template cudaError_t prog_prepare<double>(const ProgTabs &, const double *, bool, double *,
                                          double *, cudaStream_t);
template cudaError_t prog_prepare<float>(const ProgTabs &, const double *, bool, double *, float *,
                                         cudaStream_t);
template cudaError_t prog_grad<double>(const ProgTabs &, const double *, int, const double *,
                                       const double *, double *, cudaStream_t);
template cudaError_t prog_grad<float>(const ProgTabs &, const double *, int, const float *,
                                      const double *, double *, cudaStream_t);

template cudaError_t support<double>(const double *, int64_t, int64_t *, int64_t,
                                     unsigned long long *, int, cudaStream_t);
template cudaError_t support<float>(const float *, int64_t, int64_t *, int64_t,
                                    unsigned long long *, int, cudaStream_t);
template cudaError_t hpsi_scatter<double>(const SparseArgs<double> &, int, cudaStream_t);
template cudaError_t hpsi_scatter<float>(const SparseArgs<float> &, int, cudaStream_t);
template cudaError_t hpsi_support<double>(const SupRowsArgs<double> &, int, cudaStream_t);
template cudaError_t hpsi_support<float>(const SupRowsArgs<float> &, int, cudaStream_t);
cudaError_t prog_compile_big(const int64_t *list, int64_t m, const int64_t *step_len, int steps,
                             const SvOpArgs &o, const int32_t *ops, int L, const uint32_t *bits,
                             int64_t *key, uint32_t *pairs, int *npairs, int *step_l,
                             int32_t *idx_map, int *flag, cudaStream_t st)
{
    if (m <= kProgMax || m > kProgBig || steps < 1 || steps > kProgSteps)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(npairs, 0, 2 * size_t(steps) * kClusterCtas * sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_prog_keys_big<<<unsigned((m + 255) / 256), 256, 0, st>>>(list, m, step_len, steps, key,
                                                                idx_map);
    hy::count_launch();
    k_prog_tables_big<<<dim3(unsigned((m + 255) / 256), unsigned(steps)), 256, 0, st>>>(
        key, int(m), o, ops, L, bits, idx_map, pairs, npairs, npairs + steps * kClusterCtas, step_l,
        flag);
    hy::count_launch();
    return cudaGetLastError();
}

namespace {
bool big_tabs_ok(const ProgTabs &g)
{
    return g.m > kProgMax && g.m <= kProgBig && g.steps >= 1 && g.steps <= kProgSteps &&
           g.ranks == kClusterCtas && g.chunk == int((g.m + kClusterCtas - 1) / kClusterCtas);
}
}  // namespace

template <typename T>
cudaError_t prog_prepare_big(const ProgTabs &g, const double *cs, bool renorm, double *norm2,
                             T *v, cudaStream_t st)
{
    if (!big_tabs_ok(g)) return cudaErrorInvalidValue;
    size_t smem = 0;
    int cap = 0;
    const cudaError_t e = prog_smem<T>(g, size_t(g.chunk) * sizeof(T), &smem, &cap);
    if (e != cudaSuccess) return e;
    k_prog_prepare_big<T><<<kClusterCtas, 1024, smem, st>>>(g, cs, renorm ? 1 : 0, norm2, v, cap);
    hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t prog_grad_big(const ProgTabs &g, const double *cs, int L, const T *sigma,
                          const double *norm2, double *gout, cudaStream_t st)
{
    if (!big_tabs_ok(g) || L < 1) return cudaErrorInvalidValue;
    size_t smem = 0;
    int cap = 0;
    const cudaError_t e = prog_smem<T>(g, 2 * size_t(g.chunk) * sizeof(T), &smem, &cap);
    if (e != cudaSuccess) return e;
    k_prog_grad_big<T><<<unsigned(kClusterCtas * L), 1024, smem, st>>>(g, cs, sigma, norm2, gout,
                                                                       cap);
    hy::count_launch();
    return cudaGetLastError();
}

template cudaError_t prog_prepare_big<double>(const ProgTabs &, const double *, bool, double *,
                                              double *, cudaStream_t);
template cudaError_t prog_prepare_big<float>(const ProgTabs &, const double *, bool, double *,
                                             float *, cudaStream_t);
template cudaError_t prog_grad_big<double>(const ProgTabs &, const double *, int, const double *,
                                           const double *, double *, cudaStream_t);
template cudaError_t prog_grad_big<float>(const ProgTabs &, const double *, int, const float *,
                                          const double *, double *, cudaStream_t);
template cudaError_t grad_sparse<double>(const SparseGradArgs<double> &, int, cudaStream_t);
template cudaError_t grad_sparse<float>(const SparseGradArgs<float> &, int, cudaStream_t);
#define HY_SV_INST(T)                                                                       \
    template cudaError_t sv_reset<T>(const SVec<T> &, bool, int, cudaStream_t);              \
    template cudaError_t sv_copy<T>(const SVec<T> &, const SVec<T> &, int, cudaStream_t);   \
    template cudaError_t sv_excite<T>(const SVec<T> &, const SvOpArgs &, int, int, double,  \
                                      int, cudaStream_t, bool);                              \
    template cudaError_t sv_prepare<T>(const SVec<T> &, const SvOpArgs &, const int32_t *,  \
                                       const double *, int, bool, double *, int64_t *,      \
                                       cudaStream_t);                                        \
    template cudaError_t sv_grad_fwd<T>(const SVec<T> &, const SVec<T> &, const SvOpArgs &, \
                                        const int32_t *, const double *, int, const T *,    \
                                        const double *, double *, cudaStream_t);            \
    template cudaError_t sv_dot<T>(const SVec<T> &, const T *, double *, double *, int,     \
                                   cudaStream_t);                                            \
    template cudaError_t sv_scale_rsqrt<T>(const SVec<T> &, const double *, int, cudaStream_t);
HY_SV_INST(double)
HY_SV_INST(float)
#undef HY_SV_INST

}  // namespace k
}  // namespace hy
