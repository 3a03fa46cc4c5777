// hy_ranker.cu -- the learned pool ranker: per-operator features computed on
// the device, a small MLP (three hidden ReLU layers, FP32) with hand-written
// forward, backward and Adam kernels, and a top-M selection kernel.  The
// ranker has no counterpart in the paper's method: it proposes the M pool
// operators most likely to have the largest |g_k|, which are then screened
// exactly; the full screen stays the fallback and the judge.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hyperion.h"

#include "hy_kernels.cuh"

namespace hy {
void set_last_error(const std::string &msg);
}

namespace hy {
namespace k {

// ---------------------------------------------------------------------------
// occupation numbers <psi|n_P|psi> of every spin orbital (blocked order),
// normalised by <psi|psi>.  Fixed grid, per-CTA partials, ordered final sum.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_occ_partial(const T *__restrict__ psi, int64_t Na, int64_t Nb,
              const uint32_t *__restrict__ astr, const uint32_t *__restrict__ bstr,
              int n, double *__restrict__ partial)
{
    __shared__ double red[256];
    float occ[2 * 16 + 1];
#pragma unroll
    for (int i = 0; i < 33; ++i) occ[i] = 0.0f;
    for (int64_t a = blockIdx.x; a < Na; a += gridDim.x) {
        float rowsum = 0.0f;
        const T *row = psi + a * Nb;
        for (int64_t b = threadIdx.x; b < Nb; b += blockDim.x) {
            const float v = float(row[b]);
            const float w = v * v;
            rowsum += w;
            uint32_t m = bstr[b];
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if ((m >> r) & 1u) occ[16 + r] += w;
        }
        const uint32_t am = astr[a];
#pragma unroll
        for (int p = 0; p < 16; ++p)
            if ((am >> p) & 1u) occ[p] += rowsum;
        occ[32] += rowsum;
    }
    // block reduction of the 2*16+1 sums, one at a time in fixed order
    for (int i = 0; i < 33; ++i) {
        red[threadIdx.x] = double(occ[i]);
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[blockIdx.x * 33 + i] = red[0];
        __syncthreads();
    }
    (void)n;
}

// out[P] for P < 2n in blocked order: alpha p -> occ[p], beta p -> occ[16+p]
__global__ void k_occ_final(const double *__restrict__ partial, int G, int n,
                            float *__restrict__ out)
{
    const int i = threadIdx.x;
    if (i >= 33) return;
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += partial[g * 33 + i];
    __shared__ double sums[33];
    sums[i] = s;
    __syncthreads();
    const double norm = sums[32] > 0.0 ? sums[32] : 1.0;
    if (i < n) out[i] = float(sums[i] / norm);
    else if (i >= 16 && i < 16 + n) out[n + (i - 16)] = float(sums[i] / norm);
}

// The same occupations from the touched-weight partials of psi (Bw, rs of
// touched_weights), without another pass over the state: the beta
// occupation of r is sum_a Bw[a][r*n+r], the alpha occupation of p is
// sum_{a holding p} rs[a], the norm sum_a rs[a].  Block i (of 33) forms sum
// i in a fixed order; the last block to finish normalises.
__global__ void __launch_bounds__(256)
k_occ_from_weights(const float *__restrict__ Bw, const float *__restrict__ rs,
                   const uint32_t *__restrict__ astr, int64_t Na, int n, double *__restrict__ sums,
                   unsigned *__restrict__ done, float *__restrict__ out)
{
    __shared__ double red[8];
    __shared__ bool last;
    const int i = blockIdx.x, nn = n * n;
    double acc = 0.0;
    if (i == 32 || (i < 16 && i < n) || (i >= 16 && i - 16 < n))
        for (int64_t a = threadIdx.x; a < Na; a += blockDim.x) {
            if (i == 32) acc += double(rs[a]);
            else if (i < 16) acc += ((astr[a] >> i) & 1u) ? double(rs[a]) : 0.0;
            else acc += double(Bw[a * nn + (i - 16) * n + (i - 16)]);
        }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        sums[i] = t;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int j = threadIdx.x;
    if (j < 33) {
        const double norm = sums[32] > 0.0 ? sums[32] : 1.0;
        if (j < n) out[j] = float(sums[j] / norm);
        else if (j >= 16 && j < 16 + n) out[n + (j - 16)] = float(sums[j] / norm);
    }
    if (j == 0) *done = 0u;
}

cudaError_t occupations_from_weights(const float *Bw, const float *rs, const uint32_t *astr,
                                     int64_t Na, int n, double *scratch, float *out,
                                     cudaStream_t st)
{
    // scratch: 33 sums then the finished-block counter
    unsigned *done = reinterpret_cast<unsigned *>(scratch + 33);
    k_occ_from_weights<<<33, 256, 0, st>>>(Bw, rs, astr, Na, n, scratch, done, out);
    hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t occupations(const T *psi, int64_t Na, int64_t Nb, const uint32_t *astr,
                        const uint32_t *bstr, int n, double *partial, int G, float *out,
                        cudaStream_t st)
{
    k_occ_partial<T><<<G, 256, 0, st>>>(psi, Na, Nb, astr, bstr, n, partial); hy::count_launch();
    k_occ_final<<<1, 64, 0, st>>>(partial, G, n, out); hy::count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Weights of the state on the determinants an operator touches.
//   Bw[a][j*n+b] = sum_beta w(a, beta) [j in beta][b in beta],  w = psi^2
//   (or sigma^2), rs[a] = sum_beta w(a, beta)
// then
//   D[(i,a)][(j,b)] = sum_alpha [i in alpha][a not in alpha] *
//                     sum_beta w [j in beta][b not in beta]
// with i == a (j == b) meaning "no condition on the alpha (beta) string".
// The inner beta sum for j != b is Bw[.][j*n+j] - Bw[.][j*n+b].  Bw is
// symmetric in (j, b): the contraction reads the upper triangle only
// (j <= b), so the list-based weights fill only that.
// ---------------------------------------------------------------------------
// Bw is an indicator product, Bw = W I with W[a][c] = w(a, c) (N_a x N_b) and
// I[c][jb] = [j in c][b in c] (N_b x n^2): a block owns 16 alpha rows, a
// thread the pairs t and t + 128; column chunks of W and the beta masks are
// staged in shared memory and read as broadcasts, so the inner loop is
// 128 FMAs per 17 shared loads.
constexpr int kPwRows = 16, kPwChunk = 128, kPwThreads = 128;

template <typename T>
__global__ void __launch_bounds__(kPwThreads)
k_pair_weights(const T *__restrict__ psi, int64_t Na, int64_t Nb,
               const uint32_t *__restrict__ bstr, int n, float *__restrict__ Bw,
               float *__restrict__ rs)
{
    __shared__ __align__(16) float ws[kPwRows][kPwChunk];
    __shared__ __align__(16) uint32_t ms[kPwChunk];
    __shared__ float rsw[kPwThreads / 32][kPwRows];
    const int nn = n * n, t0 = threadIdx.x, t1 = threadIdx.x + kPwThreads;
    // an unused slot asks for all 32 bits: no string of < 32 electrons has them
    const uint32_t sel0 = t0 < nn ? (1u << (t0 / n)) | (1u << (t0 % n)) : 0xFFFFFFFFu;
    const uint32_t sel1 = t1 < nn ? (1u << (t1 / n)) | (1u << (t1 % n)) : 0xFFFFFFFFu;
    for (int64_t a0 = int64_t(blockIdx.x) * kPwRows; a0 < Na; a0 += int64_t(gridDim.x) * kPwRows) {
        float acc0[kPwRows], acc1[kPwRows], rsum[kPwRows];
#pragma unroll
        for (int r = 0; r < kPwRows; ++r) acc0[r] = acc1[r] = rsum[r] = 0.0f;
        for (int64_t c0 = 0; c0 < Nb; c0 += kPwChunk) {
            __syncthreads();
            const int64_t c = c0 + threadIdx.x;
            int nz = 0;
#pragma unroll 4
            for (int r = 0; r < kPwRows; ++r) {
                const int64_t a = a0 + r;
                const float v = (a < Na && c < Nb) ? float(psi[a * Nb + c]) : 0.0f;
                ws[r][threadIdx.x] = v * v;
                rsum[r] = fmaf(v, v, rsum[r]);
                nz |= v != 0.0f;
            }
            ms[threadIdx.x] = c < Nb ? bstr[c] : 0u;
            // a tile of zero weights adds nothing: sparse states skip most
            if (!__syncthreads_or(nz)) continue;
            for (int cc = 0; cc < kPwChunk; cc += 4) {
                const uint4 m4 = *reinterpret_cast<const uint4 *>(ms + cc);
                const float f00 = (m4.x & sel0) == sel0 ? 1.f : 0.f, f10 = (m4.x & sel1) == sel1 ? 1.f : 0.f;
                const float f01 = (m4.y & sel0) == sel0 ? 1.f : 0.f, f11 = (m4.y & sel1) == sel1 ? 1.f : 0.f;
                const float f02 = (m4.z & sel0) == sel0 ? 1.f : 0.f, f12 = (m4.z & sel1) == sel1 ? 1.f : 0.f;
                const float f03 = (m4.w & sel0) == sel0 ? 1.f : 0.f, f13 = (m4.w & sel1) == sel1 ? 1.f : 0.f;
#pragma unroll
                for (int r = 0; r < kPwRows; ++r) {
                    const float4 w = *reinterpret_cast<const float4 *>(&ws[r][cc]);
                    acc0[r] = fmaf(f00, w.x, fmaf(f01, w.y, fmaf(f02, w.z, fmaf(f03, w.w, acc0[r]))));
                    acc1[r] = fmaf(f10, w.x, fmaf(f11, w.y, fmaf(f12, w.z, fmaf(f13, w.w, acc1[r]))));
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kPwRows; ++r) {
            float v = rsum[r];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) rsw[threadIdx.x >> 5][r] = v;
        }
        __syncthreads();
        if (threadIdx.x < kPwRows && a0 + threadIdx.x < Na) {
            float v = 0.0f;
            for (int w = 0; w < kPwThreads / 32; ++w) v += rsw[w][threadIdx.x];
            rs[a0 + threadIdx.x] = v;
        }
#pragma unroll
        for (int r = 0; r < kPwRows; ++r) {
            const int64_t a = a0 + r;
            if (a >= Na) break;
            if (t0 < nn) Bw[a * nn + t0] = acc0[r];
            if (t1 < nn) Bw[a * nn + t1] = acc1[r];
        }
    }
}

// D[(i,a)][(j,b)] split over alpha rows: block (group, split) owns 16
// consecutive ia and sums the rows split, split + S, ...; threads own jb.
// Each row's weight x (rs, or the beta difference) is read once per block and
// added to the ia whose alpha condition the row meets, so Bw is read n^2 / 16
// times in all (once per ia before).  Partials [S][n^4].
constexpr int kPairSplits = 32, kPairGroup = 16;

__global__ void __launch_bounds__(256)
k_pair_contract(const float *__restrict__ Bw, const float *__restrict__ rs,
                const uint32_t *__restrict__ astr, const int32_t *__restrict__ rows,
                int n, float *__restrict__ part)
{
    const int nn = n * n;
    const int ia0 = blockIdx.x * kPairGroup, jb = threadIdx.x;
    const int j = jb < nn ? jb / n : 0, b = jb < nn ? jb % n : 0;
    const int ut = j <= b ? j * n + b : b * n + j;   // (j, b) in the upper triangle
    // alpha condition of ia = (i, a): i == a (none), else i occupied, a empty
    uint32_t need[kPairGroup], gone[kPairGroup];
#pragma unroll
    for (int q = 0; q < kPairGroup; ++q) {
        const int ia = ia0 + q < nn ? ia0 + q : 0, i = ia / n, aa = ia % n;
        need[q] = i == aa ? 0u : 1u << i;
        gone[q] = i == aa ? 0u : 1u << aa;
    }
    const int nrows = rows[0];
    float acc[kPairGroup];
#pragma unroll
    for (int q = 0; q < kPairGroup; ++q) acc[q] = 0.0f;
    if (jb < nn) {
#pragma unroll 4
        for (int t = blockIdx.y; t < nrows; t += gridDim.y) {
            const int64_t al = rows[1 + t];
            const uint32_t m = astr[al];
            const float x = (j == b) ? rs[al] : (Bw[al * nn + j * n + j] - Bw[al * nn + ut]);
#pragma unroll
            for (int q = 0; q < kPairGroup; ++q)
                acc[q] += ((m & need[q]) == need[q] && (m & gone[q]) == 0u) ? x : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < kPairGroup; ++q)
            if (ia0 + q < nn) part[int64_t(blockIdx.y) * nn * nn + int64_t(ia0 + q) * nn + jb] = acc[q];
    }
}

// rows[0] = number of alpha rows with nonzero weight, rows[1..] = those rows
// in ascending order (one block: per-thread counts, block scan, write), so
// the contraction skips the all-zero rows of a sparse state
__global__ void __launch_bounds__(1024)
k_pair_rows(const float *__restrict__ rs, int64_t Na, int32_t *__restrict__ rows)
{
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (Na + blockDim.x - 1) / blockDim.x;
    const int64_t lo = tid * per, hi = lo + per < Na ? lo + per : Na;
    int cnt = 0;
    for (int64_t a = lo; a < hi; ++a) cnt += rs[a] != 0.0f;
    int incl = cnt;                              // inclusive scan within the warp
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = lane < int(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += u;
        }
        wsum[lane] = v;                          // inclusive warp totals
    }
    __syncthreads();
    int pos = incl - cnt + (warp > 0 ? wsum[warp - 1] : 0);
    for (int64_t a = lo; a < hi; ++a)
        if (rs[a] != 0.0f) rows[1 + pos++] = int32_t(a);
    if (tid == blockDim.x - 1) rows[0] = pos;
}

__global__ void __launch_bounds__(256)
k_pair_reduce(const float *__restrict__ part, int64_t total, int S, float *__restrict__ D)
{
    const int64_t id = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (id >= total) return;
    double s = 0.0;
    for (int k = 0; k < S; ++k) s += double(part[int64_t(k) * total + id]);
    D[id] = float(s);
}

int pair_splits() { return kPairSplits; }

// Bw and rs of a state held as a list of its nonzero amplitudes (Bw, rs
// zeroed by the caller): every listed determinant (A, B) adds w = x^2 to
// rs[A] and to Bw[A][j*n+b] for each pair j <= b of B's electrons (the upper
// triangle, which is all the contraction reads).  O(support) instead of a
// pass over the whole state.
template <typename T>
__global__ void __launch_bounds__(256)
k_pair_weights_list(const T *__restrict__ v, const int64_t *__restrict__ list,
                    const unsigned long long *__restrict__ count, int64_t cap, int64_t Nb,
                    const uint32_t *__restrict__ bstr, int n, float *__restrict__ Bw,
                    float *__restrict__ rs)
{
    const unsigned long long c = *count;
    const int64_t m = c < (unsigned long long)cap ? int64_t(c) : cap;
    const int nn = n * n;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t d = list[t];
        const float x = float(v[d]);
        const float w = x * x;
        if (w == 0.0f) continue;
        const int64_t A = d / Nb;
        const uint32_t bm = bstr[d % Nb];
        atomicAdd(rs + A, w);
        for (uint32_t mj = bm; mj; mj &= mj - 1) {
            const int j = __ffs(mj) - 1;
            for (uint32_t mb = mj; mb; mb &= mb - 1)   // b >= j: mj's lowest bit is j
                atomicAdd(Bw + A * nn + j * n + (__ffs(mb) - 1), w);
        }
    }
}

// The listed entries grouped by alpha row (count, scan, fill with each
// entry's beta string and weight w = x^2), then one block per row sums its
// entries into the row's pairs as k_pair_weights does over a whole row: no
// atomics on Bw, each of its slots written once.
__device__ __forceinline__ int64_t tw_len(const unsigned long long *count, int64_t cap)
{
    const unsigned long long c = *count;
    return c < (unsigned long long)cap ? int64_t(c) : cap;
}

__global__ void __launch_bounds__(256)
k_tw_count(const int64_t *__restrict__ list, const unsigned long long *__restrict__ count,
           int64_t cap, int64_t Nb, int32_t *__restrict__ cnt)
{
    const int64_t m = tw_len(count, cap);
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m;
         t += int64_t(gridDim.x) * blockDim.x)
        atomicAdd(cnt + list[t] / Nb, 1);
}

// exclusive scan of the row counts (one block): ptr[0..Na], cur = ptr
__global__ void __launch_bounds__(1024)
k_tw_scan(const int32_t *__restrict__ cnt, int64_t Na, int32_t *__restrict__ ptr,
          int32_t *__restrict__ cur)
{
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (Na + blockDim.x - 1) / blockDim.x;
    const int64_t lo = tid * per, hi = lo + per < Na ? lo + per : Na;
    int c = 0;
    for (int64_t r = lo; r < hi; ++r) c += cnt[r];
    int incl = c;
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = lane < int(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += u;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int pos = incl - c + (warp > 0 ? wsum[warp - 1] : 0);
    for (int64_t r = lo; r < hi; ++r) {
        ptr[r] = pos;
        cur[r] = pos;
        pos += cnt[r];
    }
    if (tid == blockDim.x - 1) ptr[Na] = pos;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_tw_fill(const T *__restrict__ v, const int64_t *__restrict__ list,
          const unsigned long long *__restrict__ count, int64_t cap, int64_t Nb,
          const uint32_t *__restrict__ bstr, int32_t *__restrict__ cur,
          uint32_t *__restrict__ mask, float *__restrict__ w)
{
    const int64_t m = tw_len(count, cap);
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t d = list[t];
        const int pos = atomicAdd(cur + d / Nb, 1);
        const float x = float(v[d]);
        mask[pos] = bstr[d % Nb];
        w[pos] = x * x;
    }
}

constexpr int kTwThreads = 128;

__global__ void __launch_bounds__(kTwThreads)
k_tw_rows(const int32_t *__restrict__ ptr, const uint32_t *__restrict__ mask,
          const float *__restrict__ w, int64_t Na, int n, float *__restrict__ Bw,
          float *__restrict__ rs)
{
    __shared__ uint32_t ms[kTwThreads];
    __shared__ float ws[kTwThreads];
    __shared__ float red[kTwThreads / 32];
    const int nn = n * n, t0 = threadIdx.x, t1 = threadIdx.x + kTwThreads;
    // an unused slot asks for all 32 bits: no string of < 32 electrons has them
    const uint32_t sel0 = t0 < nn ? (1u << (t0 / n)) | (1u << (t0 % n)) : 0xFFFFFFFFu;
    const uint32_t sel1 = t1 < nn ? (1u << (t1 / n)) | (1u << (t1 % n)) : 0xFFFFFFFFu;
    for (int64_t A = blockIdx.x; A < Na; A += gridDim.x) {
        const int j0 = ptr[A], j1 = ptr[A + 1];
        if (j0 == j1) continue;                      // the row stays zero
        float acc0 = 0.0f, acc1 = 0.0f, rsum = 0.0f;
        for (int c0 = j0; c0 < j1; c0 += kTwThreads) {
            __syncthreads();                          // the previous chunk's readers are done
            const int j = c0 + threadIdx.x;
            const float wj = j < j1 ? w[j] : 0.0f;
            ms[threadIdx.x] = j < j1 ? mask[j] : 0u;
            ws[threadIdx.x] = wj;
            rsum += wj;
            __syncthreads();
            const int cnt = j1 - c0 < kTwThreads ? j1 - c0 : kTwThreads;
            for (int k = 0; k < cnt; ++k) {
                const uint32_t mk = ms[k];
                const float wk = ws[k];
                acc0 += (mk & sel0) == sel0 ? wk : 0.0f;
                acc1 += (mk & sel1) == sel1 ? wk : 0.0f;
            }
        }
        for (int o = 16; o > 0; o >>= 1) rsum += __shfl_down_sync(0xffffffffu, rsum, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            float s = 0.0f;
            for (int i = 0; i < kTwThreads / 32; ++i) s += red[i];
            rs[A] = s;
        }
        if (t0 < nn) Bw[A * nn + t0] = acc0;
        if (t1 < nn) Bw[A * nn + t1] = acc1;
    }
}

template <typename T>
cudaError_t touched_weights_list(const T *v, const int64_t *list, const unsigned long long *count,
                                 int64_t cap, int64_t hint, int64_t Na, int64_t Nb,
                                 const uint32_t *astr, const uint32_t *bstr, int n, float *Bw,
                                 float *rs, int32_t *rows, float *part, float *D,
                                 const TwGroups &gr, int num_sms, cudaStream_t st)
{
    const int nn = n * n;
    cudaError_t e = cudaMemsetAsync(Bw, 0, size_t(Na) * nn * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(rs, 0, size_t(Na) * sizeof(float), st);
    if (e != cudaSuccess) return e;
    int64_t g = (std::max<int64_t>(hint, 1) + 255) / 256;
    if (g > int64_t(num_sms) * 8) g = int64_t(num_sms) * 8;
    if (gr.mask && gr.cap >= cap && cap <= int64_t(INT32_MAX)) {
        e = cudaMemsetAsync(gr.cnt, 0, size_t(Na + 1) * sizeof(int32_t), st);
        if (e != cudaSuccess) return e;
        k_tw_count<<<unsigned(g), 256, 0, st>>>(list, count, cap, Nb, gr.cnt); hy::count_launch();
        k_tw_scan<<<1, 1024, 0, st>>>(gr.cnt, Na, gr.ptr, gr.cur); hy::count_launch();
        k_tw_fill<T><<<unsigned(g), 256, 0, st>>>(v, list, count, cap, Nb, bstr, gr.cur, gr.mask,
                                                 gr.w);
        hy::count_launch();
        const int64_t gb = Na < int64_t(num_sms) * 16 ? Na : int64_t(num_sms) * 16;
        k_tw_rows<<<unsigned(gb), kTwThreads, 0, st>>>(gr.ptr, gr.mask, gr.w, Na, n, Bw, rs);
        hy::count_launch();
    } else {
        k_pair_weights_list<T><<<unsigned(g), 256, 0, st>>>(v, list, count, cap, Nb, bstr, n, Bw,
                                                            rs);
        hy::count_launch();
    }
    k_pair_rows<<<1, 1024, 0, st>>>(rs, Na, rows); hy::count_launch();
    k_pair_contract<<<dim3(unsigned((nn + kPairGroup - 1) / kPairGroup), kPairSplits), 256, 0, st>>>(
        Bw, rs, astr, rows, n, part);
    hy::count_launch();
    const int64_t tot = int64_t(nn) * nn;
    k_pair_reduce<<<unsigned((tot + 255) / 256), 256, 0, st>>>(part, tot, kPairSplits, D);
    hy::count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t touched_weights(const T *psi, int64_t Na, int64_t Nb, const uint32_t *astr,
                            const uint32_t *bstr, int n, float *Bw, float *rs, int32_t *rows,
                            float *part, float *D, int num_sms, cudaStream_t st)
{
    int64_t g = (Na + kPwRows - 1) / kPwRows;
    if (g > int64_t(num_sms) * 16) g = int64_t(num_sms) * 16;
    k_pair_weights<T><<<unsigned(g), kPwThreads, 0, st>>>(psi, Na, Nb, bstr, n, Bw, rs);
    hy::count_launch();
    const int nn = n * n;
    k_pair_rows<<<1, 1024, 0, st>>>(rs, Na, rows); hy::count_launch();
    k_pair_contract<<<dim3(unsigned((nn + kPairGroup - 1) / kPairGroup), kPairSplits), 256, 0, st>>>(
        Bw, rs, astr, rows, n, part);
    hy::count_launch();
    const int64_t tot = int64_t(nn) * nn;
    k_pair_reduce<<<unsigned((tot + 255) / 256), 256, 0, st>>>(part, tot, kPairSplits, D);
    hy::count_launch();
    return cudaGetLastError();
}

template cudaError_t touched_weights<double>(const double *, int64_t, int64_t, const uint32_t *,
                                             const uint32_t *, int, float *, float *, int32_t *,
                                             float *, float *, int, cudaStream_t);
template cudaError_t touched_weights_list<double>(const double *, const int64_t *,
                                                  const unsigned long long *, int64_t, int64_t,
                                                  int64_t, int64_t, const uint32_t *,
                                                  const uint32_t *, int, float *, float *,
                                                  int32_t *, float *, float *, const TwGroups &,
                                                  int, cudaStream_t);
template cudaError_t touched_weights_list<float>(const float *, const int64_t *,
                                                 const unsigned long long *, int64_t, int64_t,
                                                 int64_t, int64_t, const uint32_t *,
                                                 const uint32_t *, int, float *, float *,
                                                 int32_t *, float *, float *, const TwGroups &,
                                                 int, cudaStream_t);
template cudaError_t touched_weights<float>(const float *, int64_t, int64_t, const uint32_t *,
                                            const uint32_t *, int, float *, float *, int32_t *,
                                            float *, float *, int, cudaStream_t);

// ---------------------------------------------------------------------------
// per-operator features (kRankerFeatures floats per operator)
// ---------------------------------------------------------------------------
// weight of one constituent's domain (x annihilated present, y created
// absent) from the touched-weight tensor D; nap / nbp alpha / beta pairs
__device__ float touched(const float *D, int n, int nap, const int *ax, const int *ay, int nbp,
                         const int *bx, const int *by)
{
    const int nn = n * n;
    if (nap <= 1 && nbp <= 1) {
        const int ia = nap ? ax[0] * n + ay[0] : 0, jb = nbp ? bx[0] * n + by[0] : 0;
        return fmaxf(D[ia * nn + jb], 0.0f);
    }
    if (nap == 2 && nbp == 0)
        return sqrtf(fmaxf(D[(ax[0] * n + ay[0]) * nn], 0.0f) *
                     fmaxf(D[(ax[1] * n + ay[1]) * nn], 0.0f));
    if (nbp == 2 && nap == 0)
        return sqrtf(fmaxf(D[bx[0] * n + by[0]], 0.0f) * fmaxf(D[bx[1] * n + by[1]], 0.0f));
    return 0.0f;
}

__global__ void __launch_bounds__(128)
k_features(const int32_t *__restrict__ desc, int64_t K, int n, const double *__restrict__ h1,
           const double *__restrict__ eri, const float *__restrict__ occ,
           const float *__restrict__ extra, const float *__restrict__ Dpsi,
           const float *__restrict__ Dsig, float *__restrict__ feat)
{
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int32_t *d = desc + 11 * k;
    const int nc = d[0], rank = d[1];
    const int c0 = d[2], c1 = d[3], a1 = d[4], a0 = d[5];
    float f[kRankerFeatures];
    for (int i = 0; i < kRankerFeatures; ++i) f[i] = 0.0f;
    const int sc0 = c0 % n, sa0 = a0 % n;
    const bool single = rank == 1;
    const int sc1 = single ? 0 : c1 % n, sa1 = single ? 0 : a1 % n;
    const bool same = !single && ((c0 < n) == (c1 < n));
    f[0] = single ? 1.0f : 0.0f;
    f[1] = same ? 1.0f : 0.0f;
    f[2] = (!single && !same) ? 1.0f : 0.0f;
    f[3] = float(nc - 1);
    f[4] = float(sa0) / n;
    f[5] = single ? -0.1f : float(sa1) / n;
    f[6] = float(sc0) / n;
    f[7] = single ? -0.1f : float(sc1) / n;
    double integral, gap;
    if (single) {
        integral = h1[sc0 * n + sa0];
        gap = h1[sc0 * n + sc0] - h1[sa0 * n + sa0];
    } else {
        auto at = [&](int p, int q, int r, int s) {
            return eri[((size_t(p) * n + q) * n + r) * n + s];
        };
        integral = at(sc0, sa0, sc1, sa1);
        if (same) integral -= at(sc0, sa1, sc1, sa0);
        gap = h1[sc0 * n + sc0] + h1[sc1 * n + sc1] - h1[sa0 * n + sa0] - h1[sa1 * n + sa1];
    }
    f[8] = float(log10(fabs(integral) + 1e-10));
    f[9] = float(gap);
    const float na0 = occ[a0], nc0 = occ[c0];
    const float na1 = single ? 1.0f : occ[a1], nc1 = single ? 0.0f : occ[c1];
    f[10] = na0 * na1 * (1.0f - nc0) * (1.0f - nc1);
    f[11] = na0 + na1 - nc0 - nc1;
    if (Dpsi && Dsig) {
        // Cauchy-Schwarz bound on |g_k| over its constituents' pairs:
        // 2 (|sigma_img| |psi_dom| + |sigma_dom| |psi_img|), relative to
        // |sigma| |psi|, and the state weight on the touched determinants
        float bound = 0.0f, wsum = 0.0f;
        for (int c = 0; c < nc; ++c) {
            const int32_t *q = d + 1 + 5 * c;
            const int modes_c[2] = {q[1], q[2]}, modes_a[2] = {q[4], q[3]};
            const int nm = q[0];
            int ax[2], ay[2], bx[2], by[2], nap = 0, nbp = 0;
            for (int u = 0; u < nm; ++u) {
                const int x = modes_a[u], y = modes_c[u];
                if (x < n) { ax[nap] = x; ay[nap] = y; ++nap; }
                else { bx[nbp] = x - n; by[nbp] = y - n; ++nbp; }
            }
            const float dp = touched(Dpsi, n, nap, ax, ay, nbp, bx, by);
            const float ip = touched(Dpsi, n, nap, ay, ax, nbp, by, bx);
            const float ds = touched(Dsig, n, nap, ax, ay, nbp, bx, by);
            const float is = touched(Dsig, n, nap, ay, ax, nbp, by, bx);
            bound += 2.0f * (sqrtf(dp * is) + sqrtf(ip * ds));
            wsum += dp + ip;
        }
        const float np2 = fmaxf(Dpsi[0], 1e-30f), ns2 = fmaxf(Dsig[0], 1e-30f);
        f[10] = log10f(bound / sqrtf(np2 * ns2) + 1e-12f);
        f[11] = log10f(wsum / np2 + 1e-12f);
    }
    if (extra)
        for (int i = 0; i < 4; ++i) f[12 + i] = extra[4 * k + i];
    float *o = feat + kRankerFeatures * k;
    for (int i = 0; i < kRankerFeatures; ++i) o[i] = f[i];
}

cudaError_t features(const int32_t *desc, int64_t K, int n, const double *h1,
                     const double *eri, const float *occ, const float *extra, const float *Dpsi,
                     const float *Dsig, float *feat, cudaStream_t st)
{
    if (K == 0) return cudaSuccess;
    k_features<<<unsigned((K + 127) / 128), 128, 0, st>>>(desc, K, n, h1, eri, occ, extra, Dpsi,
                                                          Dsig, feat); hy::count_launch();
    return cudaGetLastError();
}

template cudaError_t occupations<double>(const double *, int64_t, int64_t, const uint32_t *,
                                         const uint32_t *, int, double *, int, float *,
                                         cudaStream_t);
template cudaError_t occupations<float>(const float *, int64_t, int64_t, const uint32_t *,
                                        const uint32_t *, int, double *, int, float *,
                                        cudaStream_t);

// ---------------------------------------------------------------------------
// MLP kernels (FP32)
// ---------------------------------------------------------------------------
// C[M x N] = op(A) op(B) (+ bias[j]) (ReLU), tiles of 16 x 16.
//   A(i, k) = TA ? A[k * lda + i] : A[i * lda + k]
//   B(k, j) = TB ? B[j * ldb + k] : B[k * ldb + j]
template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
k_gemm(const float *__restrict__ A, const float *__restrict__ B, float *__restrict__ C,
       int M, int N, int Kd, int lda, int ldb, int ldc, const float *__restrict__ bias,
       int relu)
{
    __shared__ float As[16][17], Bs[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
    float acc = 0.0f;
    for (int k0 = 0; k0 < Kd; k0 += 16) {
        {
            const int ii = blockIdx.y * 16 + ty, kk = k0 + tx;
            As[ty][tx] = (ii < M && kk < Kd) ? (TA ? A[size_t(kk) * lda + ii]
                                                  : A[size_t(ii) * lda + kk])
                                             : 0.0f;
            const int kb = k0 + ty, jj = blockIdx.x * 16 + tx;
            Bs[ty][tx] = (kb < Kd && jj < N) ? (TB ? B[size_t(jj) * ldb + kb]
                                                  : B[size_t(kb) * ldb + jj])
                                             : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc += As[ty][kk] * Bs[kk][tx];
        __syncthreads();
    }
    if (i < M && j < N) {
        if (bias) acc += bias[j];
        if (relu) acc = acc > 0.0f ? acc : 0.0f;
        C[size_t(i) * ldc + j] = acc;
    }
}

template <bool TA, bool TB>
cudaError_t gemm(const float *A, const float *B, float *C, int M, int N, int Kd, int lda,
                 int ldb, int ldc, const float *bias, bool relu, cudaStream_t st)
{
    if (M == 0 || N == 0) return cudaSuccess;
    dim3 grid((N + 15) / 16, (M + 15) / 16);
    k_gemm<TA, TB><<<grid, 256, 0, st>>>(A, B, C, M, N, Kd, lda, ldb, ldc, bias, relu ? 1 : 0); hy::count_launch();
    return cudaGetLastError();
}

// dZ = dY * (Z > 0) in place on dY
__global__ void k_relu_bwd(float *__restrict__ dy, const float *__restrict__ z, int64_t m)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < m && !(z[i] > 0.0f)) dy[i] = 0.0f;
}

// db[j] = sum_i dZ[i][j] (fixed order): a block of 32 x 8 threads owns 32
// columns; each of the 8 row groups sums rows g, g + 8, ..., then the 8
// partials are added in order
__global__ void __launch_bounds__(256)
k_colsum(const float *__restrict__ dz, int M, int N, float *__restrict__ db)
{
    __shared__ float part[8][33];
    const int cx = threadIdx.x & 31, gy = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + cx;
    float s = 0.0f;
    if (j < N)
        for (int i = gy; i < M; i += 8) s += dz[size_t(i) * N + j];
    part[gy][cx] = s;
    __syncthreads();
    if (gy == 0 && j < N) {
        float t = 0.0f;
        for (int g = 0; g < 8; ++g) t += part[g][cx];
        db[j] = t;
    }
}

// loss gradient of the mean squared error on one output column; also the
// per-row squared error (for the host-side loss report)
__global__ void k_mse(const float *__restrict__ pred, const float *__restrict__ target,
                      int m, float *__restrict__ dpred, float *__restrict__ sq)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const float d = pred[i] - target[i];
    dpred[i] = 2.0f * d / float(m);
    sq[i] = d * d;
}

__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, int64_t n, float lr, float b1t, float b2t)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float b1 = 0.9f, b2 = 0.999f;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float mh = a / (1.0f - b1t), vh = b / (1.0f - b2t);
    w[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// rows of X gathered by an index list (minibatch assembly)
__global__ void k_gather_rows(const float *__restrict__ X, const int32_t *__restrict__ idx,
                              int m, int F, float *__restrict__ out)
{
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= int64_t(m) * F) return;
    const int r = int(t / F), c = int(t % F);
    out[t] = X[size_t(idx[r]) * F + c];
}

// target t_k = log10(|g_k| / max |g| + 1e-6), max over the m entries; one CTA
// (the floor keeps the fit on the operators that can compete for the top)
__global__ void __launch_bounds__(1024)
k_targets(const double *__restrict__ g, int64_t m, float *__restrict__ t)
{
    __shared__ double red[1024];
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) mx = fmax(mx, fabs(g[i]));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    const double M = red[0] > 0.0 ? red[0] : 1.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x)
        t[i] = float(log10(fabs(g[i]) / M + 1e-6));
}

// top-k of m <= kTopKMax scores (descending; ties to the lower index) by a
// bitonic sort of (score, index) pairs in shared memory; one CTA.
__global__ void __launch_bounds__(1024)
k_topk(const float *__restrict__ score, int m, int kk, int32_t *__restrict__ out)
{
    extern __shared__ unsigned char raw[];
    float *s = reinterpret_cast<float *>(raw);
    int32_t *ix = reinterpret_cast<int32_t *>(s + kTopKMax);
    int P = 1;
    while (P < m) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        s[i] = i < m ? score[i] : -INFINITY;
        ix[i] = i < m ? i : 0x7fffffff;
    }
    __syncthreads();
    // "a before b" when a.score > b.score, or equal scores and a.index < b.index
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const float si = s[i], sj = s[j];
                    const int ii = ix[i], ij = ix[j];
                    const bool i_first = si > sj || (si == sj && ii < ij);
                    if (desc != i_first) {
                        s[i] = sj; s[j] = si;
                        ix[i] = ij; ix[j] = ii;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < kk; i += blockDim.x) out[i] = ix[i];
}

}  // namespace k
}  // namespace hy

// ---------------------------------------------------------------------------
// the ranker object
// ---------------------------------------------------------------------------
struct hy_ranker {
    int F = hy::k::kRankerFeatures, H = 256;
    // layers: W0 [H][F], b0 [H], W1 [H][H], b1, W2 [H][H], b2, W3 [1][H], b3 [1]
    std::vector<size_t> woff, boff, wsz, bsz;
    size_t nparam = 0;
    float *w = nullptr, *gw = nullptr, *m1 = nullptr, *m2 = nullptr;
    int64_t step = 0;
    // dataset
    float *X = nullptr, *Y = nullptr;
    int64_t n_samples = 0, cap = 0;
    // activations for one minibatch / prediction block
    int64_t act_rows = 0;
    float *xb = nullptr, *yb = nullptr, *z[3] = {nullptr, nullptr, nullptr},
          *d[3] = {nullptr, nullptr, nullptr}, *out = nullptr, *dout = nullptr, *sq = nullptr;
    int32_t *idx = nullptr;
    // one epoch's sample order and the last epoch's per-row squared errors
    int32_t *perm = nullptr;
    float *sqall = nullptr;
    int64_t perm_cap = 0;
    bool fitted = false;
};

namespace {

hy_status rerr(hy_status s, const std::string &m)
{
    hy::set_last_error(m);
    return s;
}

hy_status rcu(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return HY_OK;
    return rerr(e == cudaErrorMemoryAllocation ? HY_ERR_OOM : HY_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define RTRY(x)                         \
    do {                                \
        hy_status s_ = (x);             \
        if (s_ != HY_OK) return s_;     \
    } while (0)

hy_status ensure_act(hy_ranker *r, int64_t rows)
{
    if (rows <= r->act_rows) return HY_OK;
    float **bufs[] = {&r->xb, &r->yb, &r->z[0], &r->z[1], &r->z[2], &r->d[0], &r->d[1],
                      &r->d[2], &r->out, &r->dout, &r->sq};
    for (float **b : bufs) {
        cudaFree(*b);
        *b = nullptr;
    }
    cudaFree(r->idx);
    r->idx = nullptr;
    const size_t R = size_t(rows);
    RTRY(rcu(cudaMalloc(&r->xb, R * r->F * 4), "ranker buffers"));
    RTRY(rcu(cudaMalloc(&r->yb, R * 4), "ranker buffers"));
    for (int l = 0; l < 3; ++l) {
        RTRY(rcu(cudaMalloc(&r->z[l], R * r->H * 4), "ranker buffers"));
        RTRY(rcu(cudaMalloc(&r->d[l], R * r->H * 4), "ranker buffers"));
    }
    RTRY(rcu(cudaMalloc(&r->out, R * 4), "ranker buffers"));
    RTRY(rcu(cudaMalloc(&r->dout, R * 4), "ranker buffers"));
    RTRY(rcu(cudaMalloc(&r->sq, R * 4), "ranker buffers"));
    RTRY(rcu(cudaMalloc(&r->idx, R * 4), "ranker buffers"));
    r->act_rows = rows;
    return HY_OK;
}

// forward pass of rows [x: m x F] -> out [m]
hy_status forward(hy_ranker *r, const float *x, int m, cudaStream_t st)
{
    namespace K = hy::k;
    const float *in = x;
    int fin = r->F;
    for (int l = 0; l < 3; ++l) {
        RTRY(rcu(K::gemm<false, true>(in, r->w + r->woff[l], r->z[l], m, r->H, fin, fin, fin,
                                      r->H, r->w + r->boff[l], true, st), "mlp forward"));
        in = r->z[l];
        fin = r->H;
    }
    return rcu(K::gemm<false, true>(in, r->w + r->woff[3], r->out, m, 1, r->H, r->H, r->H, 1,
                                    r->w + r->boff[3], false, st), "mlp forward");
}

uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

hy_status hy_ranker_create(int hidden, uint64_t seed, hy_ranker **out)
{
    if (!out) return rerr(HY_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (hidden < 8 || hidden > 4096) return rerr(HY_ERR_ARG, "hidden must be in [8, 4096]");
    hy_ranker *r = new (std::nothrow) hy_ranker;
    if (!r) return rerr(HY_ERR_OOM, "host allocation failed");
    r->H = hidden;
    const int dims_in[4] = {r->F, hidden, hidden, hidden};
    const int dims_out[4] = {hidden, hidden, hidden, 1};
    size_t off = 0;
    for (int l = 0; l < 4; ++l) {
        r->woff.push_back(off);
        r->wsz.push_back(size_t(dims_in[l]) * dims_out[l]);
        off += r->wsz.back();
        r->boff.push_back(off);
        r->bsz.push_back(size_t(dims_out[l]));
        off += r->bsz.back();
    }
    r->nparam = off;
    // He-uniform weights, zero biases (seeded SplitMix64)
    std::vector<float> w(off, 0.0f);
    uint64_t s = seed;
    for (int l = 0; l < 4; ++l) {
        const float lim = std::sqrt(6.0f / float(dims_in[l]));
        for (size_t i = 0; i < r->wsz[l]; ++i) {
            const double u = double(splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
            w[r->woff[l] + i] = float((2.0 * u - 1.0) * lim);
        }
    }
    hy_status st = rcu(cudaMalloc(&r->w, off * 4), "ranker params");
    if (st == HY_OK) st = rcu(cudaMalloc(&r->gw, off * 4), "ranker params");
    if (st == HY_OK) st = rcu(cudaMalloc(&r->m1, off * 4), "ranker params");
    if (st == HY_OK) st = rcu(cudaMalloc(&r->m2, off * 4), "ranker params");
    if (st == HY_OK) st = rcu(cudaMemcpy(r->w, w.data(), off * 4, cudaMemcpyHostToDevice), "upload");
    if (st == HY_OK) st = rcu(cudaMemset(r->m1, 0, off * 4), "memset");
    if (st == HY_OK) st = rcu(cudaMemset(r->m2, 0, off * 4), "memset");
    if (st != HY_OK) {
        hy_ranker_destroy(r);
        return st;
    }
    *out = r;
    return HY_OK;
}

hy_status hy_ranker_destroy(hy_ranker *r)
{
    if (!r) return HY_OK;
    float *bufs[] = {r->w, r->gw, r->m1, r->m2, r->X, r->Y, r->xb, r->yb, r->z[0], r->z[1],
                     r->z[2], r->d[0], r->d[1], r->d[2], r->out, r->dout, r->sq};
    for (float *b : bufs) cudaFree(b);
    cudaFree(r->idx);
    cudaFree(r->perm);
    cudaFree(r->sqall);
    delete r;
    return HY_OK;
}

hy_status hy_ranker_info(const hy_ranker *r, int64_t *n_params, int64_t *n_samples,
                         int *n_features, int *fitted)
{
    if (!r) return rerr(HY_ERR_ARG, "ranker is NULL");
    if (n_params) *n_params = int64_t(r->nparam);
    if (n_samples) *n_samples = r->n_samples;
    if (n_features) *n_features = r->F;
    if (fitted) *fitted = r->fitted ? 1 : 0;
    return HY_OK;
}

hy_status hy_ranker_get_params(const hy_ranker *r, float *host)
{
    if (!r || !host) return rerr(HY_ERR_ARG, "NULL argument");
    return rcu(cudaMemcpy(host, r->w, r->nparam * 4, cudaMemcpyDeviceToHost), "download");
}

hy_status hy_ranker_set_params(hy_ranker *r, const float *host)
{
    if (!r || !host) return rerr(HY_ERR_ARG, "NULL argument");
    RTRY(rcu(cudaMemcpy(r->w, host, r->nparam * 4, cudaMemcpyHostToDevice), "upload"));
    r->fitted = true;
    return HY_OK;
}

hy_status hy_ranker_predict(hy_ranker *r, const float *feat, int64_t m, float *score,
                            void *stream)
{
    if (!r || (m > 0 && (!feat || !score)) || m < 0) return rerr(HY_ERR_ARG, "bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t blk = 1 << 14;
    RTRY(ensure_act(r, blk));
    for (int64_t o = 0; o < m; o += blk) {
        const int mm = int(m - o < blk ? m - o : blk);
        RTRY(forward(r, feat + o * r->F, mm, st));
        RTRY(rcu(cudaMemcpyAsync(score + o, r->out, size_t(mm) * 4, cudaMemcpyDeviceToDevice, st),
                 "copy scores"));
    }
    return HY_OK;
}

hy_status hy_ranker_add_samples(hy_ranker *r, const float *feat, const double *g, int64_t m,
                                void *stream)
{
    if (!r || m < 0 || (m > 0 && (!feat || !g))) return rerr(HY_ERR_ARG, "bad arguments");
    if (m == 0) return HY_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (r->n_samples + m > r->cap) {
        int64_t nc = std::max<int64_t>(2 * r->cap, r->n_samples + m);
        nc = std::max<int64_t>(nc, 4096);
        float *X = nullptr, *Y = nullptr;
        RTRY(rcu(cudaMalloc(&X, size_t(nc) * r->F * 4), "ranker dataset"));
        if (cudaMalloc(&Y, size_t(nc) * 4) != cudaSuccess) {
            cudaFree(X);
            return rerr(HY_ERR_OOM, "ranker dataset");
        }
        if (r->n_samples) {
            RTRY(rcu(cudaMemcpyAsync(X, r->X, size_t(r->n_samples) * r->F * 4,
                                     cudaMemcpyDeviceToDevice, st), "grow dataset"));
            RTRY(rcu(cudaMemcpyAsync(Y, r->Y, size_t(r->n_samples) * 4,
                                     cudaMemcpyDeviceToDevice, st), "grow dataset"));
            RTRY(rcu(cudaStreamSynchronize(st), "sync"));
        }
        cudaFree(r->X);
        cudaFree(r->Y);
        r->X = X;
        r->Y = Y;
        r->cap = nc;
    }
    RTRY(rcu(cudaMemcpyAsync(r->X + size_t(r->n_samples) * r->F, feat, size_t(m) * r->F * 4,
                             cudaMemcpyDeviceToDevice, st), "append features"));
    hy::k::k_targets<<<1, 1024, 0, st>>>(g, m, r->Y + r->n_samples); hy::count_launch();
    RTRY(rcu(cudaGetLastError(), "targets"));
    r->n_samples += m;
    return HY_OK;
}

hy_status hy_ranker_fit(hy_ranker *r, int epochs, int batch, float lr, uint64_t seed,
                        float *loss, void *stream)
{
    namespace K = hy::k;
    if (!r || epochs < 0 || batch < 1 || !(lr > 0)) return rerr(HY_ERR_ARG, "bad arguments");
    if (r->n_samples == 0) return rerr(HY_ERR_ARG, "no training samples");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    RTRY(ensure_act(r, batch));
    const int64_t m = r->n_samples;
    if (m > r->perm_cap) {
        RTRY(rcu(cudaStreamSynchronize(st), "sync"));
        cudaFree(r->perm);
        cudaFree(r->sqall);
        r->perm = nullptr;
        r->sqall = nullptr;
        r->perm_cap = 0;
        RTRY(rcu(cudaMalloc(&r->perm, size_t(m) * 4), "ranker order"));
        RTRY(rcu(cudaMalloc(&r->sqall, size_t(m) * 4), "ranker order"));
        r->perm_cap = m;
    }
    std::vector<int32_t> perm(m);
    std::vector<float> sq(m);
    uint64_t s = seed;
    double last = 0.0;
    const int H = r->H, F = r->F;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t i = 0; i < m; ++i) perm[i] = int32_t(i);
        for (int64_t i = m - 1; i > 0; --i) {   // Fisher-Yates
            const int64_t j = int64_t(splitmix(s) % uint64_t(i + 1));
            std::swap(perm[i], perm[j]);
        }
        // one upload of the epoch's order; minibatches then run without a
        // host round trip
        RTRY(rcu(cudaMemcpyAsync(r->perm, perm.data(), size_t(m) * 4, cudaMemcpyHostToDevice, st),
                 "upload order"));
        for (int64_t o = 0; o < m; o += batch) {
            const int mb = int(std::min<int64_t>(batch, m - o));
            const int32_t *bidx = r->perm + o;
            const unsigned gx = unsigned((int64_t(mb) * F + 255) / 256);
            K::k_gather_rows<<<gx, 256, 0, st>>>(r->X, bidx, mb, F, r->xb); hy::count_launch();
            K::k_gather_rows<<<unsigned((mb + 255) / 256), 256, 0, st>>>(r->Y, bidx, mb, 1, r->yb); hy::count_launch();
            RTRY(forward(r, r->xb, mb, st));
            K::k_mse<<<unsigned((mb + 255) / 256), 256, 0, st>>>(r->out, r->yb, mb, r->dout, r->sq); hy::count_launch();
            // layer 3 (H -> 1): dW3 = dout^T z2, db3 = sum dout, d2 = dout W3
            RTRY(rcu(K::gemm<true, false>(r->dout, r->z[2], r->gw + r->woff[3], 1, H, mb, 1, H, H,
                                          nullptr, false, st), "mlp backward"));
            K::k_colsum<<<1, 256, 0, st>>>(r->dout, mb, 1, r->gw + r->boff[3]); hy::count_launch();
            RTRY(rcu(K::gemm<false, false>(r->dout, r->w + r->woff[3], r->d[2], mb, H, 1, 1, H, H,
                                           nullptr, false, st), "mlp backward"));
            for (int l = 2; l >= 0; --l) {
                const int64_t cnt = int64_t(mb) * H;
                K::k_relu_bwd<<<unsigned((cnt + 255) / 256), 256, 0, st>>>(r->d[l], r->z[l], cnt); hy::count_launch();
                const float *xin = l == 0 ? r->xb : r->z[l - 1];
                const int fin = l == 0 ? F : H;
                RTRY(rcu(K::gemm<true, false>(r->d[l], xin, r->gw + r->woff[l], H, fin, mb, H, fin,
                                              fin, nullptr, false, st), "mlp backward"));
                K::k_colsum<<<unsigned((H + 31) / 32), 256, 0, st>>>(r->d[l], mb, H,
                                                                     r->gw + r->boff[l]); hy::count_launch();
                if (l > 0)
                    RTRY(rcu(K::gemm<false, false>(r->d[l], r->w + r->woff[l], r->d[l - 1], mb, H,
                                                   H, H, H, H, nullptr, false, st),
                             "mlp backward"));
            }
            ++r->step;
            const float b1t = std::pow(0.9f, float(r->step)), b2t = std::pow(0.999f, float(r->step));
            K::k_adam<<<unsigned((r->nparam + 255) / 256), 256, 0, st>>>(
                r->w, r->gw, r->m1, r->m2, int64_t(r->nparam), lr, b1t, b2t); hy::count_launch();
            RTRY(rcu(cudaGetLastError(), "mlp step"));
            if (ep == epochs - 1)
                RTRY(rcu(cudaMemcpyAsync(r->sqall + o, r->sq, size_t(mb) * 4,
                                         cudaMemcpyDeviceToDevice, st), "loss"));
        }
    }
    if (epochs > 0) {
        RTRY(rcu(cudaMemcpyAsync(sq.data(), r->sqall, size_t(m) * 4, cudaMemcpyDeviceToHost, st),
                 "loss readback"));
        RTRY(rcu(cudaStreamSynchronize(st), "sync"));
        double tot = 0.0;
        for (int64_t i = 0; i < m; ++i) tot += sq[i];
        last = tot / double(m);
    }
    RTRY(rcu(cudaStreamSynchronize(st), "sync"));
    r->fitted = true;
    if (loss) *loss = float(last);
    return HY_OK;
}

hy_status hy_ranker_topk(const float *score, int64_t m, int64_t k, int32_t *idx, void *stream)
{
    if (m < 0 || k < 0 || k > m || (m > 0 && (!score || !idx)))
        return rerr(HY_ERR_ARG, "bad arguments");
    if (m > hy::k::kTopKMax) return rerr(HY_ERR_UNSUPPORTED, "top-k supports at most 8192 scores");
    if (k == 0) return HY_OK;
    const size_t smem = size_t(hy::k::kTopKMax) * 8;
    cudaError_t e = cudaFuncSetAttribute(hy::k::k_topk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return rcu(e, "top-k attribute");
    hy::k::k_topk<<<1, 1024, smem, static_cast<cudaStream_t>(stream)>>>(score, int(m), int(k), idx); hy::count_launch();
    return rcu(cudaGetLastError(), "top-k");
}

}  // extern "C"
