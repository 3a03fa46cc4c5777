// hy_adapt.cpp -- the ADAPT-VQE driver (include/hyperion.h, "ADAPT-VQE
// driver").  Host code only: it is a client of the library's own C ABI
// (hy_apply_excitation, hy_apply_h, hy_energy, hy_pool_gradients), so every
// sweep over the state runs in the CUDA kernels; this file holds the loop,
// the BFGS optimiser and the bookkeeping.
//
// Paper: ADAPT-VQE as described in the Numerical performance subsection
// (screen the pool by energy gradient, append the largest, re-optimise all
// parameters), with the energy of Eq. "ev" prepared from the Hartree-Fock
// state by the ansatz's exponentiated fermionic operators.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "hyperion.h"
#include "hy_internal.h"

namespace {

double now_s()
{
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

size_t esize(hy_dtype dt) { return dt == HY_F64 ? 8 : 4; }

}  // namespace

struct hy_adapt {
    const hy_ham *h = nullptr;
    const hy_pool *p = nullptr;
    hy_ranker *ranker = nullptr;
    int warm_iters = 0, epochs = 0, refresh_every = 0;
    // epochs of ranker training owed: fits run when the ranker is next used
    // (iterations that screen exactly only collect its samples)
    int fit_pending = 0;
    bool fitted_once = false;
    float *d_feat = nullptr, *d_extra = nullptr, *d_score = nullptr;
    double *d_gp = nullptr;       // proposals' exact gradients [M]
    std::vector<double> last_g;   // |g_k| when last screened (-1: never)
    std::vector<int> age;         // iterations since last screened
    std::vector<float> count, thsum;
    double last_max = 0.0;        // largest |g| of the most recent screen
    hy_adapt_config cfg{};
    int64_t N = 0, K = 0;
    int n_orb = 0;
    std::vector<int32_t> p_desc_v;       // [K][11] pool descriptors (host)
    const int32_t *p_desc = nullptr;
    // device state: [dtype][psi, sigma, phi, lam]
    void *buf[2][4] = {{nullptr, nullptr, nullptr, nullptr},
                       {nullptr, nullptr, nullptr, nullptr}};
    double *d_g = nullptr;        // screen gradients [K]
    double *d_ga = nullptr;       // ansatz gradients [max_iter]
    double *d_e = nullptr;        // scalar
    int32_t *d_ops = nullptr;     // ansatz ops [max_iter]
    int32_t *d_prop = nullptr;    // proposals [K]
    std::vector<int64_t> ops;
    std::vector<double> theta;
    std::vector<double> hinv;     // inverse-Hessian estimate (len x len)
    bool hinv_fresh = true;       // hinv is the identity (not yet scaled)
    // which (dtype, theta) the psi/sigma buffers currently hold
    int valid_dt = -1;
    std::vector<double> valid_theta;
    // the last iteration was refined in double: screen its double state
    bool screen_f64_next = false;
    // the last optimisation ran in double until its own stopping rule
    // (gradient below gtol, or no representable decrease), and theta has not
    // changed since: a double refinement would stop at once with this energy
    bool f64_settled = false;
    double e_f64_settled = 0.0;
    // sigma = H psi holds every component (false after an evaluation that
    // formed it on psi's support only, through the support Hamiltonian)
    bool sigma_full[2] = {false, false};
    // sigma was formed on psi's support only (rows of the support): the
    // reverse sweep then keeps lambda on that support too
    bool sig_support[2] = {false, false};
    bool want_full_sigma = false;        // the next evaluation must form all of sigma
    int evals = 0, evals64 = 0;
    int iter = 0;
    int64_t h2d = 0, d2h = 0;     // bytes copied host <-> device so far
    // sparse path: psi and phi of each precision as sparse vectors over
    // buf[dt][0] and buf[dt][2]; clean: the dense array and bitmap hold
    // exactly the listed support (false after dense use or an overflow)
    // sparse vectors of each precision over [psi, phi, lam, sigma] =
    // buf[dt][0, 2, 3, 1]; clean: array and bitmap hold exactly the listed
    // support (false after dense use or an overflow)
    hy::SparseState *ss[2][4] = {{nullptr, nullptr, nullptr, nullptr},
                                 {nullptr, nullptr, nullptr, nullptr}};
    bool ss_clean[2][4] = {{false, false, false, false}, {false, false, false, false}};
    bool sig_listed[2] = {false, false};   // sigma's support is listed in ss[dt][3]
    int64_t sig_count[2] = {0, 0};         // its size at the last evaluation
    // growth of lambda's support over the backward rotations, as last seen
    // (the rotations list partners: each constituent can double it)
    double lam_growth[2] = {2.0, 2.0};
    int64_t conn = 0;             // couplings per determinant (bounds sigma's support)
    // ansatz length at which a precision's support list overflowed: the
    // dense sweeps serve that precision while the ansatz is this long
    size_t sparse_fail_len[2] = {SIZE_MAX, SIZE_MAX};
    int64_t sparse_m = -1;        // support of the last evaluated state (-1: dense)
    int64_t sparse_m_last[2] = {1, 1};   // last sparse support of each precision
    bool prep_small = false;             // the last evaluation prepared psi in one CTA
                                         // (angles on the device for its theta)
    double *d_n2 = nullptr;       // tracked squared norm (float renormalisation)
    double *h_cs = nullptr, *d_cs = nullptr;   // cos, sin of the ansatz angles (pinned / device)
    int32_t *h_ops = nullptr;                  // pinned staging of the ansatz's operators
    // pinned readback slots of an evaluation (energy, support counts, the
    // ansatz gradient): its copies are queued and waited for once
    void *h_pin = nullptr;
    double *h_e = nullptr, *h_g = nullptr;
    int64_t *h_cnt = nullptr;
    // pinned staging of the screen's gradients [K] and the ranker's extra
    // features [K][4]
    double *h_gs = nullptr;
    float *h_extra = nullptr;
    double *d_one = nullptr;      // device constants {1.0, 1.0f}
    // support program of the current ansatz (small supports): compiled from
    // the first structural preparation after an append, then run by every
    // evaluation and forward gradient of the iteration
    hy::SupportProgram *prog = nullptr;
    int prog_max_steps = 0;
    std::vector<int64_t> prog_ops;       // the ansatz it was compiled for
    int64_t prog_m = 0;                  // its support size
    bool prog_grad_ok = false;           // its tables serve the forward gradient
    bool prog_support[2] = {false, false};   // ss[dt][0] lists the program's support
    // an optimiser's evaluation on a compiled program also queues that
    // point's forward gradient (read into h_g) behind the energy, and waits
    // only for the energy (ev_energy): the gradient that usually follows is
    // then already on its way
    bool spec_pending = false;
    hy_dtype spec_dt = HY_F64;
    std::vector<double> spec_theta;
    cudaEvent_t ev_energy = nullptr;
};

namespace {

hy_status set_err(hy_status s, const char *msg);

#define HY_TRY(x)                       \
    do {                                \
        hy_status s_ = (x);             \
        if (s_ != HY_OK) return s_;     \
    } while (0)

hy_status cu(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return HY_OK;
    return set_err(e == cudaErrorMemoryAllocation ? HY_ERR_OOM : HY_ERR_CUDA, what);
}

int di(hy_dtype dt) { return dt == HY_F64 ? 0 : 1; }

// host <-> device copy on the driver's stream, counted in a->h2d / a->d2h
hy_status xfer(hy_adapt *a, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind,
               cudaStream_t st, const char *what)
{
    if (kind == cudaMemcpyHostToDevice) a->h2d += int64_t(bytes);
    if (kind == cudaMemcpyDeviceToHost) a->d2h += int64_t(bytes);
    return cu(cudaMemcpyAsync(dst, src, bytes, kind, st), what);
}

// psi <- HF determinant (index 0: lowest orbitals of both spins occupied);
// the amplitude comes from a device constant, so nothing waits on the host
hy_status set_hf(hy_adapt *a, void *psi, hy_dtype dt, cudaStream_t st)
{
    HY_TRY(cu(cudaMemsetAsync(psi, 0, size_t(a->N) * esize(dt), st), "memset"));
    const void *one = dt == HY_F64 ? static_cast<const void *>(a->d_one)
                                   : static_cast<const void *>(a->d_one + 1);
    return cu(cudaMemcpyAsync(psi, one, esize(dt), cudaMemcpyDeviceToDevice, st),
              "set HF amplitude");
}

hy_status finish_energy(hy_adapt *a, const std::vector<double> &th, hy_dtype dt)
{
    ++a->evals;
    if (dt == HY_F64) ++a->evals64;
    a->valid_dt = dt;
    a->valid_theta = th;
    return HY_OK;
}

// last support up to which one CTA prepares the sparse state and the ansatz
// is compiled into a support program (up to 12,288 elements its vectors live
// in shared memory, beyond that in an L2-resident global scratch); the
// general single-CTA forward gradient (no program) stays with supports up to
// kForwardSmall, above which the reverse sweep serves
const int64_t kPrepareSmall = 65536;
const int64_t kForwardSmall = 12288;
// the support Hamiltonian is built when it holds at most this many entries
// (12 bytes each)
const int64_t kHssMaxEntries = int64_t(1) << 29;
// cost of the scatter H psi per listed amplitude over the dense sweep's cost
// per determinant, [double, float]: both scale with the couplings per
// determinant.  Measured on a GB300 at 32 qubits: the scatter's atomics into
// a sigma beyond L2 take ~175-235 ns per listed amplitude in double and ~170
// ns in float at supports of 1-5 M, the dense sweep 10 ns (double, FP64-rate
// bound) and 1.24 ns (float, tensor-core coupling) per determinant
const double kScatterPerDense[2] = {20.0, 135.0};

// The sparse evaluation: psi = U(theta)|HF> as a sparse vector (rotations
// cost O(support)), renormalised over its support in double (float states),
// sigma = H psi by the scatter, E = <psi|sigma> over the support.  *ok =
// false when the support list overflowed (nothing valid is left).
hy_status energy_sparse(hy_adapt *a, const std::vector<double> &th, hy_dtype dt,
                        cudaStream_t st, double *e, bool *ok, bool speculate)
{
    const int d = di(dt);
    hy::SparseState *S = a->ss[d][0], *G = a->ss[d][3];
    void *psi = a->buf[d][0], *sigma = a->buf[d][1];
    const size_t L = a->ops.size();
    a->prep_small = a->sparse_m_last[d] <= kPrepareSmall;
    // the support program serves this ansatz and S lists its support: only
    // the amplitudes change
    const bool prog_run = a->prep_small && L > 0 && a->prog && a->prog_support[d] &&
                          a->prog_ops == a->ops;
    bool prog_build = false;
    int64_t steps = 0;
    if (a->prep_small) {
        for (size_t l = 0; l < L; ++l) {
            a->h_cs[2 * l] = std::cos(th[l]);
            a->h_cs[2 * l + 1] = std::sin(th[l]);
        }
        if (L) HY_TRY(xfer(a, a->d_cs, a->h_cs, L * 2 * sizeof(double), cudaMemcpyHostToDevice, st,
                           "angles"));
    }
    if (prog_run) {
        HY_TRY(hy::prog_prepare(a->prog, S, a->p, a->d_ops, a->d_cs, int64_t(L), dt == HY_F32,
                                a->d_n2, st));
    } else if (a->prep_small) {
        // small support: the whole preparation in one launch, dating each
        // listed determinant when a support program is to be compiled from it
        if (!a->ss_clean[d][0]) HY_TRY(hy::sstate_reset(S, true, false, st));
        a->ss_clean[d][0] = true;
        a->prog_support[d] = false;
        if (a->prog && L > 0 && a->prog_ops != a->ops) {
            std::vector<int32_t> o32(a->ops.begin(), a->ops.end());
            steps = hy::prog_steps(a->p, o32.data(), int64_t(L));
            prog_build = steps <= a->prog_max_steps;
        }
        HY_TRY(hy::sstate_prepare(S, a->p, a->d_ops, a->d_cs, int64_t(L), dt == HY_F32 && L > 0,
                                  a->d_n2, st, prog_build ? hy::prog_step_len(a->prog) : nullptr));
    } else {
        a->prog_support[d] = false;
        HY_TRY(hy::sstate_reset(S, !a->ss_clean[d][0], true, st));
        a->ss_clean[d][0] = true;
        for (size_t l = 0; l < L; ++l)
            HY_TRY(hy::sstate_excite(S, a->p, a->ops[l], th[l], st));
        if (dt == HY_F32 && L > 0) {
            HY_TRY(hy::sstate_dot(S, psi, a->d_n2, st));
            HY_TRY(hy::sstate_scale_rsqrt(S, a->d_n2, st));
        }
    }
    // a new ansatz whose structural preparation has just been queued: read
    // its support's size, then compile its support program and support
    // Hamiltonian before sigma, so that already this first evaluation's sigma
    // is H_SS psi (the program's gradient flag comes back with the energy)
    bool compiled = false;
    int *h_flag = reinterpret_cast<int *>(&a->h_cnt[2]);
    if (prog_build) {
        HY_TRY(xfer(a, &a->h_cnt[0], hy::sstate_count(S), sizeof(int64_t), cudaMemcpyDeviceToHost,
                    st, "support count"));
        HY_TRY(cu(cudaStreamSynchronize(st), "sync"));
        const int64_t c0 = a->h_cnt[0];
        if (c0 > hy::sstate_cap(S)) {
            *ok = false;
            a->ss_clean[d][0] = false;
            a->prog_support[d] = false;
            return HY_OK;
        }
        if (c0 <= kPrepareSmall) {
            HY_TRY(hy::prog_compile(a->prog, S, c0, a->p, a->d_ops, int64_t(L), steps, st));
            HY_TRY(hy::prog_build_hss(a->prog, S, kHssMaxEntries, st));
            *h_flag = 1;
            HY_TRY(xfer(a, h_flag, hy::prog_flag(a->prog), sizeof(int), cudaMemcpyDeviceToHost, st,
                        "support program check"));
            a->prog_ops = a->ops;
            a->prog_m = c0;
            a->prog_grad_ok = false;            // until the flag is read
            a->prog_support[0] = a->prog_support[1] = false;
            a->prog_support[d] = true;
            compiled = true;
        }
    }
    // sigma: within a compiled ansatz the energy and the forward gradients
    // read it on psi's support only, so the support Hamiltonian forms just
    // that part; otherwise the scatter forms all of it.  List sigma's
    // support while the last support times the couplings (an upper bound)
    // fits its list; a list that still overflows (the support grew with a new
    // operator) is caught below and costs only the listing
    // (the program's forward gradient is the one that reads sigma on the
    // support only: without it the gradient reads sigma beyond the support)
    const bool use_hss = (prog_run || compiled) && hy::prog_hss_ready(a->prog) &&
                         (compiled || a->prog_grad_ok) && !a->want_full_sigma;
    // the energy and the gradients read sigma only through inner products
    // with psi and with d psi / d theta_l, vectors inside psi's support: sigma
    // is formed on that support alone, without atomics (rows of psi's list
    // against the listed determinants).  Only the screen (and the general
    // single-CTA forward gradient, which re-forms sigma in full when it
    // runs) read it beyond
    const bool on_support = !use_hss && !a->want_full_sigma && L > 0;
    const double est = double(std::max<int64_t>(a->sparse_m_last[d], 1)) * double(a->conn);
    // all of sigma: by the scatter, or by the dense sweep over psi's array
    // (zero off the support) once the scatter's atomics cost more
    const bool dense_sigma = !use_hss && !on_support &&
        double(a->sparse_m_last[d]) * kScatterPerDense[d] > double(a->N);
    const bool track = !use_hss && !on_support && !dense_sigma &&
                       est <= double(hy::sstate_cap(G));
    if (use_hss) {
        // the energy comes with the apply (psi on the support = S's list)
        a->ss_clean[d][3] = false;
        HY_TRY(hy::prog_hss_apply(a->prog, psi, sigma, dt, a->d_e, st));
    } else if (on_support) {
        HY_TRY(hy::sstate_reset(G, !a->ss_clean[d][3], false, st));
        a->ss_clean[d][3] = true;
        HY_TRY(hy::sstate_apply_h_support(S, G, sigma, st));
    } else if (dense_sigma) {
        a->ss_clean[d][3] = false;
        HY_TRY(hy_apply_h(a->h, psi, sigma, dt, st));
    } else if (track) {
        HY_TRY(hy::sstate_reset(G, !a->ss_clean[d][3], false, st));
        a->ss_clean[d][3] = true;
        HY_TRY(hy::sstate_apply_h(S, G, sigma, st));
    } else {
        a->ss_clean[d][3] = false;
        HY_TRY(hy::sstate_apply_h(S, nullptr, sigma, st));
    }
    a->sigma_full[d] = !use_hss && !on_support;
    a->sig_support[d] = on_support;
    if (!use_hss) HY_TRY(hy::sstate_dot(S, sigma, a->d_e, st));
    int64_t cnt[2] = {0, 0};
    a->h_cnt[1] = 0;
    HY_TRY(xfer(a, a->h_e, a->d_e, sizeof(double), cudaMemcpyDeviceToHost, st, "energy readback"));
    HY_TRY(xfer(a, &a->h_cnt[0], hy::sstate_count(S), sizeof(int64_t), cudaMemcpyDeviceToHost, st,
                "support count"));
    if (track)
        HY_TRY(xfer(a, &a->h_cnt[1], hy::sstate_count(G), sizeof(int64_t), cudaMemcpyDeviceToHost,
                    st, "support count"));
    // within a compiled ansatz whose tables serve the forward gradient, the
    // gradient the optimiser asks for next is this point's: queue it behind
    // the energy and wait for the energy alone
    if (speculate && prog_run && use_hss && a->prog_grad_ok && L > 0) {
        HY_TRY(cu(cudaEventRecord(a->ev_energy, st), "event"));
        HY_TRY(hy::prog_grad(a->prog, a->p, a->d_ops, a->d_cs, int64_t(L), sigma, dt,
                             dt == HY_F32 ? a->d_n2 : nullptr, a->d_ga, st));
        HY_TRY(xfer(a, a->h_g, a->d_ga, L * sizeof(double), cudaMemcpyDeviceToHost, st,
                    "gradient readback"));
        a->spec_pending = true;
        a->spec_dt = dt;
        a->spec_theta = th;
        HY_TRY(cu(cudaEventSynchronize(a->ev_energy), "sync"));
    } else {
        HY_TRY(cu(cudaStreamSynchronize(st), "sync"));
    }
    *e = a->h_e[0];
    cnt[0] = a->h_cnt[0];
    cnt[1] = a->h_cnt[1];
    *ok = cnt[0] <= hy::sstate_cap(S);
    if (!*ok) {
        a->spec_pending = false;
        a->ss_clean[d][0] = false;
        a->prog_support[d] = false;
        return HY_OK;
    }
    if (compiled) {
        a->prog_grad_ok = *h_flag == 0;
    } else if (a->prep_small && !prog_run && L > 0 && a->prog_ops == a->ops) {
        // a structural preparation of the compiled ansatz lists the same support
        a->prog_support[d] = cnt[0] == a->prog_m;
    }
    // sigma's values are complete either way; an overflowing list only
    // leaves its support unlisted (and its array to be cleared in full)
    a->sig_listed[d] = (track && cnt[1] <= hy::sstate_cap(G)) || on_support;
    a->sig_count[d] = on_support ? cnt[0] : cnt[1];
    if (track && !a->sig_listed[d]) a->ss_clean[d][3] = false;
    hy::sstate_set_hint(S, cnt[0]);
    if (a->sig_listed[d]) hy::sstate_set_hint(G, a->sig_count[d]);
    a->sparse_m = cnt[0];
    a->sparse_m_last[d] = cnt[0];
    return HY_OK;
}

// psi = U(theta) |HF>, sigma = H psi, returns E = <psi|sigma>; speculate:
// the caller will most likely ask for the gradient at th next
hy_status energy(hy_adapt *a, const std::vector<double> &th, hy_dtype dt,
                 cudaStream_t st, double *e, bool speculate = false)
{
    const int d = di(dt);
    a->sparse_m = -1;
    a->prep_small = false;
    a->spec_pending = false;
    if (a->cfg.sparse && a->ops.size() < a->sparse_fail_len[d]) {
        bool ok = false;
        HY_TRY(energy_sparse(a, th, dt, st, e, &ok, speculate));
        if (ok) return finish_energy(a, th, dt);
        a->sparse_fail_len[d] = a->ops.size();
    }
    void *psi = a->buf[d][0], *sigma = a->buf[d][1];
    a->ss_clean[d][0] = false;
    a->ss_clean[d][3] = false;
    a->sig_listed[d] = false;
    a->sig_support[d] = false;
    a->prog_support[d] = false;
    HY_TRY(set_hf(a, psi, dt, st));
    // float states: the squared norm is tracked through the rotations in
    // double and the state renormalised once after the last one (equal to
    // renormalising after each: the scaling commutes with the rotations)
    const bool track = dt == HY_F32 && !a->ops.empty();
    if (track)
        HY_TRY(cu(cudaMemcpyAsync(a->d_n2, a->d_one, 8, cudaMemcpyDeviceToDevice, st), "norm"));
    for (size_t l = 0; l < a->ops.size(); ++l) {
        if (track)
            HY_TRY(hy_apply_excitation_tracked(a->h, a->p, a->ops[l], th[l], psi, dt, a->d_n2, st));
        else
            HY_TRY(hy_apply_excitation(a->h, a->p, a->ops[l], th[l], psi, dt, 0, st));
    }
    if (track) HY_TRY(hy_renormalize(a->h, psi, dt, a->d_n2, st));
    HY_TRY(hy_apply_h(a->h, psi, sigma, dt, st));
    a->sigma_full[d] = true;
    HY_TRY(hy_energy(a->h, psi, sigma, dt, a->d_e, st));
    HY_TRY(xfer(a, e, a->d_e, sizeof(double), cudaMemcpyDeviceToHost, st, "energy readback"));
    HY_TRY(cu(cudaStreamSynchronize(st), "sync"));
    return finish_energy(a, th, dt);
}

// adjoint gradient at the point of the last energy() call in dt
hy_status gradient_dense(hy_adapt *a, const std::vector<double> &th, hy_dtype dt,
                         cudaStream_t st, std::vector<double> &g)
{
    const size_t j = a->ops.size(), es = esize(dt);
    const int d = di(dt);
    void *psi = a->buf[d][0], *sigma = a->buf[d][1];
    void *phi = a->buf[d][2], *lam = a->buf[d][3];
    a->ss_clean[d][1] = false;
    a->ss_clean[d][2] = false;
    HY_TRY(cu(cudaMemcpyAsync(phi, psi, size_t(a->N) * es, cudaMemcpyDeviceToDevice, st), "copy"));
    HY_TRY(cu(cudaMemcpyAsync(lam, sigma, size_t(a->N) * es, cudaMemcpyDeviceToDevice, st), "copy"));
    for (size_t l = j; l-- > 0;) {
        HY_TRY(hy::pool_gradients_unchecked(a->h, a->p, phi, lam, a->d_ops + l, 1, a->d_ga + l, dt, st));
        if (l == 0) break;
        HY_TRY(hy_apply_excitation(a->h, a->p, a->ops[l], -th[l], phi, dt, 0, st));
        HY_TRY(hy_apply_excitation(a->h, a->p, a->ops[l], -th[l], lam, dt, 0, st));
    }
    HY_TRY(xfer(a, g.data(), a->d_ga, j * sizeof(double), cudaMemcpyDeviceToHost, st,
                "gradient readback"));
    return cu(cudaStreamSynchronize(st), "sync");
}

// sigma = H psi in full for the sparse psi of the last evaluation in dt (whose
// sigma was formed on psi's support only), by the scatter
hy_status full_sigma_sparse(hy_adapt *a, int d, cudaStream_t st)
{
    hy::SparseState *S = a->ss[d][0], *G = a->ss[d][3];
    HY_TRY(hy::sstate_reset(G, !a->ss_clean[d][3], false, st));
    a->ss_clean[d][3] = false;
    HY_TRY(hy::sstate_apply_h(S, nullptr, a->buf[d][1], st));
    a->sig_support[d] = false;
    a->sig_listed[d] = false;
    a->sigma_full[d] = true;
    return HY_OK;
}

// adjoint gradient at the point of the last energy() call in dt:
// dE/dtheta_l = 2 <lam_l | A_l phi_l> with phi_l = U_l..U_1|HF> and lam_l =
// U_{l+1}^dag..U_L^dag H psi, both walked back from (psi, H psi).  After a
// sparse evaluation phi stays a sparse vector (its side costs O(support))
// and lam, which H spreads over most determinants, is rotated densely.
hy_status gradient(hy_adapt *a, const std::vector<double> &th, hy_dtype dt,
                   cudaStream_t st, std::vector<double> &g)
{
    const size_t j = a->ops.size(), es = esize(dt);
    g.assign(j, 0.0);
    if (j == 0) return HY_OK;
    if (a->sparse_m < 0) return gradient_dense(a, th, dt, st, g);
    const int d = di(dt);
    hy::SparseState *P = a->ss[d][0], *F = a->ss[d][1], *L = a->ss[d][2], *G = a->ss[d][3];
    if (a->spec_pending && a->spec_dt == dt && a->spec_theta == th && a->prog_ops == a->ops) {
        // queued with the energy at this point
        a->spec_pending = false;
        HY_TRY(cu(cudaStreamSynchronize(st), "sync"));
        std::copy(a->h_g, a->h_g + j, g.begin());
        return HY_OK;
    }
    if (a->prep_small && a->sparse_m <= kPrepareSmall && a->prog && a->prog_grad_ok &&
        a->prog_support[d] && a->prog_ops == a->ops) {
        // the support program's forward gradient: one CTA per angle
        HY_TRY(hy::prog_grad(a->prog, a->p, a->d_ops, a->d_cs, int64_t(j), a->buf[d][1], dt,
                             dt == HY_F32 ? a->d_n2 : nullptr, a->d_ga, st));
        HY_TRY(xfer(a, a->h_g, a->d_ga, j * sizeof(double), cudaMemcpyDeviceToHost, st,
                    "gradient readback"));
        HY_TRY(cu(cudaStreamSynchronize(st), "sync"));
        std::copy(a->h_g, a->h_g + j, g.begin());
        return HY_OK;
    }
    if (a->prep_small && a->sparse_m <= kForwardSmall) {
        // small support: the whole gradient in forward mode in one launch.
        // Its vectors may leave the support (a generator of several
        // constituents from an element a later constituent listed), so it
        // reads sigma in full
        if (!a->sigma_full[d]) HY_TRY(full_sigma_sparse(a, d, st));
        if (!a->ss_clean[d][1]) HY_TRY(hy::sstate_reset(F, true, false, st));
        if (!a->ss_clean[d][2]) HY_TRY(hy::sstate_reset(L, true, false, st));
        a->ss_clean[d][1] = a->ss_clean[d][2] = true;
        HY_TRY(hy::sstate_grad_forward(F, L, a->p, a->d_ops, a->d_cs, int64_t(j), a->buf[d][1],
                                       dt == HY_F32 ? a->d_n2 : nullptr, a->d_ga, st));
        int64_t cnt[2] = {0, 0};
        HY_TRY(xfer(a, g.data(), a->d_ga, j * sizeof(double), cudaMemcpyDeviceToHost, st,
                    "gradient readback"));
        HY_TRY(xfer(a, &cnt[0], hy::sstate_count(F), sizeof(int64_t), cudaMemcpyDeviceToHost, st,
                    "support count"));
        HY_TRY(xfer(a, &cnt[1], hy::sstate_count(L), sizeof(int64_t), cudaMemcpyDeviceToHost, st,
                    "support count"));
        HY_TRY(cu(cudaStreamSynchronize(st), "sync"));
        if (cnt[0] <= hy::sstate_cap(F) && cnt[1] <= hy::sstate_cap(L)) return HY_OK;
        if (cnt[0] > hy::sstate_cap(F)) a->ss_clean[d][1] = false;
        if (cnt[1] > hy::sstate_cap(L)) a->ss_clean[d][2] = false;
        return gradient_dense(a, th, dt, st, g);
    }
    // sigma formed by the support Hamiltonian for a program whose own
    // gradient cannot serve: the reverse sweep needs it in full
    if (!a->sigma_full[d] && !a->sig_support[d]) HY_TRY(full_sigma_sparse(a, d, st));
    void *sigma = a->buf[d][1], *lam = a->buf[d][3];
    HY_TRY(hy::sstate_reset(F, !a->ss_clean[d][1], false, st));
    a->ss_clean[d][1] = true;
    HY_TRY(hy::sstate_copy(F, P, st));
    hy::sstate_set_hint(F, a->sparse_m);
    // lambda starts as sigma: a sparse copy when sigma's support is listed
    // and, grown as last seen, still fits lambda's list.  When sigma was
    // formed on psi's support S only, lambda stays on S (closed rotations):
    // dE/dtheta_l = 2 <lam_l | A_l phi_l> reads lam_l only where A_l phi_l
    // lives, inside S_l (the support after l operators), and lam_l there is
    // U_{l+1}^T applied to lam_{l+1} on S_{l+1}, which holds every partner of
    // S_l under operator l + 1 -- values on S off S_l are never read
    const bool lam_closed = a->sig_support[d];
    const bool lam_sparse = lam_closed || (a->sig_listed[d] &&
        double(a->sig_count[d]) * a->lam_growth[d] <= double(hy::sstate_cap(L)));
    if (lam_sparse) {
        HY_TRY(hy::sstate_reset(L, !a->ss_clean[d][2], false, st));
        a->ss_clean[d][2] = true;
        HY_TRY(hy::sstate_copy(L, G, st));
        if (lam_closed) hy::sstate_set_hint(L, a->sig_count[d]);
    } else {
        a->ss_clean[d][2] = false;
        HY_TRY(cu(cudaMemcpyAsync(lam, sigma, size_t(a->N) * es, cudaMemcpyDeviceToDevice, st),
                  "copy"));
    }
    for (size_t l = j; l-- > 0;) {
        HY_TRY(hy::sstate_gradients(F, lam, a->p, a->d_ops + l, 1, a->sparse_m, a->d_ga + l, st));
        if (l == 0) break;
        // phi_{l-1} = U_l^T phi_l lies inside S_{l-1}, within psi's support S:
        // a partner off S holds an exact zero and would receive one, so phi's
        // rotations keep S's list (closed) instead of listing such partners
        HY_TRY(hy::sstate_excite(F, a->p, a->ops[l], -th[l], st, true));
        if (lam_sparse)
            HY_TRY(hy::sstate_excite(L, a->p, a->ops[l], -th[l], st, lam_closed));
        else
            HY_TRY(hy_apply_excitation(a->h, a->p, a->ops[l], -th[l], lam, dt, 0, st));
    }
    int64_t cnt[2] = {0, 0};
    HY_TRY(xfer(a, g.data(), a->d_ga, j * sizeof(double), cudaMemcpyDeviceToHost, st,
                "gradient readback"));
    HY_TRY(xfer(a, &cnt[0], hy::sstate_count(F), sizeof(int64_t), cudaMemcpyDeviceToHost, st,
                "support count"));
    if (lam_sparse)
        HY_TRY(xfer(a, &cnt[1], hy::sstate_count(L), sizeof(int64_t), cudaMemcpyDeviceToHost, st,
                    "support count"));
    HY_TRY(cu(cudaStreamSynchronize(st), "sync"));
    const bool f_ok = cnt[0] <= hy::sstate_cap(F), l_ok = cnt[1] <= hy::sstate_cap(L);
    if (lam_sparse && !lam_closed) {
        hy::sstate_set_hint(L, cnt[1]);
        a->lam_growth[d] = l_ok ? std::max(1.0, 1.25 * double(cnt[1]) /
                                                    double(std::max<int64_t>(a->sig_count[d], 1)))
                                : 4.0 * a->lam_growth[d];
    }
    if (f_ok && l_ok) return HY_OK;
    if (!f_ok) a->ss_clean[d][1] = false;
    if (!l_ok) a->ss_clean[d][2] = false;
    return gradient_dense(a, th, dt, st, g);   // a list overflowed: redo densely
}

// the ansatz's operators to the device, staged in pinned memory.  With wait
// false the copy is only queued: the caller's kernels that read them run on
// the same stream, and the staging slot is not written again before the
// stream has been synchronised (an ADAPT step's evaluations synchronise it)
hy_status upload_ops(hy_adapt *a, cudaStream_t st, bool wait = true)
{
    if (a->ops.empty()) return HY_OK;
    for (size_t l = 0; l < a->ops.size(); ++l) a->h_ops[l] = int32_t(a->ops[l]);
    HY_TRY(xfer(a, a->d_ops, a->h_ops, a->ops.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st,
                "upload ops"));
    return wait ? cu(cudaStreamSynchronize(st), "sync") : HY_OK;
}

double dotv(const std::vector<double> &x, const std::vector<double> &y)
{
    double s = 0.0;
    for (size_t i = 0; i < x.size(); ++i) s += x[i] * y[i];
    return s;
}

double maxabs(const std::vector<double> &x)
{
    double m = 0.0;
    for (double v : x) m = std::max(m, std::fabs(v));
    return m;
}

// remember the exact |g_k| of the operators just screened; age the rest
void note_screen(hy_adapt *a, const std::vector<int64_t> &ids, const std::vector<double> &gv)
{
    for (auto &x : a->age) ++x;
    double mx = 0.0;
    for (size_t i = 0; i < ids.size(); ++i) {
        a->last_g[ids[i]] = std::fabs(gv[i]);
        a->age[ids[i]] = 0;
        mx = std::max(mx, std::fabs(gv[i]));
    }
    a->last_max = mx;
}

// per-operator extra ranker features from the driver's bookkeeping
hy_status upload_extra(hy_adapt *a, cudaStream_t st)
{
    // stale |g| relative to the most recent screen's largest |g| (not the
    // largest ever seen, which early iterations dominate)
    const double mx = a->last_max;
    float *ex = a->h_extra;   // pinned: the previous upload finished with its iteration
    for (int64_t k = 0; k < a->K; ++k) {
        const double lg = a->last_g[k];
        ex[4 * k + 0] = lg < 0.0 ? -12.0f : float(std::log10(lg / (mx > 0 ? mx : 1.0) + 1e-12));
        ex[4 * k + 1] = float(std::min(a->age[k], 50)) / 10.0f;
        ex[4 * k + 2] = a->count[k];
        ex[4 * k + 3] = a->thsum[k];
    }
    for (size_t l = 0; l < a->ops.size(); ++l) ex[4 * a->ops[l] + 3] = 0.0f;
    for (size_t l = 0; l < a->ops.size(); ++l) ex[4 * a->ops[l] + 3] += float(std::fabs(a->theta[l]));
    return xfer(a, a->d_extra, ex, size_t(a->K) * 16, cudaMemcpyHostToDevice, st,
                "upload extra features");
}

// Relative energy decrease below which an accepted double-precision step is
// rounding noise: the Armijo test cannot reject such steps once its
// threshold e + c * alpha * slope rounds to e, and following them only
// spends evaluations.
const double kStall64 = std::ldexp(1.0, -50);

// (pool size) x (nonzero amplitudes) below which the exact sparse screen
// replaces the ranker's proposals (~10 ms on a GB300, the cost of the
// ranker's feature pass at 32 qubits)
const double kExactScreenWork = 5e9;
const double kCollectFactor = 64.0;
// the mixed-precision driver optimises in float from this many nonzero
// amplitudes on; below it an evaluation is latency-bound and costs the same
// in either precision, so it optimises in double directly and needs no
// refinement
const int64_t kFloatFrom = int64_t(1) << 20;

// cost of one atomic add of the list-based touched weights in amplitudes of
// the dense pass (the rule that picks sigma's list).  Measured at 32 qubits
// on sigma supports of 0.15-2.1 M: about 12 ps per add, against 10-15 ps per
// amplitude of the dense pass (compute-bound once most tiles are nonzero)
const double kListAddCost = 1.0;


// BFGS with backtracking (Armijo) line search on E(theta) in dt, starting
// from a->theta and a->hinv; updates both.  *e_out = final energy.  With
// stall > 0 the run also stops after an accepted step whose decrease is
// below stall * |E| (the rounding floor of a float evaluation, where further
// steps only follow noise).
hy_status bfgs(hy_adapt *a, hy_dtype dt, double gtol, int max_steps, cudaStream_t st,
               double *e_out, double stall = 0.0, bool *settled = nullptr)
{
    bool done = false;   // stopped by the gradient, the line search or a stall
    const size_t j = a->ops.size();
    std::vector<double> x = a->theta, g, gn, pdir(j), xn(j), s(j), y(j), Hy(j);
    double e = 0.0;
    HY_TRY(energy(a, x, dt, st, &e, true));
    HY_TRY(gradient(a, x, dt, st, g));
    std::vector<double> &H = a->hinv;
    const int ev_start = a->evals;
    // a full step's trial point queues its gradient with its energy unless
    // the last full step was rejected (then it most likely is again);
    // backtracked trial points always do
    bool full_ok = true;
    for (int it = 0; it < max_steps; ++it) {
        if (maxabs(g) < gtol) {
            done = true;
            break;
        }
        if (a->evals - ev_start >= a->cfg.max_evals) break;
        for (size_t r = 0; r < j; ++r) {
            double v = 0.0;
            for (size_t c = 0; c < j; ++c) v -= H[r * j + c] * g[c];
            pdir[r] = v;
        }
        double slope = dotv(g, pdir);
        if (!(slope < 0.0)) {   // not a descent direction: restart from I
            std::fill(H.begin(), H.end(), 0.0);
            for (size_t r = 0; r < j; ++r) H[r * j + r] = 1.0;
            for (size_t r = 0; r < j; ++r) pdir[r] = -g[r];
            slope = -dotv(g, g);
            a->hinv_fresh = true;
        }
        double alpha = 1.0, en = 0.0;
        bool ok = false, tried = false;
        for (int ls = 0; ls < 40; ++ls) {
            // a step whose predicted decrease is below the precision's
            // rounding floor cannot be told apart from noise: stop trying
            if (stall > 0.0 && -alpha * slope < stall * std::fabs(e)) break;
            for (size_t r = 0; r < j; ++r) xn[r] = x[r] + alpha * pdir[r];
            HY_TRY(energy(a, xn, dt, st, &en, ls > 0 || full_ok));
            tried = true;
            if (en <= e + 1e-4 * alpha * slope) {
                ok = true;
                if (ls == 0) full_ok = true;
                break;
            }
            if (ls == 0) full_ok = false;
            alpha *= 0.5;
        }
        if (!ok) {
            // no decrease representable in this precision: keep x (the
            // buffers hold x's state unless a trial point was evaluated)
            if (tried) HY_TRY(energy(a, x, dt, st, &e));
            done = true;
            break;
        }
        HY_TRY(gradient(a, xn, dt, st, gn));
        for (size_t r = 0; r < j; ++r) {
            s[r] = xn[r] - x[r];
            y[r] = gn[r] - g[r];
        }
        const double sy = dotv(s, y);
        if (sy > 1e-300) {
            if (a->hinv_fresh) {   // scale an identity start (Nocedal & Wright 6.20)
                const double sc = sy / dotv(y, y);
                for (size_t r = 0; r < j; ++r) H[r * j + r] = sc;
                a->hinv_fresh = false;
            }
            for (size_t r = 0; r < j; ++r) {
                double v = 0.0;
                for (size_t c = 0; c < j; ++c) v += H[r * j + c] * y[c];
                Hy[r] = v;
            }
            const double yHy = dotv(y, Hy), rho = 1.0 / sy;
            for (size_t r = 0; r < j; ++r)
                for (size_t c = 0; c < j; ++c)
                    H[r * j + c] += (1.0 + rho * yHy) * rho * s[r] * s[c] -
                                    rho * (Hy[r] * s[c] + s[r] * Hy[c]);
        }
        const bool stalled = stall > 0.0 && (e - en) < stall * std::fabs(e);
        x = xn;
        e = en;
        g = gn;
        if (stalled) {
            done = true;
            break;
        }
    }
    if (!done && max_steps > 0 && maxabs(g) < gtol) done = true;
    a->theta = x;
    *e_out = e;
    if (settled) *settled = done;
    return HY_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// error plumbing shared with the rest of the library (hy_api.cu)
// ---------------------------------------------------------------------------
namespace hy {
void set_last_error(const std::string &msg);
}

namespace {
hy_status set_err(hy_status s, const char *msg)
{
    hy::set_last_error(msg);
    return s;
}
}  // namespace

extern "C" {

hy_status hy_adapt_create(const hy_ham *h, const hy_pool *p, const hy_adapt_config *cfg,
                          hy_adapt **out)
{
    if (!out) return set_err(HY_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!h || !p) return set_err(HY_ERR_ARG, "handle is NULL");
    hy_adapt_config c;
    if (cfg) {
        c = *cfg;
    } else {
        c.bulk = HY_F64;
        c.max_iter = 64;
        c.eps_grad = 1e-5;
        c.gtol = 1e-9;
        c.gtol_bulk = 1e-5;
        c.max_evals = 200;
        c.refine_steps = 4;
        c.refine_every = 1;
        c.screen_top_m = 0;
        c.judge = 0;
        c.sparse = 0;
        c.sparse_cap = 0;
        c.exact_screen_work = 0.0;
        c.float_from = 0;
    }
    if ((c.bulk != HY_F64 && c.bulk != HY_F32) || c.max_iter < 1 || c.max_iter > (1 << 20) ||
        !(c.eps_grad >= 0) || !(c.gtol > 0) || !(c.gtol_bulk > 0) || c.max_evals < 1 ||
        c.refine_steps < 0 || c.refine_every < 0 || c.screen_top_m < 0 || c.sparse_cap < 0 ||
        c.float_from < 0)
        return set_err(HY_ERR_ARG, "invalid hy_adapt_config");
    hy_adapt *a = new (std::nothrow) hy_adapt;
    if (!a) return set_err(HY_ERR_OOM, "host allocation failed");
    a->h = h;
    a->p = p;
    a->cfg = c;
    hy_status s = hy_ham_info(h, &a->N, nullptr, nullptr, nullptr, nullptr);
    if (s == HY_OK) s = hy_pool_size(p, &a->K);
    if (s == HY_OK) {
        a->n_orb = hy::ham_view(h).n;
        a->p_desc_v.assign(size_t(a->K) * 11, 0);
        for (int64_t k = 0; k < a->K && s == HY_OK; ++k)
            s = hy_pool_describe(p, k, a->p_desc_v.data() + 11 * k);
        a->p_desc = a->p_desc_v.data();
    }
    auto alloc = [&](void **ptr, size_t bytes) {
        if (s != HY_OK) return;
        s = cu(cudaMalloc(ptr, bytes ? bytes : 8), "cudaMalloc (driver)");
    };
    for (int b = 0; b < 4; ++b) alloc(&a->buf[0][b], size_t(a->N) * 8);
    if (c.bulk == HY_F32)
        for (int b = 0; b < 4; ++b) alloc(&a->buf[1][b], size_t(a->N) * 4);
    alloc(reinterpret_cast<void **>(&a->d_g), size_t(a->K) * 8);
    alloc(reinterpret_cast<void **>(&a->d_ga), size_t(c.max_iter) * 8);
    alloc(reinterpret_cast<void **>(&a->d_e), 8);
    alloc(reinterpret_cast<void **>(&a->d_ops), size_t(c.max_iter) * 4);
    alloc(reinterpret_cast<void **>(&a->d_prop), size_t(a->K) * 4);
    if (c.screen_top_m > 0) {
        alloc(reinterpret_cast<void **>(&a->d_feat), size_t(a->K) * 16 * 4);
        alloc(reinterpret_cast<void **>(&a->d_extra), size_t(a->K) * 4 * 4);
        alloc(reinterpret_cast<void **>(&a->d_score), size_t(a->K) * 4);
        alloc(reinterpret_cast<void **>(&a->d_gp), size_t(a->K) * 8);
    }
    alloc(reinterpret_cast<void **>(&a->d_n2), 8);
    alloc(reinterpret_cast<void **>(&a->d_cs), size_t(c.max_iter) * 16);
    if (s == HY_OK) s = cu(cudaMallocHost(&a->h_cs, size_t(c.max_iter) * 16), "pinned angles");
    if (s == HY_OK) s = cu(cudaMallocHost(&a->h_ops, size_t(c.max_iter) * 4), "pinned ops");
    if (s == HY_OK)
        s = cu(cudaMallocHost(&a->h_pin, 64 + size_t(c.max_iter) * sizeof(double)), "pinned readbacks");
    if (s == HY_OK) s = cu(cudaMallocHost(&a->h_gs, size_t(a->K) * 8 + 8), "pinned screen");
    if (s == HY_OK && c.screen_top_m > 0)
        s = cu(cudaMallocHost(&a->h_extra, size_t(a->K) * 16 + 16), "pinned extra features");
    if (s == HY_OK) {
        a->h_e = static_cast<double *>(a->h_pin);
        a->h_cnt = reinterpret_cast<int64_t *>(static_cast<char *>(a->h_pin) + 16);
        a->h_g = reinterpret_cast<double *>(static_cast<char *>(a->h_pin) + 64);
    }
    alloc(reinterpret_cast<void **>(&a->d_one), 16);
    if (s == HY_OK)
        s = cu(cudaEventCreateWithFlags(&a->ev_energy, cudaEventDisableTiming), "event");
    if (s == HY_OK) {
        unsigned char one[16] = {};
        const double one64 = 1.0;
        const float one32 = 1.0f;
        std::memcpy(one, &one64, 8);
        std::memcpy(one + 8, &one32, 4);
        s = cu(cudaMemcpy(a->d_one, one, 16, cudaMemcpyHostToDevice), "constants");
    }
    if (c.sparse) {
        for (int d = 0; d < 2 && s == HY_OK; ++d) {
            if (!a->buf[d][0]) continue;
            // a sparse evaluation at large supports (state preparation,
            // sigma on the support, the closed reverse sweep) costs ~30 ns per
            // listed amplitude in float and ~55 ns in double at 32 qubits
            // (2.67 M listed: 77 and 150 ms), against ~250 ms for a dense
            // float evaluation (tensor-core H psi + rotations) and ~1.8 s for
            // a dense double one.  Float lists hold N/16 (near the float
            // break-even), double lists N/8 (their memory, 8 bytes an entry,
            // bounds them before the break-even)
            int64_t cap = c.sparse_cap > 0 ? std::min(c.sparse_cap, a->N)
                                           : a->N / (d == 0 ? 8 : 16);
            cap = std::max<int64_t>(cap, 1);
            const hy_dtype dt = d == 0 ? HY_F64 : HY_F32;
            for (int b = 0; b < 2 && s == HY_OK; ++b)
                s = hy::sstate_create(h, dt, a->buf[d][b == 0 ? 0 : 2], cap, &a->ss[d][b]);
            // sigma = H psi and lambda spread over <= support x couplings
            // determinants: their lists hold N/8
            const int64_t lcap = std::min(a->N, std::max(cap, a->N / 8));
            if (s == HY_OK) s = hy::sstate_create(h, dt, a->buf[d][3], lcap, &a->ss[d][2]);
            if (s == HY_OK) s = hy::sstate_create(h, dt, a->buf[d][1], lcap, &a->ss[d][3]);
        }
        a->conn = hy::ham_connections(h);
        // two constituents at most per operator
        a->prog_max_steps = int(std::min<int64_t>(254, 2 * int64_t(c.max_iter)));
        if (s == HY_OK) s = hy::prog_create(h, a->prog_max_steps, &a->prog);
    }
    a->last_g.assign(a->K, -1.0);
    a->age.assign(a->K, 0);
    a->count.assign(a->K, 0.0f);
    a->thsum.assign(a->K, 0.0f);
    if (s != HY_OK) {
        hy_adapt_destroy(a);
        return s;
    }
    *out = a;
    return HY_OK;
}

hy_status hy_adapt_destroy(hy_adapt *a)
{
    if (!a) return HY_OK;
    for (auto &row : a->buf)
        for (void *&b : row)
            if (b) cudaFree(b);
    cudaFree(a->d_g);
    cudaFree(a->d_ga);
    cudaFree(a->d_e);
    cudaFree(a->d_ops);
    cudaFree(a->d_prop);
    cudaFree(a->d_feat);
    cudaFree(a->d_extra);
    cudaFree(a->d_score);
    cudaFree(a->d_gp);
    cudaFree(a->d_n2);
    cudaFree(a->d_cs);
    if (a->h_cs) cudaFreeHost(a->h_cs);
    if (a->h_ops) cudaFreeHost(a->h_ops);
    if (a->h_pin) cudaFreeHost(a->h_pin);
    if (a->h_gs) cudaFreeHost(a->h_gs);
    if (a->h_extra) cudaFreeHost(a->h_extra);
    cudaFree(a->d_one);
    if (a->ev_energy) cudaEventDestroy(a->ev_energy);
    for (auto &row : a->ss)
        for (hy::SparseState *&x : row) hy::sstate_destroy(x);
    hy::prog_destroy(a->prog);
    delete a;
    return HY_OK;
}

hy_status hy_adapt_step(hy_adapt *a, hy_adapt_record *rec, void *stream)
{
    if (!a || !rec) return set_err(HY_ERR_ARG, "NULL argument");
    if (int64_t(a->ops.size()) >= a->cfg.max_iter)
        return set_err(HY_ERR_ARG, "ansatz is full (max_iter)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::memset(rec, 0, sizeof(*rec));
    rec->iter = a->iter;
    rec->selected = -1;
    rec->true_argmax = -1;
    rec->true_rank = -1;
    const double t0 = now_s();
    const int ev0 = a->evals, ev640 = a->evals64;
    const hy_dtype bulk = a->cfg.bulk;
    // 1. state and sigma at the current parameters.  The screen runs in the
    // bulk precision, except after an iteration refined in double: its
    // parameters are then the double-precision optimum, and screening that
    // state in double makes the selection the one plain FP64 would make
    // (float gradients differ from it by ~1e-6 relative, enough to reorder
    // near-equal operators)
    const hy_dtype sdt = a->screen_f64_next ? HY_F64 : bulk;
    if (a->valid_dt == sdt && a->valid_theta == a->theta && !a->sigma_full[di(sdt)] &&
        a->sparse_m >= 0) {
        // psi (sparse) is this point's: only sigma beyond psi's support is
        // missing (formed on the support by the last evaluation): the
        // scatter, listing sigma's support while it fits its list (as the
        // evaluation would), or the dense sweep once the scatter's atomics
        // cost more
        const int d = di(sdt);
        hy::SparseState *S = a->ss[d][0], *G = a->ss[d][3];
        const double est = double(std::max<int64_t>(a->sparse_m, 1)) * double(a->conn);
        a->sig_support[d] = false;
        a->sig_listed[d] = false;
        a->sigma_full[d] = true;
        if (double(a->sparse_m) * kScatterPerDense[d] > double(a->N)) {
            a->ss_clean[d][3] = false;
            HY_TRY(hy_apply_h(a->h, a->buf[d][0], a->buf[d][1], sdt, st));
        } else if (est <= double(hy::sstate_cap(G))) {
            HY_TRY(hy::sstate_reset(G, !a->ss_clean[d][3], false, st));
            a->ss_clean[d][3] = true;
            HY_TRY(hy::sstate_apply_h(S, G, a->buf[d][1], st));
            a->h_cnt[1] = 0;
            HY_TRY(xfer(a, &a->h_cnt[1], hy::sstate_count(G), sizeof(int64_t),
                        cudaMemcpyDeviceToHost, st, "support count"));
            HY_TRY(cu(cudaStreamSynchronize(st), "sync"));
            a->sig_listed[d] = a->h_cnt[1] <= hy::sstate_cap(G);
            a->sig_count[d] = a->h_cnt[1];
            if (a->sig_listed[d]) hy::sstate_set_hint(G, a->sig_count[d]);
            else a->ss_clean[d][3] = false;
        } else {
            HY_TRY(full_sigma_sparse(a, d, st));
        }
    } else if (a->valid_dt != sdt || a->valid_theta != a->theta || !a->sigma_full[di(sdt)]) {
        double e;
        a->want_full_sigma = true;           // the screen reads sigma beyond psi's support
        const hy_status rs = energy(a, a->theta, sdt, st, &e);
        a->want_full_sigma = false;
        HY_TRY(rs);
    }
    void *psi = a->buf[di(sdt)][0], *sigma = a->buf[di(sdt)][1];
    rec->support = a->sparse_m;
    const bool sig_listed = a->sparse_m >= 0 && a->sig_listed[di(sdt)];
    rec->sigma_support = sig_listed ? a->sig_count[di(sdt)] : -1;
    // the sparse path lists psi's support, and sigma's while it fits its list:
    // the ranker's features then take psi's touched weights from its list,
    // and sigma's while its list costs less than the pass over the dense
    // array (one atomic add per electron pair of a listed determinant,
    // counted as kListAddCost streamed amplitudes)
    const hy::SparseState *psi_list = a->sparse_m >= 0 ? a->ss[di(sdt)][0] : nullptr;
    const hy::SparseState *sigma_list =
        sig_listed && double(a->sig_count[di(sdt)]) *
                              double(hy::ham_list_weight_adds(a->h)) * kListAddCost <=
                          double(a->N)
            ? a->ss[di(sdt)][3]
            : nullptr;
    // 2. screen: full, or the ranker's top-M proposals screened exactly
    const bool ranked = a->cfg.screen_top_m > 0;
    if (ranked && !a->ranker) return set_err(HY_ERR_UNSUPPORTED, "ranked screen needs a ranker");
    // warm-up and refresh iterations select from the full screen and feed
    // (and refit) the ranker; the others screen only its proposals
    const int post = a->iter - a->warm_iters;   // ranked iteration index
    const bool refresh = ranked && post >= 0 && a->refresh_every > 0 &&
                         (post + 1) % a->refresh_every == 0;
    // in the sparse regime an exact screen over the support costs about as
    // much as the ranker's features: screen exactly (and keep feeding the
    // ranker) while K x nonzeros stays below kExactScreenWork
    const bool cheap_exact = a->sparse_m >= 0 &&
                             double(a->sparse_m) * double(a->K) <=
                                 (a->cfg.exact_screen_work == 0.0 ? kExactScreenWork
                                                                  : a->cfg.exact_screen_work);
    const double exact_work = a->cfg.exact_screen_work == 0.0 ? kExactScreenWork
                                                               : a->cfg.exact_screen_work;
    int64_t n_samples = 0;
    if (ranked) HY_TRY(hy_ranker_info(a->ranker, nullptr, &n_samples, nullptr, nullptr));
    // a ranker with nothing to learn from is not asked
    const bool use_ranker = ranked && post >= 0 && !refresh && !cheap_exact &&
                            (n_samples > 0 || a->fitted_once);
    // exact screens feed the ranker once the work of the exact screen comes
    // within kCollectFactor of the point where the ranker takes over (about
    // three iterations of support growth ahead; earlier samples would only be
    // collected, never used, and the feature pass is the costliest part of an
    // iteration with a small support)
    const bool collect = ranked && (a->sparse_m < 0 || exact_work < 0.0 ||
                                    double(a->sparse_m) * double(a->K) * kCollectFactor >
                                        exact_work);
    std::vector<double> g;
    std::vector<int64_t> cand;   // screened operators, in proposal order
    int64_t sel = -1;
    double gmax = 0.0, gn2 = 0.0;
    auto full_screen = [&]() -> hy_status {
        if (a->sparse_m >= 0)
            HY_TRY(hy::sstate_gradients(a->ss[di(sdt)][0], sigma, a->p, nullptr, a->K,
                                        a->sparse_m, a->d_g, st));
        else
            HY_TRY(hy::pool_gradients_unchecked(a->h, a->p, psi, sigma, nullptr, a->K, a->d_g, sdt, st));
        HY_TRY(xfer(a, a->h_gs, a->d_g, a->K * sizeof(double), cudaMemcpyDeviceToHost, st,
                    "screen readback"));
        HY_TRY(cu(cudaStreamSynchronize(st), "sync"));
        g.assign(a->h_gs, a->h_gs + a->K);
        return HY_OK;
    };
    auto pick = [&](const std::vector<int64_t> &ids, const std::vector<double> &gv) {
        gmax = 0.0;
        gn2 = 0.0;
        for (double v : gv) {
            gmax = std::max(gmax, std::fabs(v));
            gn2 += v * v;
        }
        sel = -1;
        for (size_t i = 0; i < gv.size(); ++i)
            if (std::fabs(gv[i]) >= gmax - 1e-12 * gmax && (sel < 0 || ids[i] < sel)) sel = ids[i];
    };
    std::vector<int64_t> all(a->K);
    for (int64_t k = 0; k < a->K; ++k) all[k] = k;
    double t_judge = 0.0;
    if (ranked) HY_TRY(upload_extra(a, st));
    rec->screen = use_ranker ? 2 : (a->sparse_m >= 0 ? 1 : 0);
    if (!use_ranker) {
        HY_TRY(full_screen());
        pick(all, g);
        if (collect) {
            HY_TRY(hy::ranker_features_impl(a->h, a->p, psi, psi_list, sigma, sigma_list, sdt,
                                            a->d_extra, a->d_feat, st));
            HY_TRY(hy_ranker_add_samples(a->ranker, a->d_feat, a->d_g, a->K, st));
            // the first fit after the warm-up, warm-started refits on the
            // grown training set at refresh iterations; both are owed until
            // the ranker's proposals are next needed
            if (a->iter + 1 >= a->warm_iters && !a->fitted_once)
                a->fit_pending = std::max(a->fit_pending, a->epochs);
            else if (refresh)
                a->fit_pending = std::max(a->fit_pending, std::max(1, a->epochs / 4));
        }
        note_screen(a, all, g);
    } else {
        const int64_t M = std::min<int64_t>(a->cfg.screen_top_m, a->K);
        if (a->fit_pending > 0 || !a->fitted_once) {
            HY_TRY(hy_ranker_fit(a->ranker, std::max(a->fit_pending, 1), 256, 1e-3f,
                                 1234 + a->iter, nullptr, st));
            a->fit_pending = 0;
            a->fitted_once = true;
        }
        HY_TRY(hy::ranker_features_impl(a->h, a->p, psi, psi_list, sigma, sigma_list, sdt,
                                        a->d_extra, a->d_feat, st));
        HY_TRY(hy_ranker_predict(a->ranker, a->d_feat, a->K, a->d_score, st));
        // proposals: the M / 4 operators with the largest Cauchy-Schwarz
        // gradient bound (feature 10, an upper bound on |g_k|), the M / 4 the
        // MLP ranks highest among those sharing two or more spatial orbitals
        // with the last appended operator (its rotation moves the gradients
        // of exactly these the most), the M / 4 with the largest stale |g_k|,
        // then the MLP's ranking until M distinct operators
        const int64_t Mb = M / 4;
        std::vector<int32_t> by_mlp(M), by_bound(Mb);
        std::vector<float> score_h(a->ops.empty() ? 0 : size_t(a->K));
        HY_TRY(hy_ranker_topk(a->d_score, a->K, M, a->d_prop, st));
        HY_TRY(xfer(a, by_mlp.data(), a->d_prop, M * 4, cudaMemcpyDeviceToHost, st,
                    "proposals readback"));
        if (!score_h.empty())
            HY_TRY(xfer(a, score_h.data(), a->d_score, size_t(a->K) * 4, cudaMemcpyDeviceToHost,
                        st, "scores readback"));
        if (Mb > 0) {
            HY_TRY(cu(cudaMemcpy2DAsync(a->d_score, sizeof(float), a->d_feat + 10,
                                        16 * sizeof(float), sizeof(float), size_t(a->K),
                                        cudaMemcpyDeviceToDevice, st), "bound column"));
            HY_TRY(hy_ranker_topk(a->d_score, a->K, Mb, a->d_prop, st));
            HY_TRY(xfer(a, by_bound.data(), a->d_prop, Mb * 4, cudaMemcpyDeviceToHost, st,
                        "proposals readback"));
        }
        HY_TRY(cu(cudaStreamSynchronize(st), "sync"));
        // the M / 4 operators with the largest |g| at their last exact
        // screen (host bookkeeping): gradients change slowly between
        // iterations, and this catches operators the MLP under-rates
        std::vector<int32_t> by_stale;
        {
            std::vector<int32_t> idx;
            for (int64_t k = 0; k < a->K; ++k)
                if (a->last_g[k] >= 0.0) idx.push_back(int32_t(k));
            const size_t ns = std::min<size_t>(size_t(Mb), idx.size());
            std::partial_sort(idx.begin(), idx.begin() + ns, idx.end(), [&](int32_t x, int32_t y) {
                return a->last_g[x] > a->last_g[y] || (a->last_g[x] == a->last_g[y] && x < y);
            });
            by_stale.assign(idx.begin(), idx.begin() + ns);
        }
        // neighbours of the last append: spatial-orbital masks of each
        // operator's constituents, two or more orbitals in common
        std::vector<int32_t> by_near;
        if (!score_h.empty()) {
            auto orbs = [&](int64_t k) {
                const int32_t *dsc = a->p_desc + 11 * k;
                uint32_t m = 0;
                for (int c = 0; c < dsc[0]; ++c)
                    for (int u = 1; u < 5; ++u) {
                        const int32_t *q = dsc + 1 + 5 * c;
                        if (q[0] == 1 && (u == 2 || u == 3)) continue;   // a single's unused slots
                        m |= 1u << (q[u] % a->n_orb);
                    }
                return m;
            };
            const uint32_t last = orbs(a->ops.back());
            std::vector<int32_t> idx;
            for (int64_t k = 0; k < a->K; ++k)
                if (__builtin_popcount(orbs(k) & last) >= 2) idx.push_back(int32_t(k));
            const size_t nn = std::min<size_t>(size_t(Mb), idx.size());
            std::partial_sort(idx.begin(), idx.begin() + nn, idx.end(), [&](int32_t x, int32_t y) {
                return score_h[x] > score_h[y] || (score_h[x] == score_h[y] && x < y);
            });
            by_near.assign(idx.begin(), idx.begin() + nn);
        }
        std::vector<int32_t> prop;
        std::vector<char> taken(a->K, 0);
        for (int32_t k : by_bound)
            if (!taken[k]) { taken[k] = 1; prop.push_back(k); }
        for (int32_t k : by_near)
            if (int64_t(prop.size()) < M && !taken[k]) { taken[k] = 1; prop.push_back(k); }
        for (int32_t k : by_stale)
            if (int64_t(prop.size()) < M && !taken[k]) { taken[k] = 1; prop.push_back(k); }
        for (int32_t k : by_mlp)
            if (int64_t(prop.size()) < M && !taken[k]) { taken[k] = 1; prop.push_back(k); }
        HY_TRY(xfer(a, a->d_prop, prop.data(), prop.size() * 4, cudaMemcpyHostToDevice, st,
                    "proposals upload"));
        const int64_t Mp = int64_t(prop.size());
        if (a->sparse_m >= 0)
            HY_TRY(hy::sstate_gradients(a->ss[di(sdt)][0], sigma, a->p, a->d_prop, Mp,
                                        a->sparse_m, a->d_gp, st));
        else
            HY_TRY(hy::pool_gradients_unchecked(a->h, a->p, psi, sigma, a->d_prop, Mp, a->d_gp, sdt, st));
        std::vector<double> gp(Mp);
        HY_TRY(xfer(a, gp.data(), a->d_gp, Mp * 8, cudaMemcpyDeviceToHost, st,
                    "proposals readback"));
        HY_TRY(cu(cudaStreamSynchronize(st), "sync"));
        cand.assign(prop.begin(), prop.end());
        pick(cand, gp);
        note_screen(a, cand, gp);
        if (std::sqrt(gn2) < a->cfg.eps_grad) {
            // fallback: never stop on the proposals alone
            rec->screen = 3;
            HY_TRY(full_screen());
            pick(all, g);
            note_screen(a, all, g);
        } else if (a->cfg.judge) {
            const double tj = now_s();
            HY_TRY(full_screen());
            double tmax = 0.0;
            int64_t targ = -1;
            for (int64_t k = 0; k < a->K; ++k)
                if (std::fabs(g[k]) > tmax + 1e-12 * tmax) {
                    tmax = std::fabs(g[k]);
                    targ = k;
                }
            rec->true_argmax = targ;
            for (size_t i = 0; i < cand.size(); ++i)
                if (cand[i] == targ) rec->true_rank = int64_t(i);
            HY_TRY(hy_ranker_add_samples(a->ranker, a->d_feat, a->d_g, a->K, st));
            t_judge = now_s() - tj;
        }
    }
    const double t1 = now_s() - t_judge;
    rec->grad_norm = std::sqrt(gn2);
    rec->t_screen = t1 - t0;
    rec->t_judge = t_judge;
    if (a->K == 0 || rec->grad_norm < a->cfg.eps_grad) {
        rec->converged = 1;
        rec->energy = rec->energy_bulk = 0.0;
        rec->t_total = now_s() - t0 - t_judge;
        return HY_OK;
    }
    rec->selected = sel;
    rec->max_grad = gmax;
    // 3. append and re-optimise
    const size_t j = a->ops.size();
    a->ops.push_back(sel);
    a->theta.push_back(0.0);
    // warm start: previous inverse Hessian, unit curvature guess for the
    // new parameter
    std::vector<double> H((j + 1) * (j + 1), 0.0);
    for (size_t r = 0; r < j; ++r)
        for (size_t c = 0; c < j; ++c) H[r * (j + 1) + c] = a->hinv[r * j + c];
    H[j * (j + 1) + j] = 1.0;
    a->hinv = H;
    if (j == 0) a->hinv_fresh = true;
    HY_TRY(upload_ops(a, st, false));
    double e = 0.0;
    a->f64_settled = false;
    if (bulk == HY_F64) {
        HY_TRY(bfgs(a, HY_F64, a->cfg.gtol, a->cfg.max_evals, st, &e, kStall64,
                    &a->f64_settled));
        a->e_f64_settled = e;
        rec->energy = rec->energy_bulk = e;
        rec->energy_bulk_err = 0.0;
    } else if ((a->sparse_m >= 0 ? a->sparse_m : a->N) * 4 <
               (a->cfg.float_from > 0 ? a->cfg.float_from : kFloatFrom)) {
        // few nonzero amplitudes (the support on the sparse path, every
        // determinant on the dense sweeps; the new operator at most
        // quadruples the support): double directly
        HY_TRY(bfgs(a, HY_F64, a->cfg.gtol, a->cfg.max_evals, st, &e, kStall64,
                    &a->f64_settled));
        a->e_f64_settled = e;
        rec->energy = rec->energy_bulk = e;
        rec->energy_bulk_err = 0.0;
        a->screen_f64_next = true;
    } else {
        double e32 = 0.0, e64 = 0.0;
        // float phase; 2^-22 |E| is a few float roundings of the energy
        HY_TRY(bfgs(a, HY_F32, a->cfg.gtol_bulk, a->cfg.max_evals, st, &e32,
                    std::ldexp(1.0, -22)));
        rec->energy_bulk = e32;
        rec->energy = e32;
        rec->energy_bulk_err = -1.0;
        a->screen_f64_next = false;
        if (a->cfg.refine_every > 0 && (a->iter + 1) % a->cfg.refine_every == 0) {
            HY_TRY(energy(a, a->theta, HY_F64, st, &e64));
            rec->energy_bulk_err = std::fabs(e32 - e64);
            if (a->cfg.refine_steps > 0)
                HY_TRY(bfgs(a, HY_F64, a->cfg.gtol, a->cfg.refine_steps, st, &e64, kStall64,
                            &a->f64_settled));
            a->e_f64_settled = e64;
            rec->energy = e64;
            a->screen_f64_next = true;
        }
    }
    rec->n_evals = a->evals - ev0;
    rec->n_evals_f64 = a->evals64 - ev640;
    rec->t_optimise = now_s() - t_judge - t1;
    rec->t_total = now_s() - t0 - t_judge;
    a->count[sel] += 1.0f;
    ++a->iter;
    return HY_OK;
}

hy_status hy_adapt_set_judge(hy_adapt *a, int judge)
{
    if (!a) return set_err(HY_ERR_ARG, "NULL argument");
    a->cfg.judge = judge ? 1 : 0;
    return HY_OK;
}

hy_status hy_adapt_set_ranker(hy_adapt *a, hy_ranker *r, int warm_iters, int epochs,
                              int refresh_every)
{
    if (!a || !r) return set_err(HY_ERR_ARG, "NULL argument");
    if (a->cfg.screen_top_m <= 0)
        return set_err(HY_ERR_ARG, "driver was created without screen_top_m");
    if (warm_iters < 1 || epochs < 1 || refresh_every < 0)
        return set_err(HY_ERR_ARG, "warm_iters and epochs must be >= 1, refresh_every >= 0");
    int fitted = 0;
    HY_TRY(hy_ranker_info(r, nullptr, nullptr, nullptr, &fitted));
    a->ranker = r;
    a->warm_iters = warm_iters;
    a->epochs = epochs;
    a->refresh_every = refresh_every;
    a->fit_pending = 0;
    a->fitted_once = fitted != 0;
    return HY_OK;
}

hy_status hy_adapt_refine(hy_adapt *a, int steps, double *e, void *stream)
{
    if (!a || !e || steps < 0) return set_err(HY_ERR_ARG, "bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (steps > 0 && a->f64_settled) {
        // the last optimisation already ended in double by its own rule at
        // this theta: refining would re-evaluate this point and stop
        *e = a->e_f64_settled;
        return HY_OK;
    }
    HY_TRY(upload_ops(a, st));
    double e64 = 0.0;
    if (steps > 0) {
        HY_TRY(bfgs(a, HY_F64, a->cfg.gtol, steps, st, &e64, kStall64, &a->f64_settled));
        a->e_f64_settled = e64;
    } else
        HY_TRY(energy(a, a->theta, HY_F64, st, &e64));
    *e = e64;
    return HY_OK;
}

hy_status hy_adapt_ansatz(const hy_adapt *a, int64_t *ops, double *thetas, int64_t cap,
                          int64_t *len)
{
    if (!a || !len) return set_err(HY_ERR_ARG, "NULL argument");
    *len = int64_t(a->ops.size());
    if (cap <= 0) return HY_OK;
    if (!ops || !thetas || cap < *len) return set_err(HY_ERR_ARG, "output too small");
    for (size_t l = 0; l < a->ops.size(); ++l) {
        ops[l] = a->ops[l];
        thetas[l] = a->theta[l];
    }
    return HY_OK;
}

hy_status hy_adapt_set_ansatz(hy_adapt *a, const int64_t *ops, const double *thetas,
                              int64_t len)
{
    if (!a || len < 0 || (len > 0 && (!ops || !thetas)))
        return set_err(HY_ERR_ARG, "bad arguments");
    if (len > a->cfg.max_iter) return set_err(HY_ERR_ARG, "ansatz longer than max_iter");
    for (int64_t l = 0; l < len; ++l)
        if (ops[l] < 0 || ops[l] >= a->K || !std::isfinite(thetas[l]))
            return set_err(HY_ERR_ARG, "invalid operator index or parameter");
    a->ops.assign(ops, ops + len);
    a->theta.assign(thetas, thetas + len);
    a->hinv.assign(size_t(len) * len, 0.0);
    for (int64_t l = 0; l < len; ++l) a->hinv[l * len + l] = 1.0;
    a->hinv_fresh = true;
    a->valid_dt = -1;
    a->screen_f64_next = false;
    a->f64_settled = false;
    a->iter = int(len);
    cudaStream_t st = nullptr;
    return upload_ops(a, st);
}

hy_status hy_adapt_evaluate(hy_adapt *a, const double *thetas, hy_dtype dt, double *e,
                            double *grad, void *stream)
{
    if (!a || !e || (!thetas && !a->ops.empty())) return set_err(HY_ERR_ARG, "NULL argument");
    if (dt != HY_F64 && !(dt == HY_F32 && a->cfg.bulk == HY_F32))
        return set_err(HY_ERR_ARG, "dtype not allocated by this driver");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<double> th(thetas, thetas + a->ops.size()), g;
    HY_TRY(upload_ops(a, st));
    HY_TRY(energy(a, th, dt, st, e));
    if (grad) {
        HY_TRY(gradient(a, th, dt, st, g));
        std::copy(g.begin(), g.end(), grad);
    }
    return HY_OK;
}

hy_status hy_adapt_io_bytes(const hy_adapt *a, int64_t *h2d, int64_t *d2h)
{
    if (!a) return set_err(HY_ERR_ARG, "NULL argument");
    if (h2d) *h2d = a->h2d;
    if (d2h) *d2h = a->d2h;
    return HY_OK;
}

hy_status hy_adapt_state(const hy_adapt *a, void *psi, hy_dtype dt, void *stream)
{
    if (!a || !psi) return set_err(HY_ERR_ARG, "NULL argument");
    if (a->valid_dt != dt) return set_err(HY_ERR_ARG, "no state of this dtype evaluated yet");
    return cu(cudaMemcpyAsync(psi, a->buf[di(dt)][0], size_t(a->N) * esize(dt),
                              cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)),
              "state copy");
}

}  // extern "C"
