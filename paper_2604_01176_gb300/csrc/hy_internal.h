// hy_internal.h -- host-side data structures shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "hyperion.h"

namespace hy {

constexpr int kMaxOrb = 16;

// Binomial coefficients C(n, k) for 0 <= n, k <= 32.
uint32_t binom(int n, int k);

// Colexicographic combinadic rank of an occupation string:
// rank = sum_i C(pos_i, i + 1) over set bits pos_0 < pos_1 < ...
uint32_t string_rank(uint32_t mask);
// Inverse of string_rank for strings of k electrons.
uint32_t string_unrank(uint32_t rank, int k);

// Packed single-excitation entry: partner string rank in bits 0..15, the
// orbital p created on the output string in bits 16..19, the orbital q
// annihilated (present in the partner) in bits 20..23, bit 31 set when the
// Jordan-Wigner sign is negative.
inline uint32_t pack_ex(uint32_t partner, int p, int q, int neg)
{
    return partner | (uint32_t(p) << 16) | (uint32_t(q) << 20) |
           (uint32_t(neg ? 1u : 0u) << 31);
}

// All strings of k electrons in n orbitals, in rank order, and for each
// output string K every single excitation K = a+_p a_q J (p in K, q not in
// K): partner J, orbitals (p, q) and sign (-1)^popcount(K & between(p, q)).
struct StringSpace {
    int n = 0, k = 0;
    int64_t N = 0;
    int nex = 0;                    // k * (n - k) entries per string
    std::vector<uint32_t> str;      // rank -> mask
    std::vector<uint32_t> ex;       // [N][nex] packed entries
    // inv[r][e]: position of string r in the entry list of its partner
    // ex[r][e] (the same excitation seen from the partner's side)
    std::vector<uint8_t> inv;       // [N][nex]
};
void build_string_space(int n, int k, StringSpace &s);

// Jordan-Wigner Pauli table grouped by X-mask.  Coefficients are kept in the
// X^x Z^z basis (real for a real Hamiltonian): H = sum_t cxz[t] X^x Z^z,
// with X^x Z^z |d> = (-1)^popcount(d & z) |d ^ x>.
struct PauliTable {
    int n_qubits = 0;
    std::vector<uint64_t> x, z;
    std::vector<double> cxz;
    std::vector<int64_t> group_off;             // n_groups + 1
    std::unordered_map<uint64_t, int64_t> group_of_x;
    // <bra|H|ket> = f_x(ket) with x = bra ^ ket.
    double element(uint64_t bra, uint64_t ket) const;
};

// Build the table from integrals; returns false with a message on failure.
bool build_pauli_table(const double *h1, const double *h2, double e_core,
                       int n, double prune_tol, PauliTable &t,
                       std::string &err);
// Check that every group has the structure of a two-body number- and
// spin-conserving Hamiltonian (what the kernel tables rely on).
bool check_two_body_structure(const PauliTable &t, int n, std::string &err);

// Kernel tables folded from the Pauli table.
//   sigma(a', b') = sum_J Ma[a'][J] psi[J][b'] + sum_J Mb[b'][J] psi[a'][J]
//     + sum_{(p,q) in X(a'), (r,s) in X(b')} sa sb V[p][q][r][s] psi[a'^pq][b'^rs]
// where X(s) holds the single excitations (p in s created, q annihilated)
// and the diagonal pairs (p, p) for occupied p.
struct CsrHost {
    int64_t rows = 0;
    std::vector<int32_t> ptr, col;
    std::vector<double> val;
};
struct KernelTables {
    CsrHost Ma, Mb;
    std::vector<double> V;   // n^4, index ((p*n+q)*n+r)*n+s
    double E0 = 0.0;         // <vacuum|H|vacuum>
};
// E0 = <vacuum|H|vacuum> and the alpha-beta coupling V from the Pauli table;
// the same-spin CSR tables are folded on the device (hy_fold.cu) and copied
// into Ma / Mb on the host only when a host consumer asks (ham_view)
void fold_coupling(const PauliTable &t, int n, KernelTables &kt);

// ---------------------------------------------------------------------------
// Operator pool.
// ---------------------------------------------------------------------------
struct PoolOpHost {
    int32_t desc[11];   // [nc, (rank, c0, c1, a1, a0) x 2]
};
void build_pool_spin_adapted(int n, int na, int nb, std::vector<PoolOpHost> &ops);
// Qubit-excitation-based pool: every spin-orbital single and double
// excitation from the Hartree-Fock occupied to the virtual spin orbitals
// that keeps S_z, one operator each (no spin complement), acting as a qubit
// excitation (no Jordan-Wigner sign)
void build_pool_qeb(int n, int na, int nb, std::vector<PoolOpHost> &ops);

// A constituent split into its alpha part and beta part: C = eps * Ca * Cb.
// Each part is a pattern id into the per-spin pattern lists, or -1 for the
// identity.
struct PatternKey {
    int nops;
    int ops[4];          // 2 * orbital + dagger, in product order
    int qubit = 0;       // 1: qubit operators (no Jordan-Wigner sign)
    bool operator==(const PatternKey &o) const;
};
struct PatternKeyHash {
    size_t operator()(const PatternKey &k) const;
};
struct PatternLists {
    // entries: bits 0..14 string S in the pattern's domain, bits 15..29
    // image S' = C S, bit 31 set for a negative sign.
    std::vector<uint32_t> entry;
    std::vector<int64_t> off;   // per pattern
    std::vector<int64_t> cnt;
    std::unordered_map<PatternKey, int, PatternKeyHash> id;
    std::vector<PatternKey> keys;   // by id
    // id of pattern k (registered on first use); finalize() then lists every
    // registered pattern's pairs (patterns in parallel, stored in id order)
    int get(const PatternKey &k);
    void finalize(const StringSpace &s);
};

// Kernel-class timing (hy_profile.cpp): records an event pair on `stream`
// around its lifetime when the class is enabled, with the algorithmic bytes
// and floating-point operations of the enclosed launches (0 where the host
// does not know them).
class ProfScope {
  public:
    ProfScope(int cls, void *stream, double bytes, double flops = 0.0);
    ~ProfScope();
    ProfScope(const ProfScope &) = delete;
    ProfScope &operator=(const ProfScope &) = delete;

  private:
    int cls_;
    void *stream_;
    double bytes_, flops_;
    void *a_;
};

// ---------------------------------------------------------------------------
// Sparse state vectors for the ADAPT driver (implemented in hy_api.cu over
// the kernels of hy_sparse.cu).  A SparseState owns a support list of
// capacity cap, a membership bitmap and device counters; the amplitudes live
// in the caller's dense array v (N amplitudes, zero off the support).  The
// count stays on the device; count() > cap means the list overflowed and the
// contents are no longer a valid sparse vector (reset(full) repairs it).
// ---------------------------------------------------------------------------
struct SparseState;
hy_status sstate_create(const hy_ham *h, hy_dtype dt, void *v, int64_t cap, SparseState **out);
void sstate_destroy(SparseState *s);
// full: zero the whole dense array and bitmap (after dense use or overflow);
// else only the listed entries.  hf: then set v = |HF> (index 0).
hy_status sstate_reset(SparseState *s, bool full, bool hf, void *stream);
hy_status sstate_copy(SparseState *dst, const SparseState *src, void *stream);
// sigma = H psi on psi's support only: sig (clean, over the array sigma)
// receives psi's list and bitmap, and sigma every listed row of H psi, from
// the couplings to listed determinants; sigma elsewhere stays zero.  Enough
// for everything that reads sigma only on psi's support (the energy, and the
// gradients, whose vectors d psi / d theta_l lie in that support).
hy_status sstate_apply_h_support(const SparseState *s, SparseState *sig, void *sigma,
                                 void *stream);
// host estimate of the count, used only to size grids
void sstate_set_hint(SparseState *s, int64_t n);
// closed: keep s's list fixed -- a pair whose other end is unlisted only
// scales its listed end (for a vector that is read on a fixed support only)
hy_status sstate_excite(SparseState *s, const hy_pool *p, int64_t k, double theta, void *stream,
                        bool closed = false);
// In one CTA: clear the support, |HF>, the rotations of ops[0..L) (device)
// with cs[2l], cs[2l+1] (device) = cos, sin theta_l, then (renorm) divide by
// the FP64 norm over the support.  For small supports (one launch instead of
// two per constituent); the state must be clean.
hy_status sstate_prepare(SparseState *s, const hy_pool *p, const int32_t *ops, const double *cs,
                         int64_t L, bool renorm, double *norm2, void *stream,
                         int64_t *step_len = nullptr);
// Support program of a fixed ansatz (see prog_compile in hy_kernels.cuh): the
// rotations as pairings of the support's elements, compiled once per ansatz
// from a structural sstate_prepare (with step_len = prog_step_len(g)) and
// then run on m-vectors in shared memory.
struct SupportProgram;
hy_status prog_create(const hy_ham *h, int max_steps, SupportProgram **out);
void prog_destroy(SupportProgram *g);
int64_t *prog_step_len(SupportProgram *g);           // device, max_steps entries
const int *prog_flag(const SupportProgram *g);        // device, set by prog_compile
// constituent rotations of ops[0..L) (host array), i.e. the program's steps
int64_t prog_steps(const hy_pool *p, const int32_t *ops_host, int64_t L);
// the largest support a program holds
int64_t prog_capacity();
// H restricted to the program's support, built from s (which lists exactly
// that support, as after prog_compile): skipped (left unbuilt) when it would
// hold more than max_nnz entries or its memory cannot be had.  prog_hss_apply
// writes sigma = H psi on the support only (the rest of sigma untouched) and,
// with dot (device) not null, *dot = <psi|sigma> in FP64.
hy_status prog_build_hss(SupportProgram *g, const SparseState *s, int64_t max_nnz, void *stream);
bool prog_hss_ready(const SupportProgram *g);
hy_status prog_hss_apply(const SupportProgram *g, const void *psi, void *sigma, hy_dtype dt,
                         double *dot, void *stream);
// compile from s (whose support, m <= prog_capacity() elements, was just
// listed by a structural sstate_prepare of ops[0..L) (device) with step_len)
hy_status prog_compile(SupportProgram *g, const SparseState *s, int64_t m, const hy_pool *p,
                       const int32_t *ops, int64_t L, int64_t steps, void *stream);
// s.v on the program's support = U_L .. U_1|HF> (renormalised as
// sstate_prepare); s's list and bits, which hold that support, are kept
hy_status prog_prepare(const SupportProgram *g, SparseState *s, const hy_pool *p,
                       const int32_t *ops, const double *cs, int64_t L, bool renorm,
                       double *norm2, void *stream);
// g_out[l] = dE/dtheta_l in forward mode (as sstate_grad_forward)
hy_status prog_grad(const SupportProgram *g, const hy_pool *p, const int32_t *ops,
                    const double *cs, int64_t L, const void *sigma, hy_dtype dt,
                    const double *norm2, double *g_out, void *stream);
// In one CTA, for small supports: g[l] (device) = dE/dtheta_l in forward mode
// (dE/dtheta_l = 2 <sigma| U_L .. U_{l+1} A_l U_l .. U_1 |HF>), with f and w
// clean scratch sparse vectors, sigma = H psi (dense), ops / cs as for
// sstate_prepare and norm2 (device, float states) the squared norm psi was
// divided by (nullptr: none)
hy_status sstate_grad_forward(SparseState *f, SparseState *w, const hy_pool *p, const int32_t *ops,
                              const double *cs, int64_t L, const void *sigma, const double *norm2,
                              double *g, void *stream);
// *out (device) = sum over the support of v * y (y dense, same dtype), FP64
hy_status sstate_dot(const SparseState *s, const void *y, double *out, void *stream);
// v <- v / sqrt(*norm2) on the support (norm2 on the device)
hy_status sstate_scale_rsqrt(SparseState *s, const double *norm2, void *stream);
// sigma = H v.  sig == nullptr: sigma (dense) is zeroed here; else sig is
// sigma's sparse state (its array must be `sigma`, reset by the caller) and
// every reached determinant is listed in it
hy_status sstate_apply_h(const SparseState *s, SparseState *sig, void *sigma, void *stream);
// g[i] = 2 <lam | A_{ops[i]} v> over the pairs with a listed end (ops device
// array or nullptr for the whole pool); m_hint ~ the support size (grid shape)
hy_status sstate_gradients(const SparseState *s, const void *lam, const hy_pool *p,
                           const int32_t *ops, int64_t n_ops, int64_t m_hint, double *g,
                           void *stream);
// hy_ranker_features, with psi's (sigma's) touched weights taken from its
// support list when psi_state (sigma_state), a sparse vector whose array is
// psi (sigma) and whose list holds its whole support, is not null
hy_status ranker_features_impl(const hy_ham *h, const hy_pool *p, const void *psi,
                               const SparseState *psi_state, const void *sigma_or_null,
                               const SparseState *sigma_state, hy_dtype dt, const float *extra,
                               float *feat, void *stream);
const int64_t *sstate_count(const SparseState *s);   // device pointer
// most determinants one determinant couples to through H (itself included):
// 1 + s_a + s_b + d_a + d_b + s_a s_b (singles s, doubles d of each spin)
int64_t ham_connections(const hy_ham *h);
// atomic adds per listed determinant of the list-based touched weights
// (its row sum and one per pair j <= b of its beta electrons)
int64_t ham_list_weight_adds(const hy_ham *h);
const int64_t *sstate_list(const SparseState *s);    // device pointer

// Read-only view of a Hamiltonian handle for the library's other
// translation units (the explicit H build reads the string spaces and the
// folded tables).
struct HamView {
    int n, na, nb, device, num_sms;
    int64_t Na, Nb, N;
    const StringSpace *A, *B;
    const KernelTables *kt;
};
// host_tables: also make the host copy of the same-spin tables (kt->Ma, Mb)
HamView ham_view(const hy_ham *h, bool host_tables = false);
void set_last_error(const std::string &msg);
void count_launch();

// hy_pool_gradients without the operator-list checks (the ADAPT driver's
// lists are built by the library and always valid)
hy_status pool_gradients_unchecked(const hy_ham *hc, const hy_pool *p, const void *psi,
                                   const void *sigma, const int32_t *ops, int64_t n_ops,
                                   double *g_out, hy_dtype dt, void *stream);
// operator lists of the public screens (hy_api.cu): host lists are checked
// here, device lists by the kernels with a deferred report
hy_status check_op_list(const hy_pool *p, const int32_t *ops, int64_t n_ops,
                        bool *device_list, void *stream);
hy_status fetch_op_list_flag(const hy_pool *p, void *stream);
int64_t sstate_cap(const SparseState *s);

}  // namespace hy
