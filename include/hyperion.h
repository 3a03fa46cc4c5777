/*
 * hyperion.h -- C ABI of the GB300 state-vector ADAPT-VQE hot path.
 *
 * The operations follow the statement of the problem in arXiv 2604.01176
 * ("High Performance Quantum Emulation for Chemistry Applications with
 * Hyperion"):
 *   - the variational energy E(theta) = <psi|H|psi> of a real molecular
 *     Hamiltonian (Method section, Eq. "ev");
 *   - H mapped to qubits by Jordan-Wigner and applied to a state held only on
 *     the particle- and S_z-conserving determinant space Omega_CIk
 *     (Sparse State-Vector Emulation section, Table 1);
 *   - the three sparse operations the paper's library provides: H times a
 *     state, inner products, and the application of an exponentiated
 *     fermionic operator (same section);
 *   - the ADAPT-VQE pool-gradient screen (Numerical performance subsection).
 *
 * Conventions shared by every call
 *   - Spin orbitals are in blocked order: qubit p is orbital p alpha for
 *     p < n_orb, qubit n_orb + p is orbital p beta.  A determinant is a
 *     2*n_orb-bit occupation mask (uint64, alpha block in the low bits).
 *   - An alpha (beta) string is an n_orb-bit mask; its rank is the
 *     colexicographic combinadic rank sum_i C(pos_i, i+1) over its set bits
 *     pos_0 < pos_1 < ...  The determinant index is
 *     I = rank(alpha) * N_beta + rank(beta); a state vector is a dense array
 *     of N_det = N_alpha * N_beta amplitudes in that order.
 *   - Precision: HY_F64 computes in double; HY_F32 keeps amplitudes and the
 *     bulk arithmetic in float with float accumulation (the float coupling
 *     of H psi runs on the tensor cores as TF32 products of split operands,
 *     FP32 accuracy; hy_ham_set_coupling).  Energies, norms, dot products
 *     and gradients are always returned in double and reduced with FP64
 *     accuracy (see hy_dot).
 *   - Ownership: the caller owns every state vector and output buffer passed
 *     in (device pointers unless stated "host") and the CUDA stream (passed
 *     as void*, NULL = legacy default stream).  The library owns the tables
 *     inside hy_ham / hy_pool and a per-handle workspace it allocates with
 *     cudaMalloc on first use (so make the first call of each kind before
 *     capturing a CUDA graph).  All launches are stream-ordered; no call
 *     synchronises the host except where stated.
 *   - Errors: every call returns hy_status; hy_last_error() gives a message
 *     for the calling thread's most recent failure.  Sizes and arguments are
 *     validated on the host before any launch; no call traps on the device.
 *   - Limits: 1 <= n_orb <= 16 (32 qubits), 0 <= n_alpha, n_beta <= n_orb.
 *   - Threading: calls on one handle must not overlap in time on different
 *     streams (they share the handle's workspace).
 */
#ifndef HYPERION_H
#define HYPERION_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HY_OK = 0,
    HY_ERR_ARG = 1,          /* invalid argument, size or shape            */
    HY_ERR_CUDA = 2,         /* a CUDA runtime call failed                 */
    HY_ERR_OOM = 3,          /* device or host allocation failed          */
    HY_ERR_TIMEOUT = 4,      /* a bounded device wait ran out              */
    HY_ERR_UNSUPPORTED = 5   /* input outside what the library implements */
} hy_status;

typedef enum { HY_F64 = 0, HY_F32 = 1 } hy_dtype;

typedef enum { HY_POOL_SPIN_ADAPTED_SD = 0, HY_POOL_QEB = 1 } hy_pool_kind;

typedef struct hy_ham hy_ham;
typedef struct hy_pool hy_pool;
typedef struct hy_ranker hy_ranker;
typedef struct hy_adapt hy_adapt;

/* Message describing the calling thread's most recent error ("" if none). */
const char *hy_last_error(void);

/* Library version string. */
const char *hy_version(void);

/* Number of kernels this library has launched in this process (including
 * the kernels of each CUDA-graph replay it issues). */
int64_t hy_launch_count(void);

/* Kernel-class timing.  hy_profile_enable(mask) clears the counters and, for
 * every class whose bit (1u << class) is set, makes the library record a
 * pair of CUDA events on the launching stream around each of its launches of
 * that class, with the algorithmic bytes and floating-point operations those
 * launches perform (0 where the host does not know them, e.g. sparse work
 * whose size lives on the device).  hy_profile_read waits for the recorded
 * events and returns, per class, the launches, the summed device
 * milliseconds, bytes and flops (any output may be NULL).  mask = 0 (the
 * default) records nothing and costs nothing.  Process-wide; calls may come
 * from several threads. */
typedef enum {
    HY_PROF_HPSI = 0,          /* dense H|psi> (hy_apply_h): 2 N s bytes,
                                  2 x connections x N flops                    */
    HY_PROF_HPSI_SPARSE = 1,   /* scatter H|psi> incl. zeroing sigma: N s      */
    HY_PROF_EXCITE = 2,        /* dense exp(theta A) pair rotations: 4 s/pair  */
    HY_PROF_SPARSE_EXCITE = 3, /* rotations of a sparse state: (12 + 4 s) bytes
                                  per listed entry and constituent, estimated
                                  from the support the host last read back     */
    HY_PROF_SCREEN = 4,        /* dense pool gradients: 4 s per pair per op    */
    HY_PROF_SCREEN_SPARSE = 5, /* support-restricted gradients (unknown)       */
    HY_PROF_REDUCE = 6,        /* dots / norms / renormalisation: s per read
                                  or written amplitude                         */
    HY_PROF_FEATURES = 7,      /* ranker features: N s bytes per pass over psi
                                  or sigma (its arithmetic skips zero tiles and
                                  is not counted)                              */
    HY_PROF_HMAT = 8,          /* H psi over the explicit H (hy_hmat_apply):
                                  the stored matrix + read psi rows + write
                                  sigma rows; 2 flops per stored entry         */
    HY_PROF_CLASSES = 9
} hy_prof_class;
hy_status hy_profile_enable(uint32_t class_mask);
hy_status hy_profile_read(int cls, int64_t *launches, double *ms, double *bytes,
                          double *flops);

/* ---------------------------------------------------------------------- */
/* Hamiltonian                                                              */
/* ---------------------------------------------------------------------- */

/* Build H from integrals (Sparse State-Vector Emulation section: fermionic
 * operators mapped to qubits and summed; Methods: the Hamiltonian is real).
 *   h1     host, n_orb*n_orb row-major one-electron integrals h_pq (symmetric)
 *   h2     host, n_orb^4 two-electron integrals in chemists' notation,
 *          (pq|rs) at ((p*n+q)*n+r)*n+s, with (pq|rs) = (qp|sr) = (rs|pq)
 *   e_core constant energy added to the diagonal
 *   prune_tol  Pauli terms with |coefficient| <= prune_tol are dropped
 *          (the paper builds its Hamiltonian with a 1e-14 threshold)
 * H = e_core + sum h_pq a+_ps a_qs + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs.
 * The build maps every term by Jordan-Wigner into a table of Pauli strings
 * grouped by X-mask, derives the kernel tables from that table, and uploads
 * them to the current CUDA device.  Returns HY_ERR_ARG for bad sizes or
 * integrals that are not symmetric to 1e-12, HY_ERR_OOM on allocation
 * failure.  *out receives an owned handle (free with hy_ham_destroy). */
hy_status hy_build_hamiltonian(const double *h1, const double *h2,
                               double e_core, int n_orb, int n_alpha,
                               int n_beta, double prune_tol, hy_ham **out);

/* Host-only build of the Jordan-Wigner Pauli table of H (no CUDA device is
 * touched; same integrals, conventions and pruning as hy_build_hamiltonian).
 * Terms are returned as in hy_ham_pauli_table.  Call with capacity 0 (or any
 * output NULL) to obtain *n_terms and *n_groups only; otherwise x, z and
 * coeff need room for capacity >= *n_terms entries and group_offsets for
 * capacity + 1.  Returns HY_ERR_ARG for bad sizes or non-symmetric
 * integrals, HY_ERR_ARG also when capacity is too small (sizes still set). */
hy_status hy_pauli_table_build(const double *h1, const double *h2,
                               double e_core, int n_orb, double prune_tol,
                               int64_t capacity, uint64_t *x, uint64_t *z,
                               double *coeff, int64_t *group_offsets,
                               int64_t *n_terms, int64_t *n_groups);

/* Partitioned Hamiltonian of the SV-MPS scheme (Partitioned SV-MPS
 * Emulation section): for a partitioning level eta the qubit chain is cut
 * into 2^eta contiguous blocks of 2 n_orb / 2^eta qubits, and
 * H = H_eta + sum B, where H_eta holds the Pauli terms of H that act inside
 * one block (the blocks' local Hamiltonians H^(i), the identity term with
 * them) and the B terms the interactions across blocks.  part = 0 builds a
 * handle for H_eta, part = 1 one for the rest, from src's Pauli table (same
 * integrals, determinant space and pruning); hy_energy on it gives the
 * exact state-vector energy <psi|H_eta|psi> of the paper's expectation-value
 * split (and <psi|B|psi>), every other call works on it as on any H.
 * interleaved = 0 cuts the library's blocked qubit order (alpha spin
 * orbitals, then beta); 1 cuts the chain with orbital p's alpha and beta
 * spin orbitals adjacent (positions 2p, 2p + 1).  The paper does not state
 * its qubit order; both are offered.  eta = 0 gives H itself (part 0).
 * HY_ERR_ARG unless 2^eta divides 2 n_orb (eta <= 5); *out receives an
 * owned handle (hy_ham_destroy). */
hy_status hy_ham_partition(const hy_ham *src, int eta, int interleaved, int part,
                           hy_ham **out);

/* Release a handle and its device memory (NULL is accepted). */
hy_status hy_ham_destroy(hy_ham *h);

/* Sizes: determinants, alpha / beta strings, X-mask groups, Pauli terms.
 * Any output pointer may be NULL. */
hy_status hy_ham_info(const hy_ham *h, int64_t *n_det, int64_t *n_alpha_str,
                      int64_t *n_beta_str, int64_t *n_groups,
                      int64_t *n_terms);

/* With enable != 0, every later hy_apply_h records a pair of CUDA events on
 * its stream around the alpha-beta coupling kernel(s); hy_ham_coupling_ms
 * waits for the last pair and returns the elapsed milliseconds (host).  Off
 * by default; the events cost nothing when off. */
hy_status hy_ham_profile(hy_ham *h, int enable);

/* Float H|psi>: phase A of the alpha-beta coupling (the dense per-string
 * product T_J = W_J G_J) on the tensor cores (impl = 0, the default:
 * tcgen05 TF32 MMAs with split hi/lo operands, FP32 accuracy) or on the FP32
 * SIMT pipes (impl = 1).  Both feed the same phase B.  A bounded wait of the
 * tensor-core kernel that runs out is returned as HY_ERR_TIMEOUT by the next
 * hy_apply_h on this handle (the kernel itself gives up, releases its tensor
 * memory and returns; the context stays usable).  impl = 2 is a test of that
 * path: the tensor-core kernel runs with its MMAs withheld, so no stage
 * barrier ever completes, every wait runs out after its limit and the
 * float H|psi> of that call is wrong. */
hy_status hy_ham_set_coupling(hy_ham *h, int impl);
hy_status hy_ham_coupling_ms(const hy_ham *h, float *ms);

/* Polls of an mbarrier before a wait of the tensor-core coupling gives up
 * (default 2^26, seconds of waiting; >= 1). */
hy_status hy_ham_set_wait_limit(hy_ham *h, int64_t polls);

/* Bytes the build of h (and of pool p, when not NULL) copied from host to
 * device memory: the kernel tables, string lists, pool patterns. */
hy_status hy_ham_upload_bytes(const hy_ham *h, const hy_pool *p, int64_t *bytes);

/* Copy the Pauli table (host outputs, caller-allocated).  Term t is
 * coeff[t] * P(x[t], z[t]) where P is the Hermitian Pauli string with X on
 * bits of x & ~z, Z on z & ~x and Y on x & z (bit j = qubit j).  Terms are
 * sorted by (x, z); group g holds terms group_offsets[g] .. [g+1]-1 and all
 * share x.  Arrays hold n_terms (x, z, coeff) and n_groups + 1 entries. */
hy_status hy_ham_pauli_table(const hy_ham *h, uint64_t *x, uint64_t *z,
                             double *coeff, int64_t *group_offsets);

/* ---------------------------------------------------------------------- */
/* The Hamiltonian stored explicitly                                        */
/* ---------------------------------------------------------------------- */

/* The paper assembles H as a sparse matrix over Omega_CIk and distributes
 * its rows (Sparse State-Vector Emulation section; Table 1 gives its size
 * per molecule).  hy_hmat_build stores the rows of the determinants whose
 * alpha string lies in [row_begin, row_end) (the same row unit as
 * hy_apply_h_rows), with every structural nonzero of those rows -- 1 + s_a
 * + s_b + d_a + d_b + s_a s_b entries per row (singles s, doubles d of each
 * spin; 5,793 at 32 qubits), explicit zeros included -- in dt (HY_F64 or
 * HY_F32 values, computed in double from the folded tables and rounded
 * once).  Layout: rows grouped by alpha string; within a group the columns
 * fall into segments, one per alpha partner (the string itself, its singles,
 * its doubles), every row of the group having the same number of entries
 * per segment; an entry is its beta column (16 bits) and its value, the
 * segment's alpha partner is stored once, and entry j of all rows of a group
 * is contiguous, so a row group is one contiguous stream.  Bytes: per alpha
 * string S * 2 + w * N_bp * (2 + sizeof(dt)) with w the row length, S = 1 +
 * s_a + d_a and N_bp = N_beta rounded up to 8 (padding rows hold zeros).
 * The device memory is checked first: HY_ERR_OOM when the matrix plus 1 GiB
 * does not fit the free memory.  The build synchronises the device.  *out
 * receives an owned handle (hy_hmat_destroy); it refers to h, which must
 * outlive it. */
typedef struct hy_hmat hy_hmat;
hy_status hy_hmat_bytes(const hy_ham *h, hy_dtype dt, int64_t row_begin,
                        int64_t row_end, int64_t *bytes, int64_t *nnz);
hy_status hy_hmat_build(const hy_ham *h, hy_dtype dt, int64_t row_begin,
                        int64_t row_end, hy_hmat **out);
hy_status hy_hmat_destroy(hy_hmat *m);
/* Stored row range, entries (rows x row length), row length, bytes. */
hy_status hy_hmat_info(const hy_hmat *m, int64_t *row_begin, int64_t *row_end,
                       int64_t *nnz, int64_t *row_len, int64_t *bytes);
/* sigma_rows = the stored rows of H times psi: psi the whole state (n_det
 * elements of the matrix's dtype, device), sigma_rows (row_end - row_begin)
 * * N_beta elements; the accumulation runs in the matrix's dtype.  One pass
 * over the stored matrix (streaming loads); psi stays resident in L2. */
hy_status hy_hmat_apply(const hy_hmat *m, const void *psi, void *sigma_rows,
                        void *stream);
/* The stored row of determinant det (its alpha string inside the stored
 * range): *len = row length; with cap >= *len, cols[j] (host) = column
 * determinant index and vals[j] (host) = value (widened to double), in
 * storage order (segments, then ascending beta columns within each). */
hy_status hy_hmat_row(const hy_hmat *m, int64_t det, int64_t *cols,
                      double *vals, int64_t cap, int64_t *len);

/* ---------------------------------------------------------------------- */
/* Determinant indexing (bit-exact)                                         */
/* ---------------------------------------------------------------------- */

/* idx[i] = index of determinant dets[i], or -1 if it is not in Omega_CIk.
 * dets, idx: device arrays of m entries. */
hy_status hy_rank(const hy_ham *h, const uint64_t *dets, int64_t *idx,
                  int64_t m, void *stream);

/* dets[i] = determinant of index idx[i] (0 when idx is out of range).
 * idx, dets: device arrays of m entries. */
hy_status hy_unrank(const hy_ham *h, const int64_t *idx, uint64_t *dets,
                    int64_t m, void *stream);

/* ---------------------------------------------------------------------- */
/* Sweeps                                                                   */
/* ---------------------------------------------------------------------- */

/* sigma = H psi on Omega_CIk (the paper's sparse H times sparse state).
 * psi, sigma: device arrays of n_det elements of the given dtype; they must
 * not alias.  The first call per dtype allocates the handle's workspace. */
hy_status hy_apply_h(const hy_ham *h, const void *psi, void *sigma,
                     hy_dtype dt, void *stream);

/* Rows [row_begin, row_end) of sigma = H psi, counted in alpha strings: the
 * block sigma[row_begin * N_beta .. row_end * N_beta) written to sigma_rows
 * (device, (row_end - row_begin) * N_beta elements of dt); psi is the whole
 * state (n_det elements) and must not overlap sigma_rows.  This is the
 * paper's distribution of H by rows of Omega_CIk with the state replicated
 * (Sparse State-Vector Emulation section, parallelisation paragraph): each
 * process forms the components of its own rows, and one all-gather of the
 * blocks (or an all-reduce of the scalars formed from them) completes the
 * operation.  Every element is computed by the same arithmetic in the same
 * order as in hy_apply_h, so blocks of any split concatenate to hy_apply_h's
 * sigma bit for bit.  The same-spin parts and the FP64 coupling cost the
 * range's share of the full sweep; the float tensor-core coupling forms its
 * per-string products for the range's strings and their single-excitation
 * partners (for a contiguous range of more than a few rows, nearly all).
 * 0 <= row_begin <= row_end <= N_alpha, else HY_ERR_ARG. */
hy_status hy_apply_h_rows(const hy_ham *h, const void *psi, void *sigma_rows,
                          hy_dtype dt, int64_t row_begin, int64_t row_end,
                          void *stream);

/* *out (device, one double) = <x|y> over a block of rows [row_begin,
 * row_end) (alpha strings), x_rows and y_rows holding that block only
 * ((row_end - row_begin) * N_beta elements each), with FP64 accuracy as
 * hy_dot: the per-process partial of a row-distributed inner product, summed
 * over processes by one all-reduce (Sparse State-Vector Emulation section). */
hy_status hy_dot_rows(const hy_ham *h, const void *x_rows, const void *y_rows,
                      hy_dtype dt, int64_t row_begin, int64_t row_end,
                      double *out, void *stream);

/* *e_out (device, one double) = <psi|sigma> with FP64 accuracy (see hy_dot); if
 * sigma_or_null is NULL, sigma = H psi is computed first into the
 * workspace.  psi is not normalised by this call. */
hy_status hy_energy(const hy_ham *h, const void *psi, const void *sigma_or_null,
                    hy_dtype dt, double *e_out, void *stream);

/* *out (device, one double) = <x|y> with FP64 accuracy: HY_F64 products
 * summed in double; HY_F32 products formed exactly (FP32 TwoProduct) and
 * summed with their rounding errors (TwoSum, the Dot2 scheme of Ogita, Rump
 * and Oishi), each run of 32 flushed into a double -- the float->double
 * conversion and FP64 add per element would bound the sweep on GB300's FP64
 * pipe.  Products near the FP32 overflow threshold are taken in double.
 * Deterministic: fixed grid and summation order for a given device. */
hy_status hy_dot(const hy_ham *h, const void *x, const void *y, hy_dtype dt,
                 double *out, void *stream);

/* Sparse states (paper: the state vector is stored sparse and H is applied
 * as a sparse matrix to a sparse vector).  psi stays a dense array over
 * Omega_CIk; these calls take the list of its nonzero amplitudes. */

/* list[0..min(count,cap)-1] (device int64) = indices of the nonzero entries
 * of psi, in no particular order; *count (device int64) = their number, even
 * when it exceeds cap (then only cap are listed). */
hy_status hy_support(const hy_ham *h, const void *psi, hy_dtype dt, int64_t *list,
                     int64_t cap, int64_t *count, void *stream);

/* sigma = H psi for a psi that is zero outside list[0..m-1] (device): sigma
 * is zeroed and every listed amplitude is scattered to all determinants H
 * connects it to (atomic adds; the summation order is not fixed, so results
 * agree with hy_apply_h to rounding).  Cost ~ m x (connections per row). */
hy_status hy_apply_h_sparse(const hy_ham *h, const void *psi, void *sigma,
                            hy_dtype dt, const int64_t *list, int64_t m,
                            void *stream);

/* hy_pool_gradients for a psi that is zero outside list[0..m-1]: only the
 * pairs of each operator with an endpoint in the list are visited (sigma
 * must be the full H psi). */
hy_status hy_pool_gradients_sparse(const hy_ham *h, const hy_pool *p,
                                   const void *psi, const void *sigma,
                                   const int64_t *list, int64_t m,
                                   const int32_t *ops_or_null, int64_t n_ops,
                                   double *g_out, hy_dtype dt, void *stream);

/* ---------------------------------------------------------------------- */
/* Operator pool, gradients and exp(theta A)                                */
/* ---------------------------------------------------------------------- */

/* HY_POOL_SPIN_ADAPTED_SD: spin-adapted singles and doubles relative to the
 * Hartree-Fock determinant (lowest n_alpha / n_beta orbitals occupied).
 * Order: singles (i<a), then same-spin doubles (i<j, a<b), then
 * opposite-spin doubles (i<=j, a<=b, couplings); an operator whose
 * constituents would share a spin orbital is split into one pool entry per
 * constituent, so every generator A_k = sum_c (C_c - C_c^dagger) is a sum of
 * commuting terms on disjoint spin orbitals.
 * HY_POOL_QEB: the qubit-excitation-based pool the paper's ADAPT-VQE runs use
 * (Numerical performance subsection): one operator per spin-orbital single
 * i -> a (same spin) and double (i, j) -> (a, b) (S_z kept) from occupied to
 * virtual spin orbitals of the Hartree-Fock determinant, each a qubit
 * excitation: C = Q+_a Q_i or Q+_a Q+_b Q_j Q_i with Q+ = (X - iY)/2 acting
 * on one qubit and no Jordan-Wigner parity string, so C maps determinant d
 * to d with the electrons moved and sign +1.  Order: alpha singles, beta
 * singles, alpha-alpha, beta-beta, alpha-beta doubles, each lexicographic in
 * (i, [j,] a [, b]).  Descriptors have the same layout as the fermionic
 * pool's (hy_pool_describe); hy_pool_qubit tells the two apart.
 * *out receives an owned pool (free with hy_pool_destroy). */
hy_status hy_pool_create(const hy_ham *h, hy_pool_kind kind, hy_pool **out);
hy_status hy_pool_destroy(hy_pool *p);
hy_status hy_pool_size(const hy_pool *p, int64_t *k);
/* *qubit = 1 for a pool of qubit excitations (HY_POOL_QEB), else 0. */
hy_status hy_pool_qubit(const hy_pool *p, int *qubit);

/* Host output desc[11]: [n_constituents, then per constituent (rank, c0, c1,
 * a1, a0)]; rank 1 is a+_{c0} a_{a0}, rank 2 is a+_{c0} a+_{c1} a_{a1}
 * a_{a0}; modes are spin orbitals in blocked order. */
hy_status hy_pool_describe(const hy_pool *p, int64_t k, int32_t *desc);

/* g_out[i] (device doubles) = 2 <sigma | A_{op_i} psi> for op_i =
 * ops_or_null[i] (int32 list of n_ops pool indices the device can read), or
 * for every pool operator in order when ops_or_null is NULL (n_ops is then
 * ignored and the pool size is used).  With sigma = H psi this is
 * dE/dtheta of exp(theta A) psi at theta = 0 (the ADAPT-VQE screen).
 * Operator lists (the same rules hold for hy_pool_gradients_sparse and
 * hy_pool_gradients_noalloc):
 *   - a list in pageable host memory is range-checked before any launch: an
 *     index outside [0, pool size) returns HY_ERR_ARG naming its position;
 *     where the device cannot read pageable memory such a list is refused;
 *   - a device, pinned or managed list may still be written by work queued
 *     on the stream, so the kernels check it: a refused entry reads nothing
 *     out of range and its gradient is returned as NaN, and the next screen
 *     call on the same pool (once the stream has passed this one) returns
 *     HY_ERR_ARG with the first refused position and index, then clears the
 *     report. */
hy_status hy_pool_gradients(const hy_ham *h, const hy_pool *p, const void *psi,
                            const void *sigma, const int32_t *ops_or_null,
                            int64_t n_ops, double *g_out, hy_dtype dt,
                            void *stream);

/* Allocation-free variant of hy_pool_gradients (the paper has no
 * counterpart: this is a deployment convenience).  For callers that cannot
 * let a library allocate device memory -- e.g. a serving process whose
 * device memory is fully reserved by another allocator, or a loop that must
 * never pay cudaFree's implicit device-wide synchronisation -- this call
 * computes exactly what hy_pool_gradients computes (same kernels, same
 * arguments, same results) but keeps its partial sums in a fixed
 * file-scope device array of 2^18 doubles (2 MiB), resident on every
 * device that loads the library until the process exits, instead of the
 * handle's workspace.  It calls no cudaMalloc or cudaFree.
 *   - Limit: the call needs n_ops * max(1, ceil(4 * SMs / n_ops)) partial
 *     sums, so n_ops may be at most 262,144; larger requests return
 *     HY_ERR_ARG before any launch, with the limit in hy_last_error().
 *   - The first call on each device resolves the array's device address
 *     (cudaGetSymbolAddress) once; make that first call before any stream
 *     capture.
 *   - Every call on a device shares the one array: calls whose launches may
 *     overlap on the GPU (different streams, or threads without ordering)
 *     race and give wrong results; serialise them.  Each call overwrites
 *     every partial it later reads, so nothing needs clearing between
 *     calls. */
hy_status hy_pool_gradients_noalloc(const hy_ham *h, const hy_pool *p,
                                    const void *psi, const void *sigma,
                                    const int32_t *ops_or_null, int64_t n_ops,
                                    double *g_out, hy_dtype dt, void *stream);

/* psi <- exp(theta A_k) psi in place: for each constituent C (sign s on the
 * pair d -> C d) and each connected pair, psi(d) <- cos psi(d) - s sin
 * psi(Cd), psi(Cd) <- cos psi(Cd) + s sin psi(d).  With renormalize != 0
 * psi is then divided by its double-precision norm (HY_F32 drift control). */
hy_status hy_apply_excitation(const hy_ham *h, const hy_pool *p, int64_t k,
                              double theta, void *psi, hy_dtype dt,
                              int renormalize, void *stream);

/* Renormalisation after each exp(theta A) (paper: Method, mixed precision --
 * the renormalisation stays in double) without a sweep over the state:
 * hy_apply_excitation_tracked applies exp(theta A_k) like
 * hy_apply_excitation (no renormalisation) and adds to the device scalar
 * *norm2 the change of ||psi||^2 over the rotated pairs, with FP64 accuracy
 * (FP64 products for HY_F64; for HY_F32 exact FP32 products summed by the
 * compensated Dot2 scheme and flushed into FP64 every 32 terms).  Untouched
 * amplitudes keep their norm, so starting from *norm2 = ||psi||^2 it tracks
 * the norm through a product of rotations; scaling commutes with the
 * rotations, so one hy_renormalize (psi <- psi / sqrt(*norm2); *norm2 is
 * read, not changed) after the last one equals renormalising after each.
 * norm2: device pointer, 8-byte aligned, ordered on `stream`. */
hy_status hy_apply_excitation_tracked(const hy_ham *h, const hy_pool *p, int64_t k,
                                      double theta, void *psi, hy_dtype dt,
                                      double *norm2, void *stream);
hy_status hy_renormalize(const hy_ham *h, void *psi, hy_dtype dt,
                         const double *norm2, void *stream);

/* Scale psi by 1 / sqrt(<psi|psi>) (norm with FP64 accuracy, as hy_dot). */
hy_status hy_normalize(const hy_ham *h, void *psi, hy_dtype dt, void *stream);

/* ---------------------------------------------------------------------- */
/* Batches of molecules                                                     */
/* ---------------------------------------------------------------------- */

/* A batch runs sigma = H psi (and the energies <psi|sigma>) for many
 * molecules of uneven size in one persistent launch: CTAs are split into
 * groups of tile.gsize threads; each group takes the next (molecule, alpha
 * row) task from a device work-list (largest molecules first) and computes
 * that output row completely, then writes its <psi|sigma> partial, which a
 * second small kernel sums per molecule in row order.  Intended for
 * molecules of up to 12 orbitals (their tables stay in L2); larger ones are
 * correct but slow.  States are packed: molecule m's amplitudes start at
 * element offsets[m] of one buffer (offsets are multiples of 32). */
typedef struct hy_batch hy_batch;

typedef struct {
    int gsize;        /* threads per group (32, 64, ..., 1024)             */
    int groups;       /* groups per CTA (gsize * groups <= 1024, <= 15)    */
    int ctas_per_sm;  /* 0: as many as occupancy allows                    */
} hy_batch_tile;

/* hams: host array of `count` handles, which must outlive the batch. */
hy_status hy_batch_create(const hy_ham *const *hams, int count, hy_batch **out);
hy_status hy_batch_destroy(hy_batch *b);
/* *total: packed state length; *n_tasks: rows of all molecules. */
hy_status hy_batch_info(const hy_batch *b, int64_t *total, int64_t *n_tasks);
/* offsets: host, count + 1 entries (the last one = total). */
hy_status hy_batch_offsets(const hy_batch *b, int64_t *offsets);
hy_status hy_batch_set_tile(hy_batch *b, const hy_batch_tile *tile);
hy_status hy_batch_get_tile(const hy_batch *b, hy_batch_tile *tile);

/* sigma = H psi for every molecule (packed device buffers of dt); if
 * energies is not NULL, energies[m] (device doubles) = <psi_m|sigma_m>.
 * Launches: one memset of the task counter, the persistent kernel, and the
 * energy kernel.  No host synchronisation (capturable). */
hy_status hy_batch_apply_h(hy_batch *b, const void *psi, void *sigma,
                           hy_dtype dt, double *energies, void *stream);

/* Same as hy_batch_apply_h, through a CUDA graph the batch captures on the
 * first call for these (psi, sigma, dt, energies, tile) and replays after. */
hy_status hy_batch_graph_launch(hy_batch *b, const void *psi, void *sigma,
                                hy_dtype dt, double *energies, void *stream);

/* Batched pool-gradient screen (the paper's screen g_k = 2<H psi|A_k psi>,
 * Numerical performance subsection, for many molecules at once).
 * hy_batch_set_pools: pools[m] (host array of `count` handles, pool m built on
 * the batch's Hamiltonian m) are attached to the batch; they must outlive it.
 * hy_batch_pool_offsets: offsets (host, count + 1): where molecule m's
 * gradients start in g of a full screen.
 * hy_batch_gradients: g (device doubles) for every molecule's listed
 * operators in one persistent launch over (molecule, operator, row chunk)
 * tasks plus one summing kernel.  psi, sigma: packed states of dt (sigma =
 * H psi, e.g. from hy_batch_apply_h).  ops = NULL: every operator of every
 * pool, g packed by hy_batch_pool_offsets.  Otherwise ops (device int32) holds
 * per-molecule lists of local pool indices, molecule m's at [op_offsets[m],
 * op_offsets[m + 1]) of ops and of g, op_offsets a device array of count + 1
 * entries, n_entries (host) = op_offsets[count].  An index outside its pool
 * gives NaN for that entry and is reported (HY_ERR_ARG, with its position)
 * by the next call on this batch.  No host synchronisation except when a
 * larger call first grows the partial-sum workspace (make the first call of
 * each size before capturing a CUDA graph). */
hy_status hy_batch_set_pools(hy_batch *b, const hy_pool *const *pools);
hy_status hy_batch_pool_offsets(const hy_batch *b, int64_t *offsets);
hy_status hy_batch_gradients(hy_batch *b, const void *psi, const void *sigma,
                             const int32_t *ops, const int64_t *op_offsets,
                             int64_t n_entries, double *g, hy_dtype dt, void *stream);

/* Autotuner: times every tile shape (gsize in 32..512, groups in 1..8,
 * within the shared-memory and barrier limits) on these buffers with CUDA
 * events (2 warm-up + 3 timed launches each), keeps the fastest as the
 * batch's tile and returns it with its mean time in *ms (host). */
hy_status hy_batch_tune(hy_batch *b, const void *psi, void *sigma, hy_dtype dt,
                        hy_batch_tile *best, double *ms, void *stream);

/* ---------------------------------------------------------------------- */
/* Learned pool ranker                                                      */
/* ---------------------------------------------------------------------- */

/* Occupation numbers <psi|n_P|psi> / <psi|psi> of the 2*n_orb spin orbitals
 * (blocked order) into occ (device floats).  One pass over psi; the sums
 * run in a fixed order.  (Used by the ranker features.) */
hy_status hy_occupations(const hy_ham *h, const void *psi, hy_dtype dt,
                         float *occ, void *stream);

/* Weights of the state on the determinants an excitation touches:
 * D[(i*n+a)*n*n + j*n+b] (device, n^4 floats) = sum over determinants with
 * i occupied and a empty in the alpha string and j occupied and b empty in
 * the beta string of |psi|^2, where i == a (j == b) drops the alpha (beta)
 * condition; D[0] = <psi|psi>.  Two passes: per alpha string the beta
 * pair weights, then their contraction over alpha strings. */
hy_status hy_touched_weights(const hy_ham *h, const void *psi, hy_dtype dt,
                             float *D, void *stream);

/* The same from the state's support: list (device, m indices, e.g. from
 * hy_support) holds every nonzero amplitude of psi (each once); O(m) work
 * instead of a pass over the whole state (the ADAPT driver's sparse path uses
 * it for psi and, while it is listed, sigma).  The entries are grouped by
 * alpha string (held by h, grown with a device synchronisation when m
 * exceeds them) and each string's pair weights summed by one block; equal to
 * hy_touched_weights up to float rounding in the order of addition. */
hy_status hy_touched_weights_sparse(const hy_ham *h, const void *psi, hy_dtype dt,
                                    const int64_t *list, int64_t m, float *D, void *stream);

/* The ranker is an addition with no counterpart in the paper's method: a
 * small MLP that predicts, per pool operator, t_k = log10(|g_k| / max|g| +
 * 1e-6) from 16 features, so that only its top-M operators are screened
 * exactly.  Features of operator k (first constituent; modes in blocked
 * order): [0..3] kind flags (single, same-spin double, opposite-spin
 * double, extra constituents); [4..7] annihilated and created spatial
 * orbitals / n_orb (-0.1 where absent); [8] log10 |integral| (h_ca for
 * singles, (c0 a0|c1 a1) minus exchange for same spin); [9] diagonal
 * one-electron gap; [10], [11] with sigma given: log10 of the
 * Cauchy-Schwarz bound 2 sum_c (|sigma_img| |psi_dom| + |sigma_dom|
 * |psi_img|) / (|sigma| |psi|) over the operator's constituents c, and
 * log10 of the state weight on the touched determinants sum_c (|psi_dom|^2
 * + |psi_img|^2) / |psi|^2 (exact for singles and opposite-spin doubles,
 * geometric mean of the two pair weights for same-spin doubles) -- without
 * sigma: the mean-field occupation product n_a0 n_a1 (1-n_c0)(1-n_c1) and
 * n_a0 + n_a1 - n_c0 - n_c1; [12..15] the caller's extra[k][0..3] (the
 * driver passes log10 of the operator's last exact |g_k| relative to the
 * largest |g| of the most recent screen, its age in iterations / 10, the
 * operator's count in the ansatz and its summed |theta|), or 0.
 * feat: device, K x 16 floats; extra: device K x 4 floats or NULL;
 * sigma_or_null: H psi in dt, or NULL. */
hy_status hy_ranker_features(const hy_ham *h, const hy_pool *p, const void *psi,
                             const void *sigma_or_null, hy_dtype dt,
                             const float *extra, float *feat, void *stream);

/* MLP 16 -> hidden -> hidden -> hidden -> 1 (ReLU), FP32, He-uniform init
 * from `seed` (SplitMix64).  The ranker owns its device parameters, Adam
 * moments and training set. */
hy_status hy_ranker_create(int hidden, uint64_t seed, hy_ranker **out);
hy_status hy_ranker_destroy(hy_ranker *r);
hy_status hy_ranker_info(const hy_ranker *r, int64_t *n_params,
                         int64_t *n_samples, int *n_features, int *fitted);
/* Parameters as one host float array of n_params entries (checkpoints). */
hy_status hy_ranker_get_params(const hy_ranker *r, float *host);
hy_status hy_ranker_set_params(hy_ranker *r, const float *host);

/* score[i] (device) = MLP(feat[i]) for m rows (device K x 16). */
hy_status hy_ranker_predict(hy_ranker *r, const float *feat, int64_t m,
                            float *score, void *stream);

/* Append m training pairs: features (device m x 16) and the exact
 * gradients g (device doubles) of one screen; the targets are normalised
 * by that screen's max |g|. */
hy_status hy_ranker_add_samples(hy_ranker *r, const float *feat,
                                const double *g, int64_t m, void *stream);

/* Adam (lr, beta 0.9 / 0.999) on the mean squared error over all samples,
 * `epochs` passes in shuffled minibatches of `batch` rows (shuffle seeded).
 * *loss (host, optional) = mean squared error of the last epoch. */
hy_status hy_ranker_fit(hy_ranker *r, int epochs, int batch, float lr,
                        uint64_t seed, float *loss, void *stream);

/* idx[0..k-1] (device int32) = indices of the k largest of m <= 8192 scores
 * (device floats), descending, ties to the lower index. */
hy_status hy_ranker_topk(const float *score, int64_t m, int64_t k,
                         int32_t *idx, void *stream);

/* Attach a ranker to a driver created with screen_top_m = M > 0.  The first
 * warm_iters iterations run the full screen and feed the ranker (features,
 * exact |g|) pairs; it is then fitted (`epochs` passes) and from then on
 * M operators are proposed and screened exactly: the M / 4 with the largest
 * gradient bound (feature 10, an upper bound on |g_k|), the M / 4 with the
 * largest |g_k| at their last exact screen, then the MLP's top ranks until M
 * distinct operators.  Every
 * refresh_every-th ranked iteration (0: never) selects from the full screen
 * instead, adds its pairs and refits the ranker (epochs / 4 passes, warm
 * start), which bounds the age of the stale-gradient features.  The full
 * screen is also the fallback, run whenever the proposals' ||g|| would stop
 * the loop, and, with cfg.judge, the judge: every ranked iteration also runs
 * it, records the rank of the true argmax and adds its pairs.  Fits are
 * owed, not run, while iterations screen exactly (warm-up, refresh, or the
 * sparse path's exact screen): the owed epochs (the largest owed so far) run
 * just before the ranker's next proposals, so a ranker that is never needed
 * is never trained.  A ranker passed in already fitted is used as is until
 * a refresh owes it a refit. */
hy_status hy_adapt_set_ranker(hy_adapt *a, hy_ranker *r, int warm_iters,
                              int epochs, int refresh_every);

/* ---------------------------------------------------------------------- */
/* ADAPT-VQE driver                                                         */
/* ---------------------------------------------------------------------- */

/* The ADAPT-VQE loop of the paper's Numerical performance subsection: start
 * from the Hartree-Fock determinant; each iteration screens the pool by
 * |g_k| = |dE/dtheta_k|, appends the operator with the largest |g_k| with
 * theta = 0 (ties go to the lowest index within 1e-12 max|g|), then
 * re-optimises every theta (here: BFGS with backtracking line search and
 * analytic adjoint gradients, warm-started from the previous parameters).
 * Each energy evaluation is E(theta) = <psi0|U(theta)^T H U(theta)|psi0>
 * (Method section); the state preparation applies the ansatz's exp(theta A)
 * in order (cost T_0 per operator of the paper's C-tilde metric) and the
 * measurement is one H psi plus one inner product (cost T_1).
 *
 * bulk = HY_F64: everything in double ("plain FP64").
 * bulk = HY_F32: state, H psi and gradients in float with float accumulation
 *   inside H psi; energies, norms and gradients reduced in double; psi is
 *   renormalised (norm in double) after every exp(theta A).  The float
 *   optimisation stops at gtol_bulk or at the float rounding floor; every
 *   refine_every-th iteration (and in hy_adapt_refine) it is followed by
 *   at most refine_steps BFGS steps in double, and that iteration's
 *   recorded energy is a double-precision evaluation with the float
 *   energy's error beside it; the next iteration then screens the pool on
 *   that double-precision state (its parameters are the double optimum, so
 *   the selection is the one plain FP64 makes; float gradients, ~1e-6
 *   relative off, can reorder near-equal operators).  Other iterations
 *   record the float-bulk energy (reduced in double) and
 *   energy_bulk_err = -1.  Iterations whose state has fewer nonzero
 *   amplitudes than float_from / 4 optimise in double directly (energy =
 *   energy_bulk in double, energy_bulk_err = 0). */
typedef struct {
    hy_dtype bulk;        /* HY_F64 or HY_F32                                  */
    int max_iter;         /* capacity of the ansatz (iterations)               */
    double eps_grad;      /* converged when ||g||_2 over the screen < eps_grad */
    double gtol;          /* optimiser: stop when max |dE/dtheta| < gtol       */
    double gtol_bulk;     /* HY_F32 only: float-phase tolerance                */
    int max_evals;        /* optimiser: cap on evaluations per iteration       */
    int refine_steps;     /* HY_F32 only: double-precision BFGS steps (>= 0)   */
    int refine_every;     /* HY_F32 only: refine in double after every k-th
                             iteration (1: every iteration; 0: only when
                             hy_adapt_refine is called)                        */
    int screen_top_m;     /* 0: full screen; M > 0: screen only the M operators
                             a ranker proposes (hy_adapt_set_ranker)           */
    int judge;            /* with screen_top_m > 0: also run the full screen
                             and report the true argmax and its rank           */
    int sparse;           /* 1: keep psi as a sparse vector (support list +
                             membership bitmap over the dense array) while its
                             support fits sparse_cap: state preparation,
                             renormalisation, energy and the adjoint's psi
                             side cost O(support), H psi is the scatter of
                             hy_apply_h_sparse where all of it is needed (the
                             screen, which visits only pairs with a listed
                             end) and otherwise H psi on the support's rows
                             only (the energy and the gradients read it
                             nowhere else; the reverse sweep then keeps its
                             vectors on the support); when the list overflows
                             the evaluation is redone with the dense sweeps,
                             which stay in use while the ansatz is at least as
                             long.  After each append an ansatz whose
                             support holds at most 65,536 determinants is
                             compiled into per-rotation lists of the pairs
                             of its support, so that the iteration's further
                             evaluations and forward-mode gradients run on
                             vectors in shared memory (one CTA's up to
                             12,288 determinants, an 8-CTA cluster's
                             beyond).  While (pool size) x
                             (support) <= 5e9 the whole pool is screened
                             exactly even when a ranker is attached (its
                             pairs still train it).
                             0: always the dense sweeps                        */
    int64_t sparse_cap;   /* support capacity of the sparse path; 0: N_det/8
                             for double and N_det/16 for float evaluations (a
                             sparse evaluation at large supports costs ~30 ns
                             (float) / ~55 ns (double) per listed amplitude at
                             32 qubits, a dense one ~1.5 ns / ~11 ns per
                             determinant)                                     */
    double exact_screen_work; /* sparse path with a ranker: screen the whole
                             pool exactly while (pool size) x (support) is at
                             most this; 0: 5e9 (the cost of the ranker's
                             feature pass at 32 qubits); < 0: never (always
                             ask the ranker, e.g. to judge it).  The exact
                             screens feed the ranker training pairs once
                             (pool size) x (support) exceeds 1/64 of this
                             (dense path: always)                            */
    int64_t float_from;   /* HY_F32 bulk: an iteration whose state has fewer
                             than float_from / 4 nonzero amplitudes at its
                             screen (its support on the sparse path, every
                             determinant on the dense sweeps) optimises in
                             double directly (no refinement needed); there
                             the evaluations are latency-bound and cost the
                             same in either precision.  0: 2^20; 1: always
                             float                                           */
} hy_adapt_config;

/* One ADAPT iteration (all times in seconds, host wall clock). */
typedef struct {
    int32_t iter;          /* 0-based iteration index                         */
    int32_t converged;     /* 1: ||g|| < eps_grad, nothing appended            */
    int64_t selected;      /* pool index appended (-1 if converged)           */
    double max_grad;       /* |g| of the selected operator                    */
    double grad_norm;      /* ||g||_2 over the screened operators             */
    double energy;         /* energy after optimisation (double precision when
                              refined, else the float-bulk energy)           */
    double energy_bulk;    /* bulk-precision energy at the bulk optimum        */
    double energy_bulk_err;/* |energy_bulk - double energy at the same theta|,
                              -1 when this iteration was not refined          */
    int32_t n_evals;       /* energy+gradient evaluations (all precisions)    */
    int32_t n_evals_f64;   /* of which in double precision                    */
    int64_t true_argmax;   /* judge: argmax of the full screen (-1 if none)   */
    int64_t true_rank;     /* judge: rank of true_argmax among the proposals
                              (0 = proposed first; -1 = not proposed)          */
    double t_screen, t_optimise, t_total;   /* judge time excluded            */
    double t_judge;        /* judge: time of the extra full screen and refit  */
    int64_t support;       /* nonzero amplitudes of psi at the screen when the
                              sparse path ran it, -1 for the dense sweeps     */
    int64_t sigma_support; /* listed nonzeros of sigma = H psi there, -1 when
                              sigma's support was not listed                  */
    int32_t screen;        /* how the operator was selected: 0 the whole pool
                              screened exactly by the dense sweep, 1 the whole
                              pool screened exactly over psi's support (sparse
                              path), 2 the ranker's proposals screened exactly,
                              3 the proposals and then the whole pool (the
                              fallback when the proposals' ||g|| would stop
                              the loop)                                        */
    int32_t pad_;
} hy_adapt_record;


/* Create a driver for (h, p); allocates its state buffers on the device.
 * cfg == NULL takes the defaults: HY_F64, max_iter 64, eps_grad 1e-5,
 * gtol 1e-9, gtol_bulk 1e-5, max_evals 200, refine_steps 4, refine_every 1,
 * full screen, dense sweeps. */
hy_status hy_adapt_create(const hy_ham *h, const hy_pool *p,
                          const hy_adapt_config *cfg, hy_adapt **out);
hy_status hy_adapt_destroy(hy_adapt *a);

/* Run one iteration on `stream` (the host waits for its results).  *rec
 * (host) receives the record.  Returns HY_ERR_ARG when the ansatz is full. */
hy_status hy_adapt_step(hy_adapt *a, hy_adapt_record *rec, void *stream);

/* HY_F32 drivers: refine the current ansatz in double precision (at most
 * `steps` BFGS steps from the current parameters) and return the double
 * energy in *e (host); the parameters are updated.  The run's final energy
 * in the mixed mode comes from this call.  When the last optimisation (of
 * hy_adapt_step or of an earlier refinement) already ran in double and
 * stopped by its own rule (max |dE/dtheta| < gtol, or no representable
 * decrease) and the parameters have not changed since, steps > 0 returns
 * that double energy without evaluating again: the refinement would
 * re-evaluate the same point and stop there.  steps = 0 always evaluates. */
hy_status hy_adapt_refine(hy_adapt *a, int steps, double *e, void *stream);

/* Turn the judge (the extra full screen of every ranked iteration, see
 * hy_adapt_set_ranker) on or off for the following iterations. */
hy_status hy_adapt_set_judge(hy_adapt *a, int judge);

/* Copy the ansatz (host arrays with room for cap entries); *len gets its
 * length.  Pass cap = 0 to query the length. */
hy_status hy_adapt_ansatz(const hy_adapt *a, int64_t *ops, double *thetas,
                          int64_t cap, int64_t *len);

/* Replace the ansatz (checkpoint / resume: the state is rebuilt from HF). */
hy_status hy_adapt_set_ansatz(hy_adapt *a, const int64_t *ops,
                              const double *thetas, int64_t len);

/* Energy and adjoint gradient of the current ansatz at `thetas` (host, len
 * = ansatz length) in `dt`; *e and grad (host, len doubles) are outputs. */
hy_status hy_adapt_evaluate(hy_adapt *a, const double *thetas, hy_dtype dt,
                            double *e, double *grad, void *stream);

/* Bytes the driver has copied host -> device (*h2d) and device -> host
 * (*d2h) since it was created: operator lists, extra ranker features, HF
 * amplitudes, energy / gradient / screen readbacks.  Either may be NULL. */
hy_status hy_adapt_io_bytes(const hy_adapt *a, int64_t *h2d, int64_t *d2h);

/* Copy the driver's current state (after the last evaluation) into psi
 * (device, n_det elements of dt). */
hy_status hy_adapt_state(const hy_adapt *a, void *psi, hy_dtype dt,
                         void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HYPERION_H */
