// hy_build.cpp -- host-side construction of everything the kernels read:
// determinant string spaces, the Jordan-Wigner Pauli table grouped by
// X-mask, the kernel tables folded from that table, and the operator pool.
//
// Paper: "Sparse State-Vector Emulation" section -- the Hamiltonian is
// assembled by summing the contributions of individual fermionic operators
// after a qubit mapping (Jordan-Wigner here) and the state lives on the
// particle- and S_z-conserving determinant space Omega_CIk.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "hy_internal.h"

namespace hy {

// ---------------------------------------------------------------------------
// combinatorics
// ---------------------------------------------------------------------------
namespace {
struct BinomTable {
    uint32_t c[33][33];
    BinomTable()
    {
        std::memset(c, 0, sizeof c);
        for (int n = 0; n <= 32; ++n) {
            c[n][0] = 1;
            for (int k = 1; k <= n; ++k)
                c[n][k] = c[n - 1][k - 1] + (k <= n - 1 ? c[n - 1][k] : 0);
        }
    }
};
const BinomTable &btab()
{
    static const BinomTable t;
    return t;
}
}  // namespace

uint32_t binom(int n, int k)
{
    if (n < 0 || k < 0 || k > n || n > 32) return 0;
    return btab().c[n][k];
}

uint32_t string_rank(uint32_t mask)
{
    uint32_t r = 0;
    int i = 0;
    while (mask) {
        int pos = __builtin_ctz(mask);
        r += binom(pos, i + 1);
        ++i;
        mask &= mask - 1;
    }
    return r;
}

uint32_t string_unrank(uint32_t rank, int k)
{
    uint32_t mask = 0;
    for (int i = k - 1; i >= 0; --i) {
        int pos = i;
        while (binom(pos + 1, i + 1) <= rank) ++pos;
        mask |= 1u << pos;
        rank -= binom(pos, i + 1);
    }
    return mask;
}

static inline uint32_t between_mask(int p, int q)
{
    int lo = p < q ? p : q, hi = p < q ? q : p;
    if (hi - lo < 2) return 0u;
    return ((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u);
}

void build_string_space(int n, int k, StringSpace &s)
{
    s.n = n;
    s.k = k;
    s.N = binom(n, k);
    s.nex = k * (n - k);
    s.str.resize(s.N);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < s.N; ++r) s.str[r] = string_unrank(uint32_t(r), k);
    s.ex.assign(size_t(s.N) * s.nex, 0u);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < s.N; ++r) {
        uint32_t K = s.str[r];
        int e = 0;
        for (int p = 0; p < n; ++p) {
            if (!((K >> p) & 1)) continue;
            for (int q = 0; q < n; ++q) {
                if ((K >> q) & 1) continue;
                uint32_t J = K ^ (1u << p) ^ (1u << q);
                int neg = __builtin_popcount(K & between_mask(p, q)) & 1;
                s.ex[size_t(r) * s.nex + e++] = pack_ex(string_rank(J), p, q, neg);
            }
        }
    }
    // inverse positions: the partner J of (r, e) lists r at the entry whose
    // orbitals are swapped (J lacks p and holds q).  A string lists its
    // excitations by occupied orbital, then by empty orbital, both ascending,
    // so that entry is (rank of q among J's occupied) * (n - k) + (rank of p
    // among J's empty orbitals)
    s.inv.assign(size_t(s.N) * s.nex, 0);
    const uint32_t full = n >= 32 ? ~0u : (1u << n) - 1u;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < s.N; ++r) {
        const uint32_t K = s.str[r];
        int e = 0;
        for (int p = 0; p < n; ++p) {
            if (!((K >> p) & 1)) continue;
            for (int q = 0; q < n; ++q) {
                if ((K >> q) & 1) continue;
                const uint32_t J = K ^ (1u << p) ^ (1u << q);
                const int oq = __builtin_popcount(J & ((1u << q) - 1u));
                const int ep = __builtin_popcount(~J & full & ((1u << p) - 1u));
                s.inv[size_t(r) * s.nex + e++] = uint8_t(oq * (n - k) + ep);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Jordan-Wigner Pauli table
// ---------------------------------------------------------------------------
// Under Jordan-Wigner with qubit j = spin orbital j,
//   a_j  = 1/2 X^{e_j} Z^{L_j} - 1/2 X^{e_j} Z^{L_j | e_j},
//   a+_j = 1/2 X^{e_j} Z^{L_j} + 1/2 X^{e_j} Z^{L_j | e_j},
// with L_j the qubits below j, and
//   (X^x1 Z^z1)(X^x2 Z^z2) = (-1)^popcount(z1 & x2) X^(x1^x2) Z^(z1^z2).
namespace {
// Coefficient accumulator keyed by (x | z << 32): open addressing with
// linear probing; every key keeps its contributions in insertion order, so
// the sums do not depend on the table's size or layout.
class PauliAcc {
  public:
    PauliAcc() : key_(size_t(1) << 16), val_(size_t(1) << 16), used_(size_t(1) << 16, 0) {}
    double &operator[](uint64_t k)
    {
        size_t h = slot(k);
        if (!used_[h]) {
            if (2 * (count_ + 1) > used_.size()) {
                grow();
                h = slot(k);
            }
            used_[h] = 1;
            key_[h] = k;
            val_[h] = 0.0;
            ++count_;
        }
        return val_[h];
    }
    size_t size() const { return count_; }
    template <typename F>
    void for_each(F &&f) const
    {
        for (size_t i = 0; i < used_.size(); ++i)
            if (used_[i]) f(key_[i], val_[i]);
    }

  private:
    size_t slot(uint64_t k) const
    {
        const size_t mask = used_.size() - 1;
        uint64_t x = k * 0x9E3779B97F4A7C15ull;
        size_t h = size_t(x >> 17) & mask;
        while (used_[h] && key_[h] != k) h = (h + 1) & mask;
        return h;
    }
    void grow()
    {
        std::vector<uint64_t> k0;
        std::vector<double> v0;
        std::vector<uint8_t> u0;
        k0.swap(key_);
        v0.swap(val_);
        u0.swap(used_);
        key_.assign(2 * u0.size(), 0);
        val_.assign(2 * u0.size(), 0.0);
        used_.assign(2 * u0.size(), 0);
        for (size_t i = 0; i < u0.size(); ++i)
            if (u0[i]) {
                const size_t h = slot(k0[i]);
                used_[h] = 1;
                key_[h] = k0[i];
                val_[h] = v0[i];
            }
    }
    std::vector<uint64_t> key_;
    std::vector<double> val_;
    std::vector<uint8_t> used_;
    size_t count_ = 0;
};

void add_operator_product(const int *mode, const int *dag, int nops, double coef, PauliAcc &acc)
{
    for (int choice = 0; choice < (1 << nops); ++choice) {
        uint64_t x = 0, z = 0;
        double c = coef;
        for (int t = 0; t < nops; ++t) {
            uint64_t e = 1ull << mode[t];
            int b = (choice >> t) & 1;
            uint64_t xt = e, zt = (e - 1) | (b ? e : 0);
            if (__builtin_popcountll(z & xt) & 1) c = -c;
            x ^= xt;
            z ^= zt;
            c *= b ? (dag[t] ? 0.5 : -0.5) : 0.5;
        }
        acc[x | (z << 32)] += c;
    }
}
}  // namespace

bool build_pauli_table(const double *h1, const double *h2, double e_core, int n,
                       double prune_tol, PauliTable &t, std::string &err)
{
    // Every product's Pauli strings share its X-mask (the XOR of its modes),
    // so the X-masks split the work: each thread accumulates the products
    // whose X-mask falls in its class, visiting them in the loop order below.
    // Every coefficient is therefore summed in exactly the serial order,
    // whatever the number of threads.
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    std::vector<PauliAcc> part(nthreads);
    auto cls = [nthreads](uint64_t x) {
        return int(((x * 0x9E3779B97F4A7C15ull) >> 40) % uint64_t(nthreads));
    };
#pragma omp parallel num_threads(nthreads)
    {
        int me = 0;
#ifdef _OPENMP
        me = omp_get_thread_num();
#endif
        PauliAcc &acc = part[me];
        if (cls(0) == me) acc[0] += e_core;
        for (int sp = 0; sp < 2; ++sp)
            for (int p = 0; p < n; ++p)
                for (int q = 0; q < n; ++q) {
                    double c = h1[p * n + q];
                    if (c == 0.0) continue;
                    int P = p + sp * n, Q = q + sp * n;
                    if (cls((1ull << P) ^ (1ull << Q)) != me) continue;
                    int mode[2] = {P, Q}, dag[2] = {1, 0};
                    add_operator_product(mode, dag, 2, c, acc);
                }
        for (int s1 = 0; s1 < 2; ++s1)
            for (int s2 = 0; s2 < 2; ++s2)
                for (int p = 0; p < n; ++p)
                    for (int q = 0; q < n; ++q)
                        for (int r = 0; r < n; ++r)
                            for (int s = 0; s < n; ++s) {
                                double c = h2[((size_t(p) * n + q) * n + r) * n + s];
                                if (c == 0.0) continue;
                                int P = p + s1 * n, Q = q + s1 * n;
                                int R = r + s2 * n, S = s + s2 * n;
                                if (P == R || Q == S) continue;   // a+a+ / aa vanish
                                const uint64_t x = (1ull << P) ^ (1ull << Q) ^ (1ull << R) ^
                                                   (1ull << S);
                                if (cls(x) != me) continue;
                                // 1/2 (pq|rs) a+_P a+_R a_S a_Q
                                int mode[4] = {P, R, S, Q}, dag[4] = {1, 1, 0, 0};
                                add_operator_product(mode, dag, 4, 0.5 * c, acc);
                            }
    }
    struct Term { uint64_t x, z; double c; };
    std::vector<Term> terms;
    bool odd_y = false;
    for (const PauliAcc &acc : part)
        acc.for_each([&](uint64_t key, double c) {
            if (std::fabs(c) <= prune_tol) return;
            uint64_t x = key & 0xffffffffull, z = key >> 32;
            if (__builtin_popcountll(x & z) & 1) odd_y = true;
            terms.push_back({x, z, c});
        });
    if (odd_y) {
        err = "Pauli term with an odd number of Y survives: the "
              "Hamiltonian is not real symmetric";
        return false;
    }
    std::sort(terms.begin(), terms.end(), [](const Term &a, const Term &b) {
        return a.x != b.x ? a.x < b.x : a.z < b.z;
    });
    t.n_qubits = 2 * n;
    t.x.resize(terms.size());
    t.z.resize(terms.size());
    t.cxz.resize(terms.size());
    t.group_off.clear();
    t.group_of_x.clear();
    for (size_t i = 0; i < terms.size(); ++i) {
        t.x[i] = terms[i].x;
        t.z[i] = terms[i].z;
        t.cxz[i] = terms[i].c;
        if (i == 0 || terms[i].x != terms[i - 1].x) {
            t.group_of_x[terms[i].x] = int64_t(t.group_off.size());
            t.group_off.push_back(int64_t(i));
        }
    }
    t.group_off.push_back(int64_t(terms.size()));
    return true;
}

double PauliTable::element(uint64_t bra, uint64_t ket) const
{
    auto it = group_of_x.find(bra ^ ket);
    if (it == group_of_x.end()) return 0.0;
    double v = 0.0;
    for (int64_t j = group_off[it->second]; j < group_off[it->second + 1]; ++j)
        v += (__builtin_popcountll(ket & z[j]) & 1) ? -cxz[j] : cxz[j];
    return v;
}

bool check_two_body_structure(const PauliTable &t, int n, std::string &err)
{
    uint64_t amask = (1ull << n) - 1;
    for (size_t g = 0; g + 1 < t.group_off.size(); ++g) {
        uint64_t x = t.x[t.group_off[g]];
        int na = __builtin_popcountll(x & amask);
        int nb = __builtin_popcountll(x >> n);
        if ((na & 1) || (nb & 1) || na + nb > 4) {
            err = "Pauli group does not conserve N_alpha / N_beta or is beyond two-body";
            return false;
        }
        uint64_t B = 0;
        for (int m = 0; m < 2 * n; ++m)
            if (!((x >> m) & 1) && (__builtin_popcountll(x >> (m + 1)) & 1))
                B |= 1ull << m;
        int w = na + nb;
        for (int64_t j = t.group_off[g]; j < t.group_off[g + 1]; ++j) {
            uint64_t rest = (t.z[j] & ~x) ^ B;
            int pr = __builtin_popcountll(rest);
            bool ok = (w == 0 && __builtin_popcountll(t.z[j]) <= 2) ||
                      (w == 2 && pr <= 1) || (w == 4 && pr == 0);
            if (!ok) {
                err = "Pauli group is not of two-body Jordan-Wigner form";
                return false;
            }
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Folding: kernel tables as matrix elements of the Pauli table.
// ---------------------------------------------------------------------------
// For a two-body H the determinant matrix element splits exactly into
//   * an alpha-only part: <(a',0)|H|(J,0)>, independent of the beta string;
//   * a beta-only part: <(0,b')|H|(0,J)> (minus the vacuum energy on the
//     diagonal so it is counted once);
//   * an alpha-beta coupling sa * sb * V[p][q][r][s], where V is read off
//     one-electron-per-spin determinants: single-excitation elements are
//     affine in the spectator occupations and the diagonal is quadratic,
//     so the differences below isolate exactly the cross terms.
// The two same-spin parts are folded on the GPU (hy_fold.cu, the same
// element formula as PauliTable::element); the host keeps E0 and V.
void fold_coupling(const PauliTable &t, int n, KernelTables &kt)
{
    kt.E0 = t.element(0, 0);
    kt.V.assign(size_t(n) * n * n * n, 0.0);
    auto a_ = [](int p) { return 1ull << p; };
    auto b_ = [n](int r) { return 1ull << (n + r); };
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
            for (int r = 0; r < n; ++r)
                for (int s = 0; s < n; ++s) {
                    double v;
                    uint64_t bra = a_(p) | b_(r), ket = a_(q) | b_(s);
                    if (p != q && r != s)
                        v = t.element(bra, ket);
                    else if (p != q)
                        v = t.element(bra, ket) - t.element(a_(p), a_(q));
                    else if (r != s)
                        v = t.element(bra, ket) - t.element(b_(r), b_(s));
                    else
                        v = t.element(bra, bra) - t.element(a_(p), a_(p)) -
                            t.element(b_(r), b_(r)) + kt.E0;
                    kt.V[((size_t(p) * n + q) * n + r) * n + s] = v;
                }
}

// ---------------------------------------------------------------------------
// Operator pool: spin-adapted singles and doubles relative to HF.
// ---------------------------------------------------------------------------
namespace {
struct PoolBuilder {
    int n, na, nb;
    std::vector<PoolOpHost> *ops;
    bool hf(int mode) const
    {
        return mode < n ? mode < na : (mode - n) < nb;
    }
    bool ok1(int c0, int a0) const { return hf(a0) && !hf(c0); }
    bool ok2(const int *t) const   // t = {2, c0, c1, a1, a0}
    {
        return hf(t[4]) && hf(t[3]) && !hf(t[1]) && !hf(t[2]);
    }
    void push(const std::vector<std::array<int, 5>> &cons)
    {
        if (cons.empty()) return;
        PoolOpHost o;
        std::memset(o.desc, 0, sizeof o.desc);
        o.desc[0] = int32_t(cons.size());
        for (size_t c = 0; c < cons.size(); ++c)
            for (int u = 0; u < 5; ++u) o.desc[1 + 5 * c + u] = cons[c][u];
        ops->push_back(o);
    }
};
}  // namespace

void build_pool_spin_adapted(int n, int na, int nb, std::vector<PoolOpHost> &ops)
{
    ops.clear();
    PoolBuilder pb{n, na, nb, &ops};
    // singles i -> a
    for (int i = 0; i < n; ++i)
        for (int a = i + 1; a < n; ++a) {
            std::vector<std::array<int, 5>> cons;
            for (int sp = 0; sp < 2; ++sp)
                if (pb.ok1(a + sp * n, i + sp * n))
                    cons.push_back({1, a + sp * n, 0, 0, i + sp * n});
            pb.push(cons);
        }
    // same-spin doubles
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            for (int a = 0; a < n; ++a)
                for (int b = a + 1; b < n; ++b) {
                    std::vector<std::array<int, 5>> cons;
                    for (int sp = 0; sp < 2; ++sp) {
                        int o = sp * n;
                        std::array<int, 5> t{2, a + o, b + o, j + o, i + o};
                        if (pb.ok2(t.data())) cons.push_back(t);
                    }
                    pb.push(cons);
                }
    // opposite-spin doubles
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j)
            for (int a = 0; a < n; ++a)
                for (int b = a; b < n; ++b) {
                    std::array<int, 5> c1{2, a, b + n, j + n, i};
                    std::array<int, 5> c2{2, a + n, b, j, i + n};
                    bool v1 = pb.ok2(c1.data()), v2 = pb.ok2(c2.data());
                    if (i < j && a < b) {
                        std::vector<std::array<int, 5>> cons;
                        if (v1) cons.push_back(c1);
                        if (v2) cons.push_back(c2);
                        pb.push(cons);
                        std::array<int, 5> d1{2, a, b + n, i + n, j};
                        std::array<int, 5> d2{2, a + n, b, i, j + n};
                        cons.clear();
                        if (pb.ok2(d1.data())) cons.push_back(d1);
                        if (pb.ok2(d2.data())) cons.push_back(d2);
                        pb.push(cons);
                    } else if (i == j && a == b) {
                        if (v1) pb.push({c1});
                    } else {
                        if (v1) pb.push({c1});
                        if (v2) pb.push({c2});
                    }
                }
}

void build_pool_qeb(int n, int na, int nb, std::vector<PoolOpHost> &ops)
{
    ops.clear();
    PoolBuilder pb{n, na, nb, &ops};
    // singles i -> a, alpha then beta
    for (int sp = 0; sp < 2; ++sp)
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < n; ++a)
                if (pb.ok1(a + sp * n, i + sp * n)) pb.push({{1, a + sp * n, 0, 0, i + sp * n}});
    // same-spin doubles (i < j) -> (a < b), alpha-alpha then beta-beta
    for (int sp = 0; sp < 2; ++sp) {
        const int o = sp * n;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j)
                for (int a = 0; a < n; ++a)
                    for (int b = a + 1; b < n; ++b) {
                        std::array<int, 5> t{2, a + o, b + o, j + o, i + o};
                        if (pb.ok2(t.data())) pb.push({t});
                    }
    }
    // opposite-spin doubles (i alpha, j beta) -> (a alpha, b beta)
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b) {
                    std::array<int, 5> t{2, a, b + n, j + n, i};
                    if (pb.ok2(t.data())) pb.push({t});
                }
}

bool PatternKey::operator==(const PatternKey &o) const
{
    if (nops != o.nops || qubit != o.qubit) return false;
    for (int i = 0; i < nops; ++i)
        if (ops[i] != o.ops[i]) return false;
    return true;
}

size_t PatternKeyHash::operator()(const PatternKey &k) const
{
    size_t h = size_t(k.nops) * 2 + size_t(k.qubit);
    for (int i = 0; i < k.nops; ++i) h = h * 131 + size_t(k.ops[i]);
    return h;
}

// Apply a product of operators (rightmost first) to one spin string of n
// modes; sign (-1)^(occupied modes below) per fermionic operator, none for
// qubit operators.
static bool apply_within_string(const PatternKey &k, uint32_t s, uint32_t &out,
                                int &neg)
{
    neg = 0;
    for (int t = k.nops - 1; t >= 0; --t) {
        int mode = k.ops[t] >> 1, dag = k.ops[t] & 1;
        uint32_t bit = 1u << mode;
        int occ = (s & bit) != 0;
        if (occ == dag) return false;
        if (!k.qubit) neg ^= __builtin_popcount(s & (bit - 1)) & 1;
        s ^= bit;
    }
    out = s;
    return true;
}

int PatternLists::get(const PatternKey &k)
{
    auto it = id.find(k);
    if (it != id.end()) return it->second;
    const int pid = int(keys.size());
    id[k] = pid;
    keys.push_back(k);
    return pid;
}

void PatternLists::finalize(const StringSpace &s)
{
    const int64_t np = int64_t(keys.size());
    std::vector<std::vector<uint32_t>> lists(np);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t pid = 0; pid < np; ++pid) {
        auto &l = lists[pid];
        for (int64_t r = 0; r < s.N; ++r) {
            uint32_t out;
            int neg;
            if (!apply_within_string(keys[pid], s.str[r], out, neg)) continue;
            const uint32_t img = string_rank(out);
            l.push_back(uint32_t(r) | (img << 15) | (uint32_t(neg) << 31));
        }
    }
    off.assign(np, 0);
    cnt.assign(np, 0);
    int64_t tot = 0;
    for (int64_t pid = 0; pid < np; ++pid) {
        off[pid] = tot;
        cnt[pid] = int64_t(lists[pid].size());
        tot += cnt[pid];
    }
    entry.resize(tot);
#pragma omp parallel for schedule(static)
    for (int64_t pid = 0; pid < np; ++pid)
        std::copy(lists[pid].begin(), lists[pid].end(), entry.begin() + off[pid]);
}

}  // namespace hy
