"""Partitioned Hamiltonian of the SV-MPS scheme in the oracle (test
infrastructure, FP64, CPU; shares no code with the CUDA path).

The paper's partitioned SV-MPS emulation (Partitioned SV-MPS Emulation
section) splits the n-qubit Hamiltonian as H = H_eta + sum B: the qubit chain
is cut into 2^eta contiguous blocks, H_eta is the sum over blocks of the
operator acting inside that block alone (a 2^(n/2^eta)-dimensional H^(i)
tensored with identities), and the B terms hold everything that couples
blocks; the expectation value splits the same way, <psi|H_eta|psi> being
evaluated exactly on the state vector.

Here H is expanded into Pauli strings from its second-quantised definition
under Jordan-Wigner (blocked order: qubit j is spin orbital j, alpha
orbitals first; |1> = occupied):
    a_j  = Z^(j-1..0) (X_j + i Y_j) / 2,   a+_j = Z^(j-1..0) (X_j - i Y_j) / 2,
written in the form c X^x Z^z (with Y = i X Z), products by
X^x1 Z^z1 X^x2 Z^z2 = (-1)^|z1 & x2| X^(x1^x2) Z^(z1^z2).  A term belongs to
H_eta when its support x | z lies inside one block of the chosen chain
order (the identity with H_eta).  The filtered operator is applied as a
dense matrix on the full 2^n space, then restricted to Omega_CIk.
"""
from __future__ import annotations

import numpy as np


def _popcount(v: int) -> int:
    return bin(v).count("1")


def _lower(j: int) -> int:
    return (1 << j) - 1


def _annihilate(j):
    e, m = 1 << j, _lower(j)
    return [(0.5, e, m), (-0.5, e, m | e)]


def _create(j):
    e, m = 1 << j, _lower(j)
    return [(0.5, e, m), (0.5, e, m | e)]


def _mul(A, B):
    out = []
    for c1, x1, z1 in A:
        for c2, x2, z2 in B:
            sg = -1.0 if _popcount(z1 & x2) & 1 else 1.0
            out.append((c1 * c2 * sg, x1 ^ x2, z1 ^ z2))
    return out


def jw_terms(h1, h2, e_core, n, tol=1e-14) -> dict:
    """{(x, z): c} with H = sum c X^x Z^z, from
    H = e_core + sum h_pq a+_ps a_qs + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs
    (chemists' notation, s, t spins); |c| <= tol dropped."""
    acc: dict = {}

    def add(terms, w):
        for c, x, z in terms:
            acc[(x, z)] = acc.get((x, z), 0.0) + w * c

    add([(1.0, 0, 0)], e_core)
    for sp in (0, 1):
        for p in range(n):
            for q in range(n):
                if h1[p, q] != 0.0:
                    add(_mul(_create(p + sp * n), _annihilate(q + sp * n)), h1[p, q])
    for s1 in (0, 1):
        for s2 in (0, 1):
            for p in range(n):
                for q in range(n):
                    for r in range(n):
                        for s in range(n):
                            v = h2[p, q, r, s]
                            if v == 0.0:
                                continue
                            P, Q, R, S = p + s1 * n, q + s1 * n, r + s2 * n, s + s2 * n
                            if P == R or Q == S:
                                continue            # a+ a+ (or a a) on one mode vanishes
                            t = _mul(_mul(_create(P), _create(R)),
                                     _mul(_annihilate(S), _annihilate(Q)))
                            add(t, 0.5 * v)
    return {k: c for k, c in acc.items() if abs(c) > tol}


def chain_position(j: int, n: int, interleaved: bool) -> int:
    """Position of spin orbital j (blocked numbering) along the chain being
    cut: itself, or 2p (alpha) / 2p + 1 (beta) for orbital p."""
    if not interleaved:
        return j
    return 2 * j if j < n else 2 * (j - n) + 1


def partition_terms(terms: dict, n: int, eta: int, interleaved: bool, part: int) -> dict:
    """The terms inside one of the 2^eta blocks (part 0, H_eta) or the rest
    (part 1)."""
    width = (2 * n) >> eta
    out = {}
    for (x, z), c in terms.items():
        sup = x | z
        blocks = {chain_position(j, n, interleaved) // width
                  for j in range(2 * n) if (sup >> j) & 1}
        inside = len(blocks) <= 1
        if inside == (part == 0):
            out[(x, z)] = c
    return out


def dense_full(terms: dict, n_qubits: int) -> np.ndarray:
    """The operator sum c X^x Z^z as a real 2^n x 2^n matrix (basis index =
    the occupation mask); X^x Z^z |d> = (-1)^|d & z| |d ^ x>.  Every c of this
    form is real: the factors of a+ and a are, and so are their products."""
    dim = 1 << n_qubits
    d = np.arange(dim, dtype=np.int64)
    H = np.zeros((dim, dim))
    for (x, z), c in terms.items():
        par = np.zeros(dim, dtype=np.int64)
        zz = d & z
        while np.any(zz):
            par ^= zz & 1
            zz >>= 1
        sgn = 1.0 - 2.0 * par
        H[d ^ x, d] += c * sgn
    return H


class Partition:
    """H_eta or its complement for an oracle.System, restricted to Omega_CIk."""

    def __init__(self, system, h1, h2, e_core, eta, interleaved=False, part=0):
        n = system.n
        self.terms = partition_terms(jw_terms(h1, h2, e_core, n), n, eta, interleaved, part)
        full = dense_full(self.terms, 2 * n)
        dets = system.dets().astype(np.int64)
        self.leak = float(np.abs(np.delete(full[:, dets], dets, axis=0)).max()) \
            if len(dets) < full.shape[0] else 0.0
        self.H = full[np.ix_(dets, dets)]
        self.trace_full = float(np.trace(full))

    def sigma(self, psi):
        return self.H @ psi

    def energy(self, psi):
        return float(psi @ self.H @ psi)
