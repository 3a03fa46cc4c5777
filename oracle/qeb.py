"""Qubit-excitation-based (QEB) operator pool of the oracle (test
infrastructure, FP64, CPU; shares no code with the CUDA path).

The paper's ADAPT-VQE runs draw their operators from a QEB pool (Numerical
performance subsection).  A qubit excitation moves electrons between spin
orbitals like a fermionic excitation but without the Jordan-Wigner parity
string: with Q+ = (X - iY)/2 on one qubit (|0> -> |1>, occupied = 1),
    single  C = Q+_a Q_i,            double  C = Q+_a Q+_b Q_j Q_i,
C maps a determinant with i (and j) occupied and a (and b) empty to the
determinant with those electrons moved, coefficient +1; the pool's
generators are A = C - C^dagger.  Reading where the paper names the pool
only: one operator per spin-orbital single (same spin) and double (S_z
kept) from the Hartree-Fock occupied to the virtual spin orbitals, in the
order alpha singles, beta singles, alpha-alpha, beta-beta, alpha-beta
doubles, each lexicographic in (i, [j,] a [, b]).

QubitSystem wraps an oracle.System and replaces its pool, exp(theta A),
A psi and gradients by the qubit versions, so oracle.adapt runs ADAPT-VQE
over the QEB pool unchanged.  Operators use the descriptor layout of the
fermionic pool, [1, rank, c0, c1, a1, a0, 0, ...], modes in blocked order.
"""
from __future__ import annotations

import numpy as np


class QubitSystem:
    def __init__(self, system):
        self.s = system
        self.n_det = system.n_det
        dets = system.dets().astype(np.uint64)
        self._dets = dets
        self._order = np.argsort(dets)
        self._sorted = dets[self._order]
        self._cache = {}

    # -- the wrapped system's Hamiltonian side --------------------------------
    def sigma(self, psi, nthreads: int = 0):
        return self.s.sigma(psi, nthreads)

    def energy(self, psi):
        return self.s.energy(psi)

    def hf_state(self):
        return self.s.hf_state()

    def fci_energy(self):
        return self.s.fci_energy()

    def dets(self):
        return self.s.dets()

    # -- the pool -----------------------------------------------------------------
    def pool(self) -> np.ndarray:
        n, na, nb = self.s.n, self.s.na, self.s.nb
        occ = [list(range(na)), list(range(nb))]
        vir = [list(range(na, n)), list(range(nb, n))]
        ops = []
        for sp in (0, 1):
            for i in occ[sp]:
                for a in vir[sp]:
                    ops.append([1, 1, a + sp * n, 0, 0, i + sp * n])
        for sp in (0, 1):
            o = sp * n
            for i in occ[sp]:
                for j in occ[sp]:
                    if j <= i:
                        continue
                    for a in vir[sp]:
                        for b in vir[sp]:
                            if b <= a:
                                continue
                            ops.append([1, 2, a + o, b + o, j + o, i + o])
        for i in occ[0]:
            for j in occ[1]:
                for a in vir[0]:
                    for b in vir[1]:
                        ops.append([1, 2, a, b + n, j + n, i])
        out = np.zeros((len(ops), 11), dtype=np.int32)
        if ops:
            out[:, :6] = np.array(ops, dtype=np.int32)
        return out

    def _pairs(self, op):
        """(domain indices, image indices) of the operator's pairs: the
        determinants holding its annihilated spin orbitals and lacking its
        created ones, and where the qubit excitation takes them."""
        key = tuple(int(v) for v in op[:6])
        if key in self._cache:
            return self._cache[key]
        rank = int(op[1])
        created = [int(op[2])] + ([int(op[3])] if rank == 2 else [])
        annihilated = [int(op[5])] + ([int(op[4])] if rank == 2 else [])
        occ_mask = np.uint64(sum(1 << m for m in annihilated))
        vir_mask = np.uint64(sum(1 << m for m in created))
        d = self._dets
        dom = np.flatnonzero(((d & occ_mask) == occ_mask) & ((d & vir_mask) == 0))
        img_det = d[dom] ^ occ_mask ^ vir_mask
        img = self._order[np.searchsorted(self._sorted, img_det)]
        assert np.array_equal(d[img], img_det)
        self._cache[key] = (dom, img)
        return dom, img

    def apply_generator(self, op, psi):
        """(C - C^dagger) psi: C|d> = |d'> adds psi_d to d', C^dagger|d'> = |d>
        subtracts psi_d' from d."""
        dom, img = self._pairs(op)
        out = np.zeros_like(psi)
        out[img] += psi[dom]
        out[dom] -= psi[img]
        return out

    def apply_excitation(self, op, theta, psi):
        """exp(theta (C - C^dagger)) psi, exactly: each pair (d, d' = C d) is
        rotated by theta (A^2 = -1 on the span of a pair, 0 elsewhere)."""
        dom, img = self._pairs(op)
        out = np.array(psi, dtype=np.float64, copy=True)
        c, s = np.cos(theta), np.sin(theta)
        x, y = psi[dom], psi[img]
        out[dom] = c * x - s * y
        out[img] = c * y + s * x
        return out

    def gradients(self, pool, psi, sigma, nthreads: int = 0):
        """g_k = dE/dtheta_k at 0 = 2 <sigma|A_k psi> for each operator."""
        return np.array([2.0 * float(sigma @ self.apply_generator(op, psi)) for op in pool])
