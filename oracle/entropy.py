"""Orbital entropies and mutual information: CPU reference (TEST INFRASTRUCTURE ONLY).

The paper orders the lattice by the pairwise mutual information I_ij
(Sec. "Cholesky decomposition for the wavefunction: compression and its
cost", ingredient (ii); the diagnostics of Legeza and of Rissler, Noack and
White).  Definitions used (the textbook ones):
  rho_i   one-orbital reduced density matrix (4 x 4, local basis
          |0>, |a>, |b>, |ab>), s_i = -tr rho_i ln rho_i;
  rho_ij  two-orbital reduced density matrix (16 x 16), s_ij likewise;
  I_ij    = s_i + s_j - s_ij  (i != j; 0 on the diagonal).
The reduced density matrices are fermionic partial traces.  The modes are
reordered so that the kept orbitals come first, with the sign of the
permutation of the occupied modes.  Only then are the remaining modes
traced out, so no Jordan-Wigner string runs through the traced part.  A
local state |a b> of orbital i is
c+_{i alpha}^a c+_{i beta}^b |vac>.

Pinned in tests/test_oracle_entropy.py: a closed-shell determinant has zero
entropies; the Hubbard dimer's I_12 equals its closed form; rho_ij is a
density matrix; its hopping element <c+_{i s} c_{j s}> equals the spin
component of the 1-RDM from fock.rdms, including between non-adjacent
orbitals (where a sign error would show).
"""
from __future__ import annotations

import numpy as np


def _reorder(full: np.ndarray, n_orb: int, first) -> np.ndarray:
    """The Fock vector with the modes of the orbitals in `first` moved to the
    front (in the given order, alpha before beta), the rest after them in
    their original order.  Returns an array of shape (4**len(first), rest)."""
    nm = 2 * n_orb
    front = [m for o in first for m in (2 * o, 2 * o + 1)]
    rest = [m for m in range(nm) if m not in front]
    new_order = front + rest                    # new position p holds old mode new_order[p]
    pos = np.empty(nm, dtype=np.int64)
    pos[new_order] = np.arange(nm)
    states = np.nonzero(full)[0]
    out = np.zeros((1 << len(front), 1 << len(rest)))
    for st in states:
        occ = [m for m in range(nm) if (st >> m) & 1]
        p = [pos[m] for m in occ]
        inv = sum(1 for a in range(len(p)) for b in range(a + 1, len(p)) if p[a] > p[b])
        f = sum(1 << k for k, m in enumerate(front) if (st >> m) & 1)
        r = sum(1 << k for k, m in enumerate(rest) if (st >> m) & 1)
        out[f, r] += (-1.0) ** inv * full[st]
    return out


def orbital_rdm(full: np.ndarray, n_orb: int, orbitals) -> np.ndarray:
    """Reduced density matrix of the orbitals (1 or 2 of them) of a
    normalised Fock-space vector.  Index bit 2k is orbital k's alpha mode
    and bit 2k+1 its beta mode."""
    X = _reorder(full, n_orb, list(orbitals))
    return X @ X.T


def entropy(rho: np.ndarray) -> float:
    w = np.linalg.eigvalsh(0.5 * (rho + rho.T))
    w = w[w > 1e-14]
    return float(-np.sum(w * np.log(w)))


def mutual_information(full: np.ndarray, n_orb: int) -> np.ndarray:
    s1 = np.array([entropy(orbital_rdm(full, n_orb, [i])) for i in range(n_orb)])
    I = np.zeros((n_orb, n_orb))
    for i in range(n_orb):
        for j in range(i + 1, n_orb):
            I[i, j] = I[j, i] = s1[i] + s1[j] - entropy(orbital_rdm(full, n_orb, [i, j]))
    return I
