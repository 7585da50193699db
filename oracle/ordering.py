"""Fiedler ordering of the orbitals: CPU reference (TEST INFRASTRUCTURE ONLY).

The paper orders the lattice by mutual information: Fiedler ordering, with
I_ij as the pre-screen that orders the lattice (Sec. "Cholesky decomposition
for the wavefunction: compression and its cost", ingredient (ii)).  The
ordering step itself is the textbook spectral one (Fiedler 1973): for
symmetric, non-negative couplings W between orbitals (the diagonal
ignored),
    L = D - W,   D_ii = sum_{j != i} W_ij   (the graph Laplacian),
f = the eigenvector of the second-smallest eigenvalue of L, and the
orbitals placed on the chain in ascending f, with equal values in index
order.  f is fixed only up to sign: of the two directions, the one whose
first orbital has the smaller index is taken.  A second eigenvalue that
equals the first (a disconnected graph) or the third (to 1e-10 of the
spectrum's scale) leaves f undefined and is an error.  order[k] is the
original orbital placed at site k; integrals follow as h'[a, b] =
h[order[a], order[b]].

This module takes W as given.  The mutual information the paper feeds it
needs two-orbital density matrices of the wavefunction, which are not
computed here.

Pinned in tests/test_oracle_ordering.py: a path graph under scrambled
labels is put back in path order; two weakly coupled clusters end up
contiguous; the FCI energy is invariant under the permutation of the
integrals.
"""
from __future__ import annotations

import numpy as np


def fiedler_order(W: np.ndarray) -> np.ndarray:
    W = np.asarray(W, dtype=np.float64)
    n = W.shape[0]
    if n <= 2:
        return np.arange(n)
    A = W.copy()
    np.fill_diagonal(A, 0.0)
    L = np.diag(A.sum(axis=1)) - A
    w, Z = np.linalg.eigh(L)
    tol = 1e-10 * max(1.0, abs(w[-1]))
    if w[1] - w[0] <= tol or w[2] - w[1] <= tol:
        raise ValueError("second Laplacian eigenvalue is degenerate (or the graph is disconnected)")
    order = np.argsort(Z[:, 1], kind="stable")
    if order[0] > order[-1]:
        order = order[::-1].copy()
    return order


def permute_integrals(h, chol, order):
    """h'[a, b] = h[order[a], order[b]], chol'[Q, a, b] = chol[Q, order[a], order[b]]."""
    o = np.asarray(order)
    return h[np.ix_(o, o)], chol[:, o][:, :, o]
