"""Brute-force Fock-space quantum chemistry (TEST INFRASTRUCTURE ONLY).

The active-space Hamiltonian in chemists' notation (the integrals the paper's
DMRG node consumes, Sec. "The DMRG-QD-NEVPT2 energy"):

    H = sum_{pq,sigma} h_pq a+_{p sigma} a_{q sigma}
        + 1/2 sum_{pqrs,sigma,tau} (pq|rs) a+_{p sigma} a+_{r tau} a_{s tau} a_{q sigma}.

Modes are spin orbitals in site-major order m = 2p + spin (spin 0 = alpha,
1 = beta).  A basis state is an integer whose bit m is the occupation n_m and
stands for prod_m (a+_m)^{n_m} |vac> with the lowest mode leftmost.  Then
a+_m |n> = (-1)^{sum_{j<m} n_j} |n + e_m>.  This is the Jordan-Wigner
definition; nothing here is clever.  Only for n_orb <= 6 (4096 states).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def n_modes(n_orb: int) -> int:
    return 2 * n_orb


def _popcount_below(states: np.ndarray, m: int) -> np.ndarray:
    mask = (1 << m) - 1
    x = states & mask
    c = np.zeros_like(x)
    while np.any(x):
        c += x & 1
        x >>= 1
    return c


def apply_string(ops, dim: int):
    """Sparse matrix of an operator string [(mode, dagger), ...]; the
    rightmost operator acts first."""
    cols = np.arange(dim, dtype=np.int64)   # original basis state (column)
    cur = cols.copy()                       # current state reached from it
    amps = np.ones(dim)
    for m, dag in reversed(ops):
        bit = 1 << m
        occ = (cur & bit) != 0
        keep = ~occ if dag else occ
        cols, cur, amps = cols[keep], cur[keep], amps[keep]
        amps = amps * (1 - 2 * (_popcount_below(cur, m) & 1))
        cur = cur ^ bit
    return sp.csr_matrix((amps, (cur, cols)), shape=(dim, dim))


def hamiltonian(h: np.ndarray, eri: np.ndarray) -> sp.csr_matrix:
    """Full Fock-space H (dimension 4^n) from h[p,q] and (pq|rs) = eri[p,q,r,s]."""
    n = h.shape[0]
    dim = 1 << (2 * n)
    H = sp.csr_matrix((dim, dim))
    acc = []
    for p in range(n):
        for q in range(n):
            if h[p, q] == 0.0:
                continue
            for s in range(2):
                acc.append(h[p, q] * apply_string([(2 * p + s, True), (2 * q + s, False)], dim))
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for ss in range(n):
                    v = eri[p, q, r, ss]
                    if v == 0.0:
                        continue
                    for s in range(2):
                        for t in range(2):
                            P, Q, R, S = 2 * p + s, 2 * q + s, 2 * r + t, 2 * ss + t
                            if P == R or Q == S:
                                continue
                            acc.append(0.5 * v * apply_string(
                                [(P, True), (R, True), (S, False), (Q, False)], dim))
    for a in acc:
        H = H + a
    return H.tocsr()


def sector_states(n_orb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """Fock basis states with the given alpha and beta electron counts."""
    dim = 1 << (2 * n_orb)
    st = np.arange(dim, dtype=np.int64)
    na = np.zeros(dim, dtype=np.int64)
    nb = np.zeros(dim, dtype=np.int64)
    for p in range(n_orb):
        na += (st >> (2 * p)) & 1
        nb += (st >> (2 * p + 1)) & 1
    return st[(na == n_alpha) & (nb == n_beta)]


def ground_state(h, eri, n_alpha, n_beta, nroots=1):
    """Lowest eigenpairs of H restricted to the (N_alpha, N_beta) sector by
    dense diagonalisation (numpy eigh).  Returns (energies, vectors, states)."""
    n = h.shape[0]
    H = hamiltonian(h, eri)
    st = sector_states(n, n_alpha, n_beta)
    Hs = H[st][:, st].toarray()
    w, v = np.linalg.eigh(Hs)
    return w[:nroots], v[:, :nroots], st


def rdms(vec: np.ndarray, states: np.ndarray, n_orb: int):
    """Spin-summed 1-RDM gamma_pq = sum_s <a+_ps a_qs> and 2-RDM
    Gamma_pqrs = sum_st <a+_ps a+_rt a_st a_qs> of a sector vector, by
    applying the operator strings of their definitions."""
    dim = 1 << (2 * n_orb)
    full = np.zeros(dim)
    full[states] = vec
    g1 = np.zeros((n_orb, n_orb))
    g2 = np.zeros((n_orb,) * 4)
    for p in range(n_orb):
        for q in range(n_orb):
            for s in range(2):
                op = apply_string([(2 * p + s, True), (2 * q + s, False)], dim)
                g1[p, q] += full @ (op @ full)
    for p in range(n_orb):
        for q in range(n_orb):
            for r in range(n_orb):
                for ss in range(n_orb):
                    for s in range(2):
                        for t in range(2):
                            P, Q, R, S = 2 * p + s, 2 * q + s, 2 * r + t, 2 * ss + t
                            if P == R or Q == S:
                                continue
                            op = apply_string([(P, True), (R, True), (S, False), (Q, False)], dim)
                            g2[p, q, r, ss] += full @ (op @ full)
    return g1, g2


def rdm3(vec: np.ndarray, states: np.ndarray, n_orb: int) -> np.ndarray:
    """Spin-summed 3-RDM Gamma3_pqrstu = sum_{s,t,v} <a+_ps a+_rt a+_tv a_uv a_st a_qs>
    by applying the operator strings of the definition (n_orb <= 4)."""
    dim = 1 << (2 * n_orb)
    full = np.zeros(dim)
    full[states] = vec
    n = n_orb
    G = np.zeros((n,) * 6)
    idx = range(n)
    for p in idx:
        for q in idx:
            for r in idx:
                for s_ in idx:
                    for t in idx:
                        for u in idx:
                            acc = 0.0
                            for a in range(2):
                                for b in range(2):
                                    for c in range(2):
                                        P, Q = 2 * p + a, 2 * q + a
                                        R, S = 2 * r + b, 2 * s_ + b
                                        T, U = 2 * t + c, 2 * u + c
                                        if len({P, R, T}) < 3 or len({Q, S, U}) < 3:
                                            continue
                                        op = apply_string([(P, True), (R, True), (T, True), (U, False), (S, False),
                                                           (Q, False)], dim)
                                        acc += full @ (op @ full)
                            G[p, q, r, s_, t, u] = acc
    return G


def spin_square(n_orb: int) -> sp.csr_matrix:
    """S^2 = S_z^2 + (S_+ S_- + S_- S_+)/2 with S_+ = sum_p a+_pa a_pb,
    S_- = sum_p a+_pb a_pa, S_z = 1/2 sum_p (n_pa - n_pb), from the operator
    strings (the textbook definition)."""
    dim = 1 << (2 * n_orb)
    Sp = sp.csr_matrix((dim, dim))
    Sm = sp.csr_matrix((dim, dim))
    Sz = sp.csr_matrix((dim, dim))
    for p in range(n_orb):
        a, b = 2 * p, 2 * p + 1
        Sp = Sp + apply_string([(a, True), (b, False)], dim)
        Sm = Sm + apply_string([(b, True), (a, False)], dim)
        Sz = Sz + 0.5 * (apply_string([(a, True), (a, False)], dim) - apply_string([(b, True), (b, False)], dim))
    return (Sz @ Sz + 0.5 * (Sp @ Sm + Sm @ Sp)).tocsr()


def from_ci(C: np.ndarray, n_orb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """Fock-space vector of a determinant-basis vector C[I_alpha, I_beta]
    (oracle/fci.py: alpha creators in ascending orbital order, then beta
    creators, strings at their colex addresses).  Each determinant is
    rewritten in this module's site-major creator order; the reordering
    passes every beta creator of orbital q over the alpha creators of the
    orbitals p > q, so its sign is (-1)^(sum_q n_q,beta #{p > q: n_p,alpha})."""
    from oracle import fci
    C = np.asarray(C, dtype=np.float64).reshape(len(fci.strings(n_orb, n_alpha)), -1)
    full = np.zeros(1 << (2 * n_orb))
    for ia, aocc in enumerate(fci.strings(n_orb, n_alpha)):
        for ib, bocc in enumerate(fci.strings(n_orb, n_beta)):
            st = sum(1 << (2 * p) for p in aocc) | sum(1 << (2 * q + 1) for q in bocc)
            ex = sum(1 for q in bocc for p in aocc if p > q)
            full[st] = (-1.0) ** ex * C[ia, ib]
    return full


def eri_from_chol(chol: np.ndarray) -> np.ndarray:
    """(pq|rs) = sum_Q L^Q_pq L^Q_rs (Sec. "The DMRG-QD-NEVPT2 energy",
    Cholesky-factorised two-electron tensor)."""
    return np.einsum("Qpq,Qrs->pqrs", chol, chol)
