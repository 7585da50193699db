"""Determinant-space full CI (TEST INFRASTRUCTURE ONLY).

The exact target of the DMRG sweep: at full bond dimension MPO-DMRG equals
FCI in the active space (Sec. "Cholesky decomposition for the wavefunction",
item (i); Sec. "The engine reproduces FCI-in-active-space"; Table "valid").

Determinants are |I_a, I_b> = (alpha creators in orbital order)(beta creators
in orbital order)|vac>.  Strings are addressed by the colexicographic rank
addr = sum_i C(o_i, i+1) over the sorted occupied orbitals o_0 < o_1 < ...
(Sec. "Computational details", device-native perturbative correction).

H C is applied with the Knowles-Handy resolution
    H = sum_pq k_pq E_pq + 1/2 sum_pqrs (pq|rs) E_pq E_rs,
    k_pq = h_pq - 1/2 sum_r (pr|rq),
and the ground state is found by Davidson (dense eigh for small spaces).
Pinned against fock.py (brute-force Jordan-Wigner H) on small spaces and
against closed forms in tests/test_oracle_fci.py.
"""
from __future__ import annotations

from itertools import combinations
from math import comb

import numpy as np


def colex_addr(occ) -> int:
    """addr = sum_i C(o_i, i+1) for sorted occupied orbitals."""
    return sum(comb(o, i + 1) for i, o in enumerate(sorted(occ)))


def strings(n: int, k: int):
    """All k-electron strings of n orbitals, as a list indexed by colex addr."""
    out = [None] * comb(n, k)
    for occ in combinations(range(n), k):
        out[colex_addr(occ)] = occ
    return out


def single_excitations(n: int, k: int):
    """Arrays (I, J, pq, sign) with E_pq |I> = sign |J> for every string I,
    occupied q and p not occupied in I - {q} (p == q included)."""
    strs = strings(n, k)
    I_l, J_l, pq_l, s_l = [], [], [], []
    for I, occ in enumerate(strs):
        occ_set = set(occ)
        for q in occ:
            rest = sorted(occ_set - {q})
            sign_q = (-1) ** sum(1 for o in occ if o < q)
            for p in range(n):
                if p in rest:
                    continue
                sign_p = (-1) ** sum(1 for o in rest if o < p)
                J = colex_addr(rest + [p])
                I_l.append(I)
                J_l.append(J)
                pq_l.append(p * n + q)
                s_l.append(sign_q * sign_p)
    return (np.array(I_l, dtype=np.int64), np.array(J_l, dtype=np.int64),
            np.array(pq_l, dtype=np.int64), np.array(s_l, dtype=np.float64))


class FCI:
    """FCI problem in the (N_alpha, N_beta) sector."""

    def __init__(self, h, eri, n_alpha, n_beta):
        self.h = np.asarray(h, dtype=np.float64)
        self.eri = np.asarray(eri, dtype=np.float64)
        self.n = n = h.shape[0]
        self.na, self.nb = n_alpha, n_beta
        self.Na, self.Nb = comb(n, n_alpha), comb(n, n_beta)
        self.exa = single_excitations(n, n_alpha)
        self.exb = single_excitations(n, n_beta)
        self.k = self.h - 0.5 * np.einsum("prrq->pq", self.eri)
        self.eri2 = self.eri.reshape(n * n, n * n)

    def apply_E_all(self, C):
        """D[pq] = E_pq C for all pq, shape (n^2, Na, Nb)."""
        n = self.n
        D = np.zeros((n * n, self.Na, self.Nb))
        I, J, pq, s = self.exa
        D[pq, J, :] = s[:, None] * C[I, :]
        I, J, pq, s = self.exb
        D[pq, :, J] += s[:, None] * C[:, I].T
        return D

    def apply_E_sum(self, G):
        """sum_pq E_pq G[pq] for G of shape (n^2, Na, Nb)."""
        out = np.zeros((self.Na, self.Nb))
        I, J, pq, s = self.exa
        np.add.at(out, J, s[:, None] * G[pq, I, :])
        I, J, pq, s = self.exb
        outT = np.zeros((self.Nb, self.Na))
        np.add.at(outT, J, s[:, None] * G[pq, :, I])
        return out + outT.T

    def sigma(self, C):
        C = C.reshape(self.Na, self.Nb)
        D = self.apply_E_all(C)
        n2 = self.n * self.n
        G = 0.5 * (self.eri2 @ D.reshape(n2, -1)).reshape(D.shape)
        one_body = np.tensordot(self.k.reshape(n2), D, axes=(0, 0))
        return self.apply_E_sum(G) + one_body

    def diagonal(self):
        """<I|H|I> for every determinant (Slater-Condon diagonal rule)."""
        n = self.n
        sa = strings(n, self.na)
        sb = strings(n, self.nb)
        oa = np.zeros((self.Na, n))
        ob = np.zeros((self.Nb, n))
        for i, o in enumerate(sa):
            oa[i, list(o)] = 1
        for i, o in enumerate(sb):
            ob[i, list(o)] = 1
        J = np.einsum("ppqq->pq", self.eri)
        K = np.einsum("pqqp->pq", self.eri)
        ha = np.diag(self.h)
        d = (oa @ ha)[:, None] + (ob @ ha)[None, :]
        # same-spin Coulomb minus exchange, opposite-spin Coulomb
        jk = J - K
        d += 0.5 * np.einsum("ip,pq,iq->i", oa, jk, oa)[:, None]
        d += 0.5 * np.einsum("ip,pq,iq->i", ob, jk, ob)[None, :]
        d += oa @ J @ ob.T
        return d

    def dense_h(self):
        """Dense H by applying sigma to unit vectors (small spaces only)."""
        N = self.Na * self.Nb
        H = np.zeros((N, N))
        for i in range(N):
            e = np.zeros(N)
            e[i] = 1.0
            H[:, i] = self.sigma(e).reshape(-1)
        return H

    def ground_state(self, tol=1e-10, max_iter=200, max_space=24, nroots=1, dense_limit=2000):
        """Lowest eigenpair(s) of H in the sector.  Dense eigh below
        dense_limit determinants, Davidson above."""
        N = self.Na * self.Nb
        if N <= dense_limit:
            w, v = np.linalg.eigh(self.dense_h())
            return w[:nroots], v[:, :nroots]
        return davidson(lambda x: self.sigma(x).reshape(-1), self.diagonal().reshape(-1),
                        tol=tol, max_iter=max_iter, max_space=max_space, nroots=nroots)

    def rdms(self, C):
        """gamma_pq = <E_pq>, Gamma_pqrs = <E_pq E_rs> - delta_qr gamma_ps
        (= sum_st <a+_ps a+_rt a_st a_qs>)."""
        n = self.n
        C = C.reshape(self.Na, self.Nb)
        D = self.apply_E_all(C).reshape(n * n, -1)
        g1 = (D @ C.reshape(-1)).reshape(n, n)
        M = D @ D.T  # M[(q,p),(r,s)] = <E_pq E_rs> with D[qp] = E_qp C
        g2 = M.reshape(n, n, n, n).transpose(1, 0, 2, 3).copy()
        for q in range(n):
            g2[:, q, q, :] -= g1
        return g1, g2


def rdm3(F, C):
    """Spin-summed 3-RDM Gamma3_pqrstu = sum_{s,t,v} <a+_ps a+_rt a+_tv a_uv a_st a_qs>,
    one of the densities the paper forms on the device for its SC-NEVPT2 step
    (Sec. "Computational details", the paragraph on the device-native
    perturbative correction), from products of excitation operators:
      E_pq E_rs E_tu = e_pqrstu + d_qt e_purs + d_st e_pqru + d_qr e_pstu
                       + d_qr d_st E_pu,
    with e_pqrs the 2-RDM operator (Gamma_pqrs = <e_pqrs>).  Small spaces
    only (n^4 vectors of the CI length)."""
    n = F.n
    C = C.reshape(F.Na, F.Nb)
    g1, g2 = F.rdms(C)
    D = F.apply_E_all(C)                                   # D[t n + u] = E_tu C
    T = np.stack([F.apply_E_all(D[tu]) for tu in range(n * n)], axis=1)   # [rs, tu] = E_rs E_tu C
    M = D.reshape(n * n, -1) @ T.reshape(n ** 4, -1).T     # row (q, p): <E_pq E_rs E_tu>
    G = M.reshape(n, n, n, n, n, n).transpose(1, 0, 2, 3, 4, 5).copy()
    d = np.eye(n)
    G -= np.einsum("qt,purs->pqrstu", d, g2)
    G -= np.einsum("st,pqru->pqrstu", d, g2)
    G -= np.einsum("qr,pstu->pqrstu", d, g2)
    G -= np.einsum("qr,st,pu->pqrstu", d, d, g1)
    return G


def davidson(matvec, diag, tol=1e-10, max_iter=200, max_space=24, nroots=1, guess=None, correction=None):
    """Plain Davidson (Davidson 1975) with the diagonal preconditioner
    t = -r / (diag - theta), two Gram-Schmidt passes and restart from the
    lowest Ritz vectors.  `correction(x, r, theta)`, when given, replaces
    the diagonal step (the members of oracle/precond.py)."""
    N = diag.shape[0]
    if guess is None:
        V = []
        for i in np.argsort(diag, kind="stable")[:max(nroots, 1)]:
            x = np.zeros(N)
            x[i] = 1.0
            V.append(x)
    else:
        V = [guess / np.linalg.norm(guess)]
    S = [matvec(v) for v in V]
    theta = None
    for _ in range(max_iter):
        Vm = np.array(V)
        Sm = np.array(S)
        Hs = Vm @ Sm.T
        Hs = 0.5 * (Hs + Hs.T)
        w, c = np.linalg.eigh(Hs)
        theta = w[:nroots]
        X = c[:, :nroots].T @ Vm
        R = c[:, :nroots].T @ Sm - theta[:, None] * X
        rn = np.linalg.norm(R, axis=1)
        if np.all(rn < tol):
            return theta, X.T
        if len(V) >= max_space:
            keep = max(nroots, 4)
            V = list(c[:, :keep].T @ Vm)
            S = list(c[:, :keep].T @ Sm)
        for i in range(nroots):
            if rn[i] < tol:
                continue
            if correction is not None:
                t = np.array(correction(X[i], R[i], theta[i]), dtype=np.float64)
            else:
                den = diag - theta[i]
                den = np.where(np.abs(den) < 1e-8, np.where(den >= 0, 1e-8, -1e-8), den)
                t = -R[i] / den
            for _ in range(2):
                for v in V:
                    t -= (v @ t) * v
            nt = np.linalg.norm(t)
            if nt < 1e-14:
                continue
            t /= nt
            V.append(t)
            S.append(matvec(t))
    return theta, X.T
