"""Symmetry-blocked two-site DMRG (TEST INFRASTRUCTURE ONLY).

Follows the paper's DMRG node: a two-site sweep in which sites (k, k+1) are
optimised against a left block and a right block, the two-site effective
Hamiltonian is solved matrix-free against the MPO by Davidson, and an SVD
decimates the enlarged bond back to chi_k, discarding Schmidt weight tau
(Fig. 2 and Sec. "Cholesky decomposition for the wavefunction"; FP64
throughout, Sec. "Computational details").  At full bond dimension the
result is FCI in the active space (Table "valid").

The paper works in the full Fock space with penalty terms (Sec. "Excited
states", Eq. dualpen); here every tensor is blocked by the left-block
quantum numbers q = (N_alpha, N_beta), which gives the same in-sector
energies.  Readings of points the paper leaves open (initial MPS, Davidson
details, truncation tie rule, sweep order) are stated where they are used.

Data layout (plain dicts of dense numpy blocks):
  bond k      dict q -> dim      (q = left-block particle numbers, k=0..n)
  site i      dict (q_l, s) -> (dim_i(q_l), dim_{i+1}(q_l + QN[s]))
  env         list over channels a of dict q_in -> block (q_in+delta_a, q_in)
  two-site    dict (q_l, s1, s2) -> (dim_k(q_l), dim_{k+2}(q_l+QN[s1]+QN[s2]))
Left environments hold the parity-dressed left operators and right
environments the right operators of the dressed MPO (see mpo.py), so every
contraction is a plain tensor product.
"""
from __future__ import annotations

from math import comb

import numpy as np

import gbd_synth
from . import fci as fci_mod
from .mpo import MPO, QN


def qadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


def qsub(a, b):
    return (a[0] - b[0], a[1] - b[1])


# ---------------------------------------------------------------- initial MPS
def exact_dims(n, k, Na, Nb):
    """Largest useful dimension of each sector at bond k: the smaller of the
    left- and right-block multiplicities."""
    out = {}
    for a in range(0, min(k, Na) + 1):
        for b in range(0, min(k, Nb) + 1):
            ra, rb = Na - a, Nb - b
            if ra < 0 or rb < 0 or ra > n - k or rb > n - k:
                continue
            left = comb(k, a) * comb(k, b)
            right = comb(n - k, ra) * comb(n - k, rb)
            d = min(left, right)
            if d > 0:
                out[(a, b)] = d
    return out


def initial_bond_dims(n, Na, Nb, M):
    """Initial bond dimensions (reading of the paper-silent initial state):
    every allowed sector populated; if the exact total exceeds M, sector q
    gets min(d_ex(q), max(1, floor(M d_ex(q) / T))) with T the exact total;
    then L->R and R->L consistency passes (dim_k(q) <= sum_s dim_{k-1}(q-s)
    and dim_k(q) <= sum_s dim_{k+1}(q+s)) repeat until nothing changes."""
    dims = []
    for k in range(n + 1):
        ex = exact_dims(n, k, Na, Nb)
        T = sum(ex.values())
        if T <= M:
            dims.append(dict(ex))
        else:
            dims.append({q: min(d, max(1, (M * d) // T)) for q, d in ex.items()})
    changed = True
    while changed:
        changed = False
        for k in range(1, n + 1):
            for q in list(dims[k]):
                sup = sum(dims[k - 1].get(qsub(q, QN[s]), 0) for s in range(4))
                if sup < dims[k][q]:
                    dims[k][q] = sup
                    changed = True
        for k in range(n - 1, -1, -1):
            for q in list(dims[k]):
                sup = sum(dims[k + 1].get(qadd(q, QN[s]), 0) for s in range(4))
                if sup < dims[k][q]:
                    dims[k][q] = sup
                    changed = True
        for k in range(n + 1):
            for q in [q for q, d in dims[k].items() if d == 0]:
                del dims[k][q]
                changed = True
    return dims


def initial_mps(n, Na, Nb, M, seed):
    """Random MPS with initial_bond_dims; entries from the counter-based
    values of gbd_synth.mps_init_block.  Not yet canonical."""
    dims = initial_bond_dims(n, Na, Nb, M)
    sites = []
    for i in range(n):
        blk = {}
        for ql, ml in dims[i].items():
            for s in range(4):
                qr = qadd(ql, QN[s])
                if qr in dims[i + 1]:
                    blk[(ql, s)] = gbd_synth.mps_init_block(seed, i, ql[0], ql[1], s, ml, dims[i + 1][qr])
        sites.append(blk)
    return dims, sites


def fused_right(site, dims_r, ql):
    """Columns (s, q_r) of sector ql, s = 0..3: [block(ql,0) | block(ql,1) | ...]."""
    parts, cols = [], []
    for s in range(4):
        if (ql, s) in site:
            parts.append(site[(ql, s)])
            cols.append((s, site[(ql, s)].shape[1]))
    return np.hstack(parts), cols


def right_canonicalize(dims, sites):
    """Make sites 1..n-1 right-orthonormal (B B^T = 1 per sector) by LQ
    factorisations from the right; site 0 keeps the norm, then normalised."""
    n = len(sites)
    for i in range(n - 1, 0, -1):
        for ql in list(dims[i]):
            Mx, cols = fused_right(sites[i], dims[i + 1], ql)
            Qt, R = np.linalg.qr(Mx.T)       # Mx = R^T Qt^T
            Q = Qt.T
            Lm = R.T
            off = 0
            for s, w in cols:
                sites[i][(ql, s)] = Q[:, off:off + w].copy()
                off += w
            for s in range(4):
                qp = qsub(ql, QN[s])
                if (qp, s) in sites[i - 1]:
                    sites[i - 1][(qp, s)] = sites[i - 1][(qp, s)] @ Lm
    nrm = np.sqrt(sum(np.sum(b * b) for b in sites[0].values()))
    for key in sites[0]:
        sites[0][key] = sites[0][key] / nrm
    return sites


# ---------------------------------------------------------------- environments
def left_boundary():
    return [{(0, 0): np.ones((1, 1))}]


def right_boundary(Na, Nb):
    return [{(Na, Nb): np.ones((1, 1))}]


def left_env_update(Lk, A, Wi, delta_k, n_right_channels):
    """L_{k+1}[b](l',l) = sum_{a,s,s'} Wd[a,b](s',s) A[s']^T L_k[a] A[s]."""
    out = {}
    for (a, b), w in Wi.items():
        if a >= len(Lk):
            continue
        da = delta_k[a]
        for sp, s in zip(*np.nonzero(w)):
            c = w[sp, s]
            for q0, Lb in Lk[a].items():
                q0p = qadd(q0, da)
                if (q0, s) not in A or (q0p, sp) not in A:
                    continue
                q = qadd(q0, QN[s])
                blk = c * (A[(q0p, sp)].T @ Lb @ A[(q0, s)])
                d = out.setdefault(b, {})
                d[q] = d.get(q, 0.0) + blk
    return [out.get(b, {}) for b in range(n_right_channels)]


def right_env_update(Rk1, B, Wi, delta_k1, n_left_channels):
    """R_k[b](r',r) = sum_{c,s,s'} Wd[b,c](s',s) B[s'] R_{k+1}[c] B[s]^T."""
    out = {}
    for (b, c), w in Wi.items():
        if c >= len(Rk1):
            continue
        dc = delta_k1[c]
        for sp, s in zip(*np.nonzero(w)):
            cf = w[sp, s]
            for q1, Rb in Rk1[c].items():
                q = qsub(q1, QN[s])
                qp = qsub(qadd(q1, dc), QN[sp])
                if (q, s) not in B or (qp, sp) not in B:
                    continue
                blk = cf * (B[(qp, sp)] @ Rb @ B[(q, s)].T)
                d = out.setdefault(b, {})
                d[q] = d.get(q, 0.0) + blk
    return [out.get(b, {}) for b in range(n_left_channels)]


# ---------------------------------------------------------------- two-site
def two_site_psi(center, B, dims_k1):
    """psi[(q_l,s1,s2)] = sum_q center[(q_l,s1)] @ B[(q,s2)], q = q_l+QN[s1]."""
    psi = {}
    for (ql, s1), C in center.items():
        q = qadd(ql, QN[s1])
        for s2 in range(4):
            if (q, s2) in B:
                psi[(ql, s1, s2)] = C @ B[(q, s2)]
    return psi


def psi_keys(dims_k, dims_k2):
    keys = []
    for ql in sorted(dims_k):
        for s1 in range(4):
            for s2 in range(4):
                qr = qadd(qadd(ql, QN[s1]), QN[s2])
                if qr in dims_k2:
                    keys.append((ql, s1, s2))
    return keys


def flatten(psi, keys, dims_k, dims_k2):
    parts = []
    for key in keys:
        ql, s1, s2 = key
        qr = qadd(qadd(ql, QN[s1]), QN[s2])
        b = psi.get(key)
        if b is None:
            b = np.zeros((dims_k[ql], dims_k2[qr]))
        parts.append(b.reshape(-1))
    return np.concatenate(parts) if parts else np.zeros(0)


def unflatten(x, keys, dims_k, dims_k2):
    psi, off = {}, 0
    for key in keys:
        ql, s1, s2 = key
        qr = qadd(qadd(ql, QN[s1]), QN[s2])
        m, r = dims_k[ql], dims_k2[qr]
        psi[key] = x[off:off + m * r].reshape(m, r)
        off += m * r
    return psi


def apply_heff(L, W1, W2, R, psi, mpo: MPO, k):
    """sigma = sum_{a,b,c} (L[a] x Wd_k[a,b] x Wd_{k+1}[b,c] x R[c]) psi,
    contracted in the order L, W_k, W_{k+1}, R."""
    dl = mpo.delta[k]
    T1 = {}
    for a, La in enumerate(L):
        for (ql, s1, s2), P in psi.items():
            if ql in La:
                qr = qadd(qadd(ql, QN[s1]), QN[s2])
                T1.setdefault(a, {})[(qadd(ql, dl[a]), s1, s2, qr)] = La[ql] @ P
    T2 = {}
    for (a, b), w in W1.items():
        if a not in T1:
            continue
        for sp, s in zip(*np.nonzero(w)):
            c = w[sp, s]
            for (qlp, s1, s2, qr), X in T1[a].items():
                if s1 != s:
                    continue
                d = T2.setdefault(b, {})
                key = (qlp, sp, s2, qr)
                d[key] = d.get(key, 0.0) + c * X
    T3 = {}
    for (b, cc), w in W2.items():
        if b not in T2:
            continue
        for sp, s in zip(*np.nonzero(w)):
            c = w[sp, s]
            for (qlp, s1p, s2, qr), X in T2[b].items():
                if s2 != s:
                    continue
                d = T3.setdefault(cc, {})
                key = (qlp, s1p, sp, qr)
                d[key] = d.get(key, 0.0) + c * X
    sigma = {}
    for cc, blocks in T3.items():
        if cc >= len(R):
            continue
        for (qlp, s1p, s2p, qr), X in blocks.items():
            if qr not in R[cc]:
                continue
            key = (qlp, s1p, s2p)
            sigma[key] = sigma.get(key, 0.0) + X @ R[cc][qr].T
    return sigma


def heff_diag(L, W1, W2, R, keys, mpo: MPO, k, dims_k, dims_k2):
    """Diagonal of H_eff: sum over channels with zero quantum-number change
    of diag(L[a]) Wd1[a,b](s1,s1) Wd2[b,c](s2,s2) diag(R[c])."""
    diag = {key: np.zeros((dims_k[key[0]], dims_k2[qadd(qadd(key[0], QN[key[1]]), QN[key[2]])]))
            for key in keys}
    by_b = {}
    for (b, c), w in W2.items():
        by_b.setdefault(b, []).append((c, w))
    for (a, b), w1 in W1.items():
        if a >= len(L) or mpo.delta[k][a] != (0, 0):
            continue
        for c, w2 in by_b.get(b, []):
            if c >= len(R) or mpo.delta[k + 2][c] != (0, 0):
                continue
            for key in keys:
                ql, s1, s2 = key
                f = w1[s1, s1] * w2[s2, s2]
                if f == 0.0:
                    continue
                qr = qadd(qadd(ql, QN[s1]), QN[s2])
                if ql in L[a] and qr in R[c]:
                    diag[key] += f * np.outer(np.diag(L[a][ql]), np.diag(R[c][qr]))
    return diag


def heff_dense(L, W1, W2, R, keys, mpo, k, dims_k, dims_k2):
    """Explicit H_eff matrix, column by column (tiny blocks only)."""
    N = sum(dims_k[kq[0]] * dims_k2[qadd(qadd(kq[0], QN[kq[1]]), QN[kq[2]])] for kq in keys)
    H = np.zeros((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        s = apply_heff(L, W1, W2, R, unflatten(e, keys, dims_k, dims_k2), mpo, k)
        H[:, i] = flatten(s, keys, dims_k, dims_k2)
    return H


# ---------------------------------------------------------------- truncation
def select_states(weights, M, cutoff=1e-12, tie=1e-10, max_discarded=0.0, m_min=1):
    """Reading of the decimation rule (Fig. 2: keep chi_k states, discard
    tau = sum of the dropped sigma^2).  weights = [(lambda, sector, j)] with
    lambda = sigma^2 of a normalised two-site state.
      1. drop lambda <= cutoff;
      2. sort by lambda descending, equal values by (sector, j) ascending;
      3. keep min(M, count); if the last kept and first dropped differ by
         <= tie, step back past the whole cluster (never split a
         near-degenerate multiplet at the cut; if every weight is in the
         cluster keep min(M, count)).
    Per-bond adaptive bond dimension (Sec. "Cholesky decomposition for the
    wavefunction", ingredient (ii): a dynamically adapted per-bond bond
    dimension), when max_discarded > 0: before step 3, take the smallest m
    whose discarded weight (everything not among the first m, the cut-off
    weights included) is <= max_discarded; extend m past a cluster it
    would split; raise it to m_min.  If that m is below min(M, count), keep
    it; otherwise step 3 applies (M caps the bond).
    Returns the kept list and tau."""
    cand = [w for w in weights if w[0] > cutoff]
    cand.sort(key=lambda w: (-w[0], w[1], w[2]))
    if max_discarded > 0.0:
        total = sum(w[0] for w in weights)
        m, kept_sum = 0, 0.0
        while m < len(cand) and total - kept_sum > max_discarded:
            kept_sum += cand[m][0]
            m += 1
        while 0 < m < len(cand) and cand[m - 1][0] - cand[m][0] <= tie:
            m += 1
        m = max(m, min(m_min, len(cand)))
        if m < min(M, len(cand)):
            kept = cand[:m]
            return kept, total - sum(w[0] for w in kept)
    nk = min(M, len(cand))
    if len(cand) > nk:
        j = nk
        while j > 0 and cand[j - 1][0] - cand[j][0] <= tie:
            j -= 1
        if j > 0:
            nk = j
    kept = cand[:nk]
    tau = sum(w[0] for w in weights) - sum(w[0] for w in kept)
    return kept, tau


def middle_blocks(psi, dims_k, dims_k2):
    """Group the two-site state by middle sector Q = q_l + QN[s1]: rows
    (q_l, s1) for s1 = 0..3, columns (s2, q_r) for s2 = 0..3."""
    Qs = sorted({qadd(ql, QN[s1]) for (ql, s1, s2) in psi})
    out = {}
    for Q in Qs:
        rows = [(qsub(Q, QN[s1]), s1) for s1 in range(4) if qsub(Q, QN[s1]) in dims_k]
        cols = [(s2, qadd(Q, QN[s2])) for s2 in range(4) if qadd(Q, QN[s2]) in dims_k2]
        mat = np.zeros((sum(dims_k[r[0]] for r in rows), sum(dims_k2[c[1]] for c in cols)))
        ro = 0
        for (ql, s1) in rows:
            co = 0
            for (s2, qr) in cols:
                b = psi.get((ql, s1, s2))
                if b is not None:
                    mat[ro:ro + dims_k[ql], co:co + dims_k2[qr]] = b
                co += dims_k2[qr]
            ro += dims_k[ql]
        out[Q] = (mat, rows, cols)
    return out


def truncate(psi, dims_k, dims_k2, M, direction, cutoff=1e-12, tie=1e-10, max_discarded=0.0, m_min=1):
    """SVD decimation of the two-site state.  direction 'L': left tensor is
    U (left-orthonormal) and S V^T moves right; 'R': right tensor is V^T and
    U S moves left.  Returns (left_site, right_site, new bond dims, tau,
    kept weights)."""
    mids = middle_blocks(psi, dims_k, dims_k2)
    svds = {}
    weights = []
    for Q, (mat, rows, cols) in mids.items():
        U, S, Vt = np.linalg.svd(mat, full_matrices=False)
        svds[Q] = (U, S, Vt)
        weights += [(S[j] ** 2, Q, j) for j in range(len(S))]
    kept, tau = select_states(weights, M, cutoff, tie, max_discarded, m_min)
    keep_idx = {}
    for lam, Q, j in kept:
        keep_idx.setdefault(Q, []).append(j)
    new_dims = {}
    left, right = {}, {}
    for Q in sorted(keep_idx):
        idx = sorted(keep_idx[Q])
        U, S, Vt = svds[Q]
        mat, rows, cols = mids[Q]
        new_dims[Q] = len(idx)
        if direction == "L":
            Lm = U[:, idx]
            Rm = S[idx, None] * Vt[idx, :]
        else:
            Lm = U[:, idx] * S[None, idx]
            Rm = Vt[idx, :]
        ro = 0
        for (ql, s1) in rows:
            left[(ql, s1)] = Lm[ro:ro + dims_k[ql], :].copy()
            ro += dims_k[ql]
        co = 0
        for (s2, qr) in cols:
            right[(Q, s2)] = Rm[:, co:co + dims_k2[qr]].copy()
            co += dims_k2[qr]
    return left, right, new_dims, tau, sorted(w[0] for w in kept)[::-1]


# ---------------------------------------------------------------- sweep
class DMRG:
    """Two-site DMRG state: MPS, MPO and environments."""

    def __init__(self, h, chol, n_elec, two_sz, M_init, seed, k_switch=None, mps=None, renv_down_to=2):
        self.h = np.asarray(h, dtype=np.float64)
        self.chol = np.asarray(chol, dtype=np.float64)
        self.eri = np.einsum("Qpq,Qrs->pqrs", self.chol, self.chol)
        self.n = n = self.h.shape[0]
        self.Na = (n_elec + two_sz) // 2
        self.Nb = (n_elec - two_sz) // 2
        self.mpo = MPO(self.h, self.eri, k_switch=k_switch)
        if mps is None:
            dims, sites = initial_mps(n, self.Na, self.Nb, M_init, seed)
            sites = right_canonicalize(dims, sites)
        else:
            dims, sites = mps
        self.dims = dims
        self.sites = sites
        self.Lenv = [None] * (n + 1)
        self.Renv = [None] * (n + 1)
        self.Lenv[0] = left_boundary()
        self.Renv[n] = right_boundary(self.Na, self.Nb)
        for k in range(n - 1, max(renv_down_to, 2) - 1, -1):
            self.Renv[k] = right_env_update(self.Renv[k + 1], self.sites[k], self.mpo.W[k],
                                            self.mpo.delta[k + 1], len(self.mpo.labels[k]))
        self.n_matvec = 0

    def heff_parts(self, k):
        return self.Lenv[k], self.mpo.W[k], self.mpo.W[k + 1], self.Renv[k + 2]

    def step(self, k, M, tol, direction, max_iter=100, max_space=24, cutoff=1e-12, tie=1e-10, max_discarded=0.0,
             m_min=1):
        """One two-site step at (k, k+1): Davidson on H_eff, decimation,
        environment update in the sweep direction."""
        n = self.n
        dk, dk2 = self.dims[k], self.dims[k + 2]
        psi = two_site_psi(self.sites[k], self.sites[k + 1], self.dims[k + 1])
        keys = psi_keys(dk, dk2)
        L, W1, W2, R = self.heff_parts(k)
        x0 = flatten(psi, keys, dk, dk2)
        diag = flatten(heff_diag(L, W1, W2, R, keys, self.mpo, k, dk, dk2), keys, dk, dk2)

        def mv(x):
            self.n_matvec += 1
            return flatten(apply_heff(L, W1, W2, R, unflatten(x, keys, dk, dk2), self.mpo, k),
                           keys, dk, dk2)

        theta, X = fci_mod.davidson(mv, diag, tol=tol, max_iter=max_iter,
                                    max_space=max_space, guess=x0)
        x = X[:, 0] / np.linalg.norm(X[:, 0])
        psi = unflatten(x, keys, dk, dk2)
        left, right, nd, tau, kept = truncate(psi, dk, dk2, M, direction, cutoff, tie, max_discarded, m_min)
        self.sites[k], self.sites[k + 1] = left, right
        self.dims[k + 1] = nd
        if direction == "L":
            self.Lenv[k + 1] = left_env_update(self.Lenv[k], left, self.mpo.W[k], self.mpo.delta[k],
                                               len(self.mpo.labels[k + 1]))
        else:
            self.Renv[k + 1] = right_env_update(self.Renv[k + 2], right, self.mpo.W[k + 1],
                                                self.mpo.delta[k + 2], len(self.mpo.labels[k + 1]))
        return float(theta[0]), tau, kept

    def sweep(self, M, tol, **kw):
        """L->R over (0,1)..(n-2,n-1), then R->L back (Fig. 2 sweep)."""
        n = self.n
        log = []
        for k in range(0, n - 1):
            log.append(("L", k) + self.step(k, M, tol, "L", **kw)[:2])
        for k in range(n - 2, -1, -1):
            log.append(("R", k) + self.step(k, M, tol, "R", **kw)[:2])
        return log

    def move_center(self, k):
        """Left-orthonormalise sites 0..k-1 of a state whose centre is site 0
        (QR per sector of bond i+1, the triangular factor moves right) and
        build the left environments up to bond k.  The state is unchanged."""
        for i in range(k):
            Qs = sorted({qadd(ql, QN[s]) for (ql, s) in self.sites[i]})
            for Q in Qs:
                rows = [(qsub(Q, QN[s]), s) for s in range(4) if (qsub(Q, QN[s]), s) in self.sites[i]]
                mat = np.vstack([self.sites[i][r] for r in rows])
                Qm, Rm = np.linalg.qr(mat)
                off = 0
                for r in rows:
                    m = self.sites[i][r].shape[0]
                    self.sites[i][r] = Qm[off:off + m, :].copy()
                    off += m
                assert Qm.shape[1] == self.dims[i + 1][Q]
                for s in range(4):
                    if (Q, s) in self.sites[i + 1]:
                        self.sites[i + 1][(Q, s)] = Rm @ self.sites[i + 1][(Q, s)]
            self.Lenv[i + 1] = left_env_update(self.Lenv[i], self.sites[i], self.mpo.W[i], self.mpo.delta[i],
                                               len(self.mpo.labels[i + 1]))

    def energy(self):
        """<psi|H_eff|psi> / <psi|psi> at bond (0,1) of the current MPS."""
        k = 0
        psi = two_site_psi(self.sites[0], self.sites[1], self.dims[1])
        keys = psi_keys(self.dims[0], self.dims[2])
        x = flatten(psi, keys, self.dims[0], self.dims[2])
        s = flatten(apply_heff(*self.heff_parts(0), psi, self.mpo, 0), keys, self.dims[0], self.dims[2])
        return float(x @ s / (x @ x))

    def to_ci(self):
        """Expand the MPS into the determinant basis of fci.py (C[Ia, Ib])."""
        return mps_to_ci(self.dims, self.sites, self.n, self.Na, self.Nb)

    def rdms(self):
        C = self.to_ci()
        C = C / np.linalg.norm(C)
        f = fci_mod.FCI(self.h, self.eri, self.Na, self.Nb)
        return f.rdms(C)


def mps_to_ci(dims, sites, n, Na, Nb):
    """Amplitude of each determinant = product of the site blocks along its
    occupations, times the sign that reorders the site-major creators
    (0a,0b,1a,1b,...) into alpha-first order: (-1)^{sum_j nb_j * #alpha at
    sites > j}."""
    # left-to-right dictionary of prefixes: (alpha bits, beta bits) -> row vector
    prefixes = {(0, 0): {(0, 0): np.ones((1, 1))}}  # q -> {(abits, bbits): vec}
    for i in range(n):
        nxt = {}
        for q, vecs in prefixes.items():
            for (ab, bb), v in vecs.items():
                for s in range(4):
                    if (q, s) not in sites[i]:
                        continue
                    qn = qadd(q, QN[s])
                    na_, nb_ = QN[s]
                    key = (ab | (na_ << i), bb | (nb_ << i))
                    nxt.setdefault(qn, {})[key] = v @ sites[i][(q, s)]
        prefixes = nxt
    C = np.zeros((comb(n, Na), comb(n, Nb)))
    for (ab, bb), v in prefixes[(Na, Nb)].items():
        aocc = [p for p in range(n) if ab >> p & 1]
        bocc = [p for p in range(n) if bb >> p & 1]
        ex = sum(sum(1 for p in aocc if p > j) for j in bocc)
        C[fci_mod.colex_addr(aocc), fci_mod.colex_addr(bocc)] = (-1) ** ex * v[0, 0]
    return C


def run(h, chol, n_elec, two_sz, M_schedule, tol_schedule, seed, k_switch=None,
        max_iter=100, max_space=24, cutoff=1e-12, tie=1e-10, max_discarded=0.0, m_min=1):
    """Full solve: initial MPS, sweeps per the schedule, final energy.
    max_discarded > 0 turns on the per-bond adaptive bond dimension of
    select_states in every decimation (M of each sweep is the cap)."""
    d = DMRG(h, chol, n_elec, two_sz, M_schedule[0], seed, k_switch=k_switch)
    sweep_E = []
    for M, tol in zip(M_schedule, tol_schedule):
        log = d.sweep(M, tol, max_iter=max_iter, max_space=max_space, cutoff=cutoff, tie=tie,
                      max_discarded=max_discarded, m_min=m_min)
        sweep_E.append(log[-1][2])
    return d, sweep_E


def canonical_blocks(d):
    """(n_sectors, triples, data) of a DMRG state in the canonical block
    exchange format of the CUDA library's test interface: per bond the sorted
    sector triples (N_alpha, N_beta, dim); per site, for each sector q_l and
    local state s with q_r = q_l + s present, one row-major block."""
    ns, tr, data = [], [], []
    for k in range(d.n + 1):
        secs = sorted(d.dims[k])
        ns.append(len(secs))
        for q in secs:
            tr += [q[0], q[1], d.dims[k][q]]
    for i in range(d.n):
        for ql in sorted(d.dims[i]):
            for s in range(4):
                qr = qadd(ql, QN[s])
                if qr not in d.dims[i + 1]:
                    continue
                b = d.sites[i].get((ql, s))
                if b is None:
                    b = np.zeros((d.dims[i][ql], d.dims[i + 1][qr]))
                data.append(b.reshape(-1))
    return np.array(ns), np.array(tr), np.concatenate(data)
