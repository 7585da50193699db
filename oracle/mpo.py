"""Matrix-product operator of the active-space Hamiltonian (TEST
INFRASTRUCTURE ONLY).

The paper's DMRG applies H as an MPO so that the dense d^L operator is
never formed (Sec. "Cholesky decomposition for the wavefunction", item (i)).
The paper does not give its construction; this module builds it term by
term from the definition of H:

  terms   H = sum_pq,s h_pq a+_ps a_qs
              + 1/2 sum_pqrs,s,t (pq|rs) a+_ps a+_rt a_st a_qs
          Every term is written as an operator string, reordered into site
          order (stable; the sign is the parity of the reordering, which
          only ever swaps operators on different spin orbitals), with the
          operators of one site multiplied in the order
          (a+_alpha, a_alpha, a+_beta, a_beta).

  channels  At bond k (left block = sites < k) a term with n_L operators on
          the left and n_R on the right passes through one channel:
             n_L = 0                      -> 'I'
             n_R = 0                      -> 'H'
             n_L = 1, or n_L = n_R = 2 with k <= k_switch
                                          -> ('B', left operators)   bare
             otherwise                    -> ('C', right operators)  complementary
          A bare channel fixes the left factor (no coefficient), a
          complementary channel fixes the right factor, so the term's
          coefficient is applied on the one site where its path first
          enters a 'C' or 'H' channel.  This is the normal/complementary
          operator MPO; k_switch = n // 2 gives the usual O(n^2) bond
          dimension, k_switch = n keeps every pair bare.

  fermions  With local basis [0, a, b, ab] (|ab> = a+_a a+_b |0>) and the
          product basis |s_0 s_1 ...> = prod_sites(local creators)|vac>,
          each entry is dressed with the local parity on its input side
          whenever the target channel is odd:  Wd[a,b] = W[a,b] P^{p(b)}.
          Then the Jordan-Wigner signs are carried entirely by the dressed
          tensors and every contraction (environment, H_eff) is a plain
          tensor product: left environments hold O_L P_L^{p}, right
          environments hold O_R.

Pinned in tests/test_oracle_mpo.py by contracting the MPO to the dense 4^n
matrix and comparing with fock.hamiltonian for n <= 4.
"""
from __future__ import annotations

import numpy as np

# local states [0, alpha, beta, alpha+beta]
QN = [(0, 0), (1, 0), (0, 1), (1, 1)]
PARITY = [0, 1, 1, 0]


def _local_matrices():
    ca_dag = np.zeros((4, 4))
    ca_dag[1, 0] = 1.0      # a+_a |0>  = |a>
    ca_dag[3, 2] = 1.0      # a+_a |b>  = |ab>
    cb_dag = np.zeros((4, 4))
    cb_dag[2, 0] = 1.0      # a+_b |0>  = |b>
    cb_dag[3, 1] = -1.0     # a+_b |a>  = a+_b a+_a|0> = -|ab>
    return {(0, True): ca_dag, (0, False): ca_dag.T.copy(),
            (1, True): cb_dag, (1, False): cb_dag.T.copy()}


LOCAL = _local_matrices()
PARITY_OP = np.diag([1.0, -1.0, -1.0, 1.0])


def op_code(site: int, spin: int, dag: bool) -> int:
    """Sort key of one operator: site, then spin, then creator first."""
    return site * 4 + spin * 2 + (0 if dag else 1)


def canonical_term(coef, ops):
    """Reorder an operator string [(site, spin, dag), ...] into op_code order.
    Returns (coef * sign, tuple(ops)).  Same-spin-orbital operators never
    swap here (a creator always precedes the annihilator of its own spin
    orbital in the terms of H), so only anticommutation signs appear."""
    keys = [op_code(*o) for o in ops]
    inv = 0
    for i in range(len(keys)):
        for j in range(i + 1, len(keys)):
            if keys[i] > keys[j]:
                inv += 1
    order = sorted(range(len(ops)), key=lambda i: keys[i])
    return coef * (-1) ** inv, tuple(ops[i] for i in order)


def hamiltonian_terms(h, eri, drop=0.0):
    """All operator-string terms of H (see module docstring)."""
    n = h.shape[0]
    terms = {}

    def add(coef, ops):
        c, t = canonical_term(coef, ops)
        terms[t] = terms.get(t, 0.0) + c

    for p in range(n):
        for q in range(n):
            if abs(h[p, q]) <= drop:
                continue
            for s in range(2):
                add(h[p, q], [(p, s, True), (q, s, False)])
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for ss in range(n):
                    v = eri[p, q, r, ss]
                    if abs(v) <= drop:
                        continue
                    for s in range(2):
                        for t in range(2):
                            if (p, s) == (r, t) or (q, s) == (ss, t):
                                continue
                            add(0.5 * v, [(p, s, True), (r, t, True), (ss, t, False), (q, s, False)])
    return [(c, t) for t, c in terms.items() if c != 0.0]


def channel(ops, k: int, k_switch: int):
    """Channel label of a (canonical) term at bond k."""
    left = tuple(o for o in ops if o[0] < k)
    right = tuple(o for o in ops if o[0] >= k)
    nl, nr = len(left), len(right)
    if nl == 0:
        return ("I",)
    if nr == 0:
        return ("H",)
    if nl == 1 or (nl == 2 and nr == 2 and k <= k_switch):
        return ("B", left)
    return ("C", right)


def label_key(lab):
    kind = {"I": 0, "H": 1, "B": 2, "C": 3}[lab[0]]
    if len(lab) == 1:
        return (kind, 0, ())
    return (kind, len(lab[1]), tuple(op_code(*o) for o in lab[1]))


def label_delta(lab):
    """(d N_alpha, d N_beta) of the left factor of a channel."""
    if lab[0] in ("I", "H"):
        return (0, 0)
    da = db = 0
    for (_, spin, dag) in lab[1]:
        d = 1 if dag else -1
        if spin == 0:
            da += d
        else:
            db += d
    if lab[0] == "C":  # left factor carries the negative of the right ops
        return (-da, -db)
    return (da, db)


def label_parity(lab):
    if lab[0] in ("I", "H"):
        return 0
    return len(lab[1]) % 2


class MPO:
    """Dressed MPO: W[i][(a, b)] is a 4x4 matrix (row = output local state,
    column = input local state) mapping channel a at bond i to channel b at
    bond i+1."""

    def __init__(self, h, eri, k_switch=None, drop=0.0):
        n = h.shape[0]
        self.n = n
        self.k_switch = n // 2 if k_switch is None else k_switch
        terms = hamiltonian_terms(h, eri, drop)
        labels = [set() for _ in range(n + 1)]
        for _, ops in terms:
            for k in range(n + 1):
                labels[k].add(channel(ops, k, self.k_switch))
        labels[0] = {("I",)}
        labels[n] = {("H",)}
        self.labels = [sorted(s, key=label_key) for s in labels]
        self.index = [{lab: i for i, lab in enumerate(ls)} for ls in self.labels]
        self.delta = [[label_delta(l) for l in ls] for ls in self.labels]
        self.parity = [[label_parity(l) for l in ls] for ls in self.labels]
        W = [dict() for _ in range(n)]
        for coef, ops in terms:
            for i in range(n):
                a = channel(ops, i, self.k_switch)
                b = channel(ops, i + 1, self.k_switch)
                loc = np.eye(4)
                for o in ops:
                    if o[0] == i:
                        loc = loc @ LOCAL[(o[1], o[2])]
                key = (self.index[i][a], self.index[i + 1][b])
                applies = a[0] in ("I", "B") and b[0] in ("C", "H")
                if applies:
                    W[i][key] = W[i].get(key, 0.0) + coef * loc
                else:
                    if key in W[i]:
                        assert np.array_equal(W[i][key], loc)
                    W[i][key] = loc
        # dress with the local parity when the target channel is odd
        for i in range(n):
            for (a, b), w in list(W[i].items()):
                if self.parity[i + 1][b]:
                    W[i][(a, b)] = w @ PARITY_OP
                if not np.any(W[i][(a, b)]):
                    del W[i][(a, b)]
        self.W = W

    def bond_dims(self):
        return [len(ls) for ls in self.labels]

    def dense(self):
        """Contract the full chain into the dense 4^n x 4^n matrix (plain
        tensor products, no further signs).  Small n only."""
        n = self.n
        envs = {0: np.ones((1, 1))}
        for i in range(n):
            new = {}
            for (a, b), w in self.W[i].items():
                if a not in envs:
                    continue
                t = np.kron(envs[a], w)
                new[b] = new.get(b, 0.0) + t
            envs = new
        return envs[0]
