"""Pins of the oracle MPO and the oracle two-site DMRG (CPU only)."""
import json
import os

import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import dmrg, fci, fock, mpo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def kron_to_fock_perm(n):
    # Kronecker index: site 0 most significant base-4 digit; Fock index:
    # sum_i s_i 4^i with s = n_alpha + 2 n_beta per site.
    dim = 4 ** n
    idx = np.zeros(dim, dtype=np.int64)
    for i in range(dim):
        digits = []
        x = i
        for _ in range(n):
            digits.append(x % 4)
            x //= 4
        digits = digits[::-1]  # s_0 .. s_{n-1}
        idx[i] = sum(d * 4 ** k for k, d in enumerate(digits))
    return idx


@pytest.mark.parametrize("n", [2, 3, 4])
def test_mpo_contracts_to_fock_hamiltonian(n):
    h, chol = make_integrals(n, 5, 7)
    eri = fock.eri_from_chol(chol)
    H = fock.hamiltonian(h, eri).toarray()
    idx = kron_to_fock_perm(n)
    Hf = H[np.ix_(idx, idx)]
    for ks in range(0, n + 1):
        Hm = mpo.MPO(h, eri, k_switch=ks).dense()
        assert np.abs(Hm - Hf).max() < 1e-12


def test_mpo_bond_dimension_formula():
    # normal/complementary operators: 2 + 4n + (8 m^2 - 2 m) pair channels,
    # m = min(k, n-k) at the switch bond k = n//2
    for n in [4, 6]:
        h, chol = make_integrals(n, 2 * n, 3)
        eri = fock.eri_from_chol(chol)
        m = mpo.MPO(h, eri)
        D = m.bond_dims()
        c = n // 2
        assert D[c] == 2 + 4 * n + 8 * c * c - 2 * c
        assert D[0] == 1 and D[n] == 1


def test_planted_mpo_sign_error_is_caught(monkeypatch):
    n = 3
    h, chol = make_integrals(n, 5, 7)
    eri = fock.eri_from_chol(chol)
    H = fock.hamiltonian(h, eri).toarray()
    idx = kron_to_fock_perm(n)
    bad = dict(mpo.LOCAL)
    m = bad[(1, True)].copy()
    m[3, 1] *= -1.0  # drop the Jordan-Wigner sign inside the site
    bad[(1, True)] = m
    bad[(1, False)] = m.T.copy()
    monkeypatch.setattr(mpo, "LOCAL", bad)
    Hm = mpo.MPO(h, eri).dense()
    assert np.abs(Hm - H[np.ix_(idx, idx)]).max() > 1e-3


def test_initial_dims_rule():
    dims = dmrg.initial_bond_dims(6, 3, 3, 64)
    assert [sum(d.values()) for d in dims] == [1, 4, 16, 64, 16, 4, 1]
    dims = dmrg.initial_bond_dims(12, 6, 6, 256)
    for k in range(1, 12):
        for q, d in dims[k].items():
            left = sum(dims[k - 1].get((q[0] - a, q[1] - b), 0) for a, b in mpo.QN)
            right = sum(dims[k + 1].get((q[0] + a, q[1] + b), 0) for a, b in mpo.QN)
            assert 0 < d <= min(left, right)
    assert max(sum(d.values()) for d in dims) <= 256 + 49


def test_initial_mps_is_right_canonical():
    n = 6
    dims, sites = dmrg.initial_mps(n, 3, 3, 20, 5)
    sites = dmrg.right_canonicalize(dims, sites)
    for i in range(1, n):
        for q in dims[i]:
            Mx, _ = dmrg.fused_right(sites[i], dims[i + 1], q)
            assert np.abs(Mx @ Mx.T - np.eye(Mx.shape[0])).max() < 1e-12
    nrm = sum(np.sum(b * b) for b in sites[0].values())
    assert abs(nrm - 1) < 1e-12


def test_heff_hermitian_and_equals_projected_fock_h():
    # H_eff = P^T H P with P the map from the two-site space to the Fock
    # space given by the left and right block bases.
    n = 4
    h, chol = make_integrals(n, 6, 2)
    eri = fock.eri_from_chol(chol)
    d = dmrg.DMRG(h, chol, 4, 0, 3, seed=7)
    # move to bond (1,2): one L->R step
    d.step(0, 3, 1e-10, "L")
    k = 1
    L, W1, W2, R = d.heff_parts(k)
    keys = dmrg.psi_keys(d.dims[k], d.dims[k + 2])
    Heff = dmrg.heff_dense(L, W1, W2, R, keys, d.mpo, k, d.dims[k], d.dims[k + 2])
    assert np.abs(Heff - Heff.T).max() < 1e-13 * max(1.0, np.abs(Heff).max())
    # columns of P: expand each two-site basis vector into the full MPS state
    N = Heff.shape[0]
    P = []
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        P.append(expand_two_site(d, k, dmrg.unflatten(e, keys, d.dims[k], d.dims[k + 2])))
    P = np.array(P).T
    Hf = fock.hamiltonian(h, eri).toarray()
    idx = kron_to_fock_perm(n)
    Hk = Hf[np.ix_(idx, idx)]
    assert np.abs(P.T @ P - np.eye(N)).max() < 1e-12
    assert np.abs(P.T @ Hk @ P - Heff).max() < 1e-12
    diag = dmrg.flatten(dmrg.heff_diag(L, W1, W2, R, keys, d.mpo, k, d.dims[k], d.dims[k + 2]),
                        keys, d.dims[k], d.dims[k + 2])
    assert np.abs(diag - np.diag(Heff)).max() < 1e-12


def expand_two_site(d, k, psi):
    """Kronecker-basis vector of the state A_0 .. A_{k-1} psi B_{k+2} .. B_{n-1}."""
    n = d.n
    left = {(0, 0): np.ones((1, 1))}  # q -> (4^i, dim_i(q)): block basis states
    for i in range(k):
        new = {}
        for (q, s), A in d.sites[i].items():
            if q in left:
                qn = (q[0] + mpo.QN[s][0], q[1] + mpo.QN[s][1])
                e = np.zeros((4, 1))
                e[s] = 1.0
                new[qn] = new.get(qn, 0.0) + np.kron(left[q], e) @ A
        left = new
    right = {(d.Na, d.Nb): np.ones((1, 1))}  # q -> (dim_i(q), 4^(n-i))
    for i in range(n - 1, k + 1, -1):
        new = {}
        for (q, s), B in d.sites[i].items():
            qn = (q[0] + mpo.QN[s][0], q[1] + mpo.QN[s][1])
            if qn in right:
                e = np.zeros((1, 4))
                e[0, s] = 1.0
                new[q] = new.get(q, 0.0) + np.kron(e, B @ right[qn])
        right = new
    out = 0.0
    for (ql, s1, s2), X in psi.items():
        qr = (ql[0] + mpo.QN[s1][0] + mpo.QN[s2][0], ql[1] + mpo.QN[s1][1] + mpo.QN[s2][1])
        mid = np.zeros(16)
        mid[s1 * 4 + s2] = 1.0
        lv = left[ql] @ X @ right[qr]  # (4^k, 4^(n-k-2))
        out = out + np.einsum("ab,m->amb", lv, mid).reshape(-1)
    return out


def test_dmrg_full_bond_equals_fci_cas6():
    with open(os.path.join(GOLDEN, "fci_cas6_m64_seed1.json")) as f:
        g = json.load(f)
    h, chol = make_integrals(6, 18, 1)
    d, sw = dmrg.run(h, chol, 6, 0, [64] * 4, [1e-9] * 4, seed=1)
    assert abs(d.energy() - g["E0"]) < 1e-10
    assert abs(sw[-1] - g["E0"]) < 1e-10
    g1, g2 = d.rdms()
    assert np.abs(g1 - np.array(g["rdm1"])).max() < 1e-7
    assert abs(np.einsum("pprr->", g2) - g["rdm2_trace"]) < 1e-9
    eri = fock.eri_from_chol(chol)
    E = np.einsum("pq,pq", h, g1) + 0.5 * np.einsum("pqrs,pqrs", eri, g2)
    assert abs(E - d.energy()) < 1e-10


def test_dmrg_energy_monotone_in_bond_dimension():
    h, chol = make_integrals(6, 18, 1)
    with open(os.path.join(GOLDEN, "fci_cas6_m64_seed1.json")) as f:
        E_fci = json.load(f)["E0"]
    Es = []
    for M in [4, 8, 16, 64]:
        d, sw = dmrg.run(h, chol, 6, 0, [M] * 3, [1e-9] * 3, seed=1)
        Es.append(d.energy())
    for a, b in zip(Es, Es[1:]):
        assert b <= a + 1e-10
    assert min(Es) >= E_fci - 1e-10


def test_select_states_tie_rule():
    w = [(0.5, (1, 0), 0), (0.2, (0, 1), 0), (0.2, (1, 0), 1), (0.1, (0, 0), 0)]
    kept, tau = dmrg.select_states(w, 2)
    # the 0.2 pair straddles the cut: the whole multiplet is dropped
    assert [k[0] for k in kept] == [0.5]
    assert abs(tau - 0.5) < 1e-15
    kept, tau = dmrg.select_states(w, 3)
    assert [k[1] for k in kept] == [(1, 0), (0, 1), (1, 0)]
    kept, _ = dmrg.select_states([(0.3, (0, 0), 0), (1e-13, (0, 1), 0)], 5)
    assert len(kept) == 1


def test_move_center_keeps_state_and_gauge():
    # left-orthonormal sites after the move, unchanged expansion coefficients
    h, chol = make_integrals(6, 8, 3)
    d = dmrg.DMRG(h, chol, 6, 0, 12, seed=2)
    C0 = d.to_ci()
    d.move_center(3)
    for i in range(3):
        for Q in d.dims[i + 1]:
            rows = [d.sites[i][(dmrg.qsub(Q, mpo.QN[s]), s)] for s in range(4)
                    if (dmrg.qsub(Q, mpo.QN[s]), s) in d.sites[i]]
            A = np.vstack(rows)
            assert np.abs(A.T @ A - np.eye(A.shape[1])).max() < 1e-12
    assert np.abs(d.to_ci() - C0).max() < 1e-12
    # H_eff at the new centre is the projected Hamiltonian: its expectation
    # value in the two-site state equals the energy of the full state
    eri = fock.eri_from_chol(chol)
    f = fci.FCI(h, eri, 3, 3)
    c = C0.reshape(-1)
    E = c @ f.sigma(c).ravel() / (c @ c)
    k = 3
    psi = dmrg.two_site_psi(d.sites[k], d.sites[k + 1], d.dims[k + 1])
    keys = dmrg.psi_keys(d.dims[k], d.dims[k + 2])
    x = dmrg.flatten(psi, keys, d.dims[k], d.dims[k + 2])
    s = dmrg.flatten(dmrg.apply_heff(*d.heff_parts(k), psi, d.mpo, k), keys, d.dims[k], d.dims[k + 2])
    assert abs(x @ s / (x @ x) - E) < 1e-11


def test_select_states_adaptive_bond_dimension():
    # the smallest m whose discarded weight is <= delta, clusters kept whole,
    # m_min as a floor, M as a cap (brute force over m)
    rng = np.random.default_rng(17)
    for trial in range(200):
        n = int(rng.integers(1, 30))
        lam = np.sort(rng.exponential(1.0, n) ** 3)[::-1]
        if trial % 5 == 0 and n > 3:
            lam[2] = lam[1]                      # a degenerate pair
        lam /= lam.sum()
        w = [(float(v), (i % 3, 0), i) for i, v in enumerate(lam)]
        delta = float(10 ** rng.uniform(-8, -1))
        M = int(rng.integers(1, n + 3))
        m_min = int(rng.integers(1, 4))
        kept, tau = dmrg.select_states(w, M, tie=1e-12, max_discarded=delta, m_min=m_min)
        order = sorted(w, key=lambda x: (-x[0], x[1], x[2]))
        disc = lambda m: sum(x[0] for x in order[m:])
        m_delta = next(m for m in range(n + 1) if disc(m) <= delta)
        while 0 < m_delta < n and order[m_delta - 1][0] - order[m_delta][0] <= 1e-12:
            m_delta += 1
        m_delta = max(m_delta, min(m_min, n))
        if m_delta < min(M, n):
            assert kept == order[:m_delta]
            assert tau <= delta + 1e-15   # extending m only lowers the discarded weight
        else:
            assert kept == dmrg.select_states(w, M, tie=1e-12)[0]
        assert abs(tau - (sum(lam) - sum(x[0] for x in kept))) < 1e-12
    # max_discarded = 0 is the fixed-M rule
    w = [(0.5, (0, 0), 0), (0.3, (0, 1), 0), (0.2, (1, 0), 0)]
    assert dmrg.select_states(w, 2) == dmrg.select_states(w, 2, max_discarded=0.0)
    # a loose target keeps fewer states than M; a tight one is capped by M
    assert len(dmrg.select_states(w, 3, max_discarded=0.25)[0]) == 2
    assert len(dmrg.select_states(w, 2, max_discarded=1e-9)[0]) == 2
