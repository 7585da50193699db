"""Pins of the brute-force Fock-space and FCI oracles against closed forms,
special cases and each other (nothing here runs on a GPU)."""
import json
import os
from math import comb

import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import fci, fock

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_hubbard_dimer_closed_form():
    # two-site Hubbard: (00|00) = (11|11) = U, h_01 = -t, one electron of
    # each spin: E0 = (U - sqrt(U^2 + 16 t^2)) / 2 (textbook result).
    for t, U in [(1.0, 4.0), (0.3, 1.0), (1.0, 0.0), (0.5, 8.0)]:
        E0 = (U - np.sqrt(U * U + 16 * t * t)) / 2
        h = np.array([[0.0, -t], [-t, 0.0]])
        eri = np.zeros((2, 2, 2, 2))
        eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
        w, _, _ = fock.ground_state(h, eri, 1, 1)
        assert abs(w[0] - E0) < 1e-12
        e, _ = fci.FCI(h, eri, 1, 1).ground_state()
        assert abs(e[0] - E0) < 1e-12


def test_one_body_only_is_orbital_sum():
    # without two-electron integrals E0 = sum of the lowest N_a plus the
    # lowest N_b eigenvalues of h.
    h, _ = make_integrals(5, 1, 11)
    eri = np.zeros((5, 5, 5, 5))
    eps = np.linalg.eigvalsh(h)
    for na, nb in [(2, 2), (3, 1), (2, 3)]:
        w, _, _ = fock.ground_state(h, eri, na, nb)
        assert abs(w[0] - (eps[:na].sum() + eps[:nb].sum())) < 1e-12
        e, _ = fci.FCI(h, eri, na, nb).ground_state()
        assert abs(e[0] - (eps[:na].sum() + eps[:nb].sum())) < 1e-12


def test_diagonal_integrals_give_determinant_energy():
    # h diagonal and only (pp|qq) nonzero: H is diagonal in the determinant
    # basis; E0 = min over determinants of
    #   sum h_pp n_p + 1/2 sum_pq (pp|qq) (n_p n_q - sum_s n_ps n_qs delta_pq)
    n = 4
    rng = np.random.default_rng(3)
    hd = rng.uniform(-2, 0, n)
    J = rng.uniform(0, 0.5, (n, n))
    J = 0.5 * (J + J.T)
    h = np.diag(hd)
    eri = np.zeros((n, n, n, n))
    for p in range(n):
        for q in range(n):
            eri[p, p, q, q] = J[p, q]
    best = np.inf
    for a in fci.strings(n, 2):
        for b in fci.strings(n, 2):
            na = np.zeros(n); nb = np.zeros(n)
            na[list(a)] = 1; nb[list(b)] = 1
            nt = na + nb
            E = hd @ nt + 0.5 * (nt @ J @ nt - (na * na + nb * nb) @ np.diag(J))
            best = min(best, E)
    w, _, _ = fock.ground_state(h, eri, 2, 2)
    assert abs(w[0] - best) < 1e-12
    e, _ = fci.FCI(h, eri, 2, 2).ground_state()
    assert abs(e[0] - best) < 1e-12


def test_colex_addressing_is_a_bijection():
    for n, k in [(6, 3), (8, 4), (12, 6)]:
        s = fci.strings(n, k)
        assert len(s) == comb(n, k)
        assert all(x is not None for x in s)
        assert all(fci.colex_addr(o) == i for i, o in enumerate(s))
    # determinant counts quoted for CAS(6,6) and CAS(12,12)
    assert comb(6, 3) ** 2 == 400
    assert comb(12, 6) ** 2 == 853776


def test_fci_matches_fock_space_energy_and_rdms():
    h, chol = make_integrals(4, 6, 5)
    eri = fock.eri_from_chol(chol)
    for na, nb in [(2, 2), (2, 1), (3, 1)]:
        w, v, st = fock.ground_state(h, eri, na, nb)
        f = fci.FCI(h, eri, na, nb)
        e, c = f.ground_state()
        assert abs(w[0] - e[0]) < 1e-12
        g1f, g2f = fock.rdms(v[:, 0], st, 4)
        g1, g2 = f.rdms(c[:, 0])
        assert np.abs(g1 - g1f).max() < 1e-11
        assert np.abs(g2 - g2f).max() < 1e-11


def test_fci_sigma_hermitian_and_diagonal():
    h, chol = make_integrals(5, 8, 9)
    eri = fock.eri_from_chol(chol)
    f = fci.FCI(h, eri, 3, 2)
    H = f.dense_h()
    assert np.abs(H - H.T).max() < 1e-13
    assert np.abs(np.diag(H) - f.diagonal().ravel()).max() < 1e-12


def test_fci_davidson_matches_dense():
    h, chol = make_integrals(6, 18, 1)
    eri = fock.eri_from_chol(chol)
    f = fci.FCI(h, eri, 3, 3)
    e_dense, _ = f.ground_state(dense_limit=10 ** 9)
    e_dav, x = fci.davidson(lambda v: f.sigma(v).ravel(), f.diagonal().ravel(), tol=1e-10)
    assert abs(e_dense[0] - e_dav[0]) < 1e-11


def test_rdm_identities():
    h, chol = make_integrals(6, 18, 1)
    eri = fock.eri_from_chol(chol)
    f = fci.FCI(h, eri, 3, 3)
    e, c = f.ground_state()
    g1, g2 = f.rdms(c[:, 0])
    N = 6
    assert abs(np.trace(g1) - N) < 1e-12
    assert abs(np.einsum("pprr->", g2) - N * (N - 1)) < 1e-11
    assert np.abs(g1 - g1.T).max() < 1e-12
    assert np.abs(g2 - g2.transpose(2, 3, 0, 1)).max() < 1e-12
    ev = np.linalg.eigvalsh(g1)
    assert ev.min() > -1e-12 and ev.max() < 2 + 1e-12
    E = np.einsum("pq,pq", h, g1) + 0.5 * np.einsum("pqrs,pqrs", eri, g2)
    assert abs(E - e[0]) < 1e-11


def test_fci_golden_cas6():
    with open(os.path.join(GOLDEN, "fci_cas6_m64_seed1.json")) as f:
        g = json.load(f)
    h, chol = make_integrals(6, 18, 1)
    eri = fock.eri_from_chol(chol)
    w, _, _ = fock.ground_state(h, eri, 3, 3, nroots=2)
    assert abs(w[0] - g["E0"]) < 1e-11
    assert abs(w[1] - g["E1"]) < 1e-11


def test_planted_sign_error_is_caught(monkeypatch):
    # a wrong sign in one single-excitation entry must break the FCI vs
    # Fock agreement: the pins above are sensitive to it.
    h, chol = make_integrals(4, 6, 5)
    eri = fock.eri_from_chol(chol)
    w, _, _ = fock.ground_state(h, eri, 2, 2)
    f = fci.FCI(h, eri, 2, 2)
    I, J, pq, s = f.exa
    s = s.copy()
    s[len(s) // 3] *= -1
    f.exa = (I, J, pq, s)
    e, _ = f.ground_state()
    assert abs(e[0] - w[0]) > 1e-6
