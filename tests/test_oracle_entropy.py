"""Pins of the orbital-entropy and mutual-information reference."""
import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import entropy, fock


def full_vector(n, na, nb, seed):
    st = fock.sector_states(n, na, nb)
    v = np.random.default_rng(seed).normal(size=st.size)
    full = np.zeros(1 << (2 * n))
    full[st] = v / np.linalg.norm(v)
    return full


def test_closed_shell_determinant_has_no_entropy():
    n = 4
    full = np.zeros(1 << (2 * n))
    full[0b00001111] = 1.0                      # orbitals 0 and 1 doubly occupied
    I = entropy.mutual_information(full, n)
    assert np.abs(I).max() < 1e-14
    for i in range(n):
        assert entropy.entropy(entropy.orbital_rdm(full, n, [i])) < 1e-14


@pytest.mark.parametrize("t,U", [(1.0, 0.0), (1.0, 4.0), (0.5, 1.0), (0.2, 5.0)])
def test_hubbard_dimer_mutual_information(t, U):
    # ground state = c_ion (|20>+|02>)/sqrt2 + c_cov singlet, with
    # c_ion^2 = (1 - U / sqrt(U^2 + 16 t^2)) / 2; each site has p(0) = p(ab) =
    # c_ion^2 / 2 and p(a) = p(b) = c_cov^2 / 2, and the pair is pure, so
    # I_12 = 2 s_1
    h = np.array([[0.0, -t], [-t, 0.0]])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
    _, v, st = fock.ground_state(h, eri, 1, 1)
    full = np.zeros(16)
    full[st] = v[:, 0]
    ci = (1 - U / np.sqrt(U * U + 16 * t * t)) / 2
    cc = 1 - ci
    s1 = -sum(p * np.log(p) for p in (ci / 2, ci / 2, cc / 2, cc / 2) if p > 0)
    I = entropy.mutual_information(full, 2)
    assert abs(I[0, 1] - 2 * s1) < 1e-12
    assert abs(entropy.entropy(entropy.orbital_rdm(full, 2, [0, 1]))) < 1e-12


def test_two_orbital_rdm_is_a_density_matrix():
    full = full_vector(4, 2, 2, 3)
    for i, j in [(0, 1), (0, 3), (2, 1)]:
        rho = entropy.orbital_rdm(full, 4, [i, j])
        assert abs(np.trace(rho) - 1) < 1e-12
        assert np.allclose(rho, rho.T, atol=1e-14)
        assert np.linalg.eigvalsh(rho).min() > -1e-12


@pytest.mark.parametrize("i,j", [(0, 1), (0, 3), (3, 1), (1, 2)])
def test_hopping_element_matches_the_fock_expectation(i, j):
    # <c+_{i alpha} c_{j alpha}> from rho_ij (local modes 0..3 = i alpha, i beta,
    # j alpha, j beta) equals the same expectation on the full Fock vector
    n = 4
    full = full_vector(n, 2, 2, 10 * i + j)
    rho = entropy.orbital_rdm(full, n, [i, j])
    for s in range(2):
        O = fock.apply_string([(s, True), (2 + s, False)], 16).toarray()
        local = float(np.sum(O * rho))
        direct = float(full @ (fock.apply_string([(2 * i + s, True), (2 * j + s, False)], 1 << (2 * n)) @ full))
        assert abs(local - direct) < 1e-12


def test_mutual_information_of_a_ground_state():
    h, chol = make_integrals(4, 6, 2)
    _, v, st = fock.ground_state(h, fock.eri_from_chol(chol), 2, 2)
    full = np.zeros(1 << 8)
    full[st] = v[:, 0]
    I = entropy.mutual_information(full, 4)
    assert np.allclose(I, I.T) and I.min() > -1e-12 and np.all(np.diag(I) == 0)
    assert I.max() > 1e-3                       # a correlated state


@pytest.mark.parametrize("n,na,nb", [(4, 2, 2), (4, 3, 1), (5, 2, 3)])
def test_ci_to_fock_reproduces_the_fock_ground_state(n, na, nb):
    # the determinant-basis ground state (fci.py, alpha-first creator order)
    # rewritten in the site-major Fock basis is the Fock-space ground state
    # (brute-force eigh of the Jordan-Wigner H) up to a global sign; a wrong
    # reordering sign breaks the equality
    from oracle import fci
    h, chol = make_integrals(n, 4, 31 + n + na)
    eri = fock.eri_from_chol(chol)
    w, v, st = fock.ground_state(h, eri, na, nb)
    f = fci.FCI(h, eri, na, nb)
    e, x = fci.davidson(lambda c: f.sigma(c).ravel(), f.diagonal().ravel(), tol=1e-12)
    assert abs(e[0] - w[0]) < 1e-10
    full = fock.from_ci(x[:, 0] / np.linalg.norm(x[:, 0]), n, na, nb)
    ref = np.zeros_like(full)
    ref[st] = v[:, 0]
    assert np.abs(abs(full @ ref) - 1.0) < 1e-10
    assert min(np.abs(full - ref).max(), np.abs(full + ref).max()) < 1e-6
