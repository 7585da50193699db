"""Pins of the excited-state reference: <S^2> from the 2-RDM against the
Jordan-Wigner S^2 operator and closed forms, and the sector spectrum against
the Hubbard dimer's closed form."""
import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import fock, states


def sector_vec(n, na, nb, seed):
    st = fock.sector_states(n, na, nb)
    v = np.random.default_rng(seed).normal(size=st.size)
    return v / np.linalg.norm(v), st


@pytest.mark.parametrize("n,na,nb", [(2, 1, 1), (3, 2, 1), (3, 1, 1), (3, 2, 2), (4, 2, 2), (3, 3, 0)])
def test_spin_square_from_rdm_matches_the_operator(n, na, nb):
    S2 = fock.spin_square(n)
    for seed in range(3):
        v, st = sector_vec(n, na, nb, seed + 10 * n + na)
        full = np.zeros(1 << (2 * n))
        full[st] = v
        ref = full @ (S2 @ full)
        _, g2 = fock.rdms(v, st, n)
        assert abs(states.spin_square_from_rdm(g2, na + nb) - ref) < 1e-12


def test_spin_square_closed_forms():
    # one electron: 3/4; a doubly occupied orbital: 0; two alpha electrons
    # (high-spin pair): S(S+1) = 2
    for n, na, nb, want in [(2, 1, 0, 0.75), (2, 0, 1, 0.75), (2, 2, 0, 2.0), (3, 3, 0, 3.75)]:
        v, st = sector_vec(n, na, nb, 1)
        _, g2 = fock.rdms(v, st, n)
        assert abs(states.spin_square_from_rdm(g2, na + nb) - want) < 1e-12
    st = fock.sector_states(2, 1, 1)
    v = (st == 0b0011).astype(float)   # orbital 0 doubly occupied
    _, g2 = fock.rdms(v, st, 2)
    assert abs(states.spin_square_from_rdm(g2, 2)) < 1e-12


@pytest.mark.parametrize("t,U", [(1.0, 4.0), (0.5, 1.0), (1.0, 0.5)])
def test_hubbard_dimer_spectrum_and_spins(t, U):
    # two sites, one electron of each spin: singlet (U - sqrt(U^2+16t^2))/2,
    # triplet 0, singlet U, singlet (U + sqrt(U^2+16t^2))/2
    h = np.array([[0.0, -t], [-t, 0.0]])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
    r = np.sqrt(U * U + 16 * t * t)
    want = sorted([((U - r) / 2, 0.0), (0.0, 2.0), (U, 0.0), ((U + r) / 2, 0.0)])
    w, s2, _ = states.sector_spectrum(h, eri, 1, 1, 4)
    assert np.allclose(w, [e for e, _ in want], atol=1e-12)
    assert np.allclose(s2, [s for _, s in want], atol=1e-12)
    singlets = states.select_roots(w, s2, 0.0, 3)
    assert [want[i][1] for i in singlets] == [0.0, 0.0, 0.0]
    assert states.select_roots(w, s2, 2.0, 1) == [[e for e, _ in want].index(0.0)]


def test_sector_spectrum_spins_are_s_of_s_plus_1():
    # S_z = 0 sector of CAS(4,4): every eigenvector is a spin eigenstate
    h, chol = make_integrals(4, 6, 3)
    w, s2, _ = states.sector_spectrum(h, fock.eri_from_chol(chol), 2, 2, 12)
    for v in s2:
        S = (np.sqrt(1 + 4 * v) - 1) / 2
        assert abs(S - round(S)) < 1e-8
