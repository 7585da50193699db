"""Pins of the 3-RDM reference: the excitation-operator route against the
operator strings of the definition, the partial-trace identity to the 2-RDM,
and the index symmetries."""
import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import fci, fock


@pytest.mark.parametrize("n,na,nb", [(3, 2, 1), (3, 1, 1), (3, 2, 2)])
def test_rdm3_matches_the_operator_definition(n, na, nb):
    h, chol = make_integrals(n, 4, n + na)
    eri = fock.eri_from_chol(chol)
    F = fci.FCI(h, eri, na, nb)
    w, v = np.linalg.eigh(F.dense_h())
    C = v[:, 0]
    G = fci.rdm3(F, C)
    # the same state in the Fock basis: FCI determinant order (alpha string,
    # beta string) -> Fock bit strings, through the ground state energy
    e, vf, st = fock.ground_state(h, eri, na, nb)
    assert abs(e[0] - w[0]) < 1e-12
    Gf = fock.rdm3(vf[:, 0], st, n)
    assert np.abs(G - Gf).max() < 1e-11


def test_rdm3_partial_trace_and_symmetries():
    h, chol = make_integrals(5, 7, 3)
    F = fci.FCI(h, fock.eri_from_chol(chol), 3, 2)
    C = np.random.default_rng(1).normal(size=F.Na * F.Nb)
    C /= np.linalg.norm(C)
    G = fci.rdm3(F, C)
    _, g2 = F.rdms(C)
    N = 5
    assert np.allclose(np.einsum("pqrstt->pqrs", G), (N - 2) * g2, atol=1e-12)
    assert np.allclose(G, G.transpose(2, 3, 0, 1, 4, 5), atol=1e-12)     # swap particles 1, 2
    assert np.allclose(G, G.transpose(4, 5, 2, 3, 0, 1), atol=1e-12)     # swap particles 1, 3
    assert np.allclose(G, G.transpose(1, 0, 3, 2, 5, 4), atol=1e-12)     # hermiticity (real C)
