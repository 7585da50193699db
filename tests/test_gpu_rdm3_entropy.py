"""Device 3-RDM and orbital entropies against the oracle.

* gbd_rdm3 of installed oracle MPSs equals oracle.fci.rdm3 of the oracle's
  own determinant expansion element by element (n <= 8), and at
  CAS(12,12) M=128 it satisfies the partial trace
  sum_u Gamma3_pqrsuu = (N - 2) Gamma_pqrs against gbd_rdms of the same state
  and the particle-swap symmetry.
* gbd_orbital_rdms equals the oracle's fermionic partial traces
  (oracle.entropy.orbital_rdm of the Fock vector), element by element;
  gbd_orbital_entropies equals oracle.entropy's entropies and mutual
  information; gbd_mi_order of a full-bond CAS(6,6) solve equals the
  oracle's Fiedler order of the FCI ground state's mutual information."""
import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import dmrg, entropy, fci, fock, ordering

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2609_09990_gb300 import build, gbdmrg
    build.build()
    return gbdmrg


def installed(G, n, ne, two_sz, nq, seed, M, k):
    h, chol = make_integrals(n, nq, seed)
    d = dmrg.DMRG(h, chol, ne, two_sz, M, seed=seed)
    for j in range(k):
        d.step(j, M, 1e-10, "L")
    ctx = G.Context(0)
    ctx.setup(h, chol, ne, two_sz, [M], [1e-10], seed=seed)
    ns, tr, data = dmrg.canonical_blocks(d)
    ctx.set_mps(ns, tr, data, k)
    C = d.to_ci()
    return ctx, d, C / np.linalg.norm(C)


CASES = [(6, 6, 0, 8, 1, 20, 2), (5, 5, 1, 6, 2, 16, 1), (8, 8, 0, 10, 3, 30, 3), (6, 4, -2, 8, 4, 24, 2)]


@pytest.mark.parametrize("n,ne,two_sz,nq,seed,M,k", CASES)
def test_rdm3_matches_oracle(G, n, ne, two_sz, nq, seed, M, k):
    ctx, d, C = installed(G, n, ne, two_sz, nq, seed, M, k)
    got = ctx.rdm3(n)
    ctx.close()
    ref = fci.rdm3(fci.FCI(d.h, d.eri, d.Na, d.Nb), C)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_rdm3_partial_trace_cas12(G):
    n, ne, nq, seed, M = 12, 12, 36, 2, 128
    h, chol = make_integrals(n, nq, seed)
    ctx = G.Context(0)
    ctx.solve(h, chol, ne, 0, [M] * 2, [1e-6] * 2, seed=seed)
    g3 = ctx.rdm3(n)
    g1, g2 = ctx.rdms(n)
    ctx.close()
    scale = np.abs(g3).max()
    assert np.abs(np.einsum("pqrsuu->pqrs", g3) - (ne - 2) * g2).max() <= 1e-10 * scale
    assert np.abs(g3 - g3.transpose(2, 3, 0, 1, 4, 5)).max() <= 1e-11 * scale
    assert np.abs(g3 - g3.transpose(1, 0, 3, 2, 5, 4)).max() <= 1e-11 * scale


@pytest.mark.parametrize("n,ne,two_sz,nq,seed,M,k", CASES[:2] + [(6, 5, 1, 8, 6, 12, 3)])
def test_orbital_rdms_and_entropies_match_oracle(G, n, ne, two_sz, nq, seed, M, k):
    ctx, d, C = installed(G, n, ne, two_sz, nq, seed, M, k)
    r1, r2 = ctx.orbital_rdms(n)
    s1, mi = ctx.orbital_entropies(n)
    ctx.close()
    full = fock.from_ci(C, n, d.Na, d.Nb)
    pr = 0
    for i in range(n):
        assert np.abs(r1[i] - entropy.orbital_rdm(full, n, [i])).max() <= 1e-12
        assert abs(s1[i] - entropy.entropy(entropy.orbital_rdm(full, n, [i]))) <= 1e-11
        for j in range(i + 1, n):
            assert np.abs(r2[pr] - entropy.orbital_rdm(full, n, [i, j])).max() <= 1e-12, (i, j)
            pr += 1
    assert np.abs(mi - entropy.mutual_information(full, n)).max() <= 1e-10


def test_mi_order_of_a_full_bond_solve(G):
    # CAS(6,6) at M = 64 keeps every state: the solve reaches the FCI ground
    # state, whose mutual information orders the orbitals (oracle: the Fock
    # space ground state and oracle.ordering)
    h, chol = make_integrals(6, 8, 5)
    ctx = G.Context(0)
    order, mi = ctx.mi_order(h, chol, 6, 0, [64] * 4, [1e-10] * 4, seed=5)
    ctx.close()
    _, v, st = fock.ground_state(h, fock.eri_from_chol(chol), 3, 3)
    full = np.zeros(1 << 12)
    full[st] = v[:, 0]
    I = entropy.mutual_information(full, 6)
    assert np.abs(mi - I).max() < 1e-8
    assert list(order) == list(ordering.fiedler_order(I))
