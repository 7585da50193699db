"""1-/2-RDMs contracted through the MPS (operator-string environments,
gbd_rdms) against the oracle and against the determinant-expansion route
(gbd_rdms_ci), and at CAS(20,20), where no determinant expansion fits,
against the identities every RDM pair satisfies:
  tr gamma = N,  sum_pr Gamma_pprr = N (N - 1),  sum_r Gamma_pqrr = (N - 1) gamma_pq,
  Gamma_pqrs = Gamma_rspq = Gamma_qpsr,  0 <= eig(gamma) <= 2,
  E = sum h_pq gamma_pq + 1/2 sum (pq|rs) Gamma_pqrs  (the solve's energy)."""
import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import dmrg, fock

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
        d.step(j, M, 1e-9, "L")
    ctx = G.Context(0)
    ctx.setup(h, chol, ne, two_sz, [M], [1e-9], seed=seed)
    ns, tr, data = dmrg.canonical_blocks(d)
    ctx.set_mps(ns, tr, data, k)
    return ctx, d


# (n, n_elec, 2 S_z, Cholesky vectors, seed, M, steps taken before the
# install: the position of the mixed-canonical centre)
CASES = [(2, 2, 0, 3, 1, 4, 0), (3, 3, 1, 4, 2, 8, 1), (4, 6, 0, 5, 3, 16, 2), (6, 6, 0, 8, 4, 24, 0),
         (6, 5, -1, 8, 5, 20, 4), (7, 4, 2, 6, 6, 18, 3), (8, 8, 0, 10, 7, 40, 5), (8, 11, 1, 10, 8, 32, 6)]


@pytest.mark.parametrize("n,ne,two_sz,nq,seed,M,k", CASES)
def test_mps_rdms_match_oracle(G, n, ne, two_sz, nq, seed, M, k):
    ctx, d = installed(G, n, ne, two_sz, nq, seed, M, k)
    r1, r2 = ctx.rdms(n)
    c1, c2 = ctx.rdms_ci(n)
    ctx.close()
    g1, g2 = d.rdms()
    assert np.abs(r1 - g1).max() < 1e-12
    assert np.abs(r2 - g2).max() < 1e-12
    assert np.abs(r1 - c1).max() < 1e-12
    assert np.abs(r2 - c2).max() < 1e-12


def test_mps_and_determinant_routes_agree_cas12(G):
    n, ne = 12, 12
    h, chol = make_integrals(n, 36, 2)
    ctx = G.Context(0)
    ctx.solve(h, chol, ne, 0, [128] * 2, [1e-6] * 2, seed=2)
    r1, r2 = ctx.rdms(n)
    c1, c2 = ctx.rdms_ci(n)
    ctx.close()
    assert np.abs(r1 - c1).max() < 1e-11
    assert np.abs(r2 - c2).max() < 1e-11 * max(1.0, np.abs(c2).max())


def check_identities(h, chol, ne, E, g1, g2, tol_e):
    n = h.shape[0]
    scale = max(1.0, np.abs(g2).max())
    assert abs(np.trace(g1) - ne) < 1e-9
    assert abs(np.einsum("pprr->", g2) - ne * (ne - 1)) < 1e-8
    assert np.abs(np.einsum("pqrr->pq", g2) - (ne - 1) * g1).max() < 1e-9 * scale
    assert np.abs(g2 - g2.transpose(2, 3, 0, 1)).max() < 1e-10 * scale
    assert np.abs(g2 - g2.transpose(1, 0, 3, 2)).max() < 1e-10 * scale
    w = np.linalg.eigvalsh(0.5 * (g1 + g1.T))
    assert w.min() > -1e-9 and w.max() < 2 + 1e-9
    eri = fock.eri_from_chol(chol)
    E_rdm = np.einsum("pq,pq", h, g1) + 0.5 * np.einsum("pqrs,pqrs", eri, g2)
    assert abs(E_rdm - E) < tol_e, (E_rdm, E)


def test_cas20_rdms_from_the_mps(G):
    # CAS(20,20) with 60 Cholesky vectors: 3.4e10 determinants, beyond the
    # determinant route; the RDMs of a short solve satisfy every identity
    # and reproduce its energy
    n, ne = 20, 20
    h, chol = make_integrals(n, 60, 4)
    ctx = G.Context(0)
    r = ctx.solve(h, chol, ne, 0, [32, 64], [1e-6] * 2, seed=4, rdms=True)
    st = ctx.stats()
    ctx.close()
    check_identities(h, chol, ne, r["energy"], r["rdm1"], r["rdm2"], 1e-8)
    assert st["rdm_ms"] > 0 and st["rdm_env_bytes"] > 0


@pytest.mark.parametrize("n,ne,two_sz,nq,seed,M,k", [CASES[1], CASES[3], CASES[4], CASES[7]])
def test_mps_orbital_rdms_match_oracle(G, n, ne, two_sz, nq, seed, M, k):
    from oracle import entropy
    ctx, d = installed(G, n, ne, two_sz, nq, seed, M, k)
    r1, r2 = ctx.orbital_rdms(n)
    c1, c2 = ctx.orbital_rdms_ci(n)
    s1, mi = ctx.orbital_entropies(n)
    ctx.close()
    C = d.to_ci()
    full = fock.from_ci(C / np.linalg.norm(C), n, d.Na, d.Nb)
    assert np.abs(r1 - c1).max() < 1e-12
    assert np.abs(r2 - c2).max() < 1e-12
    pr = 0
    for i in range(n):
        assert np.abs(r1[i] - entropy.orbital_rdm(full, n, [i])).max() < 1e-12
        for j in range(i + 1, n):
            assert np.abs(r2[pr] - entropy.orbital_rdm(full, n, [i, j])).max() < 1e-12, (i, j)
            pr += 1
    assert np.abs(mi - entropy.mutual_information(full, n)).max() < 1e-10


def test_cas20_orbital_rdms_and_mutual_information(G):
    # the one- and two-orbital RDMs of a CAS(20,20) state are density
    # matrices whose partial traces agree, and the mutual information is a
    # symmetric non-negative matrix bounded by 2 ln 4
    n, ne = 20, 20
    h, chol = make_integrals(n, 60, 4)
    ctx = G.Context(0)
    ctx.solve(h, chol, ne, 0, [32, 64], [1e-6] * 2, seed=4)
    r1, r2 = ctx.orbital_rdms(n)
    s1, mi = ctx.orbital_entropies(n)
    ctx.close()
    for i in range(n):
        assert abs(np.trace(r1[i]) - 1) < 1e-10
        assert np.abs(r1[i] - np.diag(np.diag(r1[i]))).max() == 0.0
    pr = 0
    for i in range(n):
        for j in range(i + 1, n):
            R = r2[pr].reshape(4, 4, 4, 4)   # [x'_j, x'_i, x_j, x_i]
            assert np.abs(r2[pr] - r2[pr].T).max() < 1e-12
            w = np.linalg.eigvalsh(r2[pr])
            assert w.min() > -1e-12 and abs(w.sum() - 1) < 1e-10
            assert np.abs(np.einsum("jajb->ab", R) - r1[i]).max() < 1e-11
            assert np.abs(np.einsum("ajbj->ab", R) - r1[j]).max() < 1e-11
            pr += 1
    assert np.abs(mi - mi.T).max() == 0.0
    assert mi.min() > -1e-10 and mi.max() < 2 * np.log(4)
    assert np.all((s1 >= -1e-12) & (s1 <= np.log(4) + 1e-12))
