"""1-/2-RDMs from the CUDA engine against the oracle (determinant expansion of
the same MPS + FCI string RDMs) and against FCI at full bond."""
import json
import os

import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import dmrg, fock

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def G():
    from paper_2609_09990_gb300 import build, gbdmrg
    build.build()
    return gbdmrg


@pytest.mark.parametrize("n,ne,two_sz,M,k", [(8, 8, 0, 30, 3), (5, 5, 1, 12, 2), (6, 4, -2, 10, 1), (7, 9, 1, 20, 0)])
def test_rdms_of_installed_mps_match_oracle(G, n, ne, two_sz, M, k):
    h, chol = make_integrals(n, 6, 11)
    d = dmrg.DMRG(h, chol, ne, two_sz, M, seed=5)
    for j in range(k):
        d.step(j, M, 1e-9, "L")
    g1, g2 = d.rdms()
    ctx = G.Context(0)
    ctx.setup(h, chol, ne, two_sz, [M], [1e-9], seed=5)
    ns, tr, data = dmrg.canonical_blocks(d)
    ctx.set_mps(ns, tr, data, k)
    r1, r2 = ctx.rdms(n)
    assert np.abs(r1 - g1).max() < 1e-12
    assert np.abs(r2 - g2).max() < 1e-12
    ctx.close()


def test_solve_cas6_rdms_equal_fci(G):
    with open(os.path.join(GOLDEN, "fci_cas6_m64_seed1.json")) as f:
        g = json.load(f)
    h, chol = make_integrals(6, 18, 1)
    ctx = G.Context(0)
    r = ctx.solve(h, chol, 6, 0, [64] * 4, [1e-9] * 4, seed=1, rdms=True)
    assert abs(r["energy"] - g["E0"]) < 1e-10
    # gap 0.037 Ha: RDMs are unique; first-order in the Davidson residual
    assert np.abs(r["rdm1"] - np.array(g["rdm1"])).max() < 1e-7
    assert abs(np.einsum("pprr->", r["rdm2"]) - g["rdm2_trace"]) < 1e-9
    eri = fock.eri_from_chol(chol)
    E = np.einsum("pq,pq", h, r["rdm1"]) + 0.5 * np.einsum("pqrs,pqrs", eri, r["rdm2"])
    assert abs(E - r["energy"]) < 1e-10
    ctx.close()


def test_solve_cas12_energy_and_rdm_identities(G):
    with open(os.path.join(GOLDEN, "fci_cas12_m256_seed2.json")) as f:
        g = json.load(f)
    h, chol = make_integrals(12, 36, 2)
    ctx = G.Context(0)
    tols = [1e-6, 1e-7, 1e-8, 1e-8, 1e-9, 1e-9]
    r = ctx.solve(h, chol, 12, 0, [256] * 6, tols, seed=2, rdms=True)
    # variational: never below FCI; sweeps non-increasing
    assert r["energy"] >= g["E0"] - 1e-8
    assert np.all(np.diff(r["sweep_energies"]) <= 1e-8)
    g1, g2 = r["rdm1"], r["rdm2"]
    N = 12
    assert abs(np.trace(g1) - N) < 1e-9
    assert abs(np.einsum("pprr->", g2) - N * (N - 1)) < 1e-8
    assert np.abs(g1 - g1.T).max() < 1e-10
    assert np.abs(g2 - g2.transpose(2, 3, 0, 1)).max() < 1e-10
    ev = np.linalg.eigvalsh(g1)
    assert ev.min() > -1e-10 and ev.max() < 2 + 1e-10
    eri = fock.eri_from_chol(chol)
    E = np.einsum("pq,pq", h, g1) + 0.5 * np.einsum("pqrs,pqrs", eri, g2)
    assert abs(E - r["energy"]) < 1e-9
    print("CAS(12,12) M=256: E_DMRG - E_FCI =", r["energy"] - g["E0"], "sweeps", r["sweep_energies"])
    ctx.close()
