"""Excited states by penalty deflation against the sector spectrum (dense FCI)
and its <S^2> values: at full bond dimension the deflated sweeps reach the
eigenpairs of H in the (N_alpha, N_beta) sector, in order, and the <S^2>
guard keeps only roots of the target spin."""
import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import fock, states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2609_09990_gb300 import build, gbdmrg
    build.build()
    return gbdmrg


@pytest.fixture(scope="module")
def cas66():
    h, chol = make_integrals(6, 8, 5)
    w, s2, _ = states.sector_spectrum(h, fock.eri_from_chol(chol), 3, 3, 30)
    return h, chol, w, s2


def test_lowest_roots_of_any_spin(G, cas66):
    h, chol, w, s2 = cas66
    pen = 2.0 * (w[2] - w[0]) + 1.0
    ctx = G.Context(0)
    rc, res = ctx.solve_states(h, chol, 6, 0, [64] * 8, [1e-9] * 8, 3, penalty=pen, target_s2=-1.0, max_extra=0,
                               seed=5)
    ctx.close()
    assert len(res) == 3
    assert np.allclose([r["energy"] for r in res], w[:3], rtol=0, atol=1e-8)
    assert np.allclose([r["s2"] for r in res], s2[:3], rtol=0, atol=1e-6)


def test_singlet_roots_with_the_spin_guard(G, cas66):
    h, chol, w, s2 = cas66
    sel = states.select_roots(w, s2, 0.0, 3)
    assert len(sel) == 3
    pen = 2.0 * (w[sel[-1]] - w[0]) + 1.0
    ctx = G.Context(0)
    rc, res = ctx.solve_states(h, chol, 6, 0, [64] * 8, [1e-9] * 8, 3, penalty=pen, target_s2=0.0,
                               max_extra=sel[-1] - 2 + 1, seed=5, rdms=True)
    ctx.close()
    assert rc == G.GBD_OK and len(res) == 3
    assert np.allclose([r["energy"] for r in res], w[sel], rtol=0, atol=1e-8)
    for r in res:
        assert abs(r["s2"]) < 1e-6
        # the RDMs reproduce the root's energy (E = sum h g1 + 1/2 sum (pq|rs) g2)
        eri = fock.eri_from_chol(chol)
        e = np.einsum("pq,pq", h, r["rdm1"]) + 0.5 * np.einsum("pqrs,pqrs", eri, r["rdm2"])
        assert abs(e - r["energy"]) < 1e-8


def test_too_few_roots_of_the_target_spin(G, cas66):
    # no extra attempts: a triplet among the lowest roots leaves fewer
    # singlets than asked for, reported as not converged with the found ones
    h, chol, w, s2 = cas66
    sel = states.select_roots(w, s2, 0.0, 3)
    if sel[-1] == 2:
        pytest.skip("the three lowest roots are all singlets")
    pen = 2.0 * (w[2] - w[0]) + 1.0
    ctx = G.Context(0)
    rc, res = ctx.solve_states(h, chol, 6, 0, [64] * 8, [1e-9] * 8, 3, penalty=pen, target_s2=0.0, max_extra=0,
                               seed=5, check=False)
    ctx.close()
    assert rc == G.GBD_ERR_NOCONV and len(res) < 3
    for r in res:
        assert abs(r["s2"]) < 1e-6


def test_roots_with_the_tensor_core_tiers(G, cas66):
    # BF16 -> TF32x3 Davidson tiers (forced on this small space): the same
    # singlet roots to the tiers' accuracy
    h, chol, w, s2 = cas66
    sel = states.select_roots(w, s2, 0.0, 3)
    pen = 2.0 * (w[sel[-1]] - w[0]) + 1.0
    ctx = G.Context(0)
    ctx.set_tc_min_two_site(0)
    rc, res = ctx.solve_states(h, chol, 6, 0, [64] * 8, [1e-7] * 8, 3, penalty=pen, target_s2=0.0,
                               max_extra=sel[-1] - 2 + 1, seed=5, precision=G.GBD_BF16, fp64_refine=0)
    st = ctx.stats()
    ctx.close()
    assert st["n_sigma_tc"] > 0
    assert np.allclose([r["energy"] for r in res], w[sel], rtol=0, atol=2e-6)
    assert all(abs(r["s2"]) < 1e-4 for r in res)


def test_truncated_bond_dimension_roots(G):
    # CAS(8,8) at M = 48 (full: 256): each root within a few mHa above FCI
    h, chol = make_integrals(8, 10, 6)
    w, s2, _ = states.sector_spectrum(h, fock.eri_from_chol(chol), 4, 4, 6)
    sel = states.select_roots(w, s2, 0.0, 2)
    pen = 2.0 * (w[sel[-1]] - w[0]) + 1.0
    ctx = G.Context(0)
    rc, res = ctx.solve_states(h, chol, 8, 0, [48] * 8, [1e-8] * 8, 2, penalty=pen, target_s2=0.0,
                               max_extra=sel[-1] - 1 + 2, seed=6)
    ctx.close()
    E = np.array([r["energy"] for r in res])
    assert np.all(E > w[sel] - 1e-9) and np.all(E - w[sel] < 5e-3), E - w[sel]
