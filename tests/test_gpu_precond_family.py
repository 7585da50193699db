"""The Davidson correction family on the GPU: Jacobi and Olsen corrections
element by element against the oracle, and converged energies that do not
depend on the correction (Jacobi, Olsen, inner PCG)."""
import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import fci, fock, precond

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2609_09990_gb300 import build, gbdmrg
    build.build()
    return gbdmrg


def ritz_like(n, seed):
    # unit x, sx with theta = x . sx (so r is orthogonal to x), a diagonal
    # with a few entries within the 1e-8 guard of theta
    rng = np.random.default_rng(seed)
    x = rng.normal(size=n)
    x /= np.linalg.norm(x)
    sx = rng.normal(size=n) + 3.0 * x
    theta = float(x @ sx)
    d = theta + rng.normal(size=n) * 2.0
    if n > 8:
        d[[1, 3, 5]] = theta + np.array([0.0, 4e-9, -7e-9])
    return x, sx, d, theta


@pytest.mark.parametrize("n", [1, 7, 1000, 100003])
@pytest.mark.parametrize("kind", ["diag", "olsen"])
def test_correction_matches_oracle(G, kind, n):
    x, sx, d, theta = ritz_like(n, n + 17)
    code = G.GBD_PRECOND_DIAG if kind == "diag" else G.GBD_PRECOND_OLSEN
    r, t, rr = G.correction_selftest(code, x, sx, d, theta)
    r_ref = sx - theta * x
    t_ref = precond.jacobi_correction(r_ref, d, theta) if kind == "diag" else \
        precond.olsen_correction(x, r_ref, d, theta)
    # r = sx - theta x may be evaluated with a fused multiply-add
    assert np.abs(r - r_ref).max() <= 1e-15 * (np.abs(sx).max() + abs(theta))
    assert abs(rr - r_ref @ r_ref) <= 1e-12 * (r_ref @ r_ref)
    assert np.abs(t - t_ref).max() <= 1e-12 * np.abs(t_ref).max()
    if kind == "olsen" and n > 1:
        assert abs(x @ t) <= 1e-12 * np.linalg.norm(t)


def test_converged_energy_does_not_depend_on_the_correction(G):
    # CAS(6,6) at M = 64 is exact: every correction reaches the FCI energy
    h, chol = make_integrals(6, 8, 5)
    e_fci = np.linalg.eigvalsh(fci.FCI(h, fock.eri_from_chol(chol), 3, 3).dense_h())[0]
    out = {}
    for kind in (G.GBD_PRECOND_DIAG, G.GBD_PRECOND_OLSEN, G.GBD_PRECOND_PCG):
        ctx = G.Context(0)
        r = ctx.solve(h, chol, 6, 0, [64] * 4, [1e-9] * 4, seed=5, preconditioner=kind)
        st = ctx.stats()
        assert (st["inner_matvecs"] > 0) == (kind == G.GBD_PRECOND_PCG)
        out[kind] = (r["energy"], st["davidson_iterations"])
        ctx.close()
    for kind, (e, _) in out.items():
        assert abs(e - e_fci) < 1e-9, (kind, e - e_fci)


def test_reduced_precision_solve_with_each_correction(G):
    # the TF32 -> TF32x3 tiers with every correction reach the FCI energy of
    # CAS(6,6) at M = 64 (exact) to the tiers' accuracy.  (At a truncated M
    # the corrections may settle in different, nearly degenerate two-site
    # fixed points, some 1e-5 Ha apart, so energies are compared where the
    # fixed point is unique.)
    h, chol = make_integrals(6, 8, 5)
    e_fci = np.linalg.eigvalsh(fci.FCI(h, fock.eri_from_chol(chol), 3, 3).dense_h())[0]
    for kind in (G.GBD_PRECOND_DIAG, G.GBD_PRECOND_OLSEN, G.GBD_PRECOND_PCG):
        ctx = G.Context(0)
        ctx.set_tc_min_two_site(0)
        r = ctx.solve(h, chol, 6, 0, [64] * 6, [1e-7] * 6, seed=5, precision=G.GBD_TF32, fp64_refine=0,
                      preconditioner=kind)
        st = ctx.stats()
        ctx.close()
        assert st["n_sigma_tc"] > 0
        assert abs(r["energy"] - e_fci) < 3e-6, (kind, r["energy"] - e_fci)


@pytest.mark.parametrize("case", ["near_converged", "random_mid_spectrum"])
def test_inner_pcg_correction_matches_oracle(G, case):
    # the solver's inner PCG (FP64 sigma of a real two-site step, its own
    # H_eff diagonal) against oracle.precond.pcg_correction with the oracle's
    # H_eff and diagonal, element by element; the random mid-spectrum Ritz
    # value makes the projected operator indefinite, so the curvature guard
    # ends the iteration there
    from oracle import dmrg
    from oracle import fci as fci_mod
    n, ne, nq, seed, M, k = 8, 8, 10, 3, 30, 3
    h, chol = make_integrals(n, nq, seed)
    d = dmrg.DMRG(h, chol, ne, 0, M, seed=seed)
    for j in range(k):
        d.step(j, M, 1e-10, "L")
    keys = dmrg.psi_keys(d.dims[k], d.dims[k + 2])
    L, W1, W2, R = d.heff_parts(k)

    def mv(v):
        return dmrg.flatten(dmrg.apply_heff(L, W1, W2, R, dmrg.unflatten(v, keys, d.dims[k], d.dims[k + 2]),
                                            d.mpo, k), keys, d.dims[k], d.dims[k + 2])

    diag = dmrg.flatten(dmrg.heff_diag(L, W1, W2, R, keys, d.mpo, k, d.dims[k], d.dims[k + 2]),
                        keys, d.dims[k], d.dims[k + 2])
    rng = np.random.default_rng(41)
    if case == "near_converged":
        x0 = dmrg.flatten(dmrg.two_site_psi(d.sites[k], d.sites[k + 1], d.dims[k + 1]), keys, d.dims[k],
                          d.dims[k + 2])
        _, X = fci_mod.davidson(mv, diag, tol=1e-3, guess=x0)
        x = X[:, 0] + 1e-4 * rng.standard_normal(X.shape[0])
    else:
        x = rng.standard_normal(diag.size)
    x /= np.linalg.norm(x)
    sx = mv(x)
    theta = float(x @ sx)
    r = sx - theta * x
    t_ref, nmv_ref = precond.pcg_correction(mv, x, r, diag, theta, steps=4, rel_tol=0.1)
    ctx = G.Context(0)
    ctx.setup(h, chol, ne, 0, [M], [1e-10], seed=seed)
    ns, tr, data = dmrg.canonical_blocks(d)
    ctx.set_mps(ns, tr, data, k)
    assert ctx.two_site_size(k) == x.size
    t, nmv = ctx.pcg_selftest(k, x, r, theta)
    ctx.close()
    assert nmv == nmv_ref
    assert np.abs(t - t_ref).max() <= 1e-9 * np.abs(t_ref).max(), np.abs(t - t_ref).max() / np.abs(t_ref).max()
    assert abs(x @ t) <= 1e-10 * np.linalg.norm(t)
