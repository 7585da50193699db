"""Pins of the CPU reference of the Davidson correction vectors (Jacobi,
Olsen, shift-and-invert inner PCG) against their defining properties and
against exact eigenvalues."""
import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import fci, fock, precond


def ritz_pair(H, rng, k=5):
    # lowest Ritz pair of H on a random k-dimensional subspace
    V, _ = np.linalg.qr(rng.normal(size=(H.shape[0], k)))
    w, c = np.linalg.eigh(V.T @ H @ V)
    x = V @ c[:, 0]
    return w[0], x, H @ x - w[0] * x


def random_h(n, seed, spread=3.0):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, n)) * 0.1
    return np.diag(np.sort(rng.normal(size=n) * spread)) + 0.5 * (A + A.T)


def test_guarded_denominator():
    d = np.array([1.0, 2.0, 2.0 + 5e-9, 2.0 - 5e-9, 2.0 + 1e-7])
    den = precond.guarded_den(d, 2.0)
    assert np.array_equal(den[:4], [-1.0, 1e-8, 1e-8, -1e-8])
    assert den[4] == (2.0 + 1e-7) - 2.0   # unguarded: the plain difference


def test_olsen_is_orthogonal_to_the_ritz_vector():
    rng = np.random.default_rng(3)
    for seed in range(5):
        H = random_h(60, seed)
        theta, x, r = ritz_pair(H, rng)
        t = precond.olsen_correction(x, r, np.diag(H), theta)
        assert abs(x @ t) < 1e-12 * np.linalg.norm(t)
        # the Jacobi step is not, in general
        tj = precond.jacobi_correction(r, np.diag(H), theta)
        assert abs(x @ tj) > 1e-6 * np.linalg.norm(tj)


def test_olsen_equals_jacobi_for_a_constant_diagonal():
    # eps = (x . r) / (x . x) = 0 for a Ritz pair when den is constant
    rng = np.random.default_rng(4)
    H = random_h(50, 7)
    theta, x, r = ritz_pair(H, rng)
    d = np.full(50, 3.5)
    assert np.allclose(precond.olsen_correction(x, r, d, theta), precond.jacobi_correction(r, d, theta),
                       rtol=0, atol=1e-13 * np.abs(r).max())


def test_pcg_zero_steps_is_olsen_and_many_steps_solve_the_projected_equation():
    rng = np.random.default_rng(5)
    H = random_h(40, 11)
    theta, x, r = ritz_pair(H, rng, k=3)
    d = np.diag(H)
    t0, nmv = precond.pcg_correction(lambda v: H @ v, x, r, d, theta, steps=0)
    assert nmv == 0
    assert np.allclose(t0, precond.olsen_correction(x, r, d, theta), rtol=0, atol=1e-12 * np.abs(t0).max())
    # theta above lambda_min makes A indefinite on x-perp only along the true
    # ground state; take theta below the spectrum of the complement instead
    w, U = np.linalg.eigh(H)
    x = U[:, 0] + 1e-3 * U[:, 1]
    x /= np.linalg.norm(x)
    theta = x @ H @ x
    r = H @ x - theta * x
    t, nmv = precond.pcg_correction(lambda v: H @ v, x, r, d, theta, steps=200, rel_tol=1e-13)
    P = np.eye(40) - np.outer(x, x)
    assert abs(x @ t) < 1e-12 * np.linalg.norm(t)
    res = P @ (H - theta * np.eye(40)) @ P @ t + r - (x @ r) * x
    assert np.linalg.norm(res) < 1e-10 * np.linalg.norm(r)
    assert 0 < nmv <= 40


def test_pcg_guard_stops_on_a_negative_curvature_direction():
    # A = P (H - theta) P with theta above the second eigenvalue: a direction
    # of negative curvature exists; the result stays finite and orthogonal to x
    H = np.diag(np.arange(1.0, 31.0))
    x = np.zeros(30)
    x[5] = 1.0
    theta = 6.0
    r = np.zeros(30)
    r[0] = 1e-3
    r[20] = -1e-3
    t, nmv = precond.pcg_correction(lambda v: H @ v, x, r, np.diag(H) + 0.3, theta, steps=10)
    assert np.all(np.isfinite(t)) and abs(x @ t) < 1e-15
    assert nmv >= 1


@pytest.mark.parametrize("kind", ["jacobi", "olsen", "pcg"])
def test_davidson_converges_to_the_lowest_eigenvalue(kind):
    H = random_h(200, 21, spread=2.0)
    d = np.diag(H)
    corr = {"jacobi": None,
            "olsen": lambda x, r, th: precond.olsen_correction(x, r, d, th),
            "pcg": lambda x, r, th: precond.pcg_correction(lambda v: H @ v, x, r, d, th, steps=3)[0]}[kind]
    theta, X = fci.davidson(lambda v: H @ v, d, tol=1e-9, max_iter=300, correction=corr)
    assert abs(theta[0] - np.linalg.eigvalsh(H)[0]) < 1e-10


@pytest.mark.parametrize("kind", ["olsen", "pcg"])
def test_davidson_reaches_the_fci_energy(kind):
    # CAS(6,6): every correction converges to the dense FCI ground state
    h, chol = make_integrals(6, 8, 5)
    eri = fock.eri_from_chol(chol)
    F = fci.FCI(h, eri, 3, 3)
    e_exact = np.linalg.eigvalsh(F.dense_h())[0]
    d = F.diagonal().reshape(-1)
    mv = lambda v: F.sigma(v).reshape(-1)
    corr = (lambda x, r, th: precond.olsen_correction(x, r, d, th)) if kind == "olsen" else \
        (lambda x, r, th: precond.pcg_correction(mv, x, r, d, th, steps=3)[0])
    theta, _ = fci.davidson(mv, d, tol=1e-8, max_iter=200, correction=corr)
    assert abs(theta[0] - e_exact) < 1e-10
