"""The decimation's host eigensolver (Householder tridiagonalisation on the
lower triangle, implicit QL; no GPU) against numpy's LAPACK eigensolver on
spectra like those of the reduced density matrices: random positive
semi-definite, exponentially decaying weights, exactly degenerate pairs, a
large cluster of tiny weights, and rank-deficient psi psi^T; sizes on both
sides of the threshold where its loops run in parallel blocks."""
import numpy as np
import pytest

from paper_2609_09990_gb300 import gbdmrg as G


def spectra(n, rng):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.exp(-np.arange(n) / 6.0)
    lam /= lam.sum()
    tiny = lam.copy()
    tiny[min(10, n):] = 1e-13 * (1 + 1e-6 * np.arange(n - min(10, n)))
    X = rng.standard_normal((n, n))
    Y = rng.standard_normal((n, max(1, n // 3)))
    return {
        "random": X @ X.T,
        "decaying": (Q * lam) @ Q.T,
        "pairs": (Q * np.repeat(lam[: (n + 1) // 2], 2)[:n]) @ Q.T,
        "tiny cluster": (Q * tiny) @ Q.T,
        "rank deficient": Y @ Y.T,
    }


@pytest.mark.parametrize("n", [1, 2, 3, 7, 40, 150, 300])
def test_host_eigensolver(n):
    rng = np.random.default_rng(n)
    for name, A in spectra(n, rng).items():
        A = 0.5 * (A + A.T)
        nA = np.abs(A).sum(1).max()
        w, Z = G.host_sym_eig(A)
        assert np.all(np.diff(w) >= 0), name
        assert np.abs(w - np.linalg.eigvalsh(A)).max() <= 1e-13 * nA, name
        assert np.abs(A @ Z - Z * w).max() <= 1e-13 * nA, name
        assert np.abs(Z.T @ Z - np.eye(n)).max() <= 1e-12, name


def test_host_eigensolver_vectors_match_lapack_on_separated_eigenvalues():
    rng = np.random.default_rng(9)
    n = 120
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(1.0, 2.0, n) ** 3
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    w, Z = G.host_sym_eig(A)
    wr, Zr = np.linalg.eigh(A)
    assert np.abs(w - wr).max() <= 1e-13 * lam.max()
    assert np.abs(np.abs(np.sum(Z * Zr, axis=0)) - 1).max() <= 1e-10
