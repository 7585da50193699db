"""Pins of the Fiedler ordering reference: a scrambled path graph, two
weakly coupled clusters, and the invariance of the FCI energy under the
orbital permutation."""
import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import fci, fock, ordering


@pytest.mark.parametrize("n,seed", [(5, 1), (8, 2), (13, 3)])
def test_scrambled_path_is_put_back_in_order(n, seed):
    perm = np.random.default_rng(seed).permutation(n)
    W = np.zeros((n, n))
    for i in range(n - 1):
        W[perm[i], perm[i + 1]] = W[perm[i + 1], perm[i]] = 1.0 + 0.1 * i
    order = ordering.fiedler_order(W)
    want = perm if perm[0] < perm[-1] else perm[::-1]
    assert list(order) == list(want)


def test_weakly_coupled_clusters_are_contiguous():
    rng = np.random.default_rng(4)
    n = 10
    W = rng.uniform(0.0, 0.01, (n, n))
    a = [0, 3, 5, 7, 8]
    b = [1, 2, 4, 6, 9]
    for grp in (a, b):
        for i in grp:
            for j in grp:
                W[i, j] = rng.uniform(0.5, 1.0)
    W = 0.5 * (W + W.T)
    order = list(ordering.fiedler_order(W))
    first = set(order[:5])
    assert first in (set(a), set(b))


def test_errors_and_trivial_sizes():
    assert list(ordering.fiedler_order(np.ones((2, 2)))) == [0, 1]
    W = np.zeros((4, 4))
    W[0, 1] = W[1, 0] = W[2, 3] = W[3, 2] = 1.0       # two components
    with pytest.raises(ValueError):
        ordering.fiedler_order(W)


def test_fci_energy_is_invariant_under_the_permutation():
    h, chol = make_integrals(5, 7, 8)
    order = np.array([3, 0, 4, 1, 2])
    h2, c2 = ordering.permute_integrals(h, chol, order)
    e1 = np.linalg.eigvalsh(fci.FCI(h, fock.eri_from_chol(chol), 3, 2).dense_h())[0]
    e2 = np.linalg.eigvalsh(fci.FCI(h2, fock.eri_from_chol(c2), 3, 2).dense_h())[0]
    assert abs(e1 - e2) < 1e-12
