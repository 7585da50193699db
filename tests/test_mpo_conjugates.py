"""The library's certified Hermitian-conjugate channel pairs (host code, no
GPU) against the oracle's MPO: for every pair (c, d, sign) the block
operators that the oracle's W tensors build for the two channels satisfy
O[d] = sign O[c]^T exactly, on the left blocks (sites before the bond) and
the right blocks (sites after it).  The library's channels have the oracle's
labels in the oracle's order (checked on the GPU by
test_gpu_parity.py::test_heff_and_envs_match_oracle), so channel indices
agree.  These block operators are the environments of the identity MPS: an
environment update that fills one channel of a pair with the other's
transpose is exact for every MPS exactly when this holds for every
product-basis state."""
import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import fock, mpo


def left_blocks(M):
    out = [{0: np.ones((1, 1))}]
    for i in range(M.n):
        new = {}
        for (a, b), w in M.W[i].items():
            if a in out[-1]:
                new[b] = new.get(b, 0.0) + np.kron(out[-1][a], w)
        out.append(new)
    return out


def right_blocks(M):
    n = M.n
    out = [None] * (n + 1)
    out[n] = {0: np.ones((1, 1))}
    for i in range(n - 1, -1, -1):
        new = {}
        for (a, b), w in M.W[i].items():
            if b in out[i + 1]:
                new[a] = new.get(a, 0.0) + np.kron(w, out[i + 1][b])
        out[i] = new
    return out


@pytest.mark.parametrize("n,nq,seed,ks", [(3, 4, 2, None), (4, 5, 7, None), (4, 5, 7, 0), (5, 6, 3, None),
                                          (5, 6, 3, 4)])
def test_certified_pairs_are_transposes(n, nq, seed, ks):
    from paper_2609_09990_gb300 import gbdmrg as G
    h, chol = make_integrals(n, nq, seed)
    M = mpo.MPO(h, fock.eri_from_chol(chol), k_switch=ks)
    for side, blocks in ((0, left_blocks(M)), (1, right_blocks(M))):
        npairs = 0
        for b in range(n + 1):
            part, sg = G.host_mpo_conjugates(h, chol, side, b, k_switch=ks)
            assert len(part) == len(M.labels[b])
            for c, d in enumerate(part):
                if d < 0:
                    continue
                assert part[d] == c and sg[d] == sg[c]
                zero = lambda x: np.zeros((4 ** (b if side == 0 else n - b),) * 2)
                Oc = blocks[b].get(c, zero(c))
                Od = blocks[b].get(d, zero(d))
                assert np.abs(Od - sg[c] * Oc.T).max() <= 1e-12 * max(1.0, np.abs(Oc).max()), (side, b, c, d)
                npairs += d != c
        # most channels have a partner other than themselves (at the central
        # bonds of the k_switch = n/2 MPO about 95 %)
        total = sum(len(M.labels[b]) for b in range(n + 1))
        assert npairs >= 0.5 * total


def test_certification_refuses_asymmetric_integrals():
    # an h with h_pq != h_qp: the one-body complementary channels lose their
    # partners, and no pair the library still certifies is wrong
    from paper_2609_09990_gb300 import gbdmrg as G
    n = 4
    h, chol = make_integrals(n, 5, 7)
    h = h.copy()
    h[0, 2] += 1e-3
    M = mpo.MPO(h, fock.eri_from_chol(chol))
    L = left_blocks(M)
    lost = 0
    for b in range(n + 1):
        part, sg = G.host_mpo_conjugates(h, chol, 0, b)
        lost += int(np.sum(part < 0))
        for c, d in enumerate(part):
            if d >= 0 and c in L[b] and d in L[b]:
                assert np.abs(L[b][d] - sg[c] * L[b][c].T).max() <= 1e-12
    assert lost > 0
