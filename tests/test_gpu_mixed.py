"""Reduced-precision (tensor-core) sigma and sweeps against the FP64 path and
the oracle: element-wise sigma error per dtype on installed oracle states, and
energies of full solves."""
import json
import os

import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import dmrg

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# relative bounds of ||sigma_tc - sigma_oracle|| / ||sigma_oracle||: BF16 inputs
# 2^-9 rounding, TF32 2^-12, TF32x3 ~2^-21 plus FP32 accumulation
BOUNDS = {1: 3e-3, 2: 2e-2, 3: 2e-5}


@pytest.fixture(scope="module")
def G():
    from paper_2609_09990_gb300 import build, gbdmrg
    build.build()
    return gbdmrg


@pytest.mark.parametrize("n,ne,M,k", [(8, 8, 40, 3), (10, 10, 64, 4), (6, 6, 20, 0)])
def test_tc_sigma_matches_oracle(G, n, ne, M, k):
    h, chol = make_integrals(n, 8, 13)
    d = dmrg.DMRG(h, chol, ne, 0, M, seed=3)
    for j in range(k):
        d.step(j, M, 1e-8, "L")
    ctx = G.Context(0)
    ctx.setup(h, chol, ne, 0, [M], [1e-8], seed=3)
    ns, tr, data = dmrg.canonical_blocks(d)
    ctx.set_mps(ns, tr, data, k)
    keys = dmrg.psi_keys(d.dims[k], d.dims[k + 2])
    N = ctx.two_site_size(k)
    rng = np.random.default_rng(n + k)
    x = rng.standard_normal(N)
    L, W1, W2, R = d.heff_parts(k)
    ref = dmrg.flatten(dmrg.apply_heff(L, W1, W2, R, dmrg.unflatten(x, keys, d.dims[k], d.dims[k + 2]), d.mpo, k),
                       keys, d.dims[k], d.dims[k + 2])
    for prec, bound in BOUNDS.items():
        y = ctx.apply_heff_prec(k, x, prec)
        rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        assert rel < bound, (prec, rel)
    ctx.close()


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_solve_cas6_reaches_fci(G, precision):
    with open(os.path.join(GOLDEN, "fci_cas6_m64_seed1.json")) as f:
        g = json.load(f)
    h, chol = make_integrals(6, 18, 1)
    ctx = G.Context(0)
    r = ctx.solve(h, chol, 6, 0, [64] * 4, [1e-9] * 4, seed=1, precision=precision, fp64_refine=4, rdms=True)
    assert abs(r["energy"] - g["E0"]) < 1e-9
    assert np.abs(r["rdm1"] - np.array(g["rdm1"])).max() < 1e-6
    st = ctx.stats()
    assert st["n_sigma_tc"] > 0
    ctx.close()
