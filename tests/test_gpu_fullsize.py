"""Parity at the full size of the CAS(16,16) M=512 workload: the oracle's
state at the central bond pair (7,8) is installed in the library, and
every sigma path the sweeps use is compared with the oracle's FP64 sigma,
element by element, on the same random vector."""
import numpy as np
import pytest

from gbd_synth import WORKLOADS, make_integrals
from oracle import dmrg

pytestmark = pytest.mark.gpu

# relative bounds of ||sigma - sigma_oracle|| / ||sigma_oracle|| (FP64: rounding
# order only; BF16 / TF32 inputs 2^-9 / 2^-12; TF32x3 and BF16x3 split errors
# plus the FP32 accumulation of split-K chunks)
BOUNDS = {0: 1e-12, 1: 1e-3, 2: 8e-3, 3: 1e-5, 4: 2e-5}


@pytest.fixture(scope="module")
def G():
    from paper_2609_09990_gb300 import build, gbdmrg
    build.build()
    return gbdmrg


@pytest.fixture(scope="module")
def central(G):
    wl = WORKLOADS["cas16_m512"]
    n, ne, nq, M, seed = wl["n_orb"], wl["n_elec"], wl["n_chol"], wl["M"], wl["seed"]
    h, chol = make_integrals(n, nq, seed)
    k = n // 2 - 1
    d = dmrg.DMRG(h, chol, ne, 0, M, seed=seed, k_switch=3, renv_down_to=k + 2)
    d.move_center(k)
    keys = dmrg.psi_keys(d.dims[k], d.dims[k + 2])
    ctx = G.Context(0)
    ctx.setup(h, chol, ne, 0, [M], [1e-8], seed=seed)
    ns, tr, data = dmrg.canonical_blocks(d)
    ctx.set_mps(ns, tr, data, k)
    N = ctx.two_site_size(k)
    x = np.random.default_rng(11).standard_normal(N)
    L, W1, W2, R = d.heff_parts(k)
    ref = dmrg.flatten(dmrg.apply_heff(L, W1, W2, R, dmrg.unflatten(x, keys, d.dims[k], d.dims[k + 2]), d.mpo, k),
                       keys, d.dims[k], d.dims[k + 2])
    yield ctx, k, x, ref
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4])
def test_central_sigma_matches_oracle(G, central, prec):
    ctx, k, x, ref = central
    y = ctx.apply_heff(k, x) if prec == 0 else ctx.apply_heff_prec(k, x, prec)
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert rel < BOUNDS[prec], (prec, rel)
    # element by element against the same scale
    assert np.abs(y - ref).max() <= max(10 * BOUNDS[prec], 1e-12) * np.abs(ref).max()
