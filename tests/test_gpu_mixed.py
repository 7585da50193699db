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
# 2^-9 rounding, TF32 2^-12, TF32x3 ~2^-21 and BF16x3 ~2^-16 split errors
# plus FP32 accumulation
BOUNDS = {1: 3e-3, 2: 2e-2, 3: 2e-5, 4: 5e-5}


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
    ctx.set_tc_min_two_site(0)   # small problem: force the tensor-core tiers
    r = ctx.solve(h, chol, 6, 0, [64] * 4, [1e-9] * 4, seed=1, precision=precision, fp64_refine=4, rdms=True)
    assert abs(r["energy"] - g["E0"]) < 1e-9
    assert np.abs(r["rdm1"] - np.array(g["rdm1"])).max() < 1e-6
    st = ctx.stats()
    assert st["n_sigma_tc"] > 0
    ctx.close()


def test_tile_shape_does_not_change_sigma(G):
    # the autotuned N cap only regroups columns: the same products are summed
    # in the same order, so sigma is bit-identical for every cap
    h, chol = make_integrals(10, 12, 21)
    ctx = G.Context(0)
    ctx.setup(h, chol, 10, 0, [64], [1e-8], seed=21)
    ctx.init_state()
    for k in range(3):
        ctx.run_step(k, 0, 64, 1e-6)
    x = np.random.default_rng(5).standard_normal(ctx.two_site_size(3))
    for prec in (2, 3, 4):
        ys = []
        for cap in (256, 128, 64):
            ctx.set_tc_tile(cap)
            ys.append(ctx.apply_heff_prec(3, x, prec))
        assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2]), prec
    # nor does the order in which the CTAs take the stage-B tiles
    ctx.set_tc_tile(0)
    for prec in (1, 3):
        ys = []
        for order in (0, 1, 2):
            ctx.set_tc_order(order)
            ys.append(ctx.apply_heff_prec(3, x, prec))
        assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2]), prec
    ctx.set_tc_order(0)
    ctx.close()


def test_graphs_and_autotune_do_not_change_the_solve(G):
    h, chol = make_integrals(8, 10, 22)
    out = []
    for graphs, cap in ((True, 0), (False, 64)):
        ctx = G.Context(0)
        ctx.set_tc_min_two_site(0)   # small problem: force the tensor-core tiers
        ctx.set_graphs(graphs)
        ctx.set_tc_tile(cap)
        r = ctx.solve(h, chol, 8, 0, [48] * 3, [1e-7] * 3, seed=22, precision=2, fp64_refine=0)
        st = ctx.stats()
        assert (st["graph_launches"] > 0) == graphs
        assert (st["autotune_trials"] > 0) == (cap == 0)
        out.append(r)
        ctx.close()
    assert np.array_equal(out[0]["sweep_energies"], out[1]["sweep_energies"])
    assert out[0]["energy"] == out[1]["energy"]


def test_probe_step_isolates_matvec_precision(G):
    # same input state: FP64 Davidson and mixed Davidson refined in FP64 reach
    # the same Rayleigh quotient; the mixed solve alone stays within its floor
    h, chol = make_integrals(10, 12, 23)
    ctx = G.Context(0)
    ctx.set_tc_min_two_site(0)   # small problem: force the tensor-core tiers
    ctx.setup(h, chol, 10, 0, [96], [1e-8], seed=23)
    ctx.init_state()
    for k in range(4):
        ctx.run_step(k, 0, 96, 1e-7)
    th, e_ref, r_ref = ctx.probe_step(4, 0, 0, 1e-9)
    assert r_ref < 1e-8 and abs(th - e_ref) < 1e-12
    _, e_mix, r_mix = ctx.probe_step(4, 2, 50, 1e-9)
    assert r_mix < 1e-8 and abs(e_mix - e_ref) < 1e-11
    _, e_lo, r_lo = ctx.probe_step(4, 2, 0, 1e-9)
    assert e_lo >= e_ref - 1e-12           # Rayleigh quotient: variational
    assert e_lo - e_ref < 1e-6
    ctx.close()
