"""Parity of the CUDA sweep engine (through the C ABI) with the CPU oracle.

FP64 path: H_eff application and environments agree to 1e-12 relative on
identical inputs; a two-site step (Davidson + decimation) agrees in energy
and kept weights; full solves agree with the oracle and with FCI."""
import json
import os

import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import dmrg, fock
from tests.gpu_helpers import export_mps, label_keys

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def G():
    from paper_2609_09990_gb300 import build, gbdmrg
    build.build()
    return gbdmrg


def oracle_state(n, ne, nq, seed, M, steps):
    h, chol = make_integrals(n, nq, seed)
    d = dmrg.DMRG(h, chol, ne, 0, M, seed=seed)
    for (k, dr) in steps:
        d.step(k, M, 1e-10, dr)
    return h, chol, d


@pytest.mark.parametrize("n,ne,nq,seed,M,k", [(6, 6, 18, 1, 20, 2), (6, 6, 18, 1, 64, 0), (8, 8, 10, 3, 30, 3),
                                             (5, 4, 6, 2, 12, 3)])
def test_heff_and_envs_match_oracle(G, n, ne, nq, seed, M, k):
    steps = [(j, "L") for j in range(k)]
    h, chol, d = oracle_state(n, ne, nq, seed, M, steps)
    ctx = G.Context(0)
    ctx.setup(h, chol, ne, 0, [M], [1e-10], seed=seed)
    ns, tr, data = export_mps(d)
    ctx.set_mps(ns, tr, data, k)
    # environments, channel by channel and sector by sector
    for side, bond in [(0, k), (1, k + 2)]:
        keys = list(ctx.mpo_labels(bond))
        assert keys == label_keys(d.mpo, bond)
        env = d.Lenv[bond] if side == 0 else d.Renv[bond]
        secs = sorted(d.dims[bond])
        for a in range(len(keys)):
            for si, q in enumerate(secs):
                got = ctx.env_block(side, bond, a, si)
                ref = env[a].get(q) if a < len(env) else None
                if got.size == 0:   # structurally absent block: the oracle has none either
                    assert ref is None or np.abs(ref).max() == 0
                    continue
                if ref is None:
                    ref = np.zeros_like(got)
                assert got.shape == ref.shape
                assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    # H_eff on random vectors and its diagonal
    keys2 = dmrg.psi_keys(d.dims[k], d.dims[k + 2])
    N = ctx.two_site_size(k)
    rng = np.random.default_rng(k)
    L, W1, W2, R = d.heff_parts(k)
    for _ in range(2):
        x = rng.standard_normal(N)
        y, dg = ctx.apply_heff(k, x, want_diag=True)
        ref = dmrg.flatten(dmrg.apply_heff(L, W1, W2, R, dmrg.unflatten(x, keys2, d.dims[k], d.dims[k + 2]),
                                           d.mpo, k), keys2, d.dims[k], d.dims[k + 2])
        assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
        dref = dmrg.flatten(dmrg.heff_diag(L, W1, W2, R, keys2, d.mpo, k, d.dims[k], d.dims[k + 2]),
                            keys2, d.dims[k], d.dims[k + 2])
        assert np.abs(dg - dref).max() <= 1e-12 * max(1.0, np.abs(dref).max())
    ctx.close()


def test_heff_hermitian_on_device(G):
    h, chol, d = oracle_state(6, 6, 18, 1, 20, [(0, "L"), (1, "L")])
    ctx = G.Context(0)
    ctx.setup(h, chol, 6, 0, [20], [1e-10], seed=1)
    ns, tr, data = export_mps(d)
    ctx.set_mps(ns, tr, data, 2)
    N = ctx.two_site_size(2)
    H = np.array([ctx.apply_heff(2, e) for e in np.eye(N)]).T
    assert np.abs(H - H.T).max() <= 1e-13 * np.abs(H).max()
    ctx.close()


@pytest.mark.parametrize("direction", ["L", "R"])
def test_two_site_step_matches_oracle(G, direction):
    n, ne, nq, seed, M = 8, 8, 10, 3, 24
    k = 3
    h, chol, d = oracle_state(n, ne, nq, seed, M, [(j, "L") for j in range(k)])
    ctx = G.Context(0)
    ctx.setup(h, chol, ne, 0, [M], [1e-11], seed=seed)
    ns, tr, data = export_mps(d)
    ctx.set_mps(ns, tr, data, k)
    e_lib, tau_lib, kept_lib = ctx.run_step(k, 0 if direction == "L" else 1, M, 1e-11)
    e_ref, tau_ref, kept_ref = d.step(k, M, 1e-11, direction)
    assert abs(e_lib - e_ref) < 1e-10
    assert len(kept_lib) == len(kept_ref)
    assert np.abs(np.array(kept_lib) - np.array(kept_ref)).max() < 1e-9
    assert abs(tau_lib - tau_ref) < 1e-9
    ctx.close()


def test_solve_cas6_full_bond_equals_fci_and_oracle(G):
    with open(os.path.join(GOLDEN, "fci_cas6_m64_seed1.json")) as f:
        g = json.load(f)
    h, chol = make_integrals(6, 18, 1)
    ctx = G.Context(0)
    r = ctx.solve(h, chol, 6, 0, [64] * 4, [1e-9] * 4, seed=1)
    assert abs(r["energy"] - g["E0"]) < 1e-10
    d, sw = dmrg.run(h, chol, 6, 0, [64] * 4, [1e-9] * 4, seed=1)
    assert np.abs(r["sweep_energies"] - np.array(sw)).max() < 1e-9
    ctx.close()


def test_solve_truncated_matches_oracle_sweeps(G):
    # M=8 < full bond: the truncation path, same schedule on both sides
    h, chol = make_integrals(6, 18, 1)
    ctx = G.Context(0)
    r = ctx.solve(h, chol, 6, 0, [8, 8, 8], [1e-10] * 3, seed=4)
    d, sw = dmrg.run(h, chol, 6, 0, [8, 8, 8], [1e-10] * 3, seed=4)
    assert np.abs(r["sweep_energies"] - np.array(sw)).max() < 1e-9
    assert abs(r["energy"] - d.energy()) < 1e-9
    ctx.close()


@pytest.mark.parametrize("n,ne,two_sz,M", [(2, 2, 0, 4), (3, 1, 1, 8), (4, 0, 0, 4), (4, 8, 0, 4), (5, 5, -1, 16),
                                           (6, 6, 0, 1), (6, 7, 1, 3)])
def test_edge_cases_match_oracle(G, n, ne, two_sz, M):
    h, chol = make_integrals(n, 4, 9)
    ctx = G.Context(0)
    r = ctx.solve(h, chol, ne, two_sz, [M, M], [1e-10, 1e-10], seed=2)
    d, sw = dmrg.run(h, chol, ne, two_sz, [M, M], [1e-10, 1e-10], seed=2)
    assert abs(r["energy"] - d.energy()) < 1e-9
    ctx.close()


def test_invalid_inputs_are_rejected(G):
    h, chol = make_integrals(4, 4, 1)
    ctx = G.Context(0)
    bad_h = h.copy()
    bad_h[0, 1] += 1e-6
    for kw, args in [({}, (bad_h, chol, 4, 0)), ({}, (h, chol, 9, 0)), ({}, (h, chol, 4, 1)),
                     ({}, (h, chol, 3, 5)), ({"precision": 7}, (h, chol, 4, 0)), ({"fp64_refine": -1}, (h, chol, 4, 0))]:
        with pytest.raises(G.GbdError, match="GBD_ERR_ARG"):
            ctx.solve(*args, [4], [1e-8], **kw)
    nan_h = h.copy()
    nan_h[1, 1] = np.nan
    with pytest.raises(G.GbdError, match="GBD_ERR_ARG"):
        ctx.solve(nan_h, chol, 4, 0, [4], [1e-8])
    with pytest.raises(G.GbdError, match="GBD_ERR_STATE"):
        G.Context(0).run_sweep(0)
    ctx.close()


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _solve_like(G, g, **setup):
    h, chol = make_integrals(g["n_orb"], g["n_chol"], g["seed"])
    ctx = G.Context(0)
    for k, v in setup.items():
        getattr(ctx, k)(*v)
    r = ctx.solve(h, chol, g["n_elec"], g["two_sz"], [g["M"]] * g["sweeps"], [g["tol"]] * g["sweeps"],
                  seed=g["seed"])
    bonds = [ctx.get_bond(b) for b in range(g["n_orb"] + 1)]
    ctx.close()
    return r, bonds


@pytest.mark.parametrize("name", ["dmrg_cas8_m48_adaptive1e-6.json", "dmrg_cas8_m48_adaptive1e-4.json"])
def test_adaptive_bond_dim_solve_matches_oracle(G, name):
    # per-bond adaptive bond dimension in a GPU solve (cap M = 48) against
    # the oracle's run with the same discarded-weight target (stored by
    # tests/golden/make_golden.py --dmrg): kept sector dimensions of every
    # bond bit for bit, sweep energies to 1e-9 Ha
    g = _golden(name)
    r, bonds = _solve_like(G, g, set_adaptive_bond_dim=(g["max_discarded"], g["m_min"]))
    assert np.abs(r["sweep_energies"] - np.array(g["sweep_energies"])).max() < 1e-9
    assert abs(r["energy"] - g["energy"]) < 1e-9
    for b, ref in enumerate(g["bonds"]):
        assert np.array_equal(bonds[b], np.array(ref, dtype=np.int32).reshape(-1, 3)), b


def test_fp64_sweeps_cas10_m96_match_oracle(G):
    # two FP64 sweeps of CAS(10,10) at M = 96: multi-sector tiles and both
    # FP64 GEMM kernels (register-blocked and flat), against the oracle run
    g = _golden("dmrg_cas10_m96_seed7.json")
    r, bonds = _solve_like(G, g)
    assert np.abs(r["sweep_energies"] - np.array(g["sweep_energies"])).max() < 1e-9
    assert abs(r["energy"] - g["energy"]) < 1e-9
    for b, ref in enumerate(g["bonds"]):
        assert np.array_equal(bonds[b], np.array(ref, dtype=np.int32).reshape(-1, 3)), b
