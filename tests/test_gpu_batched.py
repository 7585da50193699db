"""Batched solve of independent active spaces: every result equals the one
the single-problem entry point gives, whatever the number of workers, and
the oracle's (FCI where the bond dimension is exact, the oracle's DMRG run
at the same bond dimension otherwise); validation happens before any work;
per-problem status."""
import json
import os

import numpy as np
import pytest

from gbd_synth import make_integrals
from oracle import fock

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2609_09990_gb300 import build, gbdmrg
    build.build()
    return gbdmrg


# (n_orb, n_chol, seed, M, sweeps)
CASES = [(6, 8, 11, 32, 2), (4, 6, 12, 16, 3), (8, 10, 13, 48, 2), (5, 7, 14, 24, 2), (7, 9, 15, 40, 2)]


def problems(cases=CASES):
    out = []
    for n, nq, seed, M, ns in cases:
        h, chol = make_integrals(n, nq, seed)
        # half filling; odd electron counts take S_z = 1/2
        out.append((h, chol, n, n % 2, [M] * ns, [1e-8] * ns, {"seed": seed}))
    return out


def test_batched_equals_single_solves(G):
    ps = problems()
    single = []
    for h, chol, ne, sz, bd, tl, kw in ps:
        ctx = G.Context(0)
        single.append(ctx.solve(h, chol, ne, sz, bd, tl, rdms=True, **kw))
        ctx.close()
    for workers in (1, 3, 0):
        ctx = G.Context(0)
        rc, res = ctx.solve_batched(ps, rdms=True, workers=workers)
        ctx.close()
        assert rc == 0
        for a, b in zip(res, single):
            assert a["status"] == 0
            # same kernels, same order of arithmetic: identical numbers
            assert a["energy"] == b["energy"]
            assert np.array_equal(a["sweep_energies"], b["sweep_energies"])
            assert np.array_equal(a["rdm1"], b["rdm1"])
            assert a["n_matvec"] == b["n_matvec"]


def test_batched_energies_match_oracle(G):
    # CASES[1] (n = 4, M = 16) and CASES[3] (n = 5, M = 24) keep every state
    # of every bond: FCI.  The others are truncated: the oracle's DMRG run
    # with the same seed, M and schedule (tests/golden/make_golden.py --dmrg).
    ps = problems()
    ctx = G.Context(0)
    rc, res = ctx.solve_batched(ps, workers=0)
    ctx.close()
    assert rc == 0
    for i in (1, 3):
        h, chol, ne, sz = ps[i][:4]
        w, _, _ = fock.ground_state(h, fock.eri_from_chol(chol), (ne + sz) // 2, (ne - sz) // 2)
        assert abs(res[i]["energy"] - w[0]) < 1e-9, i
    for i, name in ((0, "dmrg_batch_n6_seed11.json"), (2, "dmrg_batch_n8_seed13.json"),
                    (4, "dmrg_batch_n7_seed15.json")):
        with open(os.path.join(GOLDEN, name)) as f:
            g = json.load(f)
        assert (g["n_orb"], g["n_chol"], g["seed"], g["M"], g["sweeps"]) == CASES[i]
        assert np.abs(res[i]["sweep_energies"] - np.array(g["sweep_energies"])).max() < 1e-9, i
        assert abs(res[i]["energy"] - g["energy"]) < 1e-9, i


def test_batched_validates_everything_first(G):
    ps = problems()
    h = ps[2][0].copy()
    h[0, 1] += 1e-3                      # not symmetric
    ps[2] = (h,) + ps[2][1:]
    ctx = G.Context(0)
    rc, res = ctx.solve_batched(ps, check=False)
    assert rc == G.GBD_ERR_ARG
    assert "problem 2" in ctx.last_error()
    # nothing ran, no result was touched
    assert all(r["status"] == 0 and r["energy"] == 0.0 and r["n_matvec"] == 0 for r in res)
    ctx.close()


def test_batched_empty_and_learned_without_weights(G):
    ctx = G.Context(0)
    rc, res = ctx.solve_batched([])
    assert rc == 0 and res == []
    ps = problems(CASES[:2])
    ps[1] = ps[1][:6] + ({"seed": 12, "preconditioner": 1},)
    rc, _ = ctx.solve_batched(ps, check=False)
    assert rc == G.GBD_ERR_STATE
    ctx.close()
