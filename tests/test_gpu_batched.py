"""Batched solve of independent active spaces: every result equals the one
the single-problem entry point gives, whatever the number of workers;
validation happens before any work; per-problem status."""
import numpy as np
import pytest

from gbd_synth import make_integrals

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
