"""Environment updates on the tensor cores (gbd_set_env_precision): the
left and right environments after a two-site step equal those of the FP64
update within the TF32x3 / BF16x3 error (same Davidson result, only the
update differs).  A whole reduced-precision solve with tensor-core
environment updates reports a genuine energy (evaluated with FP64
environments, and equal to the one its RDMs give) that is not above the FP64
solve's by more than the metric's 1e-6 Ha.  (Its sweeps may settle in
another fixed point of fixed-M DMRG: at CAS(12,12) M=256 after 4 sweeps it
ends 9e-5 Ha below the FP64 run.)"""
import numpy as np
import pytest

from gbd_synth import WORKLOADS, make_integrals
from oracle import dmrg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2609_09990_gb300 import build, gbdmrg
    build.build()
    return gbdmrg


def _step_envs(G, env_prec, direction):
    n, ne, nq, seed, M, k = 8, 8, 10, 3, 40, 3
    h, chol = make_integrals(n, nq, seed)
    d = dmrg.DMRG(h, chol, ne, 0, M, seed=seed)
    for j in range(k):
        d.step(j, M, 1e-10, "L")
    ctx = G.Context(0)
    ctx.set_tc_min_two_site(0)
    ctx.setup(h, chol, ne, 0, [M], [1e-8], seed=seed, precision=G.GBD_BF16, fp64_refine=0)
    ctx.set_env_precision(env_prec)
    ns, tr, data = dmrg.canonical_blocks(d)
    ctx.set_mps(ns, tr, data, k)
    ctx.run_step(k, direction, M, 1e-8)
    side, bond = (0, k + 1) if direction == 0 else (1, k + 1)
    blocks = {}
    for a in range(len(ctx.mpo_labels(bond))):
        for si in range(len(ctx.get_bond(bond))):
            b = ctx.env_block(side, bond, a, si)
            if b.size:
                blocks[(a, si)] = b
    ctx.close()
    return blocks


@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("env_prec,bound", [(3, 2e-5), (4, 2e-4)])
def test_tensor_core_env_update_matches_fp64(G, direction, env_prec, bound):
    ref = _step_envs(G, 0, direction)
    got = _step_envs(G, env_prec, direction)
    assert ref.keys() == got.keys()
    scale = max(np.abs(b).max() for b in ref.values())
    err = max(np.abs(got[key] - ref[key]).max() for key in ref)
    assert err <= bound * scale, err / scale


def test_whole_solve_with_tensor_core_envs_cas12(G):
    wl = WORKLOADS["cas12_m256"]
    n, ne, nq, M, seed = wl["n_orb"], wl["n_elec"], wl["n_chol"], wl["M"], wl["seed"]
    h, chol = make_integrals(n, nq, seed)
    out = {}
    for name, prec, env in (("fp64", G.GBD_FP64, 0), ("mixed", G.GBD_BF16, 0), ("mixed_tc_env", G.GBD_BF16, 3)):
        ctx = G.Context(0)
        ctx.set_env_precision(env)
        out[name] = ctx.solve(h, chol, ne, 0, [M] * 4, [1e-6] * 4, seed=seed, precision=prec, fp64_refine=0,
                              rdms=True)
        ctx.close()
    a, c = out["mixed_tc_env"], out["fp64"]
    eri = np.einsum("Qpq,Qrs->pqrs", chol, chol)
    for r in out.values():
        # the reported energy is <psi|H|psi> of the final MPS: the RDMs (from
        # its determinant expansion, no environments) give the same number
        e_rdm = np.einsum("pq,pq->", h, r["rdm1"]) + 0.5 * np.einsum("pqrs,pqrs->", eri, r["rdm2"])
        assert abs(r["energy"] - e_rdm) <= 1e-9, (r["energy"], e_rdm)
    assert a["energy"] <= c["energy"] + 1e-6, (a["energy"], c["energy"])


@pytest.mark.parametrize("M,N,K,nterms", [(30, 20, 50, 3), (300, 200, 700, 2), (129, 257, 1100, 1), (7, 133, 8, 4)])
@pytest.mark.parametrize("flags", [0, 1, 2, 3])
@pytest.mark.parametrize("prec,bound", [(3, 1e-5), (4, 2e-4)])
def test_tensor_core_gemm_plan_matches_fp64(G, M, N, K, nterms, flags, prec, bound):
    # the executor of the tensor-core environment updates on shapes with
    # several 128 x 128 tiles, K split into 512-wide pieces and chunks,
    # transposed operands, signs and a folded scale
    ctx = G.Context(0)
    err, ref = ctx.gemm_tc_selftest(M, N, K, nterms, flags, prec, seed=M + N + K + flags)
    ctx.close()
    assert ref > 0
    assert err <= bound * ref, err / ref
