"""Environment updates that compute one channel of each certified
Hermitian-conjugate pair and transpose it into the other
(gbd_set_env_conjugates): every environment block equals the one computed
channel by channel, a derived block is its partner's transpose times the
pair's sign bit for bit, and a whole solve gives the same energy with about
half the environment flops."""
import numpy as np
import pytest

from gbd_synth import make_integrals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2609_09990_gb300 import build, gbdmrg
    build.build()
    return gbdmrg


def blocks(ctx, n, bond, side):
    out = {}
    for c in range(len(ctx.mpo_labels(bond))):
        q = 0
        while True:
            try:
                b = ctx.env_block(side, bond, c, q)
            except Exception:
                break
            out[(c, q)] = b
            q += 1
    return out


def check_derived(ctx, bond, side, a):
    # a derived block is its partner's block, transposed, times the sign,
    # bit for bit
    part, sg = ctx.env_conjugates(side, bond)
    for (d, q), blk in a.items():
        c = part[d]
        if c < 0 or c == d or blk.size == 0:
            continue
        assert any(c2 == c and v.shape == blk.shape[::-1] and np.array_equal(sg[c] * v.T, blk)
                   for (c2, q2), v in a.items()), (bond, side, c, d, q)


def test_env_blocks_with_and_without_conjugates(G):
    # one installed oracle MPS (centre at bond 5) in two contexts: the
    # environments that gbd_set_mps builds from it agree block by block
    from oracle import dmrg
    n, ne, M, k = 10, 10, 48, 5
    h, chol = make_integrals(n, 20, 6)
    d = dmrg.DMRG(h, chol, ne, 0, M, seed=6)
    for j in range(k):
        d.step(j, M, 1e-9, "L")
    ns, tr, data = dmrg.canonical_blocks(d)
    ctxs = []
    for conj in (1, 0):
        ctx = G.Context(0)
        ctx.set_env_conjugates(conj)
        ctx.setup(h, chol, ne, 0, [M], [1e-9], seed=6)
        ctx.set_mps(ns, tr, data, k)
        ctxs.append(ctx)
    on, off = ctxs
    for bond, side in [(b, 0) for b in range(1, k + 1)] + [(b, 1) for b in range(k + 2, n)]:
        a, b = blocks(on, n, bond, side), blocks(off, n, bond, side)
        assert a.keys() == b.keys()
        scale = max(1.0, max(np.abs(v).max() for v in b.values() if v.size))
        for key in a:
            assert a[key].shape == b[key].shape
            if a[key].size:
                assert np.abs(a[key] - b[key]).max() <= 1e-13 * scale, (bond, side, key)
        check_derived(on, bond, side, a)
    for ctx in ctxs:
        ctx.close()


def test_tensor_core_env_derived_blocks_are_exact_transposes(G):
    # environment updates on the tensor cores (TF32x3) inside mixed-precision
    # steps: the derived channels are exact transposes, so the environments
    # of a Hermitian-conjugate pair are conjugate to the last bit
    n, ne, M = 10, 10, 48
    h, chol = make_integrals(n, 20, 6)
    ctx = G.Context(0)
    ctx.set_env_precision(3)
    ctx.setup(h, chol, ne, 0, [M] * 2, [1e-6] * 2, seed=6, precision=G.GBD_BF16)
    ctx.init_state()
    for k in range(5):
        ctx.run_step(k, 0, M, 1e-6)
    for bond in range(1, 6):
        check_derived(ctx, bond, 0, blocks(ctx, n, bond, 0))
    ctx.close()


def test_solve_same_energy_half_the_env_flops(G):
    n, ne = 12, 12
    h, chol = make_integrals(n, 36, 2)
    res = []
    for conj in (1, 0):
        ctx = G.Context(0)
        ctx.set_env_conjugates(conj)
        r = ctx.solve(h, chol, ne, 0, [128] * 2, [1e-8] * 2, seed=2)
        res.append((r["energy"], ctx.stats()["env_flops"]))
        ctx.close()
    (e_on, f_on), (e_off, f_off) = res
    assert abs(e_on - e_off) < 1e-10
    assert f_on < 0.6 * f_off
