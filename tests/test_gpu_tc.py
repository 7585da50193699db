"""Tensor-core grouped GEMM (tcgen05 + TMA) against an FP64 product of the
same operands: BF16 and TF32 inputs are compared as stored (error = FP32
accumulation only), TF32x3 against the FP64 originals."""
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(128, 16, 16, 1), (200, 48, 40, 3), (300, 256, 128, 5), (77, 8, 7, 2), (513, 300, 200, 4),
          (128, 144, 64, 9)]


@pytest.fixture(scope="module")
def G():
    from paper_2609_09990_gb300 import build, gbdmrg
    build.build()
    return gbdmrg


# Bounds from the FP32 accumulation of the tensor cores (measured ~2e-6 of
# max|C| at K*terms = 800 for BF16/TF32 as stored) plus, for TF32x3 and
# BF16x3 (prec 3), the split representation error (2^-21, 2^-16) against
# the FP64 originals.
@pytest.mark.parametrize("prec,rel", [(0, 5e-6), (1, 6e-6), (2, 2e-5), (3, 2e-5)])
@pytest.mark.parametrize("shape", SHAPES)
def test_tc_grouped_gemm(G, prec, rel, shape):
    M, N, K, nt = shape
    err, ref = G.tc_selftest(prec, M, N, K, nt, seed=M * 7 + N)
    # scale: max |C|, at least the typical size sqrt(K * nt) of a sum of
    # K * nt products of standard normal entries
    scale = max(ref, (K * nt) ** 0.5)
    assert err <= rel * scale, (err, ref)
