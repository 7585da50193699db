"""Davidson vector reduction through the C ABI against a plain PyTorch FP64
reference (device buffers from torch)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,k", [(1, 1), (1000, 3), (152073, 24), (3_000_001, 5)])
def test_multi_dot_matches_torch(n, k):
    import torch
    from paper_2609_09990_gb300 import build, gbdmrg as G
    build.build()
    g = torch.Generator(device="cpu").manual_seed(n + k)
    stride = n + 7
    V = torch.randn(k * stride, dtype=torch.float64, generator=g).cuda()
    x = torch.randn(n, dtype=torch.float64, generator=g).cuda()
    ctx = G.Context(0)
    out = ctx.multi_dot(V.data_ptr(), stride, k, x.data_ptr(), n)
    ref = torch.stack([V[j * stride:j * stride + n] @ x for j in range(k)]).cpu().numpy()
    assert np.abs(out - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()) * np.sqrt(n)
    ctx.close()
