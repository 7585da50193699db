"""The allocation-free overlap reduction (gbd_multi_dot_noalloc), for callers
that cannot allocate device memory, against the regular entry point
(gbd_multi_dot) on the same device buffers, on two calls in a row.

This file is collected last on purpose: it must pass in a fresh process and
after every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    from paper_2609_09990_gb300 import build, gbdmrg as G
    build.build()
    ctx = G.Context(0)
    stream = torch.cuda.current_stream()
    for call, (n, k) in enumerate([(152073, 24), (4099, 32)]):
        g = torch.Generator(device="cpu").manual_seed(100 + call)
        stride = n + 13
        V = torch.randn(k * stride, dtype=torch.float64, generator=g).cuda()
        x = torch.randn(n, dtype=torch.float64, generator=g).cuda()
        out = torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        G.multi_dot_noalloc(0, V.data_ptr(), stride, k, x.data_ptr(), n, out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        ref = ctx.multi_dot(V.data_ptr(), stride, k, x.data_ptr(), n)
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    # sizes beyond the fixed array are rejected
    with pytest.raises(G.GbdError, match="GBD_ERR_ARG"):
        G.multi_dot_noalloc(0, V.data_ptr(), stride, 33, x.data_ptr(), n, out.data_ptr(), None)
    ctx.close()
