"""The allocation-free overlap reduction (gbd_multi_dot_noalloc), for callers
that cannot allocate device memory, against the regular entry point
(gbd_multi_dot) and against a plain torch FP64 product on the same device
buffers, on two calls in a row.

This file is collected last on purpose: it must pass in a fresh process and
after every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(n, k, seed):
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    stride = n + 13
    V = torch.randn(k * stride, dtype=torch.float64, generator=g).cuda()
    x = torch.randn(n, dtype=torch.float64, generator=g).cuda()
    return V, x, stride


def _torch_ref(V, x, stride, k, n):
    return (V.view(k, stride)[:, :n] @ x).cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    from paper_2609_09990_gb300 import build, gbdmrg as G
    build.build()
    ctx = G.Context(0)
    stream = torch.cuda.current_stream()
    for call, (n, k) in enumerate([(152073, 24), (4099, 32)]):
        V, x, stride = _inputs(n, k, 100 + call)
        out = torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        G.multi_dot_noalloc(0, V.data_ptr(), stride, k, x.data_ptr(), n, out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        ref = ctx.multi_dot(V.data_ptr(), stride, k, x.data_ptr(), n)
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
        tref = _torch_ref(V, x, stride, k, n)
        assert np.abs(got - tref).max() <= 1e-12 * max(1.0, np.abs(tref).max())
    # sizes beyond the fixed array are rejected
    with pytest.raises(G.GbdError, match="GBD_ERR_ARG"):
        G.multi_dot_noalloc(0, V.data_ptr(), stride, 33, x.data_ptr(), n, out.data_ptr(), None)
    ctx.close()


def test_noalloc_queued_calls_empty_input_and_no_device_allocation():
    """Two calls queued on one stream with a single synchronisation at the
    end (the documented safe ordering: the second reuses the array after the
    first), n = 0 (zeros), and no change in the device's free memory over
    calls after the first (the first may load the library's device module)."""
    import torch
    from paper_2609_09990_gb300 import build, gbdmrg as G
    build.build()
    stream = torch.cuda.current_stream()
    V1, x1, s1 = _inputs(70001, 17, 7)
    V2, x2, s2 = _inputs(1 << 20, 9, 8)
    o1 = torch.full((17,), float("nan"), dtype=torch.float64, device="cuda")
    o2 = torch.full((9,), float("nan"), dtype=torch.float64, device="cuda")
    o0 = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    G.multi_dot_noalloc(0, V1.data_ptr(), s1, 17, x1.data_ptr(), 70001, o1.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    for _ in range(3):
        G.multi_dot_noalloc(0, V1.data_ptr(), s1, 17, x1.data_ptr(), 70001, o1.data_ptr(), stream.cuda_stream)
        G.multi_dot_noalloc(0, V2.data_ptr(), s2, 9, x2.data_ptr(), 1 << 20, o2.data_ptr(), stream.cuda_stream)
        G.multi_dot_noalloc(0, V1.data_ptr(), s1, 3, x1.data_ptr(), 0, o0.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    assert torch.cuda.mem_get_info(0)[0] == free0
    r1, r2 = _torch_ref(V1, x1, s1, 17, 70001), _torch_ref(V2, x2, s2, 9, 1 << 20)
    assert np.abs(o1.cpu().numpy() - r1).max() <= 1e-12 * max(1.0, np.abs(r1).max())
    assert np.abs(o2.cpu().numpy() - r2).max() <= 1e-12 * max(1.0, np.abs(r2).max())
    assert np.array_equal(o0.cpu().numpy(), np.zeros(3))
