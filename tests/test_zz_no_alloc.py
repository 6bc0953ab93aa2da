"""The allocation-free propagation entry point (heom_propagate_noalloc).

Callers that cannot allocate device memory when they propagate (a framework's
caching allocator owns the device pool, a real-time loop cannot afford a
synchronising cudaMalloc, a plug-in has buffers but no allocation rights) use
heom_propagate_noalloc, whose RK4 scratch lives in a fixed static device array.
This file checks it against the allocating device entry point,
heom_propagate_dev, on two calls in a row (the second call finds the scratch
holding the first call's data), within the FP64 tolerance of the other parity
tests.  Collected last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2601_20550_gb300.heom")


def test_noalloc_matches_allocating_entry_point():
    torch = pytest.importorskip("torch")
    import os
    if not os.path.exists(H.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    model = W.small_three_mode(n=3, depth_L=2)
    h = H.heom_build_hierarchy(model, H.FP64)
    H.heom_state_create(h, 1, H.FP64)          # any device call sets up the hierarchy tables
    branches = 3
    shape = (branches, h.n_ado, h.d, h.d)
    rng = np.random.default_rng(31)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        ref = torch.from_numpy(x).to(dev)
        wa = torch.empty_like(ref)
        wb = torch.empty_like(ref)
        H.heom_propagate_dev(h, ref.data_ptr(), wa.data_ptr(), wb.data_ptr(), branches, H.FP64,
                             0.5, 5, stream)
        got = torch.from_numpy(x).to(dev)
        H.heom_propagate_noalloc(h, got.data_ptr(), branches, 0.5, 5, stream)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.abs(g - r).max() < 1e-12 * np.abs(r).max(), call


def test_noalloc_rejects_oversize_state():
    torch = pytest.importorskip("torch")
    model, _ = W.config("c2")
    h = H.heom_build_hierarchy(model, H.FP64)
    H.heom_state_create(h, 1, H.FP64)
    per_branch = h.n_ado * h.d * h.d * 16
    branches = (16 * 1024 * 1024) // per_branch + 1
    buf = torch.empty(1, dtype=torch.float64, device="cuda:0")
    with pytest.raises(H.HeomError) as ei:
        H.heom_propagate_noalloc(h, buf.data_ptr(), branches, 0.5, 1, 0)
    assert ei.value.status == -1 and "scratch limit" in str(ei.value)
