"""Error statuses produced on purpose, without faulting or hanging the GPU.

  * HEOM_ETIMEOUT: the tensor-core stage kernel's waits are bounded in time.  With
    the limit cut to 1 ns a wait runs out at once; the kernel drains the
    tensor-core work it has committed, frees its tensor memory and returns, and
    heom_propagate reports HEOM_ETIMEOUT.  The context stays usable: with the
    default limit the same hierarchy propagates correctly afterwards.
  * HEOM_ENOMEM: the library's device allocations go through one allocator with a
    host-side failure injection (heom_debug_fail_alloc); the entry points that
    need memory report HEOM_ENOMEM and leave the caller's state untouched.
  * HEOM_ENONFINITE: an equilibrium state holding a NaN carries it through the kicks,
    the propagation and the traces; the response is checked on the host before the
    call returns.
"""
import numpy as np
import pytest

import workloads as W
from oracle import heom as OH
from oracle import model as OM

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2601_20550_gb300.heom")


@pytest.fixture(scope="module", autouse=True)
def built():
    import os
    if not os.path.exists(H.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()


def rand_state(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_tensor_core_wait_limit_reports_timeout_and_recovers():
    model = W.small_three_mode(n=3, depth_L=2)
    prob = OM.Problem(model)
    h = H.heom_build_hierarchy(model, H.TC)
    x = rand_state((3, prob.nado, prob.d, prob.d), 41)
    s = H.heom_state_create(h, 3, H.TC)
    H.heom_state_upload(s, x)
    H.heom_set_wait_limit_ns(h, 1)
    with pytest.raises(H.HeomError) as ei:
        H.heom_propagate(h, s, 0.5, 2)
    assert ei.value.status == -5, str(ei.value)
    # the default limit again: the same hierarchy and context work
    H.heom_set_wait_limit_ns(h, 2_000_000_000)
    H.heom_state_upload(s, x)
    H.heom_propagate(h, s, 0.5, 4)
    assert rel(H.heom_state_download(s), OH.propagate(prob, x, 0.5, 4)) < 2e-5
    with pytest.raises(H.HeomError) as ei:
        H.heom_set_wait_limit_ns(h, 0)
    assert ei.value.status == -1


def test_allocation_failure_reports_enomem_and_recovers():
    model = W.small_two_mode(n1=3, n2=3, depth_L=2)
    prob = OM.Problem(model)
    h = H.heom_build_hierarchy(model, H.FP64)
    x = rand_state((2, prob.nado, prob.d, prob.d), 42)
    s = H.heom_state_create(h, 2, H.FP64)
    H.heom_state_upload(s, x)
    try:
        for after in (0, 1):   # heom_propagate takes two scratch buffers
            H.heom_debug_fail_alloc(after)
            with pytest.raises(H.HeomError) as ei:
                H.heom_propagate(h, s, 0.5, 3)
            assert ei.value.status == -2, str(ei.value)
        H.heom_debug_fail_alloc(0)
        with pytest.raises(H.HeomError) as ei:
            H.heom_state_create(h, 1, H.FP64)
        assert ei.value.status == -2
        # a hierarchy whose device set-up fails part-way can be set up later
        h2 = H.heom_build_hierarchy(model, H.FP64)
        H.heom_debug_fail_alloc(3)
        with pytest.raises(H.HeomError) as ei:
            H.heom_state_create(h2, 1, H.FP64)
        assert ei.value.status == -2
    finally:
        H.heom_debug_fail_alloc(-1)
    # the failed calls left the state as it was
    assert np.array_equal(H.heom_state_download(s), x)
    H.heom_propagate(h, s, 0.5, 3)
    assert rel(H.heom_state_download(s), OH.propagate(prob, x, 0.5, 3)) < 1e-12
    s2 = H.heom_state_create(h2, 2, H.FP64)
    H.heom_state_upload(s2, x)
    H.heom_propagate(h2, s2, 0.5, 3)
    assert rel(H.heom_state_download(s2), OH.propagate(prob, x, 0.5, 3)) < 1e-12


def test_nonfinite_response_reported():
    model = W.small_two_mode(n1=2, n2=2, depth_L=1)
    h = H.heom_build_hierarchy(model, H.FP64)
    eq = H.heom_state_create(h, 1, H.FP64)
    x = np.zeros((1, h.n_ado, h.d, h.d), dtype=np.complex128)
    x[0, 0] = np.eye(h.d) / h.d
    x[0, 0, 0, 0] = np.nan
    H.heom_state_upload(eq, x)
    with pytest.raises(H.HeomError) as err:
        H.heom_response_2d(h, eq, W.grid(0.5, 2, 3, 3, (0.0,)))
    assert err.value.status == -7

