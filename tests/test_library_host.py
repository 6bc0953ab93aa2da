"""Host-side checks of libheom2dvs (no GPU needed).

  * the shared library loads and exports every entry point declared in
    include/heom2dvs.h;
  * the library's own model builder (C++: Jacobi eigensolver, sinc-DVR and
    harmonic bases, tridiagonal Pade poles) reproduces the oracle's operators,
    bath exponentials and hierarchy order;
  * invalid descriptors are rejected with HEOM_EINVAL before any device work.
"""
import ctypes as ct
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import model as OM

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
H = pytest.importorskip("paper_2601_20550_gb300.heom")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not os.path.exists(H.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "heom2dvs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(heom_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    names = declared_symbols()
    assert len(names) >= 15
    lib = ct.CDLL(H.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


MODELS = {
    "c1": lambda: W.config("c1")[0],
    "c2": lambda: W.config("c2")[0],
    "two_mode": lambda: W.small_two_mode(n1=3, n2=4, depth_L=3, K_pade=2),
    "harmonic": lambda: W.harmonic_bo(n_levels=6, K_pade=3),
}


@pytest.mark.parametrize("name", sorted(MODELS))
def test_host_model_matches_oracle(name):
    model = MODELS[name]()
    h = H.heom_build_hierarchy(model)
    prob = OM.Problem(model)
    assert (h.d, h.n_ado, h.n_exp) == (prob.d, prob.nado, prob.bath.D)
    ops = H.heom_get_operators(h)
    sH = np.abs(prob.sys.H).max()
    assert np.abs(ops["H"] - prob.sys.H).max() < 1e-11 * sH
    smu = np.abs(prob.sys.mu).max()
    assert np.abs(ops["mu"] - prob.sys.mu).max() < 1e-11 * smu
    assert np.abs(ops["mu_plus"] - prob.sys.mu_plus).max() < 1e-11 * smu
    bath = ops["bath"]
    assert np.array_equal(bath[:, 0].astype(int), prob.bath.mode_of)
    assert np.allclose(bath[:, 1], prob.bath.nu, rtol=1e-12, atol=0)
    assert np.allclose(bath[:, 2], prob.bath.a, rtol=1e-10, atol=1e-14 * np.abs(prob.bath.a).max())
    assert np.allclose(bath[:, 3], (prob.bath.b / 1j).real, rtol=1e-12, atol=0)
    assert np.array_equal(ops["ado"], np.array(prob.hier.n))
    for s, md in enumerate(model["modes"]):
        E, qk = H.heom_get_mode(h, s, md["n_levels"])
        assert np.allclose(E, prob.sys.E[s], rtol=1e-12, atol=1e-12 * np.abs(E).max())
        for k in range(1, 5):
            ref = prob.sys.q[s][k]
            assert np.abs(qk[k - 1] - ref).max() < 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("mutate", [
    lambda m: m["modes"][0].update(n_levels=0),
    lambda m: m["modes"][0].update(n_prim=1, n_levels=2),
    lambda m: m["modes"][0].update(K_pade=9),
    lambda m: m["modes"][0].update(potential="harmonic", omega_cm=-5.0),
    lambda m: m["pairs"][0].update(t=7),
    lambda m: m.update(T_K=0.0),
])
def test_invalid_descriptors_rejected(mutate):
    model = W.small_two_mode()
    mutate(model)
    with pytest.raises(H.HeomError) as ei:
        H.heom_build_hierarchy(model)
    assert ei.value.status == -1


def test_new_entry_points_reject_bad_arguments_on_host():
    """Argument checks that run before any device work (no GPU needed)."""
    import ctypes as ct
    L = H.lib()
    h = H.heom_build_hierarchy(W.small_two_mode())
    out = ct.c_void_p()
    its = ct.c_int(0)
    # steady state: tol, restart, max_iter and steps_per_matvec are validated first
    for tol, restart, max_iter, k in ((0.0, 30, 10, 0), (1e-10, 1, 10, 0), (1e-10, 30, 0, 0), (1e-10, 30, 10, -1)):
        rc = L.heom_steady_state(h.h, tol, restart, max_iter, 0.5, k, ct.byref(out), ct.byref(its))
        assert rc == -1 and not out.value
    # batched and gradient entry points: null arguments
    g = H.marshal_grid(W.grid(0.5, 2, 3, 3, (0.0,)))
    assert L.heom_response_2d_batched(None, None, 1, ct.byref(g), None, None, None) == -1
    assert L.heom_response_2d_grad(h.h, None, ct.byref(g), None, 64, None, None) == -1
    # a hierarchy that has not propagated has no tuned launch shapes
    assert H.heom_get_tuning(h) == []
    assert L.heom_get_tuning(None, 0, None, None, None, None) == 0
    assert L.heom_state_copy_out(None, None) == -1
    # the coupling-kernel shape override takes 0 .. count - 1, or -1 to tune again
    count = H.heom_tc_shape_count()
    assert count == 17
    assert L.heom_debug_force_tc_shape(count) == -1 and L.heom_debug_force_tc_shape(-2) == -1
    assert L.heom_debug_force_tc_shape(count - 1) == 0 and L.heom_debug_force_tc_shape(-1) == 0
    assert H.heom_get_tc_shape(h, 1) is None


def test_c5_batch_sets_are_seeded_and_uneven():
    a, b = W.c5_batch(), W.c5_batch()
    assert a == b and len(a) == 16
    dims = {tuple(md["n_levels"] for md in m["modes"]) for m in a}
    assert len(dims) > 4 and all(set(x) <= {4, 5, 6} for x in dims)
    base, _ = W.config("c5")
    for m in a:
        for md, md0 in zip(m["modes"], base["modes"]):
            assert abs(md["gamma_cm"] / md0["gamma_cm"] - 1) <= 0.05
    # the library builds the smallest set's hierarchy on the host
    small = min(a, key=lambda m: np.prod([md["n_levels"] for md in m["modes"]]))
    small = dict(small, depth_L=2)
    h = H.heom_build_hierarchy(small)
    assert h.d == int(np.prod([md["n_levels"] for md in small["modes"]]))


def test_noalloc_rejects_bad_pointers_before_any_launch():
    """heom_propagate_noalloc checks its arguments before it touches the device:
    a state pointer that is not 16-byte aligned (complex128) and a non-finite dt
    are rejected with HEOM_EINVAL (no GPU needed; the pointers are never used)."""
    import ctypes as ct
    L = H.lib()
    h = H.heom_build_hierarchy(W.small_two_mode())
    rc = L.heom_propagate_noalloc(h.h, ct.c_void_p(0x10008), 1, 0.5, 1, None)
    assert rc == -1 and "aligned" in H.heom_last_error()
    for dt in (float("inf"), float("nan"), 0.0, -0.5):
        rc = L.heom_propagate_noalloc(h.h, ct.c_void_p(0x10000), 1, dt, 1, None)
        assert rc == -1 and "bad arguments" in H.heom_last_error()


def test_unstable_step_rejected_before_any_device_work():
    """dt outside the RK4 stability region of the model returns HEOM_EUNSTABLE from
    the host-side pre-check, before the device is touched (no GPU needed)."""
    import ctypes as ct
    L = H.lib()
    h = H.heom_build_hierarchy(W.config("c2")[0])
    p = ct.c_void_p(0x10000)
    rc = L.heom_propagate_dev(h.h, p, p, p, 1, 0, 10.0, 1, None)
    assert rc == -4 and "stability" in H.heom_last_error()
    out = ct.c_void_p()
    assert L.heom_equilibrate(h.h, 10.0, 100.0, 0.0, ct.byref(out)) == -4 and not out.value
    # a stable step passes the pre-check (and then needs the device)
    assert L.heom_propagate_dev(h.h, p, p, p, 1, 0, 0.5, 0, None) != -4


def test_source_tag_names_the_stage_kernels_source():
    """heom_source_tag is the SHA-256 prefix of the stage kernels' sources the library was
    built from, so a stored traffic capture matches only the kernels it measured."""
    import hashlib
    import os
    csrc = os.path.join(os.path.dirname(H.__file__), "csrc")
    h = hashlib.sha256()
    for name in ("tc_stage.cu", "tc_stage.h"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    assert H.heom_source_tag() == h.hexdigest()[:16]

