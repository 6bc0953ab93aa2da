"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances
  FP64 path : 1e-10 relative to the max-norm of the compared quantity.
  FP32 path : states after a few steps within 2e-5 of the max-norm; spectra
              within 1e-4 of the spectrum max-norm.
Sizes span several thread blocks with ragged tails (d = 6, 9, 12, 64, 125;
n1, n3 not multiples of anything), plus the full workload shapes in the batched
launch configuration, checked on sampled branches.
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


def rand_state(shape, seed, hermitian=False):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if hermitian:
        x = x + np.conj(np.swapaxes(x, -1, -2))
    return x


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("name,model_fn", [
    ("two_mode", lambda: W.small_two_mode(n1=3, n2=3, depth_L=3, K_pade=2)),
    ("three_mode", lambda: W.small_three_mode(n=2, depth_L=2)),
    ("c1", lambda: W.config("c1")[0]),
])
def test_propagate_fp64(name, model_fn):
    model = model_fn()
    prob = OM.Problem(model)
    h = H.heom_build_hierarchy(model)
    x = rand_state((3, prob.nado, prob.d, prob.d), 11)
    s = H.heom_state_create(h, 3, H.FP64)
    H.heom_state_upload(s, x)
    H.heom_propagate(h, s, 0.5, 6)
    got = H.heom_state_download(s)
    ref = OH.propagate(prob, x, 0.5, 6)
    assert rel(got, ref) < 1e-12


def test_propagate_fp32():
    model = W.small_two_mode(n1=4, n2=3, depth_L=3)
    prob = OM.Problem(model)
    h = H.heom_build_hierarchy(model, H.FP32)
    x = rand_state((2, prob.nado, prob.d, prob.d), 12)
    s = H.heom_state_create(h, 2, H.FP32)
    H.heom_state_upload(s, x)
    H.heom_propagate(h, s, 0.5, 4)
    got = H.heom_state_download(s)
    ref = OH.propagate(prob, x, 0.5, 4)
    assert rel(got, ref) < 2e-5


@pytest.mark.parametrize("precision", [1, 2])
def test_propagate_coupling_basis(precision):
    """FP32 (CUDA cores) and tensor-core paths, both in the coupling eigenbasis."""
    model = W.small_three_mode(n=3, depth_L=2)
    prob = OM.Problem(model)
    h = H.heom_build_hierarchy(model, precision)
    x = rand_state((3, prob.nado, prob.d, prob.d), 14)
    s = H.heom_state_create(h, 3, precision)
    H.heom_state_upload(s, x)
    H.heom_propagate(h, s, 0.5, 4)
    got = H.heom_state_download(s)
    ref = OH.propagate(prob, x, 0.5, 4)
    assert rel(got, ref) < 2e-5


@pytest.mark.parametrize("precision", [1, 2])
def test_kicks_and_trace_coupling_basis(precision):
    model = W.small_two_mode(n1=3, n2=4, depth_L=2)
    prob = OM.Problem(model)
    h = H.heom_build_hierarchy(model, precision)
    x = rand_state((2, prob.nado, prob.d, prob.d), 15)
    s = H.heom_state_create(h, 2, precision)
    H.heom_state_upload(s, x)
    tr = H.heom_trace(h, s, 3)
    assert rel(tr, (1j) ** 3 * OH.trace_mu(prob, x)) < 1e-6
    H.heom_kick(h, s, 1)
    assert rel(H.heom_state_download(s), OH.kick(x, prob.sys.mu_plus)) < 1e-6


def test_kicks_and_trace():
    model = W.small_two_mode(n1=3, n2=4, depth_L=2)
    prob = OM.Problem(model)
    h = H.heom_build_hierarchy(model)
    x = rand_state((2, prob.nado, prob.d, prob.d), 13)
    for which, K in ((0, prob.sys.mu), (1, prob.sys.mu_plus), (2, prob.sys.mu_minus)):
        s = H.heom_state_create(h, 2, H.FP64)
        H.heom_state_upload(s, x)
        H.heom_kick(h, s, which)
        assert rel(H.heom_state_download(s), OH.kick(x, K)) < 1e-13
    s = H.heom_state_create(h, 2, H.FP64)
    H.heom_state_upload(s, x)
    tr = H.heom_trace(h, s, 3)
    assert rel(tr, (1j) ** 3 * OH.trace_mu(prob, x)) < 1e-13


def test_equilibrate_fixed_time():
    model = W.small_two_mode(n1=3, n2=3, depth_L=3)
    prob = OM.Problem(model)
    h = H.heom_build_hierarchy(model)
    eq = H.heom_equilibrate(h, 0.5, 50.0, 0.0)
    got = H.heom_state_download(eq)
    ref, _, _ = OH.equilibrate(prob, 0.5, t_eq_fs=50.0)
    assert rel(got, ref) < 1e-11


def test_equilibrate_tolerance_mode():
    model = W.harmonic_bo(omega_cm=300.0, n_levels=6, lambda_cm=60.0, gamma_cm=150.0,
                          depth_L=2, K_pade=1)
    prob = OM.Problem(model)
    h = H.heom_build_hierarchy(model)
    eq = H.heom_equilibrate(h, 1.0, 20000.0, 1e-10)
    assert eq.converged
    ref, _, conv = OH.equilibrate(prob, 1.0, tol=1e-13, t_max_fs=20000.0, check_every=500)
    assert rel(H.heom_state_download(eq), ref) < 1e-8
    # an unreachable tolerance reports HEOM_ENOTCONV but still returns the state
    eq2 = H.heom_equilibrate(h, 1.0, 200.0, 1e-14)
    assert not eq2.converged


@pytest.mark.parametrize("model_fn,grid", [
    (lambda: W.small_two_mode(n1=3, n2=3, depth_L=2),
     W.grid(0.5, 4, 7, 5, (0.0, 6.0), t_eq_fs=30.0)),
    (lambda: W.small_three_mode(n=2, depth_L=2), W.grid(0.5, 3, 5, 6, (2.0,), t_eq_fs=10.0)),
])
def test_response_2d_fp64_small(model_fn, grid):
    model = model_fn()
    prob = OM.Problem(model)
    _, _, RI, RII, SC = H.spectrum_2d(model, grid, H.FP64)
    _, RIo, RIIo, SCo = OH.spectrum_2d(prob, grid)
    scale = max(np.abs(RIo).max(), np.abs(RIIo).max())
    assert np.abs(RI - RIo).max() < 1e-10 * scale
    assert np.abs(RII - RIIo).max() < 1e-10 * scale
    assert np.abs(SC - SCo).max() < 1e-10 * np.abs(SCo).max()


def test_response_2d_c1_full():
    model, grid = W.config("c1")
    prob = OM.Problem(model)
    _, _, RI, RII, SC = H.spectrum_2d(model, grid, H.FP64)
    _, RIo, RIIo, SCo = OH.spectrum_2d(prob, grid)
    scale = max(np.abs(RIo).max(), np.abs(RIIo).max())
    assert np.abs(RI - RIo).max() < 1e-10 * scale
    assert np.abs(RII - RIIo).max() < 1e-10 * scale
    assert np.abs(SC - SCo).max() < 1e-10 * np.abs(SCo).max()


def test_response_2d_fp32_spectrum():
    model = W.small_two_mode(n1=3, n2=3, depth_L=2)
    grid = W.grid(0.5, 4, 16, 16, (0.0,), t_eq_fs=30.0)
    prob = OM.Problem(model)
    _, _, RI, RII, SC = H.spectrum_2d(model, grid, H.FP32)
    _, RIo, RIIo, SCo = OH.spectrum_2d(prob, grid)
    assert np.abs(SC - SCo).max() < 1e-4 * np.abs(SCo).max()


def test_response_2d_tc_spectrum():
    """Tensor-core path: S_C within 1e-4 of the FP64 oracle's max-norm."""
    model = W.small_three_mode(n=3, depth_L=2)
    grid = W.grid(0.5, 8, 24, 24, (0.0,), t_eq_fs=40.0)
    prob = OM.Problem(model)
    _, _, RI, RII, SC = H.spectrum_2d(model, grid, H.TC)
    _, RIo, RIIo, SCo = OH.spectrum_2d(prob, grid)
    scale = max(np.abs(RIo).max(), np.abs(RIIo).max())
    assert np.abs(RI - RIo).max() < 1e-4 * scale
    assert np.abs(SC - SCo).max() < 1e-4 * np.abs(SCo).max()


def test_response_1d():
    model = W.harmonic_bo(omega_cm=1000.0, n_levels=8, lambda_cm=50.0, gamma_cm=200.0,
                          depth_L=2, K_pade=1)
    prob = OM.Problem(model)
    h = H.heom_build_hierarchy(model)
    eq = H.heom_equilibrate(h, 0.25, 40.0, 0.0)
    R1, I = H.heom_response_1d(h, eq, 0.25, 8, 32)
    ref_eq, _, _ = OH.equilibrate(prob, 0.25, t_eq_fs=40.0)
    R1o = OH.response_1d(prob, ref_eq, 0.25, 8, 32)
    assert rel(R1, R1o) < 1e-11
    w = np.ones(32)
    w[0] = 0.5
    Io = (2.0 * np.fft.ifft(w * R1o) * 32).imag
    assert rel(I, Io) < 1e-11


@pytest.mark.parametrize("name,precision,tol,branches", [
    ("c2", 0, 1e-11, 256),
    ("c3", 1, 2e-5, 256),
    ("c3", 2, 2e-5, 256),
])
def test_full_size_batched_step_sampled(name, precision, tol, branches):
    """Full workload shape in the bench's batched launch (all branches at once),
    through the device-pointer entry point on a torch stream; one RK4 step,
    sampled branches against the oracle."""
    torch = pytest.importorskip("torch")
    model, grid = W.config(name)
    h = H.heom_build_hierarchy(model, precision)
    nado, d = h.n_ado, h.d
    cdt = torch.complex128 if precision == 0 else torch.complex64
    dev = torch.device("cuda:0")
    y = torch.zeros((branches, nado, d, d), dtype=cdt, device=dev)
    wa = torch.empty_like(y)
    wb = torch.empty_like(y)
    rng = np.random.default_rng(21)
    samples = [0, branches - 1]
    xs = {}
    for b in samples:
        xs[b] = rng.standard_normal((nado, d, d)) + 1j * rng.standard_normal((nado, d, d))
        if precision == 0:
            y[b].copy_(torch.from_numpy(xs[b]))
        else:
            # complex64 device states live in the coupling eigenbasis
            st = H.heom_state_create(h, 1, precision)
            H.heom_state_upload(st, xs[b][None])
            H.heom_state_export_dev(st, y[b].data_ptr())
            torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    H.heom_propagate_dev(h, y.data_ptr(), wa.data_ptr(), wb.data_ptr(), branches, precision,
                         grid["dt_fs"], 1, stream.cuda_stream)
    torch.cuda.synchronize()
    prob = OM.Problem(model)
    for b in samples:
        if precision == 0:
            got = y[b].cpu().numpy().astype(np.complex128)
        else:
            st = H.heom_state_create(h, 1, precision)
            H.heom_state_import_dev(st, y[b].data_ptr())
            torch.cuda.synchronize()
            got = H.heom_state_download(st)[0]
        ref = OH.rk4_step(prob, xs[b][None], grid["dt_fs"])[0]
        assert rel(got, ref) < tol
    # a branch that started at zero stays zero
    assert float(y[branches // 2].abs().max()) == 0.0


def test_rows_and_spectrum_assembly():
    """Row blocks of heom_response_2d_rows assemble the full response, and
    heom_spectrum_2d on the assembled R gives the oracle's S_C."""
    model = W.small_two_mode(n1=3, n2=2, depth_L=2)
    grid = W.grid(0.5, 4, 7, 6, (0.0, 4.0), t_eq_fs=20.0)
    prob = OM.Problem(model)
    h = H.heom_build_hierarchy(model)
    eq = H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0)
    from paper_2601_20550_gb300.shard import row_range
    parts = [H.heom_response_2d_rows(h, eq, grid, *row_range(grid["n1"], 3, r)) for r in range(3)]
    RI = np.concatenate([p[0] for p in parts], axis=1)
    RII = np.concatenate([p[1] for p in parts], axis=1)
    _, RIo, RIIo, SCo = OH.spectrum_2d(prob, grid)
    scale = max(np.abs(RIo).max(), np.abs(RIIo).max())
    assert np.abs(RI - RIo).max() < 1e-10 * scale
    assert np.abs(RII - RIIo).max() < 1e-10 * scale
    SC = H.heom_spectrum_2d(RI, RII, grid["dt_fs"] * grid["steps_per_sample"])
    assert np.abs(SC - SCo).max() < 1e-10 * np.abs(SCo).max()


def test_response_2d_batched_parameter_sets():
    """Two parameter sets of different basis size on one grid, in one call."""
    grid = W.grid(0.5, 3, 5, 6, (0.0, 3.0), t_eq_fs=20.0)
    models = [W.small_two_mode(n1=3, n2=3, depth_L=2), W.small_three_mode(n=2, depth_L=2)]
    hs = [H.heom_build_hierarchy(m) for m in models]
    eqs = [H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0) for h in hs]
    RI, RII, SC = H.heom_response_2d_batched(hs, eqs, grid)
    assert RI.shape == (2, 2, 5, 6)
    for i, m in enumerate(models):
        _, RIo, RIIo, SCo = OH.spectrum_2d(OM.Problem(m), grid)
        scale = max(np.abs(RIo).max(), np.abs(RIIo).max())
        assert np.abs(RI[i] - RIo).max() < 1e-10 * scale
        assert np.abs(RII[i] - RIIo).max() < 1e-10 * scale
        assert np.abs(SC[i] - SCo).max() < 1e-10 * np.abs(SCo).max()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (2, 1e-4)])
@pytest.mark.parametrize("n1,n3,depth_L", [(1, 1, 2), (1, 7, 2), (6, 1, 2), (4, 5, 0)])
def test_response_2d_degenerate_grids(precision, tol, n1, n3, depth_L):
    """Single-sample axes and the zero-depth hierarchy (no bath auxiliaries)."""
    model = W.small_two_mode(n1=3, n2=3, depth_L=depth_L)
    grid = W.grid(0.5, 3, n1, n3, (0.0,), t_eq_fs=15.0)
    _, _, RI, RII, SC = H.spectrum_2d(model, grid, precision)
    _, RIo, RIIo, SCo = OH.spectrum_2d(OM.Problem(model), grid)
    scale = max(np.abs(RIo).max(), np.abs(RIIo).max())
    assert np.abs(RI - RIo).max() < tol * scale
    assert np.abs(RII - RIIo).max() < tol * scale
    assert np.abs(SC - SCo).max() <= tol * np.abs(SCo).max() + 1e-300


@pytest.mark.gpu
def test_autotuner_picks_a_shape_once():
    """The first propagation of a size tunes the stage-kernel launch; later ones reuse it."""
    model = W.small_two_mode(n1=3, n2=3, depth_L=2)
    h = H.heom_build_hierarchy(model, H.FP64)
    s = H.heom_state_create(h, 3, H.FP64)
    H.heom_state_upload(s, rand_state((3, h.n_ado, h.d, h.d), 4, hermitian=True))
    H.heom_propagate(h, s, 0.5, 4)
    first = H.heom_get_tuning(h)
    total = 3 * h.n_ado * h.d * h.d
    entry = [e for e in first if e[0] == 0 and e[1] == total]
    assert len(entry) == 1 and entry[0][2] in (64, 128, 256) and entry[0][3] >= 1
    H.heom_propagate(h, s, 0.5, 4)
    assert H.heom_get_tuning(h) == first


@pytest.mark.gpu
def test_tensor_core_coupling_shapes_and_tuning():
    """Every coupling-kernel shape of the tensor-core path gives the same response bit
    for bit (and the oracle's within the mixed-path tolerance); the autotuner records
    one shape per launch size (kind 2) and keeps it."""
    model = W.small_three_mode(n=3, depth_L=2)
    grid = W.grid(0.5, 4, 6, 5, (0.0,), t_eq_fs=20.0)
    h = H.heom_build_hierarchy(model, H.TC)
    eq = H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0)
    got = []
    try:
        for shape in range(H.heom_tc_shape_count()):
            H.heom_debug_force_tc_shape(shape)
            got.append(H.heom_response_2d(h, eq, grid))
    finally:
        H.heom_debug_force_tc_shape(-1)
    for ri, rii, sc in got[1:]:
        assert np.array_equal(ri, got[0][0]) and np.array_equal(rii, got[0][1]) and np.array_equal(sc, got[0][2])
    assert [e for e in H.heom_get_tuning(h) if e[0] == 2] == []   # forced shapes are not recorded
    RI, RII, SC = H.heom_response_2d(h, eq, grid)
    assert np.array_equal(RI, got[0][0]) and np.array_equal(SC, got[0][2])
    tuned = [e for e in H.heom_get_tuning(h) if e[0] == 2]
    B = 2 * grid["n1"]
    assert len(tuned) == 1 and tuned[0][1] == B * h.n_ado * h.d * h.d
    rpt, groups, ados, pf = H.heom_get_tc_shape(h, tuned[0][1])
    assert (rpt, groups, ados, pf) in ((8, 2, 1, 0), (4, 2, 1, 0), (8, 1, 1, 0), (4, 2, 2, 0), (4, 2, 4, 0),
                                       (4, 1, 4, 0), (2, 2, 8, 0), (4, 1, 8, 0), (8, 1, 1, 1), (4, 2, 1, 1),
                                       (8, 2, 1, 1), (4, 2, 4, 1), (16, 1, 1, 1), (4, 1, 1, 1),
                                       (8, 1, 1, 3), (4, 1, 1, 3), (4, 2, 1, 3))
    assert tuned[0][2] == 128 * groups
    assert tuned[0][3] == B * -(-h.n_ado // ados) * -(-h.d // (rpt * groups))
    H.heom_response_2d(h, eq, grid)
    assert [e for e in H.heom_get_tuning(h) if e[0] == 2] == tuned
    _, RIo, RIIo, SCo = OH.spectrum_2d(OM.Problem(model), grid)
    scale = max(np.abs(RIo).max(), np.abs(RIIo).max())
    assert np.abs(RI - RIo).max() < 1e-4 * scale
    assert np.abs(SC - SCo).max() < 1e-4 * np.abs(SCo).max()


@pytest.mark.gpu
def test_batched_one_launch_equals_per_set():
    """Three FP64 sets of different basis size advanced together match per-set calls."""
    grid = W.grid(0.5, 3, 5, 4, (0.0, 2.0), t_eq_fs=12.0)
    models = [W.small_two_mode(n1=3, n2=3, depth_L=2), W.small_three_mode(n=2, depth_L=2),
              W.small_two_mode(n1=4, n2=3, depth_L=3)]
    hs = [H.heom_build_hierarchy(m) for m in models]
    eqs = [H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0) for h in hs]
    assert len({h.d for h in hs}) == 3
    n0 = H.heom_launch_count()
    RI, RII, SC = H.heom_response_2d_batched(hs, eqs, grid)
    launches_batched = H.heom_launch_count() - n0
    n0 = H.heom_launch_count()
    for i, (h, eq) in enumerate(zip(hs, eqs)):
        ri, rii, sc = H.heom_response_2d(h, eq, grid)
        scale = max(np.abs(ri).max(), np.abs(rii).max())
        assert np.abs(RI[i] - ri).max() <= 1e-14 * scale
        assert np.abs(RII[i] - rii).max() <= 1e-14 * scale
        assert np.abs(SC[i] - sc).max() <= 1e-14 * np.abs(sc).max()
    launches_single = H.heom_launch_count() - n0
    assert launches_batched < launches_single


@pytest.mark.gpu
def test_batched_tensor_core_sets_one_launch():
    """Three tensor-core parameter sets of different basis size advance together (one
    tensor-core and one coupling-kernel launch per RK4 stage for all sets): the results
    equal the per-set calls bit for bit and the oracle within the mixed-path tolerance."""
    grid = W.grid(0.5, 4, 6, 5, (0.0, 2.0), t_eq_fs=20.0)
    models = [W.small_three_mode(n=3, depth_L=2), W.small_three_mode(n=2, depth_L=2),
              W.small_two_mode(n1=4, n2=3, depth_L=3)]
    hs = [H.heom_build_hierarchy(m, H.TC) for m in models]
    assert len({h.d for h in hs}) == 3
    eqs = [H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0) for h in hs]
    n0 = H.heom_launch_count()
    RI, RII, SC = H.heom_response_2d_batched(hs, eqs, grid)
    launches_batched = H.heom_launch_count() - n0
    n0 = H.heom_launch_count()
    for i, (h, eq) in enumerate(zip(hs, eqs)):
        ri, rii, sc = H.heom_response_2d(h, eq, grid)
        assert np.array_equal(RI[i], ri) and np.array_equal(RII[i], rii) and np.array_equal(SC[i], sc)
    launches_single = H.heom_launch_count() - n0
    assert launches_batched < launches_single
    for i, m in enumerate(models):
        _, RIo, RIIo, SCo = OH.spectrum_2d(OM.Problem(m), grid)
        scale = max(np.abs(RIo).max(), np.abs(RIIo).max())
        assert np.abs(RI[i] - RIo).max() < 1e-4 * scale
        assert np.abs(SC[i] - SCo).max() < 1e-4 * np.abs(SCo).max()


@pytest.mark.gpu
def test_batched_tensor_core_repeated_hierarchy():
    """A tensor-core hierarchy named twice in one batch (its scale workspace serves one
    set at a time) runs set by set and gives the single-set result for both entries."""
    grid = W.grid(0.5, 4, 5, 4, (0.0,), t_eq_fs=20.0)
    h = H.heom_build_hierarchy(W.small_three_mode(n=2, depth_L=2), H.TC)
    eq = H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0)
    RI, RII, SC = H.heom_response_2d_batched([h, h], [eq, eq], grid)
    ri, rii, sc = H.heom_response_2d(h, eq, grid)
    for i in range(2):
        assert np.array_equal(RI[i], ri) and np.array_equal(RII[i], rii) and np.array_equal(SC[i], sc)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 2])
def test_repeated_calls_are_bitwise_identical(precision):
    """Every reduction (traces, maxima, Fourier sums) runs in a fixed order and no result
    depends on a launch shape, so a repeated call (the second one with the shapes the
    first one tuned) returns the same bits."""
    model = W.small_two_mode(n1=3, n2=3, depth_L=2)
    grid = W.grid(0.5, 4, 6, 5, (0.0, 4.0), t_eq_fs=20.0)
    h = H.heom_build_hierarchy(model, precision)
    eq = H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0)
    first = H.heom_response_2d(h, eq, grid)
    second = H.heom_response_2d(h, eq, grid)
    for a, b in zip(first, second):
        assert np.array_equal(a, b)


@pytest.mark.gpu
def test_steady_state_krylov():
    """GMRES steady state against the oracle's direct null-vector solve."""
    model = W.harmonic_bo(omega_cm=300.0, n_levels=5, lambda_cm=60.0, gamma_cm=150.0,
                          depth_L=2, K_pade=1)
    model["modes"][0]["g3_cm"] = -40.0
    model["modes"][0]["n_prim"] = 12
    model["modes"][0]["V_SL"] = 0.2
    x = OH.steady_state(OM.Problem(model))
    h = H.heom_build_hierarchy(model)
    s, its = H.heom_steady_state(h, tol=1e-12, restart=30, max_iter=3000)
    assert s.converged and its > 0
    got = H.heom_state_download(s)
    assert np.max(np.abs(got - x)) < 1e-9 * np.max(np.abs(x))


@pytest.mark.gpu
def test_steady_state_two_modes():
    """A two-mode model whose slowest relaxation takes ~4e4 fs (stiff for propagation)."""
    model = W.small_two_mode(n1=3, n2=3, depth_L=2)
    x = OH.steady_state(OM.Problem(model))
    h = H.heom_build_hierarchy(model)
    s, its = H.heom_steady_state(h, tol=1e-12, restart=60, max_iter=900, dt_fs=0.5, steps_per_matvec=2000)
    assert s.converged, its
    a = H.heom_state_download(s)
    assert abs(np.trace(a[0, 0]) - 1.0) < 1e-10
    assert np.max(np.abs(a - x)) < 1e-8 * np.max(np.abs(x))


def _neighbours(hier, ados):
    out = set(ados)
    for i in ados:
        for j in range(hier.D):
            for f in (hier.up, hier.down):
                k = f(i, j)
                if k >= 0:
                    out.add(k)
    return out


@pytest.mark.gpu
def test_c5_full_size_step_sampled():
    """c5 at full size (d = 216, 24310 ADOs, 18 GB per FP64 state): one RK4 step of a
    state that is non-zero on one ADO, against the oracle's classic RK4 evaluated on the
    dependency cone of that ADO (per-ADO right-hand sides); a distant ADO stays zero."""
    torch = pytest.importorskip("torch")
    model, grid = W.config("c5")
    h = H.heom_build_hierarchy(model, H.FP64)
    prob = OM.Problem(model)
    hier, dt = prob.hier, grid["dt_fs"]
    n = 5000
    rng = np.random.default_rng(55)
    x = (rng.standard_normal((h.d, h.d)) + 1j * rng.standard_normal((h.d, h.d)))[None]
    y = torch.zeros((1, h.n_ado, h.d, h.d), dtype=torch.complex128, device="cuda")
    y[0, n].copy_(torch.from_numpy(x[0]))
    wa, wb = torch.empty_like(y), torch.empty_like(y)
    H.heom_propagate_dev(h, y.data_ptr(), wa.data_ptr(), wb.data_ptr(), 1, H.FP64, dt, 1,
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = y[0, n].cpu().numpy()
    N1 = _neighbours(hier, {n})
    N2 = _neighbours(hier, N1)
    far = next(i for i in range(h.n_ado) if i not in _neighbours(hier, _neighbours(hier, N2)))
    assert float(y[0, far].abs().max()) == 0.0
    del y, wa, wb
    zero = np.zeros_like(x)
    yv = {n: x}

    def getter(d):
        return lambda k: d.get(k, zero)

    k1 = {m: OH.rhs_one(prob, getter(yv), m) for m in N1}
    u2 = {m: yv.get(m, zero) + 0.5 * dt * k1[m] for m in N1}
    k2 = {m: OH.rhs_one(prob, getter(u2), m) for m in N2}
    u3 = {m: yv.get(m, zero) + 0.5 * dt * k2[m] for m in N2}
    k3 = {m: OH.rhs_one(prob, getter(u3), m) for m in N1}
    u4 = {m: yv.get(m, zero) + dt * k3[m] for m in N1}
    k4 = OH.rhs_one(prob, getter(u4), n)
    ref = (x + dt / 6.0 * (k1[n] + 2 * k2[n] + 2 * k3[n] + k4))[0]
    assert rel(got, ref) < 1e-11


@pytest.mark.gpu
def test_state_creation_ordered_after_pending_work():
    """A state created and filled while earlier GPU work is still queued on the
    caller's (legacy default) stream keeps its contents: the library zeroes new
    states on its own stream before the call returns, and its stream is ordered
    with the legacy stream.  (A zeroing memset left on the legacy stream once
    landed after the broadcast into the new state.)"""
    torch = pytest.importorskip("torch")
    model = W.small_three_mode(n=3, depth_L=2)
    for precision in (0, 2):
        h = H.heom_build_hierarchy(model, precision)
        eq = H.heom_equilibrate(h, 0.5, 10.0, 0.0)
        ref = H.heom_state_download(eq)
        a = torch.randn(8192, 8192, device="cuda:0")
        for _ in range(24):          # queued work (hundreds of ms), not synchronised
            a = a @ a
            a = a / a.norm()
        s = H.heom_state_create(h, 2, precision)
        H.heom_state_broadcast(eq, s)
        got = H.heom_state_download(s)
        torch.cuda.synchronize()
        assert np.abs(got[0] - ref[0]).max() < 1e-6 * np.abs(ref).max()
        assert np.abs(got[1] - ref[0]).max() < 1e-6 * np.abs(ref).max()


@pytest.mark.gpu
def test_c5_batch_uneven_sets_against_oracle():
    """Sets of the seeded c5 batch (levels per mode drawn from {4, 5, 6}, jittered
    parameters) with uneven basis sizes in one heom_response_2d_batched call, at depth 1
    and a short grid, against the oracle's response per set."""
    sets = W.c5_batch()
    dims = [int(np.prod([md["n_levels"] for md in m["modes"]])) for m in sets]
    pick = [int(np.argmin(dims)), int(np.argmax(dims))]
    pick.append(next(i for i in range(len(sets)) if dims[i] not in (dims[pick[0]], dims[pick[1]])))
    models = [dict(sets[i], depth_L=1) for i in pick]
    assert len({dims[i] for i in pick}) == 3
    grid = W.grid(0.25, 2, 3, 3, (0.0, 0.5), t_eq_fs=1.0)
    hs = [H.heom_build_hierarchy(m) for m in models]
    eqs = [H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0) for h in hs]
    RI, RII, SC = H.heom_response_2d_batched(hs, eqs, grid)
    for i, m in enumerate(models):
        _, RIo, RIIo, SCo = OH.spectrum_2d(OM.Problem(m), grid)
        scale = max(np.abs(RIo).max(), np.abs(RIIo).max())
        assert np.abs(RI[i] - RIo).max() < 1e-10 * scale
        assert np.abs(RII[i] - RIIo).max() < 1e-10 * scale
        assert np.abs(SC[i] - SCo).max() < 1e-10 * np.abs(SCo).max()
