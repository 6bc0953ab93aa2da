"""GPU parity of the 2D-misfit gradient (heom_response_2d_grad, discrete adjoint)
against the oracle's loss and its central-difference gradient, and against
central differences of the library's own forward loss at a larger size."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as OA

H = pytest.importorskip("paper_2601_20550_gb300.heom")


@pytest.fixture(scope="module", autouse=True)
def built():
    H.lib()


def lib_grad(model, grid, S_ref, ckpt=64):
    h = H.heom_build_hierarchy(model, H.FP64)
    eq = H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0)
    return H.heom_response_2d_grad(h, eq, grid, S_ref, ckpt)


def ref_spectrum(model, grid, seed):
    th = OA.theta_of(model)
    rng = np.random.default_rng(seed)
    return OA.spectrum(OA.with_theta(model, th * (1 + 0.05 * rng.uniform(-1, 1, th.size))), grid)


def test_theta_maps_agree():
    for model in (W.small_two_mode(), W.small_three_mode(), W.config("c4")[0]):
        assert np.array_equal(H.theta_of(model), OA.theta_of(model))


@pytest.mark.gpu
@pytest.mark.parametrize("grid,ckpt", [
    (W.grid(0.5, 3, 4, 5, (0.0,), t_eq_fs=15.0), 64),
    (W.grid(0.5, 2, 3, 4, (0.0, 1.5), t_eq_fs=10.0), 3),     # two t2, checkpoints inside every span
])
def test_grad_matches_oracle(grid, ckpt):
    model = W.small_two_mode(n1=3, n2=3, depth_L=2)
    S_ref = ref_spectrum(model, grid, 5)
    loss, g = lib_grad(model, grid, S_ref, ckpt)
    loss_o = OA.loss(model, grid, S_ref)
    g_o, _ = OA.grad_fd(model, grid, S_ref)
    assert abs(loss - loss_o) < 1e-9 * loss_o
    # compare theta_i d loss / d theta_i: every entry on the same footing
    w = np.maximum(np.abs(OA.theta_of(model)), 1.0)
    assert np.max(np.abs((g - g_o) * w)) < 1e-6 * np.max(np.abs(g_o * w)), (g, g_o)
    missing = [i for i in range(12) if OA._slot(model, i) is None]
    assert np.all(g[missing] == 0.0)


@pytest.mark.gpu
def test_grad_three_modes_against_library_fd():
    model = W.small_three_mode(n=2, depth_L=2)
    grid = W.grid(0.5, 4, 8, 8, (0.0,), t_eq_fs=20.0)
    th = H.theta_of(model)
    rng = np.random.default_rng(9)
    m_ref = H.with_theta(model, th * (1 + 0.05 * rng.uniform(-1, 1, th.size)))
    h = H.heom_build_hierarchy(m_ref, H.FP64)
    eq = H.heom_equilibrate(h, 0.5, 20.0, 0.0)
    S_ref = H.heom_response_2d(h, eq, grid)[2]
    loss, g = lib_grad(model, grid, S_ref, 8)

    def lib_loss(t):
        hh = H.heom_build_hierarchy(H.with_theta(model, t), H.FP64)
        e = H.heom_equilibrate(hh, 0.5, 20.0, 0.0)
        return float(np.sum((H.heom_response_2d(hh, e, grid)[2] - S_ref) ** 2))

    assert abs(loss - lib_loss(th)) < 1e-12 * loss
    w = np.maximum(np.abs(th), 1.0)

    def central(i, step):
        tp, tm = th.copy(), th.copy()
        tp[i] += step
        tm[i] -= step
        return (lib_loss(tp) - lib_loss(tm)) / (2 * step)

    for i in (0, 4, 7, 11):
        step = 1e-3 * w[i]
        fd = (4 * central(i, step / 2) - central(i, step)) / 3     # Richardson: O(step^4)
        assert abs(g[i] - fd) * w[i] < 1e-7 * np.max(np.abs(g * w)), (i, g[i], fd)


@pytest.mark.gpu
def test_autograd_wrapper():
    torch = pytest.importorskip("torch")
    from paper_2601_20550_gb300.autograd import SpectrumMisfit
    model = W.small_two_mode(n1=3, n2=3, depth_L=2)
    grid = W.grid(0.5, 3, 4, 5, (0.0,), t_eq_fs=15.0)
    S_ref = ref_spectrum(model, grid, 6)
    theta = torch.tensor(H.theta_of(model), dtype=torch.float64, requires_grad=True)
    loss = SpectrumMisfit.apply(theta, model, grid, S_ref, 64)
    (gt,) = torch.autograd.grad(loss * 3.0, theta)
    l2, g2 = lib_grad(model, grid, S_ref)
    assert abs(float(loss) - l2) < 1e-12 * l2
    assert np.allclose(gt.numpy(), 3.0 * g2, rtol=1e-12, atol=0.0)
