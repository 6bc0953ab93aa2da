"""Pins of the oracle's 2D-misfit gradient (oracle/adjoint.py).

  * parameter map: theta round-trips through the model description; absent
    modes and pairs read as 0 and are left alone.
  * the central difference quotient is second order: halving h divides its
    change by ~4, so the quoted gradient is the derivative to O(h^2).
  * the meaning of the damping entry (gamma varied with zeta fixed) against the
    closed-form linear response of the harmonic Brownian oscillator.
"""
import math

import numpy as np

import workloads as W
from oracle import adjoint as OA
from oracle import heom as Hm
from oracle import model as M


def tiny():
    model = W.small_two_mode(n1=3, n2=3, depth_L=2)
    grid = W.grid(0.5, 3, 4, 5, (0.0,), t_eq_fs=15.0)
    return model, grid


def test_theta_roundtrip():
    model, _ = tiny()
    th = OA.theta_of(model)
    assert th[0] == model["modes"][0]["morse_D_cm"] and th[1] == model["modes"][1]["g3_cm"]
    assert th[2] == 0.0 and th[5] == 0.0 and th[11] == 0.0       # no third mode or pair
    assert th[3] == model["pairs"][0]["g_s2t_cm"]
    assert th[6] == model["modes"][0]["V_SL"] and th[10] == model["modes"][1]["gamma_cm"]
    t2 = th * 1.01
    t2[2] = 5.0                                                   # ignored: no third mode
    m2 = OA.with_theta(model, t2)
    back = OA.theta_of(m2)
    mask = np.array([OA._slot(model, i) is not None for i in range(OA.N_THETA)])
    assert np.allclose(back[mask], t2[mask]) and np.all(back[~mask] == 0.0)
    assert model["modes"][0]["morse_D_cm"] == th[0]             # the input is not modified


def test_fd_gradient_second_order():
    model, grid = tiny()
    th = OA.theta_of(model)
    rng = np.random.default_rng(11)
    S_ref = OA.spectrum(OA.with_theta(model, th * (1 + 0.05 * rng.uniform(-1, 1, th.size))), grid)
    which = [0, 9]
    g1, _ = OA.grad_fd(model, grid, S_ref, rel=4e-3, which=which)
    g2, _ = OA.grad_fd(model, grid, S_ref, rel=2e-3, which=which)
    g3, _ = OA.grad_fd(model, grid, S_ref, rel=1e-3, which=which)
    for i in which:
        assert g3[i] != 0.0
        ratio = (g1[i] - g2[i]) / (g2[i] - g3[i])
        assert 3.0 < ratio < 5.5, (i, ratio)


def brownian_chi(t, w, zeta, gam):
    P = [1.0, gam, w * w + zeta * gam, w * w * gam]
    dP = np.polyder(P)
    return np.real(sum(w * (s + gam) * np.exp(s * t) / np.polyval(dP, s) for s in np.roots(P)))


def test_gamma_entry_against_closed_form():
    """d R1 / d gamma (zeta fixed) of the oracle against the closed form's derivative."""
    model = W.harmonic_bo(omega_cm=1000.0, n_levels=10, lambda_cm=50.0, gamma_cm=200.0,
                          depth_L=3, K_pade=1, mu1=1.3)
    md = model["modes"][0]
    th = OA.theta_of(model)
    h = 2.0                                                       # cm^-1
    R = []
    for sgn in (+1, -1):
        t = th.copy()
        t[9] += sgn * h
        prob = M.Problem(OA.with_theta(model, t))
        rho_eq, _, _ = Hm.equilibrate(prob, 0.25, t_eq_fs=100.0)
        R.append(Hm.response_1d(prob, rho_eq, 0.25, 8, 48))
    dR = (R[0] - R[1]) / (2 * h)
    c = M.CM_TO_RADFS
    w, zeta, gam = md["omega_cm"] * c, md["zeta_cm"] * c, md["gamma_cm"] * c
    t = np.arange(48) * 2.0
    ref = md["mu1"] ** 2 * (brownian_chi(t, w, zeta, gam + h * c) - brownian_chi(t, w, zeta, gam - h * c)) / (2 * h)
    assert np.max(np.abs(dR - ref)) < 5e-5 * np.max(np.abs(ref))
    assert math.isfinite(float(np.max(np.abs(ref)))) and np.max(np.abs(ref)) > 0
