"""Pins of the oracle's model layer against closed forms and brute force.

Each test checks oracle/model.py against something other than itself:
  * Morse levels: the analytic Morse spectrum.
  * Harmonic basis: textbook ladder-operator matrix elements, and the second-order
    perturbative shift of a cubic anharmonicity.
  * Pade decomposition: hand-derived N = 1 values, the Bernoulli series it must
    match to order 2N, its Matsubara limit and the accuracy of coth.
  * Bath coefficients: the Drude correlation function from its defining
    integral (fluctuation-dissipation theorem) by quadrature.
  * Hierarchy: binomial count and brute-force neighbour consistency.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
from scipy.special import comb

import workloads as W
from oracle import model as M


def test_morse_levels_closed_form():
    # E_n = w (n + 1/2) - w^2/(4D) (n + 1/2)^2, exact for the Morse potential
    w, D = 3650.0 * M.CM_TO_RADFS, 4.0e4 * M.CM_TO_RADFS
    E, qk = M.morse_basis(w, D, -5.0, 11.0, 240, 6)
    n = np.arange(6) + 0.5
    exact = w * n - w ** 2 / (4 * D) * n ** 2
    assert np.max(np.abs(E - exact)) < 1e-9 * w
    # q^2 is the square of q in the complete grid basis: <0|q^2|0> >= <0|q|0>^2
    assert qk[2][0, 0] > qk[1][0, 0] ** 2
    # sign convention: <n-1|q|n> > 0
    assert all(qk[1][i - 1, i] > 0 for i in range(1, 6))


def test_morse_harmonic_limit():
    # very deep well: matrix elements approach the harmonic ones
    w, D = 1000.0 * M.CM_TO_RADFS, 1.0e8 * M.CM_TO_RADFS
    E, qk = M.morse_basis(w, D, -9.0, 9.0, 240, 4)
    for n in range(3):
        assert abs(qk[1][n, n + 1] - math.sqrt((n + 1) / 2)) < 2e-3
        assert abs(qk[2][n, n] - (n + 0.5)) < 5e-3


def test_harmonic_basis_ladder():
    w = 1500.0 * M.CM_TO_RADFS
    E, qk = M.cubic_basis(w, 0.0, 8, 8)
    assert np.allclose(E, w * (np.arange(8) + 0.5), rtol=0, atol=1e-14)
    for n in range(7):
        assert abs(qk[1][n, n + 1] - math.sqrt((n + 1) / 2)) < 1e-14
    for n in range(8):
        # exact projection of q^2 and q^4 onto the truncated basis
        assert abs(qk[2][n, n] - (n + 0.5)) < 1e-13
        assert abs(qk[4][n, n] - 0.75 * (2 * n * n + 2 * n + 1)) < 1e-12


def test_cubic_second_order_shift():
    # V = alpha q^3, alpha = g3/6: Delta E_n = -(alpha^2/w)(30 n^2 + 30 n + 11)/8 + O(alpha^4)
    w = 1500.0 * M.CM_TO_RADFS
    g3 = 30.0 * M.CM_TO_RADFS
    E, _ = M.cubic_basis(w, g3, 40, 4)
    alpha = g3 / 6.0
    for n in range(4):
        pt2 = -(alpha ** 2 / w) * (30 * n * n + 30 * n + 11) / 8.0
        shift = E[n] - w * (n + 0.5)
        assert abs(shift - pt2) < 2e-3 * abs(pt2)


def test_pade_N1_by_hand():
    # [0/1] Pade of 1/12 - y/720: (1/12)/(1 + y/60) = 5/(y + 60) -> xi^2 = 60, 2 eta = 5
    xi, eta = M.pade_bose(1)
    assert abs(xi[0] - math.sqrt(60.0)) < 1e-13
    assert abs(eta[0] - 2.5) < 1e-13


@pytest.mark.parametrize("N", [2, 3, 4])
def test_pade_matches_bernoulli_series(N):
    from sympy import bernoulli
    xi, eta = M.pade_bose(N)
    # sum_k 2 eta_k / (y + xi_k^2) = sum_m y^m sum_k 2 eta_k (-1)^m / xi_k^(2m+2)
    for m in range(2 * N):
        approx = sum(2 * eta[k] * (-1) ** m / xi[k] ** (2 * m + 2) for k in range(N))
        exact = float(bernoulli(2 * m + 2)) / math.factorial(2 * m + 2)
        assert abs(approx - exact) <= 1e-10 * abs(exact)


def test_pade_matsubara_limit_and_coth():
    xi, eta = M.pade_bose(6)
    assert abs(xi[0] - 2 * math.pi) < 1e-9 and abs(eta[0] - 1.0) < 1e-9
    assert abs(xi[1] - 4 * math.pi) < 1e-4
    # coth(x/2) = 2/x + sum_k 4 eta_k x / (x^2 + xi_k^2)
    x = np.linspace(0.1, 6.0, 50)
    for N, tol in ((1, 5e-2), (2, 5e-4), (3, 2e-6), (4, 2e-9)):
        xi, eta = M.pade_bose(N)
        approx = 2 / x + sum(4 * eta[k] * x / (x ** 2 + xi[k] ** 2) for k in range(N))
        assert np.max(np.abs(approx - 1 / np.tanh(x / 2))) < tol


def test_bath_correlation_against_quadrature():
    # C(t) = (1/pi) int_0^inf J(w) [coth(beta w/2) cos wt - i sin wt] dw with
    # J(w) = m zeta gamma^2 w/(w^2+gamma^2) (Eq. drude without the 1/2pi, reading 3).
    # The Drude C(t) is log-divergent at t = 0, so t > 0 only.
    model = W.harmonic_bo(omega_cm=1200.0, lambda_cm=40.0, gamma_cm=150.0, K_pade=6, T_K=300.0)
    bath = M.Bath(model)
    md = model["modes"][0]
    w0 = md["omega_cm"] * M.CM_TO_RADFS
    zeta = md["zeta_cm"] * M.CM_TO_RADFS
    gam = md["gamma_cm"] * M.CM_TO_RADFS
    beta = bath.beta
    lam = (1.0 / w0) * zeta * gam / 2.0

    def J(w):
        if w < 1e-12:
            return 0.0
        return (1.0 / w0) * zeta * gam ** 2 / (w + gam ** 2 / w)

    def Jcoth(w):
        if w < 1e-8:
            return (1.0 / w0) * zeta * 2.0 / beta
        return J(w) / math.tanh(beta * w / 2.0)

    for t in (8.0, 20.0, 60.0):
        re = si.quad(Jcoth, 0, np.inf, weight="cos", wvar=t, limlst=200)[0] / math.pi
        im = -si.quad(J, 0, np.inf, weight="sin", wvar=t, limlst=200)[0] / math.pi
        C = bath.correlation(0, t)
        # the imaginary part (dissipation, Eq. L1) is exact: -lambda gamma exp(-gamma t)
        assert abs(C.imag - (-lam * gam * math.exp(-gam * t))) < 1e-12 * lam * gam
        assert abs(C.imag - im) < 1e-6 * lam * gam
        # the real part (fluctuation, Eq. L2) carries the Pade approximation of coth
        assert abs(C.real - re) < 1e-4 * lam * gam


@pytest.mark.parametrize("D,L", [(2, 6), (3, 4), (6, 4), (6, 6)])
def test_hierarchy_count_and_neighbours(D, L):
    h = M.Hierarchy(D, L)
    assert len(h) == comb(L + D, D, exact=True)
    for i in range(len(h)):
        for j in range(D):
            u = h.up(i, j)
            if u >= 0:
                assert h.down(u, j) == i
            else:
                assert sum(h.n[i]) == L
            dn = h.down(i, j)
            assert (dn >= 0) == (h.n[i][j] > 0)
    # canonical order: level-major
    assert all(sum(a) <= sum(b) for a, b in zip(h.n, h.n[1:]))


def test_system_operators_structure():
    model = W.small_two_mode()
    s = M.System(model)
    assert s.d == 9
    assert np.allclose(s.H, s.H.T) and np.allclose(s.mu, s.mu.T)
    # uncoupled, bath-free model: H is the Kronecker sum of the mode energies
    model0 = W.small_two_mode()
    model0["pairs"][0].update(g_st_cm=0.0, g_s2t_cm=0.0, g_st2_cm=0.0)
    for md in model0["modes"]:
        md["zeta_cm"] = 0.0
    s0 = M.System(model0)
    ksum = np.add.outer(s0.E[0], s0.E[1]).reshape(-1)
    assert np.allclose(s0.H, np.diag(ksum), atol=1e-14)
    # mu_plus raises the total excitation number, and mu = mu_plus + mu_minus + mu_0
    for a in range(s.d):
        for b in range(s.d):
            if s.mu_plus[a, b] != 0:
                assert s.N[a] > s.N[b]
    mu0 = np.where(s.N[:, None] == s.N[None, :], s.mu, 0.0)
    assert np.allclose(s.mu_plus + s.mu_minus + mu0, s.mu)


def test_pair_coupling_operator():
    # U = g q_s q_t + (g21 q_s^2 q_t + g12 q_s q_t^2)/6 in the product basis (Eq. Potential ss')
    model = W.small_two_mode()
    for md in model["modes"]:
        md["zeta_cm"] = 0.0
    pr = model["pairs"][0]
    s = M.System(model)
    E0 = np.add.outer(s.E[0], s.E[1]).reshape(-1)
    U = s.H - np.diag(E0)
    q0, q1 = s.q[0], s.q[1]
    c = M.CM_TO_RADFS
    n0, n1 = s.dims
    for a0 in range(n0):
        for a1 in range(n1):
            for b0 in range(n0):
                for b1 in range(n1):
                    ref = (pr["g_st_cm"] * c * q0[1][a0, b0] * q1[1][a1, b1]
                           + pr["g_s2t_cm"] * c / 6 * q0[2][a0, b0] * q1[1][a1, b1]
                           + pr["g_st2_cm"] * c / 6 * q0[1][a0, b0] * q1[2][a1, b1])
                    assert abs(U[a0 * n1 + a1, b0 * n1 + b1] - ref) < 1e-15
