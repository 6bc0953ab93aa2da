"""Pins of the oracle's square-linear coupling, counter term and nonlinear dipole.

These terms vanish in the Brownian-oscillator and harmonic pins (V_SL = 0,
mu2 = 0), so they are pinned here against mathematics the oracle does not use:

  * Nonlinear dipole (Eq. NLdip).  Without a bath the hierarchy decouples and
    R1(t) = 2 sum_n |<0|mu|n>|^2 sin(w_n0 t) on |0><0| (Eq. R1).  For a harmonic
    mode with mu = mu1 q + mu2 q^2 / 2 the ladder algebra gives <0|q|1> = 1/sqrt(2)
    and <0|q^2|2> = 1/sqrt(2), so R1 = 2[(mu1^2/2) sin wt + (mu2^2/8) sin 2wt];
    for two harmonic modes with the cross term mu_st q_s q_t the extra term is
    2 (mu_st^2/4) sin((w_s + w_t) t).  Compared with the RK4 amplification factor
    in place of exp(-i w dt), which makes the closed form exact to rounding.
  * Coupling operator and counter term (Eqs. h_int, counterterm, counter2).  For a
    harmonic mode the oracle's V_s and (H_S' - H_A)/Lambda are compared with
    matrix elements written from the ladder operators: q, q^2 in closed form, and
    V^2 as the square of V formed in a basis 12 states larger, then truncated
    (so no expansion of (V_LL q + V_SL q^2/2)^2 is shared with the oracle).
  * Pure dephasing (SL coupling only, two kept levels).  In the two lowest levels
    of a harmonic mode q^2 and q^4 are diagonal, so V = (V_SL/2) diag(1/2, 3/2)
    and H_S' are diagonal and every ADO is proportional to |1><0|.  The
    hierarchy then closes on a generating function, and the coherence obeys
      ln rho_10(t) = -i w' t - sum_j Delta (Re c_j Delta + i Im c_j Sigma)
                                  [t/nu_j - (1 - exp(-nu_j t))/nu_j^2],
    with Delta = V_1 - V_0 = V_SL/2, Sigma = V_1 + V_0 = V_SL and
    w' = w + Lambda (V_SL^2/4) (<1|q^4|1> - <0|q^4|0>) = w + 3 Lambda V_SL^2/4
    (the exact projection of V^2, reading 9); this is the cumulant solution of
    the Gaussian pure-dephasing problem for the factorised initial state.  The
    truncated hierarchy reaches it as the depth grows.
"""
import math

import numpy as np

import workloads as W
from oracle import heom as Hm
from oracle import model as M


def rk4_factor(z):
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


def harmonic(omega_cm, n_levels, **kw):
    return W.mode("cubic", omega_cm, g3_cm=0.0, n_levels=n_levels, n_prim=n_levels, **kw)


# ---------------------------------------------------------------------------
# Nonlinear dipole
# ---------------------------------------------------------------------------
def test_quadratic_dipole_linear_response_closed_form():
    mu1, mu2 = 0.8, 0.3
    md = harmonic(1200.0, 4, lambda_cm=0.0, V_LL=0.0, V_SL=0.0, mu1=mu1, mu2=mu2)
    model = {"modes": [md], "pairs": [], "T_K": 300.0, "depth_L": 1}
    prob = M.Problem(model)
    dt, m, n = 0.5, 4, 40
    rho = Hm.initial_state(prob)
    R1 = Hm.response_1d(prob, rho, dt, m, n)
    w = 1200.0 * M.CM_TO_RADFS
    steps = m * np.arange(n)
    ref = np.zeros(n)
    for amp, freq in ((mu1 ** 2 / 2, w), (mu2 ** 2 / 8, 2 * w)):
        ref += -2 * amp * np.imag(rk4_factor(-1j * freq * dt) ** steps)
    assert np.abs(R1.imag).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(R1.real - ref).max() < 1e-12 * np.abs(ref).max()
    # the mu2 term is not negligible here: a dropped 1/2 would change R1 by > 1%
    assert 3 * mu2 ** 2 / 8 > 0.01 * mu1 ** 2 / 2


def test_dipole_cross_term_linear_response_closed_form():
    ms, mt, mst = 0.7, 0.5, 0.4
    ws_cm, wt_cm = 1500.0, 900.0
    m0 = harmonic(ws_cm, 3, lambda_cm=0.0, V_LL=0.0, V_SL=0.0, mu1=ms, mu2=0.0)
    m1 = harmonic(wt_cm, 3, lambda_cm=0.0, V_LL=0.0, V_SL=0.0, mu1=mt, mu2=0.0)
    model = {"modes": [m0, m1], "pairs": [W.pair(0, 1, mu_st=mst)], "T_K": 300.0, "depth_L": 1}
    prob = M.Problem(model)
    dt, m, n = 0.5, 4, 40
    R1 = Hm.response_1d(prob, Hm.initial_state(prob), dt, m, n)
    ws, wt = ws_cm * M.CM_TO_RADFS, wt_cm * M.CM_TO_RADFS
    steps = m * np.arange(n)
    ref = np.zeros(n)
    for amp, freq in ((ms ** 2 / 2, ws), (mt ** 2 / 2, wt), (mst ** 2 / 4, ws + wt)):
        ref += -2 * amp * np.imag(rk4_factor(-1j * freq * dt) ** steps)
    assert np.abs(R1.real - ref).max() < 1e-12 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# Coupling operator and counter term
# ---------------------------------------------------------------------------
def ladder_q_powers(n):
    """q and q^2 of the first n harmonic states from the ladder closed forms."""
    q = np.zeros((n, n))
    q2 = np.zeros((n, n))
    for k in range(n):
        q2[k, k] = k + 0.5
        if k + 1 < n:
            q[k, k + 1] = q[k + 1, k] = math.sqrt((k + 1) / 2.0)
        if k + 2 < n:
            q2[k, k + 2] = q2[k + 2, k] = math.sqrt((k + 1) * (k + 2)) / 2.0
    return q, q2


def test_coupling_operator_and_counter_term_ladder_elements():
    n, big = 5, 17
    vll, vsl = 0.3, 0.7
    md = harmonic(1000.0, n, lambda_cm=30.0, V_LL=vll, V_SL=vsl)
    prob = M.Problem({"modes": [md], "pairs": [], "T_K": 300.0, "depth_L": 1})
    q, q2 = ladder_q_powers(big)
    V_big = vll * q + 0.5 * vsl * q2
    V_ref = V_big[:n, :n]
    V2_ref = (V_big @ V_big)[:n, :n]
    V = prob.sys.V[0]
    assert np.abs(V - V_ref).max() < 1e-12
    Lam = prob.sys.Lam[0]
    counter = (prob.sys.H - np.diag(prob.sys.E[0])) / Lam
    assert np.abs(counter - V2_ref).max() < 1e-11 * np.abs(V2_ref).max()
    # the exact projection differs from the square of the truncated V
    assert np.abs(V2_ref - V_ref @ V_ref).max() > 0.1


# ---------------------------------------------------------------------------
# Pure dephasing by the square-linear coupling
# ---------------------------------------------------------------------------
def pure_dephasing_model(V_SL, depth_L):
    md = harmonic(300.0, 2, V_LL=0.0, V_SL=V_SL, mu1=1.0, K_pade=1)
    return {"modes": [md], "pairs": [], "T_K": 300.0, "depth_L": depth_L}


def pure_dephasing_closed_form(prob, V_SL, t):
    b = prob.bath
    w = prob.sys.E[0][1] - prob.sys.E[0][0]
    w_shift = w + prob.sys.Lam[0] * (V_SL ** 2 / 4.0) * (15.0 / 4.0 - 3.0 / 4.0)
    delta, sigma = V_SL / 2.0, V_SL
    lnf = -1j * w_shift * t
    for j in range(b.D):
        c = b.a[j] + 1j * (b.b[j] / 1j).real
        g = t / b.nu[j] - (1.0 - np.exp(-b.nu[j] * t)) / b.nu[j] ** 2
        lnf = lnf - delta * (c.real * delta + 1j * c.imag * sigma) * g
    return np.exp(lnf)


def coherence_history(prob, dt, t_end, n_samples):
    rho = np.zeros((1, prob.nado, 2, 2), dtype=complex)
    rho[0, 0, 1, 0] = 1.0
    per = int(round(t_end / dt)) // n_samples
    out, ts = [], []
    for k in range(n_samples):
        rho = Hm.propagate(prob, rho, dt, per)
        out.append(rho[0, 0, 1, 0])
        ts.append((k + 1) * per * dt)
    # the state stays a multiple of |1><0| in every ADO
    assert np.abs(rho[0, :, 0, :]).max() == 0 and np.abs(rho[0, :, 1, 1]).max() == 0
    return np.array(out), np.array(ts)


def test_square_linear_pure_dephasing_closed_form():
    V_SL = 1.0
    prob = M.Problem(pure_dephasing_model(V_SL, 8))
    f, ts = coherence_history(prob, 0.25, 200.0, 4)
    ref = pure_dephasing_closed_form(prob, V_SL, ts)
    # visible dephasing and bath-induced phase: the test is not dominated by free rotation
    assert np.abs(ref[-1]) < 0.6
    assert np.abs(f - ref).max() < 1e-8
    # RK4 at half the step is closer by ~2^4 (the residual is time discretisation)
    f2, _ = coherence_history(prob, 0.5, 200.0, 4)
    e1, e2 = np.abs(f - ref).max(), np.abs(f2 - ref).max()
    assert 8.0 < e2 / e1 < 24.0


def test_square_linear_pure_dephasing_depth_convergence():
    V_SL = 1.0
    errs = []
    for L in (2, 4, 6):
        prob = M.Problem(pure_dephasing_model(V_SL, L))
        f, ts = coherence_history(prob, 0.25, 200.0, 2)
        errs.append(np.abs(f - pure_dephasing_closed_form(prob, V_SL, ts)).max())
    assert errs[0] > errs[1] > errs[2]
