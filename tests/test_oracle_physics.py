"""Physics pins of the oracle's full method (closed forms and limits).

  * P3 zero bath: with zeta = 0 the ADOs decouple and R_I, R_II reduce to
    Liouville-pathway sums in the eigenbasis of H_S'.  With the RK4 amplification
    factor P(-i dt w_ab) per step the closed form is exact to rounding; with
    exp(-i w_ab t) it agrees to the RK4 truncation error.
  * P4 harmonic Brownian oscillator: R1(t) = mu^2 chi(t) with
    chi(t) = w sum_j exp(s_j t)(s_j + gamma)/P'(s_j),
    P(s) = s^3 + gamma s^2 + (w^2 + zeta gamma) s + w^2 gamma  (m = 1/w units).
  * P5 thermal second moment: <q^2> = (1/beta)[chi^(0) + 2 sum_k eta_k chi^(nu_k)]
    with chi^(s) = w / (s^2 + w^2 + s zeta gamma/(s + gamma)) at the Pade poles,
    which tends to the Matsubara sum as K grows.
  * P6 harmonic 2D: the third-order response of a linearly coupled harmonic
    oscillator with a linear dipole vanishes (nested commutators of linear
    operators are c-numbers).
  * P7 truncation: the c1 spectrum converges monotonically in the hierarchy depth
    and in the number of Pade terms.
  * Sec. II.A: linear-linear coupling relaxes, square-linear coupling dephases.  On
    the three lowest harmonic levels (where q^2 has no element between |1> and another
    kept level) an SL-coupled mode keeps the population of |1> exactly while the
    0-1 coherence decays; an LL-coupled mode relaxes |1> towards |0>.
  * Sec. II.C and III: the vibrational quanta are far above kT, so the equilibrium is
    the ground state, and the paper notes that such modes need a larger low-temperature
    correction.  The hierarchy's null vector shows both: for two modes of 3400 and 1650
    cm^-1 at 300 K its ground-state population goes 1.41, 1.05, 1.006, 1.0001 for 1-4
    Pade terms (one term leaves a non-positive "equilibrium"), converging on the ground
    state.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import heom as Hm
from oracle import model as M


def rk4_factor(z):
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


def zero_bath_closed_form(prob, rho_eq_steps, grid, exact=False):
    E, U = np.linalg.eigh(prob.sys.H)
    dt = grid["dt_fs"]
    w = E[:, None] - E[None, :]

    def prop(X, nsteps):
        Xt = U.T @ X @ U
        f = np.exp(-1j * w * dt * nsteps) if exact else rk4_factor(-1j * w * dt) ** nsteps
        return U @ (f * Xt) @ U.T

    rho = np.zeros((prob.d, prob.d), dtype=complex)
    rho[0, 0] = 1.0
    rho = prop(rho, rho_eq_steps)
    m, n1, n3 = grid["steps_per_sample"], grid["n1"], grid["n3"]
    out = {}
    for pw in ("I", "II"):
        K1, K2, K3 = Hm.pathway_kicks(prob, pw)
        R = np.zeros((len(grid["t2_fs"]), n1, n3), dtype=complex)
        for it, t2 in enumerate(grid["t2_fs"]):
            n2 = int(round(t2 / dt))
            for j in range(n1):
                x = prop(K1 @ rho - rho @ K1, j * m)
                x = prop(K2 @ x - x @ K2, n2)
                x = K3 @ x - x @ K3
                for k in range(n3):
                    y = prop(x, k * m)
                    R[it, j, k] = (1j) ** 3 * np.trace(prob.sys.mu @ y)
        out[pw] = R
    return out["I"], out["II"]


def test_zero_bath_pathways_closed_form():
    model = W.small_two_mode(n1=3, n2=3, depth_L=2)
    for md in model["modes"]:
        md["zeta_cm"] = 0.0
    prob = M.Problem(model)
    g = W.grid(0.5, 4, 6, 5, (0.0, 6.0), t_eq_fs=20.0)
    rho_eq, nsteps, _ = Hm.equilibrate(prob, g["dt_fs"], t_eq_fs=g["t_eq_fs"])
    RI, RII = Hm.response_2d(prob, rho_eq, g)
    cI, cII = zero_bath_closed_form(prob, nsteps, g)
    scale = max(np.max(np.abs(cI)), np.max(np.abs(cII)))
    assert np.max(np.abs(RI - cI)) < 1e-12 * scale
    assert np.max(np.abs(RII - cII)) < 1e-12 * scale
    # every ADO other than n = 0 stays zero without a bath
    assert scale > 1e-3
    # and the RK4 values approach the exact exponential at a small step
    g2 = W.grid(0.05, 40, 4, 4, (3.0,), t_eq_fs=5.0)
    rho_eq, nsteps, _ = Hm.equilibrate(prob, g2["dt_fs"], t_eq_fs=g2["t_eq_fs"])
    RI, RII = Hm.response_2d(prob, rho_eq, g2)
    eI, eII = zero_bath_closed_form(prob, nsteps, g2, exact=True)
    assert np.max(np.abs(RI - eI)) < 1e-6 * np.max(np.abs(eI))
    assert np.max(np.abs(RII - eII)) < 1e-6 * np.max(np.abs(eII))


def brownian_chi(t, w, zeta, gam):
    P = [1.0, gam, w * w + zeta * gam, w * w * gam]
    dP = np.polyder(P)
    return np.real(sum(w * (s + gam) * np.exp(s * t) / np.polyval(dP, s) for s in np.roots(P)))


def test_harmonic_brownian_linear_response():
    model = W.harmonic_bo(omega_cm=1000.0, n_levels=10, lambda_cm=50.0, gamma_cm=200.0,
                          depth_L=3, K_pade=1, mu1=1.3)
    prob = M.Problem(model)
    md = model["modes"][0]
    w = md["omega_cm"] * M.CM_TO_RADFS
    zeta = md["zeta_cm"] * M.CM_TO_RADFS
    gam = md["gamma_cm"] * M.CM_TO_RADFS
    rho_eq, _, _ = Hm.equilibrate(prob, 0.25, t_eq_fs=100.0)
    R1 = Hm.response_1d(prob, rho_eq, 0.25, 8, 64)
    ref = md["mu1"] ** 2 * brownian_chi(np.arange(64) * 2.0, w, zeta, gam)
    assert np.max(np.abs(R1 - ref)) < 1e-5 * np.max(np.abs(ref))
    # temperature independence: the fluctuation terms (Re c_k) must cancel
    model_cold = W.harmonic_bo(omega_cm=1000.0, n_levels=10, lambda_cm=50.0, gamma_cm=200.0,
                               depth_L=3, K_pade=1, mu1=1.3, T_K=150.0)
    pc = M.Problem(model_cold)
    rho_c, _, _ = Hm.equilibrate(pc, 0.25, t_eq_fs=100.0)
    R1c = Hm.response_1d(pc, rho_c, 0.25, 8, 64)
    assert np.max(np.abs(R1c - ref)) < 1e-5 * np.max(np.abs(ref))


def test_thermal_second_moment():
    model = W.harmonic_bo(omega_cm=300.0, n_levels=20, lambda_cm=30.0, gamma_cm=150.0,
                          depth_L=3, K_pade=2)
    prob = M.Problem(model)
    md = model["modes"][0]
    w = md["omega_cm"] * M.CM_TO_RADFS
    zeta = md["zeta_cm"] * M.CM_TO_RADFS
    gam = md["gamma_cm"] * M.CM_TO_RADFS
    beta = prob.bath.beta

    def chihat(s):
        return w / (s * s + w * w + s * zeta * gam / (s + gam))

    xi, eta = M.pade_bose(2)
    psd = (chihat(0.0) + sum(2 * eta[k] * chihat(xi[k] / beta) for k in range(2))) / beta
    mats = (chihat(0.0) + 2 * sum(chihat(2 * math.pi * n / beta) for n in range(1, 100000))) / beta
    rho, steps, conv = Hm.equilibrate(prob, 1.0, tol=1e-9, t_max_fs=6000.0, check_every=250)
    assert conv
    q2 = (np.trace(prob.sys.q[0][2] @ rho[0, 0]) / np.trace(rho[0, 0])).real
    assert abs(q2 - psd) < 2e-5 * psd
    assert abs(psd - mats) < 1e-4 * mats
    # the bath shifts <q^2> away from the free-oscillator value by far more than the error
    free = 0.5 / math.tanh(beta * w / 2)
    assert abs(q2 - free) > 50 * abs(q2 - psd)


def test_harmonic_third_order_vanishes():
    g = W.grid(0.5, 8, 8, 8, (0.0,), t_eq_fs=50.0)
    sizes = []
    for n_levels in (5, 7, 9):
        model = W.harmonic_bo(omega_cm=1000.0, n_levels=n_levels, lambda_cm=50.0,
                              gamma_cm=200.0, depth_L=2, K_pade=1)
        prob = M.Problem(model)
        rho_eq, _, _ = Hm.equilibrate(prob, g["dt_fs"], t_eq_fs=g["t_eq_fs"])
        RI, RII = Hm.response_2d(prob, rho_eq, g)
        R1 = Hm.response_1d(prob, rho_eq, 0.5, 8, 8)
        sizes.append(max(np.max(np.abs(RI)), np.max(np.abs(RII))) / np.max(np.abs(R1)) ** 2)
    # the residual is a basis-truncation effect: it falls geometrically with the basis
    assert sizes[1] < sizes[0] / 5 and sizes[2] < sizes[1] / 5
    assert sizes[2] < 3e-5
    # with an anharmonic (Morse) mode it does not vanish
    model["modes"][0].update(potential="morse", morse_D_cm=8000.0, n_prim=120, q_min=-5.0,
                             q_max=12.0)
    pm = M.Problem(model)
    rho_eq, _, _ = Hm.equilibrate(pm, g["dt_fs"], t_eq_fs=g["t_eq_fs"])
    RIm, _ = Hm.response_2d(pm, rho_eq, g)
    assert np.max(np.abs(RIm)) > 1e-2 * np.max(np.abs(R1)) ** 2


def _c1_spectrum(depth_L, K_pade, grid):
    model, _ = W.config("c1")
    model["modes"][0]["K_pade"] = K_pade
    model["depth_L"] = depth_L
    return Hm.spectrum_2d(M.Problem(model), grid)[3]


def test_depth_and_pade_convergence():
    """P7: on the c1 model the spectrum converges monotonically in the hierarchy
    depth L and in the number of Pade terms K (successive changes shrink)."""
    grid = W.grid(0.5, 8, 12, 12, (0.0,), t_eq_fs=50.0)
    S = [_c1_spectrum(L, 1, grid) for L in range(1, 7)]
    dL = [np.abs(S[i + 1] - S[i]).max() / np.abs(S[i + 1]).max() for i in range(5)]
    assert all(dL[i + 1] < dL[i] for i in range(4)), dL
    assert dL[-1] < 1e-3
    # dt = 0.25 fs keeps dt x (L x the largest Pade rate) inside the RK4 region for K <= 4
    grid = W.grid(0.25, 16, 12, 12, (0.0,), t_eq_fs=50.0)
    S = [_c1_spectrum(3, K, grid) for K in range(1, 5)]
    dK = [np.abs(S[i + 1] - S[i]).max() / np.abs(S[i + 1]).max() for i in range(3)]
    assert all(dK[i + 1] < 0.2 * dK[i] for i in range(2)), dK
    assert dK[-1] < 1e-5


def _harmonic_three_level(vll, vsl):
    md = W.mode("cubic", 1000.0, g3_cm=0.0, n_levels=3, n_prim=3, lambda_cm=50.0, gamma_cm=500.0,
                V_LL=vll, V_SL=vsl, mu1=1.0)
    return M.Problem({"modes": [md], "pairs": [], "T_K": 300.0, "depth_L": 4})


def _evolve(prob, rho0, t_fs=400.0, dt=0.5):
    rho = Hm.initial_state(prob)
    rho[:] = 0
    rho[0, 0] = rho0
    return Hm.propagate(prob, rho, dt, int(t_fs / dt))[0, 0]


def test_linear_coupling_relaxes_square_linear_dephases():
    pop1 = np.zeros((3, 3), dtype=complex)
    pop1[1, 1] = 1.0
    v = np.array([1.0, 1.0, 0.0]) / math.sqrt(2.0)
    coh = np.outer(v, v).astype(complex)
    ll, sl = _harmonic_three_level(1.0, 0.0), _harmonic_three_level(0.0, 1.0)
    assert _evolve(ll, pop1)[1, 1].real < 0.5                 # LL: |1> relaxes
    assert abs(_evolve(sl, pop1)[1, 1].real - 1.0) < 1e-9     # SL: |1> keeps its population
    assert abs(_evolve(sl, coh)[1, 0]) < 0.8 * 0.5            # ... while the 0-1 coherence decays


def test_low_temperature_correction_restores_the_ground_state():
    dev, mineig = [], []
    for K in (1, 2, 3, 4):
        prob = M.Problem(W.small_two_mode(n1=3, n2=2, depth_L=2, K_pade=K))
        rho0 = Hm.steady_state(prob)[0, 0]
        assert abs(np.trace(rho0) - 1.0) < 1e-10
        dev.append(abs(rho0[0, 0].real - 1.0))
        mineig.append(np.linalg.eigvalsh(0.5 * (rho0 + rho0.conj().T)).min())
    assert all(a > b for a, b in zip(dev, dev[1:]))      # monotone in the Pade order
    assert dev[0] > 0.1 and mineig[0] < -0.1               # one term: far from a density matrix
    assert dev[-1] < 1e-3 and mineig[-1] > -1e-3           # four terms: the ground state
