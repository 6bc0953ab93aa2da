"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only *names* parameter sets: mode potentials, bath and coupling
strengths, dipole elements, basis truncation, hierarchy depth and the time
grid, all in the units the interface takes (cm^-1, K, fs).  It holds none of
the method's arithmetic (no unit conversion, no basis, no bath coefficients,
no hierarchy): each side turns these numbers into operators with its own code.

The parameters follow the multi-mode anharmonic Brownian (MAB) model of
Sec. II.A (Eqs. Total Hamiltonian to h_int) and the Drude bath of Eq. drude.
Where the paper gives no number the choice is stated next to it.

Model dictionary (mirrors ``heom_model`` in include/heom2dvs.h)::

    {"modes": [mode, ...], "pairs": [pair, ...], "T_K": float, "depth_L": int}
    mode = {"potential": "morse" | "cubic", "omega_cm", "g3_cm", "morse_D_cm",
            "n_levels", "n_prim", "q_min", "q_max",
            "zeta_cm", "gamma_cm", "V_LL", "V_SL", "mu1", "mu2", "K_pade"}
    pair = {"s", "t", "g_st_cm", "g_s2t_cm", "g_st2_cm", "mu_st"}

Grid dictionary (mirrors ``heom_grid``)::

    {"dt_fs", "steps_per_sample", "n1", "n3", "t2_fs": [...], "t_eq_fs"}
"""
import copy

import numpy as np

# Bath strength used for every mode where the paper's tables do not apply:
# reorganisation energy lambda = m*zeta*gamma/2 = zeta*gamma/(2*omega) of 25 cm^-1
# with gamma = 100 cm^-1 (the Drude width named for the single-mode workload).
LAMBDA_CM = 25.0
GAMMA_CM = 100.0


def zeta_for(lambda_cm, gamma_cm, omega_cm):
    """zeta (cm^-1) that gives reorganisation energy ``lambda_cm`` (parameter recipe)."""
    return 2.0 * lambda_cm * omega_cm / gamma_cm


def mode(potential, omega_cm, *, D_cm=0.0, g3_cm=0.0, n_levels=4, n_prim=300,
         q_min=-6.0, q_max=14.0, lambda_cm=LAMBDA_CM, gamma_cm=GAMMA_CM,
         V_LL=0.1, V_SL=1.0, mu1=1.0, mu2=0.0, K_pade=1):
    return {
        "potential": potential, "omega_cm": float(omega_cm), "g3_cm": float(g3_cm),
        "morse_D_cm": float(D_cm), "n_levels": int(n_levels), "n_prim": int(n_prim),
        "q_min": float(q_min), "q_max": float(q_max),
        "zeta_cm": zeta_for(lambda_cm, gamma_cm, omega_cm), "gamma_cm": float(gamma_cm),
        "V_LL": float(V_LL), "V_SL": float(V_SL), "mu1": float(mu1), "mu2": float(mu2),
        "K_pade": int(K_pade),
    }


def pair(s, t, g_st=0.0, g_s2t=0.0, g_st2=0.0, mu_st=0.0):
    return {"s": int(s), "t": int(t), "g_st_cm": float(g_st), "g_s2t_cm": float(g_s2t),
            "g_st2_cm": float(g_st2), "mu_st": float(mu_st)}


def grid(dt_fs, m, n1, n3, t2_fs=(0.0,), t_eq_fs=200.0):
    return {"dt_fs": float(dt_fs), "steps_per_sample": int(m), "n1": int(n1), "n3": int(n3),
            "t2_fs": [float(t) for t in t2_fs], "t_eq_fs": float(t_eq_fs)}


# ---------------------------------------------------------------------------
# Water-like three-mode model (asymmetric stretch 1, symmetric stretch 1', bend 2)
# ---------------------------------------------------------------------------
# Frequencies 3650 / 3750 / 1600 cm^-1; Morse depths 1e4 cm^-1 (stretches, the value
# named for the single-mode workload) and 2e4 cm^-1 (bend).  The square-linear
# coupling V_SL = 0.1 keeps the counter term Lambda <V^2> of the highest kept
# stretch levels (<q^4> ~ 5e3 at 5 levels, ~3e4 at 6) small enough that the
# Bohr-frequency spread of H_S' stays inside the RK4 stability region at the
# workloads' dt; with V_SL = 1 the spread at 5 levels per mode is 6.2e4 cm^-1
# (dt * spread = 5.9 at dt = 0.5 fs, beyond the RK4 limit of 2.8).
# Dipole ratios follow the linear dipole column of the three-mode table (3.3 : 3.3 : 1.8 -> 1 : 1 : 0.545); the quadratic
# stretch dipole is 1.2e-2 / 3.3 of the linear one; the stretch-bend dipole cross
# terms follow the 2.0e-3 entries of the pair table on the same scale.  The cubic
# pair couplings are drawn from numpy's default_rng(2601), U(-50, 50) cm^-1, in pair
# order (1,1'), (1,2), (1',2), g_{s^2 s'} before g_{s s'^2} for each pair.
WATER_OMEGA = (3650.0, 3750.0, 1600.0)
WATER_MORSE_D = (1.0e4, 1.0e4, 2.0e4)
WATER_MU1 = (1.0, 1.0, 0.545)
WATER_MU2 = (0.0036, 0.0036, 0.0)
WATER_PAIR_MU = {(0, 1): 0.0, (0, 2): 6.0e-4, (1, 2): 6.0e-4}
WATER_V_SL = 0.1
WATER_V_LL = 0.1


def water_pairs(seed=2601):
    rng = np.random.default_rng(seed)
    out = []
    for (s, t) in ((0, 1), (0, 2), (1, 2)):
        g_s2t, g_st2 = rng.uniform(-50.0, 50.0, size=2)
        out.append(pair(s, t, 0.0, g_s2t, g_st2, WATER_PAIR_MU[(s, t)]))
    return out


def water_model(n_levels, depth_L, K_pade=1, n_prim=300, T_K=300.0):
    modes = []
    for s in range(3):
        modes.append(mode("morse", WATER_OMEGA[s], D_cm=WATER_MORSE_D[s], n_levels=n_levels,
                          n_prim=n_prim, q_min=-5.0, q_max=20.0, V_LL=WATER_V_LL,
                          V_SL=WATER_V_SL, mu1=WATER_MU1[s], mu2=WATER_MU2[s], K_pade=K_pade))
    return {"modes": modes, "pairs": water_pairs(), "T_K": float(T_K), "depth_L": int(depth_L)}


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------
def c1():
    """Single Morse mode (D = 1e4 cm^-1, omega = 3600 cm^-1), its 6 lowest states,
    LL+SL coupling to a Drude bath (gamma = 100 cm^-1, 300 K), one Pade term
    (2 exponentials), depth 6 -> 28 ADOs of 6x6; dt 0.5 fs, 64x64 grid, t2 = 0."""
    m = mode("morse", 3600.0, D_cm=1.0e4, n_levels=6, n_prim=200, q_min=-4.0, q_max=16.0,
             V_LL=0.1, V_SL=0.05, mu1=1.0, mu2=0.0036, K_pade=1)
    model = {"modes": [m], "pairs": [], "T_K": 300.0, "depth_L": 6}
    return model, grid(0.5, 8, 64, 64, (0.0,), t_eq_fs=200.0)


def c2():
    """Three water-like Morse modes, 4 levels each (d = 64), one Pade term per
    mode (6 exponentials), depth 4 -> 210 ADOs; 128x128 grid, t2 in {0, 100} fs."""
    return water_model(4, 4), grid(0.5, 8, 128, 128, (0.0, 100.0), t_eq_fs=200.0)


def c3():
    """Same three modes at 5 levels (d = 125), depth 6 -> 924 ADOs; all 128 t1
    branches per pathway propagated together in mixed precision; t2 = 0."""
    return water_model(5, 6), grid(0.5, 8, 128, 128, (0.0,), t_eq_fs=200.0)


def c4():
    """The c2 model on a 64x64 grid at t2 = 0 (gradient workload)."""
    return water_model(4, 4), grid(0.5, 8, 64, 64, (0.0,), t_eq_fs=200.0)


def c5():
    """Three modes at 6 levels (d = 216), two Pade terms per mode (9 exponentials),
    depth 8 -> 24310 ADOs; dt 0.25 fs, m = 16, 256x256 grid, t2 in {0, 50, 200} fs."""
    return (water_model(6, 8, K_pade=2),
            grid(0.25, 16, 256, 256, (0.0, 50.0, 200.0), t_eq_fs=200.0))


def c5_batch(n_sets=16, seed=2605):
    """The c5 batch of parameter sets with uneven basis sizes: per set, every mode
    gets n_s levels drawn from {4, 5, 6}, and its anharmonicity, V_SL and gamma and
    each pair's cubic couplings a factor 1 + 0.05 U(-1, 1) (seeded).  Returns a
    list of model dicts (the grid is c5's)."""
    rng = np.random.default_rng(seed)
    base, _ = c5()
    out = []
    for _ in range(n_sets):
        m = copy.deepcopy(base)
        for md in m["modes"]:
            md["n_levels"] = int(rng.choice([4, 5, 6]))
            for key in ("morse_D_cm", "V_SL", "gamma_cm"):
                md[key] = float(md[key] * (1 + 0.05 * rng.uniform(-1, 1)))
        for pr in m["pairs"]:
            for key in ("g_s2t_cm", "g_st2_cm"):
                pr[key] = float(pr[key] * (1 + 0.05 * rng.uniform(-1, 1)))
        out.append(m)
    return out


# ---------------------------------------------------------------------------
# The paper's own water parameter sets (Sec. IV, Tables (i), (ii) and FitAll2)
# ---------------------------------------------------------------------------
# The tables give dimensionless ("tilde") values against the unit frequency
# omega_0 = 4000 cm^-1.  Readings (the printed normalisations are partly garbled):
#   * omega_s = nu_s (the table's frequency column); gamma_s = (gamma_s/omega_0) omega_0.
#   * zeta_s = zeta~_s (nu_s/omega_0)^2 omega_0 (the printed definition solved for zeta_s).
#   * V_LL = V~_LL omega_0/nu_s (zero in every table), V_SL = V~_SL.
#   * Every power of q_s in a potential or dipole term carries one factor nu_s/omega_0:
#     g_{s^3} = g~ (nu_s/omega_0)^3 omega_0, g_{ss'} = g~ (nu_s nu_s'/omega_0^2) omega_0,
#     g_{s^2 s'} = g~ (nu_s/omega_0)^2 (nu_s'/omega_0) omega_0, g_{s s'^2} likewise,
#     mu_s = mu~_s nu_s/omega_0, mu_ss = mu~_ss (nu_s/omega_0)^2, mu_ss' = mu~_ss' nu_s nu_s'/omega_0^2
#     (mu in units of the paper's undefined mu_0; spectra are compared after normalisation).
#     The mu_ss relation is the printed one; the printed g_{s^3} relation is the inverse,
#     which puts the lowest four levels of the unbounded cubic wells far outside the
#     harmonic range (bend fundamental above 1e5 cm^-1), whereas this reading puts the
#     stretch fundamental at 3398 cm^-1, where the paper places its diagonal peak.
#   * The two-mode caption's pair entries, written with the index 1', belong to the
#     stretch-bend pair (1, 2); FitAll2's "-2,6 x 10^-2" is -2.6e-2.
#   * T = 300 K (not printed); cubic modes in a harmonic basis of 16 states (the four
#     kept levels converge to 1 cm^-1 there, and no state of the unbounded side of the
#     cubic enters; a much larger primitive basis finds such states first).
PAPER_OMEGA0_CM = 4000.0
# Table (i), two-mode model, rows (1) stretch and (2) bend:
#   nu_s (cm^-1), gamma_s/omega_0, zeta~, V~_LL, V~_SL, g~_{s^3}, mu~_s, mu~_ss
PAPER_TABLE_I = ((3520.0, 5.0e-3, 9.0, 0.0, 1.0, -5.0e-1, 3.3, 1.2e-2),
                 (1710.0, 2e-2, 0.8, 0.0, 1.0, -7e-1, 1.8, 0.0))
# its caption's pair entries: g~_ss' (not given: 0), g~_{s^2 s'}, g~_{s s'^2}, mu~_ss'
PAPER_TABLE_I_PAIRS = {(0, 1): (0.0, 0.0, 0.2, 2.0e-3)}
# Table (ii), three-mode model, rows (1) asymmetric stretch, (1') symmetric stretch, (2) bend
PAPER_TABLE_II = ((3570.0, 5.0e-3, 9.0, 0.0, 1.0, -5.0e-1, 3.3, 1.2e-2),
                  (3470.0, 5.0e-3, 9.0, 0.0, 1.0, -5.0e-1, 3.3, 1.2e-2),
                  (1710.0, 2e-2, 0.8, 0.0, 1.0, -7e-1, 1.8, 0.0))
# Table FitAll2, pairs 1-1', 1-2, 1'-2: g~_ss', g~_{s^2 s'}, g~_{s s'^2}, mu~_ss'
PAPER_FITALL2 = {(0, 1): (-5e-3, 0.32, -4.2e-3, 0.0),
                 (0, 2): (1e-7, -2.6e-2, 4e-4, 2.0e-3),
                 (1, 2): (-8e-4, 1.2e-1, -1.2e-2, 2.0e-3)}


def paper_water_model(n_modes=2, n_levels=4, depth_L=3, K_pade=1, n_prim=16, T_K=300.0):
    """The paper's two-mode (Table (i)) or three-mode (Tables (ii) and FitAll2)
    water model with cubic potentials, read as stated above."""
    rows, prs = ((PAPER_TABLE_I, PAPER_TABLE_I_PAIRS) if n_modes == 2 else
                 (PAPER_TABLE_II, PAPER_FITALL2))
    w0 = PAPER_OMEGA0_CM
    modes = []
    for nu, gam, zt, vll, vsl, g3, mu, muss in rows:
        r = nu / w0
        md = mode("cubic", nu, g3_cm=g3 * r ** 3 * w0, n_levels=n_levels, n_prim=n_prim,
                  gamma_cm=gam * w0, V_LL=vll / r, V_SL=vsl, mu1=mu * r, mu2=muss * r ** 2,
                  K_pade=K_pade)
        md["zeta_cm"] = float(zt * r ** 2 * w0)
        modes.append(md)
    pairs = []
    for (s, t), (g, g21, g12, mst) in sorted(prs.items()):
        rs, rt = rows[s][0] / w0, rows[t][0] / w0
        pairs.append(pair(s, t, g * rs * rt * w0, g21 * rs ** 2 * rt * w0, g12 * rs * rt ** 2 * w0,
                          mst * rs * rt))
    return {"modes": modes, "pairs": pairs, "T_K": float(T_K), "depth_L": int(depth_L)}


def paper_water_grid(n=128, t2_fs=(0.0, 50.0, 100.0)):
    """2D grid for the paper's water demonstrations: dt = 0.25 fs (the paper's three-mode
    step), samples every 4 fs (m = 16; Nyquist 4170 cm^-1, above the stretch band),
    n x n samples, t2 = 0, 50 and 100 fs."""
    return grid(0.25, 16, n, n, t2_fs, t_eq_fs=200.0)


CONFIGS = {"c1": c1, "c2": c2, "c3": c3, "c4": c4, "c5": c5}


def config(name):
    model, g = CONFIGS[name]()
    return copy.deepcopy(model), copy.deepcopy(g)


# ---------------------------------------------------------------------------
# Small models for tests (all seeded / explicit)
# ---------------------------------------------------------------------------
def harmonic_bo(omega_cm=1000.0, n_levels=10, lambda_cm=50.0, gamma_cm=200.0, depth_L=3,
                K_pade=1, T_K=300.0, mu1=1.0):
    """One harmonic mode, LL coupling only, linear dipole (Brownian oscillator)."""
    m = mode("cubic", omega_cm, g3_cm=0.0, n_levels=n_levels, n_prim=n_levels,
             lambda_cm=lambda_cm, gamma_cm=gamma_cm, V_LL=1.0, V_SL=0.0, mu1=mu1, mu2=0.0,
             K_pade=K_pade)
    return {"modes": [m], "pairs": [], "T_K": float(T_K), "depth_L": int(depth_L)}


def small_two_mode(n1=3, n2=3, depth_L=2, K_pade=1, seed=7):
    """Two coupled anharmonic modes (one Morse, one cubic) with LL+SL coupling,
    quadratic dipoles and a random cubic pair coupling; d = n1*n2."""
    rng = np.random.default_rng(seed)
    g = rng.uniform(-60.0, 60.0, size=3)
    m0 = mode("morse", 3400.0, D_cm=3.0e4, n_levels=n1, n_prim=160, q_min=-5.0, q_max=11.0,
              V_LL=0.15, V_SL=0.4, mu1=1.0, mu2=0.01, K_pade=K_pade)
    m1 = mode("cubic", 1650.0, g3_cm=-120.0, n_levels=n2, n_prim=n2 + 8, lambda_cm=40.0,
              gamma_cm=150.0, V_LL=0.2, V_SL=0.3, mu1=0.6, mu2=0.0, K_pade=K_pade)
    return {"modes": [m0, m1], "pairs": [pair(0, 1, g[0], g[1], g[2], 0.002)],
            "T_K": 300.0, "depth_L": int(depth_L)}


def small_three_mode(n=2, depth_L=2, K_pade=1):
    """Scaled-down water model: three Morse modes with ``n`` levels each."""
    return water_model(n, depth_L, K_pade=K_pade, n_prim=160)
