"""Pins for the 2D correlation spectrum's sign convention and the paper's water tables.

  * Two-level closed form: a mode reduced to its two lowest harmonic levels, with no
    bath, carries exactly the 0 -> 1 -> 0 pathways.  From Eqs. RFTIRI, echo and
    virtual-echo, R_I = -2 i mu01^4 exp(i w (t1 - t3)) and R_II = -2 i mu01^4
    exp(-i w (t1 + t3)), independent of t2 (the population difference is stationary).
    With w on the Fourier grid, w = 2 pi p0 / (N dtau), the trapezoid sums of Eqs.
    2D-rephasing and 2D-nonrephasing and the flip of Eq. correlation-spectrum give
        S_C(q, p) = -4 mu01^4 dtau^2 a(q - p0) a(p - p0),
        a(0) = N - 1/2,  a(x != 0 mod N) = -1/2,
    so the printed equations make the 0 -> 1 -> 0 diagonal peak negative.
  * 1D IR with three and with four levels per mode (Sec. IV.A: the paper finds the two
    representations' linear absorption spectra nearly identical): the two-mode model's
    spectra over 1000-4100 cm^-1 correlate to better than 0.99, put their peaks in the
    same frequency bins and give the same bend/stretch band ratio within 10 %.
  * The workload's table constants equal the numbers printed in Sec. IV's Tables (i),
    (ii) and FitAll2, kept as text in tests/golden/paper_water_tables.txt.
  * Table readings (workloads.paper_water_model): the isolated cubic stretch of
    Table (i) has its fundamental at the paper's diagonal stretch peak (about
    3400 cm^-1) and the bend near its 1710 cm^-1; the printed direction of the
    g_{s^3} normalisation would put the bend's lowest levels outside the cubic well.
"""
import math

import numpy as np

import workloads as W
from oracle import heom as Hm
from oracle import model as M

C_CM_PER_FS = 2.99792458e-5


def two_level_model(omega_cm, mu1):
    md = W.mode("cubic", omega_cm, g3_cm=0.0, n_levels=2, n_prim=2, mu1=mu1, K_pade=1)
    md["zeta_cm"] = 0.0
    return {"modes": [md], "pairs": [], "T_K": 300.0, "depth_L": 1}


def test_two_level_correlation_spectrum_closed_form():
    N, dtau, p0 = 16, 4.0, 3
    omega_cm = p0 / (N * dtau * C_CM_PER_FS)        # w = 2 pi p0 / (N dtau)
    mu1 = 1.3
    model = two_level_model(omega_cm, mu1)
    prob = M.Problem(model)
    grid = W.grid(0.125, 32, N, N, (0.0, 8.0), t_eq_fs=4.0)
    rho_eq, RI, RII, SC = Hm.spectrum_2d(prob, grid)
    mu01 = mu1 / math.sqrt(2.0)                    # <0|q|1> of the harmonic basis
    t = np.arange(N) * dtau
    w = omega_cm * 2.0 * math.pi * C_CM_PER_FS
    t1, t3 = np.meshgrid(t, t, indexing="ij")
    cI = -2j * mu01 ** 4 * np.exp(1j * w * (t1 - t3))
    cII = -2j * mu01 ** 4 * np.exp(-1j * w * (t1 + t3))
    for it in range(2):
        # RK4 phase error over up to 2 x 15 x 32 steps of w dt = 0.037
        assert np.abs(RI[it] - cI).max() < 1e-6 * np.abs(cI).max()
        assert np.abs(RII[it] - cII).max() < 1e-6 * np.abs(cII).max()
    a = np.full(N, -0.5)
    a[0] = N - 0.5
    q = np.arange(N)
    ref = -4.0 * mu01 ** 4 * dtau ** 2 * np.outer(a[(q - p0) % N], a[(q - p0) % N])
    for it in range(2):
        assert np.abs(SC[it] - ref).max() < 1e-5 * np.abs(ref).max()
    assert SC[0, p0, p0] < 0 and SC[0, p0, p0] == SC[0].min()


def test_paper_table_readings():
    model = W.paper_water_model(2)
    stretch, bend = model["modes"]
    E, _ = M.mode_basis(stretch)
    w01 = (E[1] - E[0]) / M.CM_TO_RADFS
    assert abs(w01 - 3400.0) < 10.0
    E, _ = M.mode_basis(bend)
    assert abs((E[1] - E[0]) / M.CM_TO_RADFS - 1710.0) < 10.0
    # the anharmonic shifts are negative and of a vibrational size (tens to hundreds of cm^-1)
    for md in (stretch, bend):
        E, _ = M.mode_basis(md)
        shift = ((E[2] - E[1]) - (E[1] - E[0])) / M.CM_TO_RADFS
        assert -400.0 < shift < -1.0
    # the printed direction of the cubic normalisation, g = g~ (omega_0/nu)^3 omega_0
    inv = dict(bend)
    inv["g3_cm"] = -0.7 * (4000.0 / 1710.0) ** 3 * 4000.0
    E, _ = M.mode_basis(inv)
    assert (E[1] - E[0]) / M.CM_TO_RADFS > 1.0e4
    # the three-mode tables build (d = 64) with every pair of FitAll2
    m3 = W.paper_water_model(3)
    assert len(m3["modes"]) == 3 and len(m3["pairs"]) == 3
    assert M.Problem(W.paper_water_model(3, depth_L=1)).d == 64


def linear_spectrum(model, n=256, dt=0.5, m=8):
    prob = M.Problem(model)
    rho, _, _ = Hm.equilibrate(prob, dt, t_eq_fs=100.0)
    R1 = Hm.response_1d(prob, rho, dt, m, n)
    dtau = dt * m
    w = np.ones(n)
    w[0] = 0.5
    om = np.arange(n) / (n * dtau * C_CM_PER_FS)
    ph = np.exp(2j * math.pi * np.outer(np.arange(n), np.arange(n)) / n)
    return om, (dtau * (ph @ (w * R1))).imag


def test_three_and_four_levels_give_nearly_the_same_linear_spectrum():
    spectra = {nl: linear_spectrum(W.paper_water_model(2, n_levels=nl, depth_L=2)) for nl in (3, 4)}
    om = spectra[3][0]
    sel = (om > 1000.0) & (om < 4100.0)
    a, b = spectra[3][1][sel], spectra[4][1][sel]
    assert np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)) > 0.99

    def peaks(x):
        big = np.abs(x) > 0.15 * np.abs(x).max()
        return [i for i in range(1, len(x) - 1) if big[i] and abs(x[i]) >= abs(x[i - 1]) and abs(x[i]) >= abs(x[i + 1])]

    assert peaks(a) == peaks(b) and len(peaks(a)) >= 1
    ratio = []
    for nl in (3, 4):
        I = spectra[nl][1]
        ratio.append(I[(om > 1400) & (om < 2000)].sum() / I[(om > 3000) & (om < 3900)].sum())
    assert ratio[0] > 0 and abs(ratio[0] - ratio[1]) < 0.1 * abs(ratio[1])



def read_golden_tables():
    """tests/golden/paper_water_tables.txt: the numbers of Sec. IV's Tables (i), (ii), FitAll2."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_water_tables.txt")
    modes, pairs, omega0 = {"i": [], "ii": []}, {"i": [], "ii": []}, None
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "omega_0":
            omega0 = float(f[1])
        elif f[0] == "mode":
            modes[f[1]].append(tuple(float(x) for x in f[3:]))
        elif f[0] == "pair":
            pairs[f[1]].append(tuple(float(x) for x in f[3:]))
    return omega0, modes, pairs


def test_workload_tables_match_the_printed_values():
    omega0, modes, pairs = read_golden_tables()
    assert omega0 == W.PAPER_OMEGA0_CM
    assert [tuple(r) for r in W.PAPER_TABLE_I] == modes["i"]
    assert [tuple(r) for r in W.PAPER_TABLE_II] == modes["ii"]
    assert [W.PAPER_TABLE_I_PAIRS[k] for k in sorted(W.PAPER_TABLE_I_PAIRS)] == pairs["i"]
    assert [W.PAPER_FITALL2[k] for k in sorted(W.PAPER_FITALL2)] == pairs["ii"]
