"""The paper's own water parameter sets (Sec. IV, Tables (i), (ii), FitAll2) on the GPU.

  * Reduced grids: the FP64 path against the oracle (R_I, R_II and S_C to 1e-10 of
    their largest magnitude) for the two-mode and three-mode tables with cubic
    potentials and four levels per mode.
  * The two-level closed form of the correlation spectrum (see
    test_oracle_water.py) through the C ABI.
  * The qualitative feature the paper describes for the two-mode stretch region:
    the 0 -> 1 -> 0 pathway on the diagonal and the 0 -> 1 -> 2 pathway at lower
    Omega_3 (by the anharmonic shift) with opposite signs.  Under the printed
    Eqs. RFTIRI to correlation-spectrum the 0 -> 1 -> 0 feature is negative (the
    closed form), so the test asks for a negative diagonal extremum in the stretch
    band and, on its Omega_1 row, a positive one 1 to 8 frequency bins lower (32.6 to
    260 cm^-1 on the 256 x 256 grid of 4 fs samples).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import heom as OH
from oracle import model as OM

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2601_20550_gb300.heom")

C_CM_PER_FS = 2.99792458e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import os
    if not os.path.exists(H.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()


@pytest.mark.parametrize("n_modes, depth_L, n, t2", [(2, 2, 12, (0.0, 50.0, 100.0)), (3, 1, 6, (0.0, 50.0))])
def test_paper_tables_fp64_against_oracle(n_modes, depth_L, n, t2):
    model = W.paper_water_model(n_modes, depth_L=depth_L)
    grid = W.paper_water_grid(n, t2)
    _, _, RI, RII, SC = H.spectrum_2d(model, grid, H.FP64)
    _, RIo, RIIo, SCo = OH.spectrum_2d(OM.Problem(model), grid)
    scale = max(np.abs(RIo).max(), np.abs(RIIo).max())
    assert np.abs(RI - RIo).max() < 1e-10 * scale
    assert np.abs(RII - RIIo).max() < 1e-10 * scale
    assert np.abs(SC - SCo).max() < 1e-10 * np.abs(SCo).max()


def test_two_level_closed_form_through_the_library():
    N, dtau, p0, mu1 = 16, 4.0, 3, 1.3
    md = W.mode("cubic", p0 / (N * dtau * C_CM_PER_FS), g3_cm=0.0, n_levels=2, n_prim=2, mu1=mu1)
    md["zeta_cm"] = 0.0
    model = {"modes": [md], "pairs": [], "T_K": 300.0, "depth_L": 1}
    _, _, _, _, SC = H.spectrum_2d(model, W.grid(0.125, 32, N, N, (0.0, 8.0), t_eq_fs=4.0), H.FP64)
    a = np.full(N, -0.5)
    a[0] = N - 0.5
    q = np.arange(N)
    ref = -4.0 * (mu1 / math.sqrt(2.0)) ** 4 * dtau ** 2 * np.outer(a[(q - p0) % N], a[(q - p0) % N])
    assert np.abs(SC - ref).max() < 1e-5 * np.abs(ref).max()


def stretch_features(S, om):
    """Negative extremum of S in the stretch window, and the positive extremum on its
    Omega_1 row at lower Omega_3."""
    sel = np.where((om > 3200.0) & (om < 3700.0))[0]
    sub = S[np.ix_(sel, sel)]
    i, j = np.unravel_index(np.argmin(sub), sub.shape)
    q, p = sel[i], sel[j]
    below = np.arange(max(p - 12, 0), p)
    k = below[np.argmax(S[q, below])]
    return q, p, k


@pytest.mark.parametrize("depth_L", [4])
def test_two_mode_stretch_pathway_signs(depth_L):
    model = W.paper_water_model(2, depth_L=depth_L)
    grid = W.paper_water_grid(256, (0.0, 50.0, 100.0))
    _, _, _, _, SC = H.spectrum_2d(model, grid, H.FP64)
    n = grid["n1"]
    om = np.arange(n) / (n * 4.0 * C_CM_PER_FS)
    for it in range(len(grid["t2_fs"])):
        S = SC[it]
        q, p, k = stretch_features(S, om)
        neg, pos = S[q, p], S[q, k]
        print("L=%d t2=%g: diagonal %.3g at (%.0f, %.0f), below %.3g at Omega_3 = %.0f"
              % (depth_L, grid["t2_fs"][it], neg, om[q], om[p], pos, om[k]))
        assert neg < 0 and abs(p - q) <= 1           # 0 -> 1 -> 0 on the diagonal
        assert pos > 0.3 * abs(neg)                  # 0 -> 1 -> 2, opposite sign
        assert 1 <= p - k <= 8                       # at lower Omega_3 by the anharmonic shift
