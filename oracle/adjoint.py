"""Oracle: the 2D-spectrum misfit and its gradient by central differences.

Test infrastructure only (see the package docstring).

The loss follows the inverse-problem use of the 2D correlation spectrum: the
squared L2 misfit between the model's S_C (Eq. correlation-spectrum, every t2 of
the grid) and a reference spectrum on the same grid,

    loss(theta) = sum_{t2, p, q} (S_C(theta)[t2, p, q] - S_ref[t2, p, q])^2 .

theta holds twelve fields of the model description (the parameters the paper's
fits vary: anharmonicities, mode-mode couplings, system-bath coupling strengths
and bath damping), in this order:

    0-2   anharmonicity of mode s: Morse depth D_s (morse) or cubic g3_s (cubic)
    3-5   cubic mode-mode coupling g_{s^2 t} of pair p (pairs in model order)
    6-8   square system-bath coupling strength V_SL of mode s
    9-11  Drude damping gamma_s of mode s (zeta_s held fixed, so the
          reorganisation energy lambda_s = zeta_s gamma_s / (2 omega_s) moves with it)

Entries for modes or pairs the model does not have are ignored (gradient 0).

The gradient is the definition itself, evaluated by second-order central
differences with step h_i = rel * max(|theta_i|, 1): every loss evaluation runs
the whole oracle procedure (equilibration over the grid's t_eq, both pathways,
Fourier sums).  Pins (tests/test_oracle_adjoint.py): the error of the difference
quotient falls as h^2 (ratio ~4 per halving), and for the harmonic Brownian
oscillator the gamma-derivative of the linear response matches the derivative
of its closed form.
"""
import copy

import numpy as np

from . import heom as OH
from . import model as OM

N_THETA = 12


def _slot(model, i):
    """(container, key) of theta_i in ``model``, or None if the model lacks it."""
    modes, pairs = model["modes"], model["pairs"]
    grp, k = divmod(i, 3)
    if grp == 1:
        return (pairs[k], "g_s2t_cm") if k < len(pairs) else None
    if k >= len(modes):
        return None
    md = modes[k]
    if grp == 0:
        return (md, "morse_D_cm") if md["potential"] == "morse" else (md, "g3_cm")
    return (md, "V_SL") if grp == 2 else (md, "gamma_cm")


def theta_of(model):
    """The twelve parameters of ``model`` (0 where it has no such field)."""
    th = np.zeros(N_THETA)
    for i in range(N_THETA):
        s = _slot(model, i)
        if s is not None:
            th[i] = s[0][s[1]]
    return th


def with_theta(model, theta):
    """Copy of ``model`` with its parameter fields set from ``theta``."""
    out = copy.deepcopy(model)
    for i in range(N_THETA):
        s = _slot(out, i)
        if s is not None:
            s[0][s[1]] = float(theta[i])
    return out


def spectrum(model, grid):
    """S_C [n_t2][n1][n3] of the whole 2D procedure (Sec. II.C.2)."""
    _, _, _, S = OH.spectrum_2d(OM.Problem(model), grid)
    return S


def loss(model, grid, S_ref):
    """Squared L2 misfit of S_C against S_ref over every t2 and frequency pair."""
    return float(np.sum((spectrum(model, grid) - S_ref) ** 2))


def grad_fd(model, grid, S_ref, rel=1e-4, which=None):
    """Central-difference gradient of ``loss`` with respect to theta.

    Returns (g, h): g[i] = (loss(theta + h_i e_i) - loss(theta - h_i e_i)) / (2 h_i)
    for the entries in ``which`` (default: every entry the model has), 0 elsewhere.
    """
    th = theta_of(model)
    g = np.zeros(N_THETA)
    h = rel * np.maximum(np.abs(th), 1.0)
    idx = [i for i in range(N_THETA) if _slot(model, i) is not None]
    if which is not None:
        idx = [i for i in idx if i in which]
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h[i]
        tm[i] -= h[i]
        g[i] = (loss(with_theta(model, tp), grid, S_ref) - loss(with_theta(model, tm), grid, S_ref)) / (2 * h[i])
    return g, h
