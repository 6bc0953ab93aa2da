"""Oracle: HEOM right-hand side, RK4, equilibrium, kicks, traces and spectra.

Test infrastructure only (see the package docstring).  FP64, dense matrices,
a plain Python loop over hierarchy elements.  States are complex arrays of
shape (B, N_ADO, d, d): B independent branches (a batch of the same linear
problem), ADOs in the canonical order of ``model.Hierarchy``.

Pins (tests/test_oracle_heom.py, tests/test_oracle_physics.py):
  * rhs, rk4_step: one step equals sum_{j<=4} (dt L)^j/j! with an independently
    assembled sparse Liouvillian; convergence to expm at O(dt^4).
  * rhs invariants: tr rho_0 conserved, Hermiticity preserved.
  * response_1d: harmonic Brownian oscillator closed form; zero-bath closed form.
  * response_2d: zero-bath Liouville-pathway closed form (eigenbasis); vanishing
    third-order response of the harmonic oscillator; one-sided kicks on |0><0|.
  * equilibrate: thermal <q^2> of a low-frequency oscillator (Matsubara / Pade sum);
    null vector of the Liouvillian.
  * steady_state: the null vector of the independently assembled Liouvillian and the
    long-time limit of the propagation.
  * dft2d / correlation spectrum: brute-force single-frequency signals.
"""
import math

import numpy as np


def comm(A, X):
    """A^x X = A X - X A (Sec. II.B hyperoperators)."""
    return A @ X - X @ A


def acomm(A, X):
    """A^o X = A X + X A."""
    return A @ X + X @ A


def rhs_one(prob, get, i):
    """Eq. HEOM_DB for ADO i alone; get(k) returns ADO k of every branch, shape (B, d, d).

    d rho_n/dt = -(i H_S'^x + sum_j n_j nu_j) rho_n
                 - i sum_j n_j Theta_j rho_{n - e_j}
                 - i sum_j V_{s(j)}^x rho_{n + e_j},
    with Theta_j = a_j V^x + b_j V^o (Eqs. Pade1, Pade2) and rho = 0 outside the
    index set.
    """
    sysm, bath, hier = prob.sys, prob.bath, prob.hier
    n = hier.n[i]
    r = get(i)
    decay = sum(n[j] * bath.nu[j] for j in range(hier.D))
    acc = -1j * comm(sysm.H, r) - decay * r
    for j in range(hier.D):
        Vs = sysm.V[bath.mode_of[j]]
        dn = hier.down(i, j)
        if dn >= 0:
            rd = get(dn)
            theta = bath.a[j] * comm(Vs, rd) + bath.b[j] * acomm(Vs, rd)
            acc = acc - 1j * n[j] * theta
        up = hier.up(i, j)
        if up >= 0:
            acc = acc - 1j * comm(Vs, get(up))
    return acc


def rhs(prob, rho):
    """Eq. HEOM_DB for every ADO of every branch (``rhs_one`` over the index set)."""
    out = np.empty_like(rho)
    for i in range(prob.nado):
        out[:, i] = rhs_one(prob, lambda k: rho[:, k], i)
    return out


def rk4_step(prob, rho, dt):
    """Classic fourth-order Runge-Kutta step (Sec. III: 'Runge-Kutta method')."""
    k1 = rhs(prob, rho)
    k2 = rhs(prob, rho + 0.5 * dt * k1)
    k3 = rhs(prob, rho + 0.5 * dt * k2)
    k4 = rhs(prob, rho + dt * k3)
    return rho + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def propagate(prob, rho, dt, n_steps):
    for _ in range(n_steps):
        rho = rk4_step(prob, rho, dt)
    return rho


def initial_state(prob, branches=1):
    """rho_{n=0} = |0><0| (product ground state), all other ADOs zero (Sec. II.C.1)."""
    rho = np.zeros((branches, prob.nado, prob.d, prob.d), dtype=complex)
    rho[:, 0, 0, 0] = 1.0
    return rho


def equilibrate(prob, dt, t_eq_fs=None, tol=None, t_max_fs=None, check_every=100):
    """Propagate the factorised initial state to equilibrium (Sec. II.C.1).

    Either a fixed time ``t_eq_fs`` (round(t_eq/dt) steps), or until
    max_n ||RHS(rho)_n||_F <= tol * ||rho_0||_F, checked every ``check_every``
    steps, up to ``t_max_fs``.  Returns (rho_eq, steps_taken, converged).
    """
    rho = initial_state(prob)
    if t_eq_fs is not None:
        n = int(round(t_eq_fs / dt))
        return propagate(prob, rho, dt, n), n, True
    n_max = int(round(t_max_fs / dt))
    steps = 0
    while steps < n_max:
        rho = propagate(prob, rho, dt, min(check_every, n_max - steps))
        steps += min(check_every, n_max - steps)
        f = rhs(prob, rho)
        res = max(np.linalg.norm(f[0, i]) for i in range(prob.nado))
        if res <= tol * np.linalg.norm(rho[0, 0]):
            return rho, steps, True
    return rho, steps, False


def steady_state(prob):
    """Stationary hierarchy by a direct solve (alternative to the propagation of Sec. II.C.1).

    The definition written out: L x = 0 with tr x_0 = 1, where L is the
    right-hand side of Eq. HEOM_DB as a matrix on vec(rho).  L is built column by
    column from ``rhs`` applied to unit states (tiny problems only), the first
    equation is replaced by the trace condition, and the dense system is solved.
    """
    shape = (1, prob.nado, prob.d, prob.d)
    n = prob.nado * prob.d * prob.d
    L = np.zeros((n, n), dtype=complex)
    e = np.zeros(n, dtype=complex)
    for k in range(n):
        e[k] = 1.0
        L[:, k] = rhs(prob, e.reshape(shape)).reshape(n)
        e[k] = 0.0
    A = L.copy()
    b = np.zeros(n, dtype=complex)
    A[0, :] = 0.0
    for a in range(prob.d):
        A[0, a * prob.d + a] = 1.0
    b[0] = 1.0
    return np.linalg.solve(A, b).reshape(shape)


def kick(rho, M):
    """(M)^x applied to every ADO of every branch (Sec. II.C procedure)."""
    return M @ rho - rho @ M


def trace_mu(prob, rho):
    """tr{mu rho_0} for every branch (n = 0 element only)."""
    return np.einsum("ab,zba->z", prob.sys.mu, rho[:, 0])


def pathway_kicks(prob, pathway):
    """One-sided dipoles for the rephasing (I) and non-rephasing (II) signals.

    R_I : kicks mu_minus, mu_plus, mu_plus  (k_I = k3 + k2 - k1)
    R_II: kicks mu_plus, mu_minus, mu_plus  (k_II = k3 - k2 + k1)
    (Eqs. echo, virtual-echo, read through excitation manifolds: mu_plus raises
    the total excitation number, mu_minus lowers it.)
    """
    mp, mm = prob.sys.mu_plus, prob.sys.mu_minus
    return (mm, mp, mp) if pathway == "I" else (mp, mm, mp)


def response_2d(prob, rho_eq, grid):
    """R_I and R_II on the (t2, t1, t3) grid (Eqs. RFTIRI, echo, virtual-echo).

    R(t3, t2, t1) = i^3 tr{mu G(t3) K3^x G(t2) K2^x G(t1) K1^x rho_eq}, with
    t1 = j*m*dt (j < n1), t3 = k*m*dt (k < n3), t2 from grid["t2_fs"] (a multiple
    of dt).  The t1 branches are carried as a batch.  Returns complex arrays
    R_I, R_II of shape (n_t2, n1, n3).
    """
    dt, m = grid["dt_fs"], grid["steps_per_sample"]
    n1, n3 = grid["n1"], grid["n3"]
    t2s = grid["t2_fs"]
    order = np.argsort(t2s)
    out = {}
    for pw in ("I", "II"):
        K1, K2, K3 = pathway_kicks(prob, pw)
        R = np.zeros((len(t2s), n1, n3), dtype=complex)
        trunk = kick(rho_eq, K1)
        snaps = []
        for j in range(n1):
            if j > 0:
                trunk = propagate(prob, trunk, dt, m)
            snaps.append(trunk[0])
        rho2 = kick(np.stack(snaps), K2)
        t_now = 0
        for it in order:
            n2 = int(round(t2s[it] / dt))
            rho2 = propagate(prob, rho2, dt, n2 - t_now)
            t_now = n2
            rho3 = kick(rho2, K3)
            for k in range(n3):
                if k > 0:
                    rho3 = propagate(prob, rho3, dt, m)
                R[it, :, k] = (1j) ** 3 * trace_mu(prob, rho3)
        out[pw] = R
    return out["I"], out["II"]


def dft2d(R, dtau):
    """Trapezoid double Fourier sum of Eqs. 2D-rephasing / 2D-nonrephasing.

    S(q, p) = Im[ dtau^2 sum_{b,a} w_b w_a exp(+i (Omega1_q t1_b + Omega3_p t3_a)) R[b, a] ]
    with t_j = j dtau, w_0 = 1/2, w_j = 1 otherwise, Omega_p = 2 pi p / (N dtau).
    R has shape (n1, n3); S has shape (n1, n3) indexed [Omega1 index q, Omega3 index p].
    """
    n1, n3 = R.shape
    w1 = np.ones(n1)
    w1[0] = 0.5
    w3 = np.ones(n3)
    w3[0] = 0.5
    S = np.zeros((n1, n3))
    for q in range(n1):
        for p in range(n3):
            ph1 = np.exp(2j * math.pi * q * np.arange(n1) / n1)
            ph3 = np.exp(2j * math.pi * p * np.arange(n3) / n3)
            S[q, p] = (dtau ** 2 * np.sum(np.outer(w1 * ph1, w3 * ph3) * R)).imag
    return S


def correlation_spectrum(R_I, R_II, dtau):
    """S_C(Omega3, Omega1) = S_R(Omega3, -Omega1) + S_NR(Omega3, Omega1).

    Eq. correlation-spectrum; -Omega1_q is the index (n1 - q) mod n1.  Inputs of
    shape (n_t2, n1, n3); returns S_C, S_R, S_NR of the same shape.
    """
    nt2, n1, n3 = R_I.shape
    SR = np.stack([dft2d(R_I[i], dtau) for i in range(nt2)])
    SNR = np.stack([dft2d(R_II[i], dtau) for i in range(nt2)])
    flip = (-np.arange(n1)) % n1
    SC = SR[:, flip, :] + SNR
    return SC, SR, SNR


def response_1d(prob, rho_eq, dt, m, n):
    """R^(1)(t) = i tr{mu G(t) mu^x rho_eq} at t = k*m*dt, k < n (Eq. R1)."""
    rho = kick(rho_eq, prob.sys.mu)
    out = np.zeros(n, dtype=complex)
    for k in range(n):
        if k > 0:
            rho = propagate(prob, rho, dt, m)
        out[k] = 1j * trace_mu(prob, rho)[0]
    return out


def spectrum_2d(prob, grid):
    """Whole 2D procedure: equilibrate, R_I/R_II, S_C (Sec. II.C.2)."""
    rho_eq, _, _ = equilibrate(prob, grid["dt_fs"], t_eq_fs=grid["t_eq_fs"])
    R_I, R_II = response_2d(prob, rho_eq, grid)
    dtau = grid["dt_fs"] * grid["steps_per_sample"]
    S_C, _, _ = correlation_spectrum(R_I, R_II, dtau)
    return rho_eq, R_I, R_II, S_C
