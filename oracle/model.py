"""Oracle: the MAB model as matrices, the Drude/Pade bath and the hierarchy.

Test infrastructure only (see the package docstring).  FP64 throughout.

Units: hbar = 1, time in fs, energies as angular frequencies in rad/fs.  The
mode coordinates q_s are dimensionless with mass m_s = 1/omega_s, so that the
harmonic part of Eq. Potentials reads omega_s*(p^2 + q^2)/2.

Pins (tests/test_oracle_model.py):
  * Morse levels against the closed form E_n = w(n+1/2) - w^2/(4D) (n+1/2)^2.
  * Harmonic basis: q, q^2 matrix elements against sqrt((n+1)/2), n+1/2.
  * Pade coefficients: N = 1 by hand (xi = sqrt(60), eta = 5/2); matching of the
    Bernoulli series to order 2N; convergence to the Matsubara values 2*pi*k.
  * Bath coefficients: the Drude correlation function by direct quadrature.
  * Hierarchy size C(L+D, D) and neighbour consistency by brute force.
  * System (tests/test_oracle_couplings.py): V_s and the counter term Lambda <V_s^2>
    for V_SL != 0 against ladder-operator matrix elements (V^2 squared in a larger
    basis); the square-linear pure-dephasing closed form; the quadratic and
    cross-mode dipole terms through the zero-bath linear response.
  * Physics (tests/test_oracle_physics.py): LL coupling relaxes and SL coupling
    dephases; the equilibrium converges on the ground state as Pade terms are added
    (quanta far above kT).
  * The paper's water tables (tests/test_oracle_water.py): the printed numbers
    (tests/golden/paper_water_tables.txt), the stretch fundamental at the paper's
    diagonal peak, three- and four-level linear spectra nearly identical.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import sympy

# 1 cm^-1 as an angular frequency in rad/fs: 2*pi*c with c = 2.99792458e-5 cm/fs.
CM_TO_RADFS = 2.0 * math.pi * 2.99792458e-5
# Boltzmann constant in cm^-1 / K (CODATA 2018).
KB_CM_PER_K = 0.6950348005


# ---------------------------------------------------------------------------
# Mode eigenbases (Eqs. System Hamiltonian, Potentials; Sec. II.A eigenstates)
# ---------------------------------------------------------------------------
def _fix_signs(U, q):
    """Sign convention for the kept eigenvectors (columns of U).

    Ground state: its largest-magnitude component is positive.  Excited state n:
    <n-1|q|n> > 0.  Both conventions are interface choices (results that are
    traces do not depend on them); the library uses the same ones.
    """
    U = U.copy()
    i0 = np.argmax(np.abs(U[:, 0]))
    if U[i0, 0] < 0:
        U[:, 0] = -U[:, 0]
    for n in range(1, U.shape[1]):
        if U[:, n - 1] @ q @ U[:, n] < 0:
            U[:, n] = -U[:, n]
    return U


def morse_basis(omega, D, q_min, q_max, n_prim, n_levels):
    """Lowest ``n_levels`` eigenstates of H = omega p^2/2 + D (1 - exp(-a q))^2.

    a = sqrt(omega / (2 D)) makes the harmonic limit omega q^2 / 2.  The
    Hamiltonian is represented on a uniform sinc-DVR grid of ``n_prim`` points
    spanning [q_min, q_max] (Colbert and Miller, JCP 96, 1982 (1992)): kinetic
    matrix (omega/2)/dx^2 * (-1)^(i-j) * (pi^2/3 if i == j else 2/(i-j)^2) and a
    diagonal potential.  Returns energies E[n] and the matrices of q^k
    (k = 1..4) in the kept eigenbasis, projected from the grid operators.
    """
    a = math.sqrt(omega / (2.0 * D))
    x = np.linspace(q_min, q_max, n_prim)
    dx = x[1] - x[0]
    T = np.zeros((n_prim, n_prim))
    for i in range(n_prim):
        for j in range(n_prim):
            if i == j:
                T[i, j] = math.pi ** 2 / 3.0
            else:
                T[i, j] = (-1.0) ** (i - j) * 2.0 / (i - j) ** 2
    T *= 0.5 * omega / dx ** 2
    Hm = T + np.diag(D * (1.0 - np.exp(-a * x)) ** 2)
    E, U = np.linalg.eigh(Hm)
    qprim = np.diag(x)
    U = _fix_signs(U[:, :n_levels], qprim)
    qk = {k: U.T @ np.diag(x ** k) @ U for k in (1, 2, 3, 4)}
    return E[:n_levels].copy(), qk


def cubic_basis(omega, g3, n_prim, n_levels):
    """Lowest eigenstates of omega (p^2 + q^2)/2 + g3 q^3 / 6 in a harmonic basis.

    The primitive basis is the first ``n_prim`` harmonic-oscillator states, with
    q = (a + a^dagger)/sqrt(2).  q^k (k <= 4) is projected exactly onto that
    basis by forming it in a basis 4 states larger and truncating.
    """
    M = n_prim + 4
    ann = np.diag(np.sqrt(np.arange(1, M, dtype=float)), 1)
    qM = (ann + ann.T) / math.sqrt(2.0)
    qpow = {1: qM}
    for k in (2, 3, 4):
        qpow[k] = qpow[k - 1] @ qM
    proj = {k: qpow[k][:n_prim, :n_prim] for k in qpow}
    Hm = omega * np.diag(np.arange(n_prim) + 0.5) + (g3 / 6.0) * proj[3]
    E, U = np.linalg.eigh(Hm)
    U = _fix_signs(U[:, :n_levels], proj[1])
    qk = {k: U.T @ proj[k] @ U for k in proj}
    return E[:n_levels].copy(), qk


def mode_basis(md):
    """Energies (rad/fs) and q^k matrices for one mode dictionary."""
    w = md["omega_cm"] * CM_TO_RADFS
    if md["potential"] == "morse":
        return morse_basis(w, md["morse_D_cm"] * CM_TO_RADFS, md["q_min"], md["q_max"],
                           md["n_prim"], md["n_levels"])
    if md["potential"] == "cubic":
        return cubic_basis(w, md["g3_cm"] * CM_TO_RADFS, md["n_prim"], md["n_levels"])
    raise ValueError("unknown potential %r" % md["potential"])


# ---------------------------------------------------------------------------
# Product basis and the system operators (Eqs. Total Hamiltonian .. sys_interaction)
# ---------------------------------------------------------------------------
def embed(ops, dims):
    """Kronecker product I x .. x ops[s] x .. x I; mode 0 is the slowest index."""
    out = np.ones((1, 1))
    for s, n in enumerate(dims):
        out = np.kron(out, ops.get(s, np.eye(n)))
    return out


class System:
    """H_S' (with counter terms), V_s, mu and the raising/lowering parts of mu.

    * H_S' = sum_s H_A^(s) + sum_{s<s'} U_ss' + sum_s Lambda_s V_s^2
      (Eqs. Total Hamiltonian, Potential ss', counter Hamiltonian, counter2), with
      H_A^(s) diagonal in its own eigenbasis and every U_ss' and V_s^2 element kept.
    * V_s = V_LL q_s + V_SL q_s^2 / 2 (Eq. h_int).
    * Lambda_s = m_s zeta_s gamma_s / 2 = zeta_s gamma_s / (2 omega_s) (Eq. counterterm).
    * mu = sum_s mu_s q_s + (1/2) sum_{s,s'} mu_ss' q_s q_s' (Eq. NLdip), with
      mu_ss on the diagonal (mode dict "mu2") and mu_ss' = mu_s's (pair "mu_st").
    * Excitation number N = sum_s n_s of each product state; mu_plus keeps the
      elements <a|mu|b> with N(a) > N(b), mu_minus = mu_plus^T.
    """

    def __init__(self, model):
        self.model = model
        modes = model["modes"]
        self.dims = [md["n_levels"] for md in modes]
        self.d = int(np.prod(self.dims))
        self.E = []
        self.q = []
        for md in modes:
            E, qk = mode_basis(md)
            self.E.append(E)
            self.q.append(qk)
        d, dims = self.d, self.dims
        H = np.zeros((d, d))
        self.V = []
        self.Lam = []
        for s, md in enumerate(modes):
            qk = self.q[s]
            H += embed({s: np.diag(self.E[s])}, dims)
            vll, vsl = md["V_LL"], md["V_SL"]
            Vs = vll * qk[1] + 0.5 * vsl * qk[2]
            V2 = vll ** 2 * qk[2] + vll * vsl * qk[3] + 0.25 * vsl ** 2 * qk[4]
            lam = (md["zeta_cm"] * md["gamma_cm"] / (2.0 * md["omega_cm"])) * CM_TO_RADFS
            self.Lam.append(lam)
            H += lam * embed({s: V2}, dims)
            self.V.append(embed({s: Vs}, dims))
        for pr in model["pairs"]:
            s, t = pr["s"], pr["t"]
            qs, qt = self.q[s], self.q[t]
            g = pr["g_st_cm"] * CM_TO_RADFS
            g21 = pr["g_s2t_cm"] * CM_TO_RADFS
            g12 = pr["g_st2_cm"] * CM_TO_RADFS
            H += g * embed({s: qs[1], t: qt[1]}, dims)
            H += (g21 / 6.0) * embed({s: qs[2], t: qt[1]}, dims)
            H += (g12 / 6.0) * embed({s: qs[1], t: qt[2]}, dims)
        self.H = H
        mu = np.zeros((d, d))
        for s, md in enumerate(modes):
            mu += md["mu1"] * embed({s: self.q[s][1]}, dims)
            mu += 0.5 * md["mu2"] * embed({s: self.q[s][2]}, dims)
        for pr in model["pairs"]:
            s, t = pr["s"], pr["t"]
            # (1/2)(mu_st q_s q_t + mu_ts q_t q_s) with mu_ts = mu_st
            mu += pr["mu_st"] * embed({s: self.q[s][1], t: self.q[t][1]}, dims)
        self.mu = mu
        levels = np.array(list(itertools.product(*[range(n) for n in dims])))
        self.N = levels.sum(axis=1) if len(dims) else np.zeros(1, dtype=int)
        self.mu_plus = np.where(self.N[:, None] > self.N[None, :], mu, 0.0)
        self.mu_minus = self.mu_plus.T.copy()


# ---------------------------------------------------------------------------
# Pade spectrum decomposition of the Bose function (Sec. II.B, Hu-Xu-Yan [N-1/N])
# ---------------------------------------------------------------------------
def pade_bose(N):
    """Poles xi_k and weights eta_k of the [N-1/N] Pade decomposition.

    1/(1 - exp(-x)) ~ 1/x + 1/2 + sum_k 2 eta_k x / (x^2 + xi_k^2).
    Written out from the definition: with y = x^2 the remainder
    (1/(1-e^-x) - 1/x - 1/2)/x = sum_{m>=1} B_{2m}/(2m)! y^(m-1) is replaced by its
    [N-1/N] Pade approximant P(y)/Q(y), built in exact rational arithmetic from
    the first 2N series coefficients.  The roots of Q are y = -xi_k^2 and the
    residues of P/Q there are 2 eta_k.  Returns (xi, eta) sorted by xi.
    """
    if N == 0:
        return np.zeros(0), np.zeros(0)
    c = [Fraction(sympy.bernoulli(2 * m)) / math.factorial(2 * m) for m in range(1, 2 * N + 1)]
    # Unknowns q_1..q_N of Q = 1 + sum q_i y^i: coefficients N..2N-1 of Q*g vanish.
    A = sympy.zeros(N, N)
    rhs = sympy.zeros(N, 1)
    for r in range(N):
        k = N + r
        for i in range(1, N + 1):
            A[r, i - 1] = sympy.Rational(c[k - i].numerator, c[k - i].denominator)
        rhs[r] = -sympy.Rational(c[k].numerator, c[k].denominator)
    qv = A.LUsolve(rhs)
    qc = [sympy.Integer(1)] + [qv[i] for i in range(N)]
    pc = []
    for k in range(N):
        pc.append(sum(qc[i] * sympy.Rational(c[k - i].numerator, c[k - i].denominator)
                      for i in range(0, k + 1)))
    y = sympy.symbols("y")
    Q = sum(qc[i] * y ** i for i in range(N + 1))
    P = sum(pc[i] * y ** i for i in range(N))
    dQ = sympy.diff(Q, y)
    xi, eta = [], []
    for r in sympy.Poly(Q, y).nroots(n=40):
        r = sympy.re(r)
        xi.append(float(sympy.sqrt(-r)))
        eta.append(float((P.subs(y, r) / dQ.subs(y, r)) / 2))
    order = np.argsort(xi)
    return np.array(xi)[order], np.array(eta)[order]


class Bath:
    """Exponential terms of every mode's bath (Eqs. L1, L2, Pade1, Pade2).

    For mode s with K_s Pade terms there are K_s + 1 exponentials j, in the
    order (mode 0: k = 0..K_0), (mode 1: k = 0..K_1), ...  Each carries
      nu_j   : nu_0 = gamma_s, nu_k = xi_k / beta (Pade frequencies),
      a_j    : coefficient of V_s^x in Theta_j,
      b_j    : coefficient of V_s^o in Theta_j,
    with, in the paper's notation (m_s = 1/omega_s, hbar = 1),
      Theta_0 = -i (m zeta gamma^2 / 2) V^o
                + (m zeta gamma / beta) (1 + sum_k 2 eta_k gamma^2/(gamma^2 - nu_k^2)) V^x
      Theta_k = -(m zeta gamma^2 / beta) 2 eta_k nu_k / (gamma^2 - nu_k^2) V^x.
    """

    def __init__(self, model):
        kT = KB_CM_PER_K * model["T_K"] * CM_TO_RADFS
        beta = 1.0 / kT
        self.beta = beta
        self.mode_of, self.nu, self.a, self.b = [], [], [], []
        for s, md in enumerate(model["modes"]):
            w = md["omega_cm"] * CM_TO_RADFS
            zeta = md["zeta_cm"] * CM_TO_RADFS
            gam = md["gamma_cm"] * CM_TO_RADFS
            m = 1.0 / w
            xi, eta = pade_bose(md["K_pade"])
            nuk = xi / beta
            corr = 1.0 + sum(2.0 * eta[k] * gam ** 2 / (gam ** 2 - nuk[k] ** 2)
                             for k in range(len(xi)))
            self.mode_of.append(s)
            self.nu.append(gam)
            self.a.append(m * zeta * gam / beta * corr)
            self.b.append(-1j * m * zeta * gam ** 2 / 2.0)
            for k in range(len(xi)):
                self.mode_of.append(s)
                self.nu.append(nuk[k])
                self.a.append(-(m * zeta * gam ** 2 / beta) * 2.0 * eta[k] * nuk[k]
                              / (gam ** 2 - nuk[k] ** 2))
                self.b.append(0.0)
        self.D = len(self.nu)
        self.nu = np.array(self.nu)
        self.a = np.array(self.a, dtype=float)
        self.b = np.array(self.b, dtype=complex)

    def correlation(self, s, t):
        """C_s(t) = sum_j c_j exp(-nu_j t) with c_j = a_j + i * (b_j / i) for mode s.

        The operator Theta_j = Re(c_j) V^x + i Im(c_j) V^o, so Re c_j = a_j and
        Im c_j = b_j / i.  Used by the pins only.
        """
        out = 0.0 + 0.0j
        for j in range(self.D):
            if self.mode_of[j] == s:
                cj = self.a[j] + 1j * (self.b[j] / 1j).real
                out += cj * np.exp(-self.nu[j] * t)
        return out


# ---------------------------------------------------------------------------
# Hierarchy index set (Sec. II.B, Eq. HEOM_DB and the text after it)
# ---------------------------------------------------------------------------
class Hierarchy:
    """All multi-indices n in N^D with sum(n) <= L, in canonical order.

    Canonical order: ascending by (sum(n), n) with n compared as a tuple.  This
    order is part of the interface (state arrays use it).
    """

    def __init__(self, D, L):
        self.D, self.L = D, L
        idx = [n for n in itertools.product(range(L + 1), repeat=D) if sum(n) <= L]
        idx.sort(key=lambda n: (sum(n), n))
        self.n = idx
        self.index = {n: i for i, n in enumerate(idx)}

    def __len__(self):
        return len(self.n)

    def up(self, i, j):
        n = list(self.n[i])
        n[j] += 1
        return self.index.get(tuple(n), -1)

    def down(self, i, j):
        n = list(self.n[i])
        if n[j] == 0:
            return -1
        n[j] -= 1
        return self.index[tuple(n)]


class Problem:
    """Everything the HEOM needs for one model: system, bath, hierarchy."""

    def __init__(self, model):
        self.model = model
        self.sys = System(model)
        self.bath = Bath(model)
        self.hier = Hierarchy(self.bath.D, model["depth_L"])
        self.d = self.sys.d
        self.nado = len(self.hier)
