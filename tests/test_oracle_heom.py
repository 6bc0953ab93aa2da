"""Pins of the oracle's propagation layer (RK4, RHS invariants, equilibrium, kicks, DFT).

  * P1: on a linear ODE one classic RK4 step is the 4th-order Taylor polynomial of
    the generator; checked with a Liouvillian assembled as an explicit sparse matrix
    in Liouville space (Kronecker superoperators), and the trajectory converges to
    the matrix exponential at O(dt^4).
  * P2: tr rho_0 is conserved and Hermiticity of every ADO is preserved.
  * P8: the propagated equilibrium equals the normalised null vector of the
    Liouvillian (dense solve).
  * Kicks: the first one-sided kick on |0><0| produces only |0><N=1| coherences and
    equals -rho mu there (the worked example of the 2D procedure).
  * DFT: the trapezoid double sum equals an FFT, and a single rephasing /
    non-rephasing frequency lands on the diagonal of S_C.
"""
import math

import numpy as np
import scipy.linalg as sl
import scipy.sparse as sp

import workloads as W
from oracle import heom as Hm
from oracle import model as M


def liouvillian(prob):
    """Sparse matrix of Eq. HEOM_DB on vec(rho) (row-major, ADO-major)."""
    d, N = prob.d, prob.nado
    I = sp.identity(d, format="csr")

    def left(A):
        return sp.kron(sp.csr_matrix(A), I)

    def right(A):
        return sp.kron(I, sp.csr_matrix(A.T))

    Hx = left(prob.sys.H) - right(prob.sys.H)
    blocks = [[None] * N for _ in range(N)]
    for i, n in enumerate(prob.hier.n):
        decay = sum(n[j] * prob.bath.nu[j] for j in range(prob.bath.D))
        blocks[i][i] = -1j * Hx - decay * sp.identity(d * d)
        for j in range(prob.bath.D):
            V = prob.sys.V[prob.bath.mode_of[j]]
            Vx = left(V) - right(V)
            Vo = left(V) + right(V)
            dn = prob.hier.down(i, j)
            if dn >= 0:
                t = -1j * n[j] * (prob.bath.a[j] * Vx + prob.bath.b[j] * Vo)
                blocks[i][dn] = t if blocks[i][dn] is None else blocks[i][dn] + t
            up = prob.hier.up(i, j)
            if up >= 0:
                t = -1j * Vx
                blocks[i][up] = t if blocks[i][up] is None else blocks[i][up] + t
    return sp.bmat(blocks, format="csr")


def random_state(prob, seed, branches=1, hermitian=False):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((branches, prob.nado, prob.d, prob.d)) \
        + 1j * rng.standard_normal((branches, prob.nado, prob.d, prob.d))
    if hermitian:
        x = x + np.conj(np.swapaxes(x, -1, -2))
    return x


def test_rk4_is_taylor_polynomial():
    prob = M.Problem(W.small_two_mode(depth_L=2))
    L = liouvillian(prob)
    rho = random_state(prob, 1)
    dt = 0.4
    got = Hm.rk4_step(prob, rho, dt).reshape(-1)
    v = rho.reshape(-1)
    term, ref = v.copy(), v.copy()
    for j in range(1, 5):
        term = (dt / j) * (L @ term)
        ref = ref + term
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))


def test_rk4_converges_to_expm_at_fourth_order():
    prob = M.Problem(W.small_two_mode(n1=2, n2=2, depth_L=2))
    L = liouvillian(prob).toarray()
    rho = random_state(prob, 2)
    T = 8.0
    exact = sl.expm(L * T) @ rho.reshape(-1)
    errs = []
    for nsteps in (32, 64):
        got = Hm.propagate(prob, rho, T / nsteps, nsteps).reshape(-1)
        errs.append(np.max(np.abs(got - exact)))
    ratio = errs[0] / errs[1]
    assert 13.0 < ratio < 19.0, ratio


def test_trace_and_hermiticity_preserved():
    prob = M.Problem(W.small_two_mode(depth_L=3))
    rho = random_state(prob, 3, hermitian=True)
    tr0 = np.trace(rho[0, 0])
    out = Hm.propagate(prob, rho, 0.5, 40)
    assert abs(np.trace(out[0, 0]) - tr0) < 1e-12 * abs(tr0)
    herm = np.max(np.abs(out - np.conj(np.swapaxes(out, -1, -2))))
    assert herm < 1e-12 * np.max(np.abs(out))


def test_equilibrium_is_null_vector():
    # low-frequency, strongly damped oscillator with a cubic term: fast relaxation
    model = W.harmonic_bo(omega_cm=300.0, n_levels=6, lambda_cm=60.0, gamma_cm=150.0,
                          depth_L=2, K_pade=1)
    model["modes"][0]["g3_cm"] = -40.0
    model["modes"][0]["n_prim"] = 12
    model["modes"][0]["V_SL"] = 0.2
    prob = M.Problem(model)
    L = liouvillian(prob).toarray()
    # null vector: L x = 0, tr rho_0 = 1 (replace one row by the trace constraint)
    n = L.shape[0]
    A = L.copy()
    b = np.zeros(n, dtype=complex)
    A[0, :] = 0
    for a in range(prob.d):
        A[0, a * prob.d + a] = 1.0
    b[0] = 1.0
    x = np.linalg.solve(A, b).reshape(1, prob.nado, prob.d, prob.d)
    rho, steps, conv = Hm.equilibrate(prob, 1.0, tol=1e-11, t_max_fs=20000.0, check_every=500)
    assert conv
    assert np.max(np.abs(rho - x)) < 1e-8 * np.max(np.abs(x))


def test_steady_state_direct_solve():
    """oracle.steady_state against the independently assembled Liouvillian's null
    vector, the propagated equilibrium, and the trace and Hermiticity it must carry."""
    model = W.harmonic_bo(omega_cm=300.0, n_levels=5, lambda_cm=60.0, gamma_cm=150.0,
                          depth_L=2, K_pade=1)
    model["modes"][0]["g3_cm"] = -40.0
    model["modes"][0]["n_prim"] = 12
    model["modes"][0]["V_SL"] = 0.2
    prob = M.Problem(model)
    x = Hm.steady_state(prob)
    L = liouvillian(prob)
    v = x.reshape(-1)
    assert np.max(np.abs(L @ v)) < 1e-10 * np.max(np.abs(v))
    assert abs(np.trace(x[0, 0]) - 1.0) < 1e-12
    assert np.max(np.abs(x[0, 0] - x[0, 0].conj().T)) < 1e-10
    rho, _, conv = Hm.equilibrate(prob, 1.0, tol=1e-11, t_max_fs=20000.0, check_every=500)
    assert conv and np.max(np.abs(rho - x)) < 1e-8 * np.max(np.abs(x))


def test_first_kick_on_ground_state():
    prob = M.Problem(W.small_two_mode())
    rho = Hm.initial_state(prob)
    K1, _, _ = Hm.pathway_kicks(prob, "I")
    out = Hm.kick(rho, K1)[0, 0]
    ref = -(rho[0, 0] @ prob.sys.mu)
    for a in range(prob.d):
        for b in range(prob.d):
            if a == 0 and prob.sys.N[b] > 0:
                assert abs(out[a, b] - ref[a, b]) < 1e-15
            else:
                assert out[a, b] == 0
    K1, _, _ = Hm.pathway_kicks(prob, "II")
    out = Hm.kick(rho, K1)[0, 0]
    ref = prob.sys.mu @ rho[0, 0]
    for a in range(prob.d):
        for b in range(prob.d):
            if b == 0 and prob.sys.N[a] > 0:
                assert abs(out[a, b] - ref[a, b]) < 1e-15
            else:
                assert out[a, b] == 0


def test_dft2d_equals_fft():
    rng = np.random.default_rng(5)
    R = rng.standard_normal((12, 10)) + 1j * rng.standard_normal((12, 10))
    dtau = 4.0
    S = Hm.dft2d(R, dtau)
    Rw = R.copy()
    Rw[0, :] *= 0.5
    Rw[:, 0] *= 0.5
    ref = (dtau ** 2 * np.fft.ifft2(Rw) * R.size).imag
    assert np.max(np.abs(S - ref)) < 1e-12 * np.max(np.abs(ref))


def test_correlation_spectrum_diagonal_peak():
    n, dtau = 32, 4.0
    p0 = 5
    w = 2 * math.pi * p0 / (n * dtau)
    t = np.arange(n) * dtau
    decay = np.exp(-t / 60.0)
    # rephasing signal oscillates with opposite phase in t1 and t3, non-rephasing with equal
    RI = (np.outer(np.exp(+1j * w * t) * decay, np.exp(-1j * w * t) * decay) * 1j)[None]
    RII = (np.outer(np.exp(-1j * w * t) * decay, np.exp(-1j * w * t) * decay) * 1j)[None]
    SC, SR, SNR = Hm.correlation_spectrum(RI, RII, dtau)
    # with exp(+i Omega t) transforms the peaks sit at Omega3 = w; S_R at Omega1 = -w
    q, p = np.unravel_index(np.argmax(SC[0]), SC[0].shape)
    assert (q, p) == (p0, p0)
    # S_R peaks at Omega1 = -Omega3: the -Omega1 flip in S_C puts it on the diagonal
    qr, pr = np.unravel_index(np.argmax(np.abs(SR[0])), SR[0].shape)
    assert (qr + pr) % n == 0
