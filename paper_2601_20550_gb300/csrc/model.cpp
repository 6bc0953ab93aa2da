// Host-side model builder: mode eigenbases, system operators, bath exponentials
// and the hierarchy index tables (Sec. II.A-B of arXiv 2601.20550).
//
// Everything here runs once per model on the CPU in double precision and is
// small (d <= a few hundred, tables of a few 10^4 entries); the results are
// uploaded to the device by api.cu.
#include "model.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <unordered_map>

namespace heom {

// 1 cm^-1 as an angular frequency in rad/fs (2 pi c, c = 2.99792458e-5 cm/fs).
static const double kCmToRadFs = 2.0 * M_PI * 2.99792458e-5;
// Boltzmann constant in cm^-1 per K.
static const double kBoltzmannCm = 0.6950348005;

// ---------------------------------------------------------------------------
// Dense symmetric eigensolver: cyclic Jacobi rotations.  A (n x n, row-major) is
// destroyed; on return w holds ascending eigenvalues and the columns of Z the
// eigenvectors.
// ---------------------------------------------------------------------------
void jacobi_eigh(std::vector<double> &A, int n, std::vector<double> &w, std::vector<double> &Z) {
  Z.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  auto a = [&](int i, int j) -> double & { return A[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += a(i, i) * a(i, i);
      for (int j = i + 1; j < n; ++j) off += a(i, j) * a(i, j);
    }
    if (off <= 1e-30 * diag || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = a(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        double app = a(p, p), aqq = a(q, q);
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        // rotate rows/columns p and q
        for (int k = 0; k < n; ++k) {
          double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double zkp = Z[(size_t)k * n + p], zkq = Z[(size_t)k * n + q];
          Z[(size_t)k * n + p] = c * zkp - s * zkq;
          Z[(size_t)k * n + q] = s * zkp + c * zkq;
        }
      }
    }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return a(x, x) < a(y, y); });
  w.resize(n);
  std::vector<double> Zs((size_t)n * n);
  for (int c = 0; c < n; ++c) {
    w[c] = a(order[c], order[c]);
    for (int r = 0; r < n; ++r) Zs[(size_t)r * n + c] = Z[(size_t)r * n + order[c]];
  }
  Z.swap(Zs);
}

// C = A^T B A restricted: out (k x k) = U^T M U with U (n x k) column-major in a
// row-major n x n array (first k columns used).
static std::vector<double> project(const std::vector<double> &M, const std::vector<double> &U,
                                   int n, int k) {
  std::vector<double> MU((size_t)n * k, 0.0), out((size_t)k * k, 0.0);
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < n; ++l) {
      double m = M[(size_t)i * n + l];
      if (m == 0.0) continue;
      for (int c = 0; c < k; ++c) MU[(size_t)i * k + c] += m * U[(size_t)l * n + c];
    }
  for (int r = 0; r < k; ++r)
    for (int i = 0; i < n; ++i) {
      double u = U[(size_t)i * n + r];
      for (int c = 0; c < k; ++c) out[(size_t)r * k + c] += u * MU[(size_t)i * k + c];
    }
  return out;
}

// Sign convention of the kept eigenvectors: ground state with its largest
// component positive, state n with <n-1|q|n> > 0 (q the primitive q matrix).
static void fix_signs(std::vector<double> &U, int n, int k, const std::vector<double> &qprim) {
  auto col_flip = [&](int c) {
    for (int r = 0; r < n; ++r) U[(size_t)r * n + c] = -U[(size_t)r * n + c];
  };
  int imax = 0;
  for (int r = 1; r < n; ++r)
    if (std::fabs(U[(size_t)r * n]) > std::fabs(U[(size_t)imax * n])) imax = r;
  if (U[(size_t)imax * n] < 0) col_flip(0);
  for (int c = 1; c < k; ++c) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
      double qi = 0.0;
      for (int l = 0; l < n; ++l) qi += qprim[(size_t)i * n + l] * U[(size_t)l * n + c];
      s += U[(size_t)i * n + c - 1] * qi;
    }
    if (s < 0) col_flip(c);
  }
}

// Eigenbasis of one mode (Eqs. System Hamiltonian, Potentials): energies and the
// matrices of q^1..q^4 in the kept states, projected from the primitive basis.
static void build_mode(const heom_mode &md, ModeBasis &out) {
  const int k = md.n_levels;
  const int n = md.n_prim;
  const double w = md.omega_cm * kCmToRadFs;
  std::vector<double> Hm((size_t)n * n, 0.0), qprim[5];
  for (int p = 1; p <= 4; ++p) qprim[p].assign((size_t)n * n, 0.0);
  if (md.potential == 1) {
    // Morse on a sinc-DVR grid (Colbert-Miller kinetic matrix)
    const double D = md.morse_D_cm * kCmToRadFs;
    const double a = std::sqrt(w / (2.0 * D));
    const double dx = (md.q_max - md.q_min) / (n - 1);
    const double tk = 0.5 * w / (dx * dx);
    for (int i = 0; i < n; ++i) {
      double x = md.q_min + i * dx;
      for (int j = 0; j < n; ++j) {
        int m = i - j;
        double t = (m == 0) ? M_PI * M_PI / 3.0 : 2.0 / (double)(m * m);
        if (m & 1) t = -t;
        Hm[(size_t)i * n + j] = tk * t;
      }
      double e = 1.0 - std::exp(-a * x);
      Hm[(size_t)i * n + i] += D * e * e;
      double xp = 1.0;
      for (int p = 1; p <= 4; ++p) {
        xp *= x;
        qprim[p][(size_t)i * n + i] = xp;
      }
    }
  } else {
    // harmonic basis; q^p formed in a basis 4 larger, then truncated (exact projection)
    const int M = n + 4;
    std::vector<double> q((size_t)M * M, 0.0), cur, nxt((size_t)M * M);
    for (int i = 0; i + 1 < M; ++i) {
      double v = std::sqrt((i + 1) / 2.0);
      q[(size_t)i * M + i + 1] = v;
      q[(size_t)(i + 1) * M + i] = v;
    }
    cur = q;
    for (int p = 1; p <= 4; ++p) {
      if (p > 1) {
        std::fill(nxt.begin(), nxt.end(), 0.0);
        for (int i = 0; i < M; ++i)
          for (int l = 0; l < M; ++l) {
            double c = cur[(size_t)i * M + l];
            if (c == 0.0) continue;
            for (int j = 0; j < M; ++j) nxt[(size_t)i * M + j] += c * q[(size_t)l * M + j];
          }
        cur = nxt;
      }
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) qprim[p][(size_t)i * n + j] = cur[(size_t)i * M + j];
    }
    const double g3 = md.g3_cm * kCmToRadFs;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        Hm[(size_t)i * n + j] = (g3 / 6.0) * qprim[3][(size_t)i * n + j] + (i == j ? w * (i + 0.5) : 0.0);
  }
  std::vector<double> evals, U;
  jacobi_eigh(Hm, n, evals, U);
  fix_signs(U, n, k, qprim[1]);
  out.n = k;
  out.E.assign(evals.begin(), evals.begin() + k);
  for (int p = 1; p <= 4; ++p) out.q[p] = project(qprim[p], U, n, k);
}

// Kronecker embedding helpers on the product basis (mode 0 slowest).
struct Product {
  std::vector<int> dims, stride;
  int d = 1;
  explicit Product(const std::vector<int> &dm) : dims(dm), stride(dm.size()) {
    d = 1;
    for (int s = (int)dm.size() - 1; s >= 0; --s) {
      stride[s] = d;
      d *= dm[s];
    }
  }
  int digit(int a, int s) const { return (a / stride[s]) % dims[s]; }
  // element <a| A_s x B_t |b> (other modes identity); t may equal -1 (single mode)
  double elem(int a, int b, int s, const std::vector<double> &A, int t, const std::vector<double> &B) const {
    for (int u = 0; u < (int)dims.size(); ++u) {
      if (u == s || u == t) continue;
      if (digit(a, u) != digit(b, u)) return 0.0;
    }
    double v = A[(size_t)digit(a, s) * dims[s] + digit(b, s)];
    if (t >= 0) v *= B[(size_t)digit(a, t) * dims[t] + digit(b, t)];
    return v;
  }
};

// ---------------------------------------------------------------------------
// Pade spectrum decomposition of the Bose function, [N-1/N] scheme
// (Hu, Xu and Yan, JCP 133, 101106 (2010); JCP 134, 244106 (2011)):
//   1/(1-e^-x) ~ 1/x + 1/2 + sum_k 2 eta_k x/(x^2 + xi_k^2).
// The poles xi_k are 2/lambda for the positive eigenvalues lambda of the 2N x 2N
// symmetric tridiagonal matrix with off-diagonal 1/sqrt((2m+1)(2m+3)), m = 1..2N-1.
// The weights follow from matching the first N Taylor coefficients of the
// remainder, sum_k 2 eta_k (-1)^m / xi_k^(2m+2) = B_(2m+2)/(2m+2)!.
// ---------------------------------------------------------------------------
void pade_bose(int N, std::vector<double> &xi, std::vector<double> &eta) {
  xi.clear();
  eta.clear();
  if (N <= 0) return;
  if (N > 8) throw std::invalid_argument("K_pade > 8 is not supported");
  const int M = 2 * N;
  std::vector<double> T((size_t)M * M, 0.0), w, Z;
  for (int m = 1; m < M; ++m) {
    double v = 1.0 / std::sqrt((2.0 * m + 1.0) * (2.0 * m + 3.0));
    T[(size_t)(m - 1) * M + m] = v;
    T[(size_t)m * M + m - 1] = v;
  }
  jacobi_eigh(T, M, w, Z);
  for (int i = 0; i < M; ++i)
    if (w[i] > 0) xi.push_back(2.0 / w[i]);
  std::sort(xi.begin(), xi.end());
  // Bernoulli numbers B_2 .. B_18 divided by (2m)!
  static const double bern[9] = {1.0 / 6, -1.0 / 30, 1.0 / 42, -1.0 / 30, 5.0 / 66,
                                 -691.0 / 2730, 7.0 / 6, -3617.0 / 510, 43867.0 / 798};
  std::vector<long double> A((size_t)N * N), b(N);
  for (int m = 0; m < N; ++m) {
    long double fact = 1.0L;
    for (int i = 2; i <= 2 * m + 2; ++i) fact *= i;
    b[m] = (long double)bern[m] / fact;
    for (int k = 0; k < N; ++k)
      A[(size_t)m * N + k] = 2.0L * ((m & 1) ? -1.0L : 1.0L) / powl((long double)xi[k], 2 * m + 2);
  }
  // Gaussian elimination with partial pivoting (long double)
  for (int c = 0; c < N; ++c) {
    int p = c;
    for (int r = c + 1; r < N; ++r)
      if (fabsl(A[(size_t)r * N + c]) > fabsl(A[(size_t)p * N + c])) p = r;
    if (p != c) {
      for (int j = 0; j < N; ++j) std::swap(A[(size_t)c * N + j], A[(size_t)p * N + j]);
      std::swap(b[c], b[p]);
    }
    for (int r = c + 1; r < N; ++r) {
      long double f = A[(size_t)r * N + c] / A[(size_t)c * N + c];
      for (int j = c; j < N; ++j) A[(size_t)r * N + j] -= f * A[(size_t)c * N + j];
      b[r] -= f * b[c];
    }
  }
  std::vector<long double> x(N);
  for (int r = N - 1; r >= 0; --r) {
    long double s = b[r];
    for (int j = r + 1; j < N; ++j) s -= A[(size_t)r * N + j] * x[j];
    x[r] = s / A[(size_t)r * N + r];
  }
  for (int k = 0; k < N; ++k) eta.push_back((double)x[k]);
}

// ---------------------------------------------------------------------------
Model build_model(const heom_model &m) {
  if (m.n_modes < 1 || m.n_modes > 8 || !m.modes) throw std::invalid_argument("n_modes must be 1..8");
  if (m.depth_L < 0 || m.depth_L > 64) throw std::invalid_argument("depth_L out of range");
  if (!(m.T_K > 0)) throw std::invalid_argument("T_K must be > 0");
  Model M;
  M.n_modes = m.n_modes;
  M.depth = m.depth_L;
  M.precision = m.precision;
  std::vector<int> dims;
  for (int s = 0; s < m.n_modes; ++s) {
    const heom_mode &md = m.modes[s];
    if (md.n_levels < 1 || md.n_prim < md.n_levels || md.n_prim > 4000)
      throw std::invalid_argument("need 1 <= n_levels <= n_prim <= 4000");
    if (md.potential == 1 && !(md.morse_D_cm > 0 && md.q_max > md.q_min))
      throw std::invalid_argument("Morse mode needs D > 0 and q_max > q_min");
    if (md.potential != 0 && md.potential != 1) throw std::invalid_argument("potential must be 0 or 1");
    if (!(md.omega_cm > 0) || md.gamma_cm < 0 || md.zeta_cm < 0 || md.K_pade < 0 || md.K_pade > 8)
      throw std::invalid_argument("bad mode parameters");
    ModeBasis mb;
    build_mode(md, mb);
    M.modes.push_back(mb);
    dims.push_back(md.n_levels);
  }
  Product P(dims);
  const int d = P.d;
  M.d = d;
  M.dims = dims;
  M.stride = P.stride;
  // ---- system operators (Eqs. Total Hamiltonian, Potential ss', counter2, NLdip)
  M.H.assign((size_t)d * d, 0.0);
  M.mu.assign((size_t)d * d, 0.0);
  std::vector<double> none;
  for (int s = 0; s < m.n_modes; ++s) {
    const heom_mode &md = m.modes[s];
    const ModeBasis &mb = M.modes[s];
    const int n = mb.n;
    std::vector<double> hloc((size_t)n * n, 0.0), Vs((size_t)n * n), V2((size_t)n * n), muloc((size_t)n * n);
    const double lam = md.zeta_cm * md.gamma_cm / (2.0 * md.omega_cm) * kCmToRadFs;
    for (int i = 0; i < n * n; ++i) {
      Vs[i] = md.V_LL * mb.q[1][i] + 0.5 * md.V_SL * mb.q[2][i];
      V2[i] = md.V_LL * md.V_LL * mb.q[2][i] + md.V_LL * md.V_SL * mb.q[3][i] + 0.25 * md.V_SL * md.V_SL * mb.q[4][i];
      hloc[i] = lam * V2[i];
      muloc[i] = md.mu1 * mb.q[1][i] + 0.5 * md.mu2 * mb.q[2][i];
    }
    for (int i = 0; i < n; ++i) hloc[(size_t)i * n + i] += mb.E[i];
    M.Vloc.push_back(Vs);
    M.lambda.push_back(lam);
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        M.H[(size_t)a * d + b] += P.elem(a, b, s, hloc, -1, none);
        M.mu[(size_t)a * d + b] += P.elem(a, b, s, muloc, -1, none);
      }
  }
  for (int p = 0; p < m.n_pairs; ++p) {
    const heom_pair &pr = m.pairs[p];
    if (pr.s < 0 || pr.t < 0 || pr.s >= m.n_modes || pr.t >= m.n_modes || pr.s == pr.t)
      throw std::invalid_argument("bad pair indices");
    const ModeBasis &A = M.modes[pr.s], &B = M.modes[pr.t];
    const double g = pr.g_st_cm * kCmToRadFs, g21 = pr.g_s2t_cm * kCmToRadFs, g12 = pr.g_st2_cm * kCmToRadFs;
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        double v = g * P.elem(a, b, pr.s, A.q[1], pr.t, B.q[1]) +
                   (g21 / 6.0) * P.elem(a, b, pr.s, A.q[2], pr.t, B.q[1]) +
                   (g12 / 6.0) * P.elem(a, b, pr.s, A.q[1], pr.t, B.q[2]);
        M.H[(size_t)a * d + b] += v;
        M.mu[(size_t)a * d + b] += pr.mu_st * P.elem(a, b, pr.s, A.q[1], pr.t, B.q[1]);
      }
  }
  // raising part of mu: total excitation number of a above that of b
  M.mu_plus.assign((size_t)d * d, 0.0);
  std::vector<int> N(d, 0);
  for (int a = 0; a < d; ++a)
    for (int s = 0; s < m.n_modes; ++s) N[a] += P.digit(a, s);
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b)
      if (N[a] > N[b]) M.mu_plus[(size_t)a * d + b] = M.mu[(size_t)a * d + b];
  // ---- bath exponentials (Eqs. L1, L2, Pade1, Pade2), C(t) = sum_j c_j e^{-nu_j t}
  const double kT = kBoltzmannCm * m.T_K * kCmToRadFs;
  M.beta = 1.0 / kT;
  for (int s = 0; s < m.n_modes; ++s) {
    const heom_mode &md = m.modes[s];
    const double gam = md.gamma_cm * kCmToRadFs;
    const double lam = M.lambda[s];
    std::vector<double> xi, eta;
    pade_bose(md.K_pade, xi, eta);
    double corr = 1.0;
    for (size_t k = 0; k < xi.size(); ++k) {
      double nu = xi[k] * kT;
      corr += 2.0 * eta[k] * gam * gam / (gam * gam - nu * nu);
    }
    M.exp_mode.push_back(s);
    M.exp_nu.push_back(gam);
    M.exp_re.push_back(2.0 * lam * kT * corr);   // lambda gamma cot_PSD(beta gamma / 2)
    M.exp_im.push_back(-lam * gam);
    for (size_t k = 0; k < xi.size(); ++k) {
      double nu = xi[k] * kT;
      M.exp_mode.push_back(s);
      M.exp_nu.push_back(nu);
      M.exp_re.push_back(-4.0 * lam * gam * kT * eta[k] * nu / (gam * gam - nu * nu));
      M.exp_im.push_back(0.0);
    }
  }
  M.n_exp = (int)M.exp_nu.size();
  build_hierarchy(M);
  build_coupling_basis(M);
  return M;
}

// ---------------------------------------------------------------------------
// Coupling eigenbasis.  Each V_s acts on mode s only, so the product of the
// per-mode eigenbases of v_s diagonalises every V_s at once.  In that basis
// V_s^x X and V_s^o X are elementwise: (lam_s[a_s] -+ lam_s[b_s]) X_ab.  The
// transformation is orthogonal; H_S' and mu become dense d x d matrices.
// ---------------------------------------------------------------------------
static std::vector<double> similarity(const std::vector<double> &U, const std::vector<double> &X, int d) {
  // U^T X U
  std::vector<double> T((size_t)d * d, 0.0), out((size_t)d * d, 0.0);
  for (int c = 0; c < d; ++c)
    for (int a = 0; a < d; ++a) {
      double u = U[(size_t)c * d + a];
      if (u == 0.0) continue;
      for (int b = 0; b < d; ++b) T[(size_t)a * d + b] += u * X[(size_t)c * d + b];
    }
  for (int a = 0; a < d; ++a)
    for (int c = 0; c < d; ++c) {
      double t = T[(size_t)a * d + c];
      if (t == 0.0) continue;
      for (int b = 0; b < d; ++b) out[(size_t)a * d + b] += t * U[(size_t)c * d + b];
    }
  return out;
}

void build_coupling_basis(Model &M) {
  const int d = M.d;
  std::vector<std::vector<double>> Us;
  M.vb_lam.clear();
  for (int s = 0; s < M.n_modes; ++s) {
    const int n = M.dims[s];
    std::vector<double> A = M.Vloc[s], w, Z;
    jacobi_eigh(A, n, w, Z);
    M.vb_lam.push_back(w);
    Us.push_back(Z);
  }
  M.vb_U.assign((size_t)d * d, 0.0);
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double v = 1.0;
      for (int s = 0; s < M.n_modes && v != 0.0; ++s) {
        int as = (a / M.stride[s]) % M.dims[s], bs = (b / M.stride[s]) % M.dims[s];
        v *= Us[s][(size_t)as * M.dims[s] + bs];
      }
      M.vb_U[(size_t)a * d + b] = v;
    }
  M.vb_H = similarity(M.vb_U, M.H, d);
  M.vb_mu = similarity(M.vb_U, M.mu, d);
  M.vb_mu_plus = similarity(M.vb_U, M.mu_plus, d);
}

// ---------------------------------------------------------------------------
// Hierarchy (Sec. II.B): all n in N^D with sum(n) <= L, canonical order
// ascending by (sum, tuple); neighbour tables and the per-mode coupling lists.
// ---------------------------------------------------------------------------
static void enumerate_level(int D, int level, std::vector<int> &cur, int pos,
                            std::vector<std::vector<int>> &out) {
  if (pos == D - 1) {
    cur[pos] = level;
    out.push_back(cur);
    return;
  }
  for (int v = 0; v <= level; ++v) {
    cur[pos] = v;
    enumerate_level(D, level - v, cur, pos + 1, out);
  }
}

void build_hierarchy(Model &M) {
  const int D = M.n_exp, L = M.depth;
  if (D > 16) throw std::invalid_argument("more than 16 exponentials");
  std::vector<std::vector<int>> all;
  std::vector<int> cur(D, 0);
  for (int level = 0; level <= L; ++level) enumerate_level(D, level, cur, 0, all);
  // within a level, enumerate_level yields lexicographic order of the tuple
  const int N = (int)all.size();
  if ((long long)N * D > (1LL << 30)) throw std::invalid_argument("hierarchy too large");
  M.n_ado = N;
  auto key = [&](const std::vector<int> &v) {
    uint64_t k = 0;
    for (int j = 0; j < D; ++j) k = k * 65u + (uint64_t)v[j];
    return k;
  };
  std::unordered_map<uint64_t, int> index;
  index.reserve(N * 2);
  for (int i = 0; i < N; ++i) index[key(all[i])] = i;
  M.ado.assign((size_t)N * D, 0);
  M.up.assign((size_t)N * D, -1);
  M.down.assign((size_t)N * D, -1);
  M.decay.assign(N, 0.0);
  for (int i = 0; i < N; ++i) {
    std::vector<int> v = all[i];
    double g = 0.0;
    for (int j = 0; j < D; ++j) {
      M.ado[(size_t)i * D + j] = v[j];
      g += v[j] * M.exp_nu[j];
      v[j] += 1;
      auto it = index.find(key(v));
      if (it != index.end()) M.up[(size_t)i * D + j] = it->second;
      v[j] -= 2;
      if (v[j] >= 0) M.down[(size_t)i * D + j] = index[key(v)];
      v[j] += 1;
    }
    M.decay[i] = g;
  }
  // coupling lists per (ado, mode): A_s = sum cA w_m, B_s = sum cB w_m over
  // up-neighbours (cA = 1, cB = 0) and down-neighbours (cA = n_j Re c_j, cB = n_j Im c_j)
  M.nb_off.assign((size_t)N * M.n_modes + 1, 0);
  M.nb_idx.clear();
  M.nb_cA.clear();
  M.nb_cB.clear();
  for (int i = 0; i < N; ++i)
    for (int s = 0; s < M.n_modes; ++s) {
      M.nb_off[(size_t)i * M.n_modes + s] = (int)M.nb_idx.size();
      for (int j = 0; j < D; ++j) {
        if (M.exp_mode[j] != s) continue;
        int u = M.up[(size_t)i * D + j];
        if (u >= 0) {
          M.nb_idx.push_back(u);
          M.nb_cA.push_back(1.0);
          M.nb_cB.push_back(0.0);
        }
        int dn = M.down[(size_t)i * D + j];
        if (dn >= 0) {
          int nj = M.ado[(size_t)i * D + j];
          M.nb_idx.push_back(dn);
          M.nb_cA.push_back(nj * M.exp_re[j]);
          M.nb_cB.push_back(nj * M.exp_im[j]);
        }
      }
    }
  M.nb_off[(size_t)N * M.n_modes] = (int)M.nb_idx.size();
}

}  // namespace heom
