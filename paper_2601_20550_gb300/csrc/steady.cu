// Stationary hierarchy by restarted GMRES (heom_steady_state); the vector
// kernels are in krylov.cuh.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <future>
#include <memory>
#include <vector>

#include <cuda_runtime.h>

#include "adjoint.cuh"
#include "internal.h"
#include "krylov.cuh"

using namespace heom;

namespace heom {

// Inner products <V_j, w> for j < k (V holds basis vectors of length n back to back).
static std::vector<std::complex<double>> multi_dot(const double2 *V, int64_t n, int k, const double2 *w,
                                                   DeviceBuffer &partial, cudaStream_t st) {
  multi_dot_kernel<<<kKrylovBlocks, 256, 0, st>>>(V, n, k, w, (double2 *)partial.p);
  count_launch(1);
  LAUNCH_CHECK();
  std::vector<double2> hp((size_t)kKrylovBlocks * k);
  CUDA_TRY(cudaMemcpyAsync(hp.data(), partial.p, hp.size() * 16, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<std::complex<double>> out(k, 0.0);
  for (int b = 0; b < kKrylovBlocks; ++b)
    for (int j = 0; j < k; ++j) out[j] += std::complex<double>(hp[(size_t)b * k + j].x, hp[(size_t)b * k + j].y);
  return out;
}

// w += sum_j c_j V_j
static void multi_axpy(double2 *w, const double2 *V, int64_t n, const std::vector<std::complex<double>> &c,
                       DeviceBuffer &coef, cudaStream_t st) {
  const int k = (int)c.size();
  if (k == 0) return;
  std::vector<double2> hc(k);
  for (int j = 0; j < k; ++j) hc[j] = make_double2(c[j].real(), c[j].imag());
  CUDA_TRY(cudaMemcpyAsync(coef.p, hc.data(), k * 16, cudaMemcpyHostToDevice, st));
  multi_axpy_kernel<<<grid_for(n), 256, 0, st>>>(w, V, n, k, (const double2 *)coef.p);
  count_launch(1);
  LAUNCH_CHECK();
  CUDA_TRY(cudaStreamSynchronize(st));
}

// out = L x (one branch, FP64 product basis)
static void apply_L(heom_hier *h, const double2 *x, double2 *out, int64_t n, cudaStream_t st) {
  CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)n * 16, st));
  stage_kernel<double><<<grid_for(n), 256, 0, st>>>(x, out, out, 1.0, h->dm64, n);
  count_launch(1);
  LAUNCH_CHECK();
}

}  // namespace heom

extern "C" heom_status heom_steady_state(heom_hier *h, double tol, int restart, int max_iter, double dt_fs,
                                         int steps_per_matvec, heom_state **rho_eq, int *iterations) {
  PhaseRange phase("heom: steady state");
  if (!h || !rho_eq || !(tol > 0) || restart < 2 || max_iter < 1 || steps_per_matvec < 0)
    return fail(HEOM_EINVAL, "bad steady-state arguments");
  *rho_eq = nullptr;
  {
    heom_status e = guarded([&]() -> heom_status {
      ensure_device(h);
      return HEOM_OK;
    });
    if (e != HEOM_OK) return e;
  }
  heom_state *s = nullptr;
  heom_status st0 = heom_state_create(h, 1, HEOM_FP64, &s);
  if (st0 != HEOM_OK) return st0;
  int its = 0;
  heom_status rc = guarded([&]() -> heom_status {
    using cd = std::complex<double>;
    const Model &M = h->M;
    cudaStream_t st = h->stream;
    const int64_t n = (int64_t)M.n_ado * M.d * M.d;
    const int m = restart;
    double2 *x = (double2 *)s->buf.p;
    const double one[2] = {1.0, 0.0};
    CUDA_TRY(cudaMemcpyAsync(x, one, 16, cudaMemcpyHostToDevice, st));   // x = |0><0|, tr x_0 = 1
    DeviceBuffer V((size_t)(m + 1) * n * 16), w((size_t)n * 16), partial((size_t)kKrylovBlocks * (m + 1) * 16),
        coef((size_t)(m + 1) * 16);
    double2 *Vp = (double2 *)V.p, *wp = (double2 *)w.p;
    auto vec = [&](int j) { return Vp + (int64_t)j * n; };
    // the operator whose null vector is sought: L itself, or G^k - 1 with G the RK4
    // step of dt (same null vector; its spectrum is far less spread for stiff hierarchies)
    DeviceBuffer sa(steps_per_matvec > 0 ? (size_t)n * 16 : 16), sb(steps_per_matvec > 0 ? (size_t)n * 16 : 16);
    if (steps_per_matvec > 0) stability_check(h, dt_fs);
    auto apply_A = [&](const double2 *in, double2 *out) {
      if (steps_per_matvec == 0) {
        apply_L(h, in, out, n, st);
        return;
      }
      CUDA_TRY(cudaMemcpyAsync(out, in, (size_t)n * 16, cudaMemcpyDeviceToDevice, st));
      rk4_steps<double>(h, out, (double2 *)sa.p, (double2 *)sb.p, 1, dt_fs, steps_per_matvec, st, HEOM_FP64);
      axpy_kernel<<<grid_for(n), 256, 0, st>>>(out, in, -1.0, n);
      count_launch(1);
      LAUNCH_CHECK();
    };
    // the reference scale: ||x_0||_F of the starting state (= 1)
    const double scale = 1.0;
    while (its < max_iter) {
      // r = -L x; every vector of range(L) has tr(.)_0 = 0 (tr rho_0 is conserved),
      // so the corrections keep tr x_0 = 1
      apply_L(h, x, vec(0), n, st);
      const double resL = std::sqrt(multi_dot(vec(0), n, 1, vec(0), partial, st)[0].real());
      if (!std::isfinite(resL)) throw Fail{HEOM_ENONFINITE, "steady-state residual is not finite"};
      if (resL <= tol * scale) return HEOM_OK;
      if (steps_per_matvec > 0) apply_A(x, vec(0));
      const double beta = std::sqrt(multi_dot(vec(0), n, 1, vec(0), partial, st)[0].real());
      zscal_kernel<<<grid_for(n), 256, 0, st>>>(vec(0), n, -1.0 / beta, 0.0);
      count_launch(1);
      std::vector<std::vector<cd>> H(m + 1, std::vector<cd>(m, 0.0));
      std::vector<cd> cs(m), sn(m), g(m + 1, 0.0);
      g[0] = beta;
      int k = 0;
      for (; k < m && its < max_iter; ++k, ++its) {
        apply_A(vec(k), wp);
        // classical Gram-Schmidt, twice
        for (int pass = 0; pass < 2; ++pass) {
          std::vector<cd> hk = multi_dot(Vp, n, k + 1, wp, partial, st);
          std::vector<cd> neg(k + 1);
          for (int j = 0; j <= k; ++j) {
            H[j][k] += hk[j];
            neg[j] = -hk[j];
          }
          multi_axpy(wp, Vp, n, neg, coef, st);
        }
        const double hn = std::sqrt(multi_dot(wp, n, 1, wp, partial, st)[0].real());
        H[k + 1][k] = hn;
        if (hn > 0) {
          CUDA_TRY(cudaMemcpyAsync(vec(k + 1), wp, (size_t)n * 16, cudaMemcpyDeviceToDevice, st));
          zscal_kernel<<<grid_for(n), 256, 0, st>>>(vec(k + 1), n, 1.0 / hn, 0.0);
          count_launch(1);
        }
        // apply the previous rotations to column k, then a new one
        for (int j = 0; j < k; ++j) {
          const cd t = std::conj(cs[j]) * H[j][k] + std::conj(sn[j]) * H[j + 1][k];
          H[j + 1][k] = -sn[j] * H[j][k] + cs[j] * H[j + 1][k];
          H[j][k] = t;
        }
        const double a = std::abs(H[k][k]), b = std::abs(H[k + 1][k]), r = std::hypot(a, b);
        if (r == 0) {
          cs[k] = 1.0;
          sn[k] = 0.0;
        } else {
          cs[k] = H[k][k] / r;
          sn[k] = H[k + 1][k] / r;
        }
        H[k][k] = r;
        H[k + 1][k] = 0.0;
        g[k + 1] = -sn[k] * g[k];
        g[k] = std::conj(cs[k]) * g[k];
        if (std::abs(g[k + 1]) <= (steps_per_matvec > 0 ? 1e-3 : 1.0) * tol * scale || hn == 0) {
          ++k;
          ++its;
          break;
        }
      }
      // y = R^{-1} g, x += V y
      std::vector<cd> y(k, 0.0);
      for (int i = k - 1; i >= 0; --i) {
        cd acc = g[i];
        for (int j = i + 1; j < k; ++j) acc -= H[i][j] * y[j];
        y[i] = acc / H[i][i];
      }
      multi_axpy(x, Vp, n, y, coef, st);
    }
    apply_L(h, x, wp, n, st);
    const double res = std::sqrt(multi_dot(wp, n, 1, wp, partial, st)[0].real());
    if (res <= tol * scale) return HEOM_OK;
    g_last_error = "steady-state tolerance not reached within max_iter";
    return HEOM_ENOTCONV;
  });
  if (iterations) *iterations = its;
  if (rc == HEOM_OK || rc == HEOM_ENOTCONV) {
    *rho_eq = s;
    return rc;
  }
  heom_free_state(s);
  return rc;
}
