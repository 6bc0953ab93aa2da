// Gradient of the 2D-spectrum misfit over twelve model parameters
// (heom_response_2d_grad): reverse mode through the FP64 procedure with
// checkpoints; the adjoint kernels are in adjoint.cuh.
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

using namespace heom;

// ===========================================================================
// Gradient of the 2D-spectrum misfit (discrete adjoint of the FP64 path)
// ===========================================================================
namespace heom {

// The twelve model parameters of the gradient: anharmonicity of mode s (Morse
// depth, or g3 of a cubic mode), cubic coupling g_{s^2 t} of pair p, square
// system-bath coupling V_SL of mode s, Drude damping gamma_s (zeta_s fixed).
static double *theta_slot(heom_model &m, std::vector<heom_mode> &modes, std::vector<heom_pair> &pairs, int i) {
  const int grp = i / 3, k = i % 3;
  if (grp == 1) return k < (int)pairs.size() ? &pairs[k].g_s2t_cm : nullptr;
  if (k >= (int)modes.size()) return nullptr;
  heom_mode &md = modes[k];
  if (grp == 0) return md.potential == 1 ? &md.morse_D_cm : &md.g3_cm;
  return grp == 2 ? &md.V_SL : &md.gamma_cm;
}

// Adjoint RHS tables: L^H has H -> -H and every coupling entry n <- m with
// (cA, cB) turned into m <- n with (-cA, cB); entry_exp maps each forward entry
// to its exponential (down-neighbours) or -1 (up-neighbours).
static void ensure_adjoint(heom_hier *h) {
  if (h->adj_ready) return;
  const Model &M = h->M;
  const int N = M.n_ado, S = M.n_modes, D = M.n_exp;
  std::vector<int> eexp;
  eexp.reserve(M.nb_idx.size());
  for (int i = 0; i < N; ++i)
    for (int s = 0; s < S; ++s)
      for (int j = 0; j < D; ++j) {
        if (M.exp_mode[j] != s) continue;
        if (M.up[(size_t)i * D + j] >= 0) eexp.push_back(-1);
        if (M.down[(size_t)i * D + j] >= 0) eexp.push_back(j);
      }
  if (eexp.size() != M.nb_idx.size()) throw Fail{HEOM_EINVAL, "coupling tables out of order"};
  if (D > kAdjMaxExp) throw Fail{HEOM_EINVAL, "too many exponentials for the gradient"};
  int nvl = 0;
  for (int s = 0; s < S; ++s) nvl += M.dims[s] * M.dims[s];
  if (nvl > kAdjMaxVl) throw Fail{HEOM_EINVAL, "mode bases too large for the gradient"};
  std::vector<int> off((size_t)N * S + 1, 0), idx(M.nb_idx.size());
  std::vector<double> cA(M.nb_idx.size()), cB(M.nb_idx.size());
  for (int n = 0; n < N; ++n)
    for (int s = 0; s < S; ++s)
      for (int q = M.nb_off[(size_t)n * S + s]; q < M.nb_off[(size_t)n * S + s + 1]; ++q)
        off[(size_t)M.nb_idx[q] * S + s + 1]++;
  for (size_t k = 1; k < off.size(); ++k) off[k] += off[k - 1];
  std::vector<int> fill(off.begin(), off.end() - 1);
  for (int n = 0; n < N; ++n)
    for (int s = 0; s < S; ++s)
      for (int q = M.nb_off[(size_t)n * S + s]; q < M.nb_off[(size_t)n * S + s + 1]; ++q) {
        const int pos = fill[(size_t)M.nb_idx[q] * S + s]++;
        idx[pos] = n;
        cA[pos] = -M.nb_cA[q];
        cB[pos] = M.nb_cB[q];
      }
  std::vector<double> Hneg(M.H.size());
  for (size_t k = 0; k < Hneg.size(); ++k) Hneg[k] = -M.H[k];
  DevModel<double> a = h->dm64;
  a.H = h->up(Hneg);
  a.nb_off = h->up(off);
  a.nb_idx = h->up(idx);
  a.nb_cA = h->up(cA);
  a.nb_cB = h->up(cB);
  h->dm_adj = a;
  h->adj_ado = h->up(M.ado);
  h->adj_entry_exp = h->up(eexp);
  h->adj_ready = true;
}

// Offsets of the model gradients in one device array.
struct GradLayout {
  int64_t H, v, re, im, nu, mup, mum, mu, total;
};

static GradLayout grad_layout(const Model &M) {
  GradLayout L{};
  const int64_t dd = (int64_t)M.d * M.d;
  int nvl = 0;
  for (int s = 0; s < M.n_modes; ++s) nvl += M.dims[s] * M.dims[s];
  L.H = 0;
  L.v = dd;
  L.re = L.v + nvl;
  L.im = L.re + M.n_exp;
  L.nu = L.im + M.n_exp;
  L.mup = L.nu + M.n_exp;
  L.mum = L.mup + dd;
  L.mu = L.mum + dd;
  L.total = L.mu + dd;
  return L;
}

struct AdjCtx {
  heom_hier *h;
  cudaStream_t st;
  double *G;
  GradLayout L;
  double2 *W4, *W3, *W2, *A;   // RK4 stage and adjoint-stage scratch (branch capacity cap)
  int cap;                     // branches the scratch holds
  int64_t per;
};

static void comm_grad(AdjCtx &c, const double2 *g, const double2 *w, int64_t items, double ph_re, double ph_im,
                      double alpha, double *G) {
  const int d = c.h->M.d, tiles = (d + 15) / 16;
  const int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(items, std::max(1, 2432 / (tiles * tiles))));
  // Re(-i x) = Im x (Hamiltonian term); Re(1 x) = Re x (kicks)
  if (ph_re == 0.0 && ph_im == -1.0)
    comm_grad_kernel<true><<<(unsigned)(tiles * tiles * chunks), 256, 0, c.st>>>(g, w, items, d, alpha, G);
  else if (ph_re == 1.0 && ph_im == 0.0)
    comm_grad_kernel<false><<<(unsigned)(tiles * tiles * chunks), 256, 0, c.st>>>(g, w, items, d, alpha, G);
  else
    throw Fail{HEOM_EINVAL, "unsupported gradient phase"};
  count_launch(1);
  LAUNCH_CHECK();
}

// Model gradients from one (adjoint, forward) pair of an RK4 stage.
static void grad_pair(AdjCtx &c, const double2 *g, const double2 *w, int branches, double alpha) {
  const Model &M = c.h->M;
  const int64_t items = (int64_t)branches * M.n_ado;
  comm_grad(c, g, w, items, 0.0, -1.0, alpha, c.G + c.L.H);
  coupling_grad_kernel<<<(unsigned)std::min<int64_t>(items, 152 * 16), 256, 0, c.st>>>(
      g, w, c.h->dm64, c.h->adj_ado, M.n_exp, c.h->adj_entry_exp, items, alpha, c.G + c.L.v, c.G + c.L.re,
      c.G + c.L.im, c.G + c.L.nu);
  count_launch(1);
  LAUNCH_CHECK();
}

static void stage64(AdjCtx &c, const DevModel<double> &dm, const double2 *w, const double2 *y, double2 *out,
                    double alpha, int branches) {
  const int64_t total = (int64_t)branches * c.per;
  stage_kernel<double><<<grid_for(total), 256, 0, c.st>>>(w, y, out, alpha, dm, total);
  count_launch(1);
  LAUNCH_CHECK();
}

static void axpy64(AdjCtx &c, double2 *y, const double2 *x, double a, int64_t n) {
  axpy_kernel<<<grid_for(n), 256, 0, c.st>>>(y, x, a, n);
  count_launch(1);
  LAUNCH_CHECK();
}

// One RK4 step backwards (Horner form): given the forward state y_t and lam =
// adjoint of y_{t+1}, leave the adjoint of y_t in lam and add the model
// gradients.  Forward: w4 = y + dt/4 L y, w3 = y + dt/3 L w4, w2 = y + dt/2 L w3,
// y' = y + dt L w2.
static void back_step(AdjCtx &c, const double2 *y, double2 *lam, int B, double dt) {
  const DevModel<double> &F = c.h->dm64, &Ad = c.h->dm_adj;
  const int64_t n = (int64_t)B * c.per;
  const size_t bytes = (size_t)n * 16;
  stage64(c, F, y, y, c.W4, dt / 4, B);
  stage64(c, F, c.W4, y, c.W3, dt / 3, B);
  stage64(c, F, c.W3, y, c.W2, dt / 2, B);
  grad_pair(c, lam, c.W2, B, dt);                       // y' = y + dt L w2
  CUDA_TRY(cudaMemsetAsync(c.A, 0, bytes, c.st));
  stage64(c, Ad, lam, c.A, c.A, dt, B);                 // w2bar = dt L^H lam
  grad_pair(c, c.A, c.W3, B, dt / 2);
  CUDA_TRY(cudaMemsetAsync(c.W2, 0, bytes, c.st));
  stage64(c, Ad, c.A, c.W2, c.W2, dt / 2, B);           // w3bar = dt/2 L^H w2bar
  grad_pair(c, c.W2, c.W4, B, dt / 3);
  axpy64(c, lam, c.A, 1.0, n);
  axpy64(c, lam, c.W2, 1.0, n);
  CUDA_TRY(cudaMemsetAsync(c.W3, 0, bytes, c.st));
  stage64(c, Ad, c.W2, c.W3, c.W3, dt / 3, B);          // w4bar = dt/3 L^H w3bar
  grad_pair(c, c.W3, y, B, dt / 4);
  axpy64(c, lam, c.W3, 1.0, n);
  stage64(c, Ad, c.W3, lam, lam, dt / 4, B);            // + dt/4 L^H w4bar
}

// Reverse sweep over a span of N RK4 steps from `start` (B branches):
// checkpoints every M steps, each segment recomputed into a ring before it is
// walked backwards.  lam holds the adjoint of y_N on entry (the caller adds the
// source at N) and the adjoint of y_0 on exit; source(t, y_t, lam) adds the
// sources at t < N after the step out of t has been reversed.
static void backprop_span(AdjCtx &c, const double2 *start, int64_t N, int B, double dt, int M, double2 *lam,
                          const std::function<void(int64_t, const double2 *, double2 *)> &source) {
  if (N <= 0) return;
  const size_t sz = (size_t)B * c.per * 16;
  const int64_t n_ck = (N - 1) / M + 1;    // checkpoints at 0, M, ..., (n_ck - 1) M
  std::vector<std::unique_ptr<DeviceBuffer>> ck;
  for (int64_t k = 1; k < n_ck; ++k) ck.emplace_back(new DeviceBuffer(sz));
  DeviceBuffer cur(sz);
  CUDA_TRY(cudaMemcpyAsync(cur.p, start, sz, cudaMemcpyDeviceToDevice, c.st));
  for (int64_t k = 1; k < n_ck; ++k) {
    rk4_steps<double>(c.h, (double2 *)cur.p, c.W4, c.W3, B, dt, M, c.st, HEOM_FP64);
    CUDA_TRY(cudaMemcpyAsync(ck[k - 1]->p, cur.p, sz, cudaMemcpyDeviceToDevice, c.st));
  }
  const int ring_n = (int)std::min<int64_t>(M, N);
  std::vector<std::unique_ptr<DeviceBuffer>> ring;
  for (int r = 0; r < ring_n; ++r) ring.emplace_back(new DeviceBuffer(sz));
  for (int64_t seg = n_ck - 1; seg >= 0; --seg) {
    const int64_t s0 = seg * M, len = std::min<int64_t>(M, N - s0);
    const void *src = seg == 0 ? (const void *)start : ck[seg - 1]->p;
    CUDA_TRY(cudaMemcpyAsync(ring[0]->p, src, sz, cudaMemcpyDeviceToDevice, c.st));
    for (int64_t u = 1; u < len; ++u) {
      CUDA_TRY(cudaMemcpyAsync(ring[u]->p, ring[u - 1]->p, sz, cudaMemcpyDeviceToDevice, c.st));
      rk4_steps<double>(c.h, (double2 *)ring[u]->p, c.W4, c.W3, B, dt, 1, c.st, HEOM_FP64);
    }
    for (int64_t t = s0 + len - 1; t >= s0; --t) {
      const double2 *y = (const double2 *)ring[t - s0]->p;
      back_step(c, y, lam, B, dt);
      if (source) source(t, y, lam);
    }
  }
}

// Adjoint of the 2D Fourier sums of dft2d_sc_kernel: Rbar = i conj(F) Sbar for
// S = Im(F R), per t2 and pathway ([n1][n3] each).
static void dft2d_adjoint(const double *Sbar, int n1, int n3, double dtau, std::vector<double> &RbarI,
                          std::vector<double> &RbarII) {
  const double tp = 2.0 * M_PI;
  // E[q][k] = sum_p Sbar[q][p] exp(-i 2 pi p k / n3)
  std::vector<double> Er((size_t)n1 * n3), Ei((size_t)n1 * n3);
  for (int q = 0; q < n1; ++q)
    for (int k = 0; k < n3; ++k) {
      double sr = 0, si = 0;
      for (int p = 0; p < n3; ++p) {
        const double ph = tp * (double)((long long)p * k % n3) / n3;
        sr += Sbar[(size_t)q * n3 + p] * std::cos(ph);
        si -= Sbar[(size_t)q * n3 + p] * std::sin(ph);
      }
      Er[(size_t)q * n3 + k] = sr;
      Ei[(size_t)q * n3 + k] = si;
    }
  RbarI.assign((size_t)n1 * n3 * 2, 0.0);
  RbarII.assign((size_t)n1 * n3 * 2, 0.0);
  for (int j = 0; j < n1; ++j)
    for (int k = 0; k < n3; ++k) {
      double ar = 0, ai = 0, br = 0, bi = 0;
      for (int q = 0; q < n1; ++q) {
        const int qf = (n1 - q) % n1;
        const double phr = tp * (double)((long long)qf * j % n1) / n1, phn = tp * (double)((long long)q * j % n1) / n1;
        const double er = Er[(size_t)q * n3 + k], ei = Ei[(size_t)q * n3 + k];
        // E exp(-i ph)
        ar += er * std::cos(phr) + ei * std::sin(phr);
        ai += ei * std::cos(phr) - er * std::sin(phr);
        br += er * std::cos(phn) + ei * std::sin(phn);
        bi += ei * std::cos(phn) - er * std::sin(phn);
      }
      const double w = dtau * dtau * (j == 0 ? 0.5 : 1.0) * (k == 0 ? 0.5 : 1.0);
      // Rbar = i w (sum): i (x + i y) = -y + i x
      RbarI[((size_t)j * n3 + k) * 2] = -w * ai;
      RbarI[((size_t)j * n3 + k) * 2 + 1] = w * ar;
      RbarII[((size_t)j * n3 + k) * 2] = -w * bi;
      RbarII[((size_t)j * n3 + k) * 2 + 1] = w * br;
    }
}

}  // namespace heom

extern "C" heom_status heom_response_2d_grad(heom_hier *h, const heom_state *rho_eq, const heom_grid *g,
                                             const double *S_ref, int ckpt_every, double *loss, double *dtheta) {
  PhaseRange phase("heom: adjoint gradient");
  heom_status a = check_response_args(h, rho_eq, g);
  if (a != HEOM_OK) return a;
  if (!S_ref || !loss || !dtheta || ckpt_every < 1) return fail(HEOM_EINVAL, "bad gradient arguments");
  if (h->M.precision != HEOM_FP64) return fail(HEOM_EINVAL, "the gradient needs a hierarchy built with HEOM_FP64");
  if (rho_eq->eq_steps < 0) return fail(HEOM_EINVAL, "rho_eq must come from heom_equilibrate");
  return guarded([&]() -> heom_status {
    ensure_device(h);
    stability_check(h, g->dt_fs);
    stability_check(h, rho_eq->eq_dt);
    ensure_adjoint(h);
    const Model &M = h->M;
    cudaStream_t st = h->stream;
    // d(model matrices)/d theta by fourth-order central differences of the host model
    // build, (8 (M(+h) - M(-h)) - (M(+2h) - M(-2h))) / (12 h), relative step 1e-3: the
    // 4 x 12 builds run on host threads while the GPU does the reverse pass
    struct Build {
      int i;
      double step;
      std::future<Model> p1, m1, p2, m2;
    };
    auto model_at = [h](int i, double delta) {
      heom_model md = h->desc;
      std::vector<heom_mode> mds = h->desc_modes;
      std::vector<heom_pair> ps = h->desc_pairs;
      *theta_slot(md, mds, ps, i) += delta;
      md.modes = mds.data();
      md.pairs = ps.empty() ? nullptr : ps.data();
      return build_model(md);
    };
    std::vector<Build> builds;
    for (int i = 0; i < 12; ++i) {
      heom_model md0 = h->desc;
      std::vector<heom_mode> m0 = h->desc_modes;
      std::vector<heom_pair> p0 = h->desc_pairs;
      double *v0 = theta_slot(md0, m0, p0, i);
      if (!v0) continue;
      Build b;
      b.i = i;
      b.step = 1e-3 * std::max(std::fabs(*v0), 1.0);
      b.p1 = std::async(std::launch::async, model_at, i, b.step);
      b.m1 = std::async(std::launch::async, model_at, i, -b.step);
      b.p2 = std::async(std::launch::async, model_at, i, 2 * b.step);
      b.m2 = std::async(std::launch::async, model_at, i, -2 * b.step);
      builds.push_back(std::move(b));
    }
    const int d = M.d, n1 = g->n1, n3 = g->n3, m = g->steps_per_sample, nt2 = g->n_t2, Mck = ckpt_every;
    const double dt = g->dt_fs, dtau = dt * m;
    const int64_t per = (int64_t)M.n_ado * d * d, dd = (int64_t)d * d;
    const size_t sz1 = (size_t)per * 16;
    std::vector<int64_t> n2(nt2);
    for (int i = 0; i < nt2; ++i) {
      const double r = g->t2_fs[i] / dt;
      n2[i] = (int64_t)std::llround(r);
      if (g->t2_fs[i] < 0 || std::fabs(r - n2[i]) > 1e-6) throw Fail{HEOM_EINVAL, "t2 must be a non-negative multiple of dt"};
    }
    // ---- forward: R and S_C, loss and the adjoint of S_C (host)
    const size_t blk = (size_t)n1 * n3;
    DeviceBuffer Rdev((size_t)nt2 * 2 * blk * 16), SCdev((size_t)nt2 * blk * 8);
    CUDA_TRY(cudaMemsetAsync(Rdev.p, 0, Rdev.bytes, st));
    response_2d_rows_impl<double>(h, rho_eq, g, 0, n1, (double2 *)Rdev.p);
    for (int it = 0; it < nt2; ++it) {
      double2 *RI = (double2 *)Rdev.p + (int64_t)it * 2 * blk;
      dft2d_sc_kernel<<<(unsigned)((blk + 255) / 256), 256, 0, st>>>(RI, RI + blk, n1, n3, dtau,
                                                                     (double *)SCdev.p + (int64_t)it * blk);
      count_launch(1);
      LAUNCH_CHECK();
    }
    std::vector<double> SC((size_t)nt2 * blk);
    CUDA_TRY(cudaMemcpyAsync(SC.data(), SCdev.p, SCdev.bytes, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    double L2 = 0;
    std::vector<double> Sbar(SC.size());
    for (size_t k = 0; k < SC.size(); ++k) {
      const double r = SC[k] - S_ref[k];
      L2 += r * r;
      Sbar[k] = 2.0 * r;
    }
    if (!std::isfinite(L2)) throw Fail{HEOM_ENONFINITE, "loss is not finite"};
    std::vector<double> Rbar((size_t)nt2 * 2 * blk * 2), tI, tII;
    for (int it = 0; it < nt2; ++it) {
      dft2d_adjoint(Sbar.data() + (size_t)it * blk, n1, n3, dtau, tI, tII);
      std::memcpy(Rbar.data() + (size_t)it * 2 * blk * 2, tI.data(), blk * 16);
      std::memcpy(Rbar.data() + ((size_t)it * 2 + 1) * blk * 2, tII.data(), blk * 16);
    }
    DeviceBuffer Rbar_d(Rbar.size() * 8);
    CUDA_TRY(cudaMemcpyAsync(Rbar_d.p, Rbar.data(), Rbar_d.bytes, cudaMemcpyHostToDevice, st));
    // ---- gradient accumulators and scratch
    AdjCtx c{};
    c.h = h;
    c.st = st;
    c.L = grad_layout(M);
    c.per = per;
    DeviceBuffer Gd((size_t)c.L.total * 8);
    CUDA_TRY(cudaMemsetAsync(Gd.p, 0, Gd.bytes, st));
    c.G = (double *)Gd.p;
    // branch chunk: J t1 rows (2J branches) per pass, sized to the free memory
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    const int64_t N3 = (int64_t)(n3 - 1) * m;
    int64_t n2max = 0;
    for (int64_t v : n2) n2max = std::max(n2max, v);
    const int64_t span_max = std::max<int64_t>(N3, n2max);
    const double states_per_branch = 8.0 + (double)std::min<int64_t>(Mck, std::max<int64_t>(1, span_max)) +
                                     (double)(span_max / Mck + 1) + 2.0;
    const double budget = 0.6 * (double)free_b - (double)(2 * n1 + 8) * sz1;
    int J = n1;
    while (J > 1 && 2.0 * J * states_per_branch * sz1 > budget) J = (J + 1) / 2;
    if (2.0 * J * states_per_branch * sz1 > budget) throw Fail{HEOM_ENOMEM, "gradient state does not fit in device memory"};
    const int cap = 2 * J;
    DeviceBuffer W4((size_t)cap * sz1), W3((size_t)cap * sz1), W2((size_t)cap * sz1), Ab((size_t)cap * sz1);
    c.W4 = (double2 *)W4.p;
    c.W3 = (double2 *)W3.p;
    c.W2 = (double2 *)W2.p;
    c.A = (double2 *)Ab.p;
    c.cap = cap;
    // ---- trunk T_j = G^{j m} mu-^x rho_eq, j < n1
    DeviceBuffer Tst((size_t)n1 * sz1), Tbar((size_t)n1 * sz1);
    CUDA_TRY(cudaMemsetAsync(Tbar.p, 0, Tbar.bytes, st));
    double2 *T = (double2 *)Tst.p, *Tb = (double2 *)Tbar.p;
    kick_into<double>(h, (const double2 *)rho_eq->buf.p, T, 1, 2, st);
    for (int j = 1; j < n1; ++j) {
      CUDA_TRY(cudaMemcpyAsync(T + (int64_t)j * per, T + (int64_t)(j - 1) * per, sz1, cudaMemcpyDeviceToDevice, st));
      rk4_steps<double>(h, T + (int64_t)j * per, c.W4, c.W3, 1, dt, m, st, HEOM_FP64);
    }
    const double c_re = 0.0, c_im = -1.0;   // i^3
    DeviceBuffer BR((size_t)cap * sz1), Y0((size_t)cap * sz1), lam((size_t)cap * sz1), tmp((size_t)cap * sz1),
        tmp2((size_t)cap * sz1);
    for (int it = 0; it < nt2; ++it) {
      const double2 *RbI = (const double2 *)Rbar_d.p + (int64_t)it * 2 * blk, *RbII = RbI + blk;
      for (int j0 = 0; j0 < n1; j0 += J) {
        const int nj = std::min(J, n1 - j0), B = 2 * nj;
        double2 *br = (double2 *)BR.p, *y0 = (double2 *)Y0.p, *lm = (double2 *)lam.p;
        double2 *t1 = (double2 *)tmp.p, *t2b = (double2 *)tmp2.p;
        // forward: second kick of both pathways, t2, third kick
        for (int j = 0; j < nj; ++j) {
          kick2_pair_kernel<double><<<grid_for(per), 256, 0, st>>>(T + (int64_t)(j0 + j) * per, br + (int64_t)j * per,
                                                                  br + (int64_t)(nj + j) * per, h->mup64, h->mum64, d, per);
          count_launch(1);
          LAUNCH_CHECK();
        }
        CUDA_TRY(cudaMemcpyAsync(t1, br, (size_t)B * sz1, cudaMemcpyDeviceToDevice, st));   // F = G^{n2} BR
        rk4_steps<double>(h, t1, c.W4, c.W3, B, dt, n2[it], st, HEOM_FP64);
        kick_into<double>(h, t1, y0, B, 1, st);                                              // Y0 = mu+^x F
        // t3: traces at t = k m; lam starts with the source of the last sample
        CUDA_TRY(cudaMemsetAsync(lm, 0, (size_t)B * sz1, st));
        auto trace_src = [&](int64_t t, const double2 *y, double2 *l) {
          if (t % m) return;
          const int k = (int)(t / m);
          trace_adjoint_kernel<<<(unsigned)((dd + 255) / 256), 256, 0, st>>>(
              l, y, RbI + (int64_t)j0 * n3 + k, n3, h->mu64, d, per, nj, c_re, c_im, c.G + c.L.mu);
          trace_adjoint_kernel<<<(unsigned)((dd + 255) / 256), 256, 0, st>>>(
              l + (int64_t)nj * per, y + (int64_t)nj * per, RbII + (int64_t)j0 * n3 + k, n3, h->mu64, d, per, nj,
              c_re, c_im, c.G + c.L.mu);
          count_launch(2);
          LAUNCH_CHECK();
        };
        {
          // state at the last sample, for its trace source
          DeviceBuffer yN((size_t)B * sz1);
          CUDA_TRY(cudaMemcpyAsync(yN.p, y0, (size_t)B * sz1, cudaMemcpyDeviceToDevice, st));
          rk4_steps<double>(h, (double2 *)yN.p, c.W4, c.W3, B, dt, N3, st, HEOM_FP64);
          trace_src(N3, (const double2 *)yN.p, lm);
          CUDA_TRY(cudaStreamSynchronize(st));
        }
        backprop_span(c, y0, N3, B, dt, Mck, lm, trace_src);
        // third kick: Fbar = mu-^x Y0bar; d/d mu+
        comm_grad(c, lm, t1, (int64_t)B * M.n_ado, 1.0, 0.0, 1.0, c.G + c.L.mup);
        kick_into<double>(h, lm, t2b, B, 2, st);
        // t2
        backprop_span(c, br, n2[it], B, dt, Mck, t2b, nullptr);
        // second kicks: I_j = mu+^x T_j, II_j = mu-^x (-T_j^dagger)
        double2 *Tj = T + (int64_t)j0 * per, *Tbj = Tb + (int64_t)j0 * per;
        const int64_t nI = (int64_t)nj * per;
        comm_grad(c, t2b, Tj, (int64_t)nj * M.n_ado, 1.0, 0.0, 1.0, c.G + c.L.mup);
        kick_into<double>(h, t2b, t1, nj, 2, st);
        axpy64(c, Tbj, t1, 1.0, nI);
        neg_dagger_kernel<<<grid_for(nI), 256, 0, st>>>(Tj, t1, d, nI);                     // U = -T^dagger
        count_launch(1);
        comm_grad(c, t2b + nI, t1, (int64_t)nj * M.n_ado, 1.0, 0.0, 1.0, c.G + c.L.mum);
        kick_into<double>(h, t2b + nI, t1, nj, 1, st);                                      // Ubar = mu+^x IIbar
        neg_dagger_kernel<<<grid_for(nI), 256, 0, st>>>(t1, y0, d, nI);
        count_launch(1);
        LAUNCH_CHECK();
        axpy64(c, Tbj, y0, 1.0, nI);
      }
    }
    // ---- trunk: sources Tbar_j at t = j m; then the first kick and the equilibration
    double2 *lm = (double2 *)lam.p;
    const int64_t N1 = (int64_t)(n1 - 1) * m;
    CUDA_TRY(cudaMemcpyAsync(lm, Tb + (int64_t)(n1 - 1) * per, sz1, cudaMemcpyDeviceToDevice, st));
    auto trunk_src = [&](int64_t t, const double2 *, double2 *l) {
      if (t % m) return;
      axpy64(c, l, Tb + (t / m) * per, 1.0, per);
    };
    backprop_span(c, T, N1, 1, dt, Mck, lm, trunk_src);
    comm_grad(c, lm, (const double2 *)rho_eq->buf.p, M.n_ado, 1.0, 0.0, 1.0, c.G + c.L.mum);
    double2 *eqbar = (double2 *)tmp.p;
    kick_into<double>(h, lm, eqbar, 1, 1, st);                                             // (mu-^x)^H = mu+^x
    DeviceBuffer rho0(sz1);
    CUDA_TRY(cudaMemsetAsync(rho0.p, 0, sz1, st));
    const double one[2] = {1.0, 0.0};
    CUDA_TRY(cudaMemcpyAsync(rho0.p, one, 16, cudaMemcpyHostToDevice, st));
    backprop_span(c, (const double2 *)rho0.p, rho_eq->eq_steps, 1, rho_eq->eq_dt, Mck, eqbar, nullptr);
    std::vector<double> G(c.L.total);
    CUDA_TRY(cudaMemcpyAsync(G.data(), Gd.p, Gd.bytes, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    // ---- chain rule to the twelve parameters
    for (int i = 0; i < 12; ++i) dtheta[i] = 0.0;
    for (Build &b : builds) {
      const Model P1 = b.p1.get(), M1 = b.m1.get(), P2 = b.p2.get(), M2 = b.m2.get();
      const double inv = 1.0 / (12 * b.step);
      auto dv = [&](double p1, double m1, double p2, double m2) { return (8 * (p1 - m1) - (p2 - m2)) * inv; };
      double s = 0;
      for (int64_t k = 0; k < dd; ++k) {
        const int64_t kt = (k % d) * d + k / d;   // mu- = (mu+)^T
        s += G[c.L.H + k] * dv(P1.H[k], M1.H[k], P2.H[k], M2.H[k]);
        s += G[c.L.mup + k] * dv(P1.mu_plus[k], M1.mu_plus[k], P2.mu_plus[k], M2.mu_plus[k]);
        s += G[c.L.mu + k] * dv(P1.mu[k], M1.mu[k], P2.mu[k], M2.mu[k]);
        s += G[c.L.mum + k] * dv(P1.mu_plus[kt], M1.mu_plus[kt], P2.mu_plus[kt], M2.mu_plus[kt]);
      }
      int64_t o = 0;
      for (int sm = 0; sm < M.n_modes; ++sm)
        for (size_t k = 0; k < P1.Vloc[sm].size(); ++k, ++o)
          s += G[c.L.v + o] * dv(P1.Vloc[sm][k], M1.Vloc[sm][k], P2.Vloc[sm][k], M2.Vloc[sm][k]);
      for (int j = 0; j < M.n_exp; ++j) {
        s += G[c.L.re + j] * dv(P1.exp_re[j], M1.exp_re[j], P2.exp_re[j], M2.exp_re[j]);
        s += G[c.L.im + j] * dv(P1.exp_im[j], M1.exp_im[j], P2.exp_im[j], M2.exp_im[j]);
        s += G[c.L.nu + j] * dv(P1.exp_nu[j], M1.exp_nu[j], P2.exp_nu[j], M2.exp_nu[j]);
      }
      dtheta[b.i] = s;
    }
    *loss = L2;
    for (int i = 0; i < 12; ++i)
      if (!std::isfinite(dtheta[i])) throw Fail{HEOM_ENONFINITE, "gradient is not finite"};
    return HEOM_OK;
  });
}

