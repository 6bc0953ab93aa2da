// CUDA kernels of the HEOM-2DVS hot path (generic CUDA-core versions).
//
// State layout in HBM: [branch][ado][d][d] complex, row-major, ADO stride d*d,
// complex as (re, im) pairs (double2 for FP64, float2 for the mixed paths).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace heom {

template <typename R> struct CxT;
template <> struct CxT<double> { using type = double2; };
template <> struct CxT<float> { using type = float2; };

constexpr int kMaxModes = 8;

// Device view of the model (all pointers are device pointers).
template <typename R>
struct DevModel {
  int d, n_ado, n_modes;
  int dims[kMaxModes], stride[kMaxModes], vloc_off[kMaxModes];
  const R *H;        // d x d
  const R *vloc;     // concatenated n_s x n_s blocks
  const double *decay;   // [n_ado] sum_j n_j nu_j
  const int *nb_off;     // [n_ado * n_modes + 1]
  const int *nb_idx;     // neighbour ADO index
  const R *nb_cA, *nb_cB;
};

// ---------------------------------------------------------------------------
// Fused RK4 stage (Eq. HEOM_DB right-hand side, Horner form of the RK4 step):
//   out = y + alpha * L(w)
// L(w)_n = -i [H, w_n] - gamma_n w_n + sum_s ( -i [V_s, A_s] + {V_s, B_s} ),
// A_s = sum cA w_m, B_s = sum cB w_m over the coupling list of (n, s):
// up-neighbours n + e_j with (cA, cB) = (1, 0) and down-neighbours n - e_j with
// (n_j Re c_j, n_j Im c_j).  V_s acts on mode s of the product index only.
// One thread per output element; out may alias y (each element is read and
// written by the same thread) but not w.
// ---------------------------------------------------------------------------
// One element e of the fused stage (branch, ADO, row, column flattened).
template <typename R>
__device__ __forceinline__ void stage_element(const typename CxT<R>::type *__restrict__ w,
                                              const typename CxT<R>::type *y, typename CxT<R>::type *out,
                                              R alpha, const DevModel<R> &M, int64_t e) {
  using C = typename CxT<R>::type;
  const int d = M.d;
  const int64_t dd = (int64_t)d * d;
  const int64_t el = e % dd;
  const int64_t bn = e / dd;
  const int n = (int)(bn % M.n_ado);
  const int64_t br = bn / M.n_ado;
  const int a = (int)(el / d), b = (int)(el % d);
  const C *wb = w + br * M.n_ado * dd;
  const C *wn = wb + (int64_t)n * dd;
  R re = 0, im = 0;
  const R *Ha = M.H + (int64_t)a * d;
  // Each product is its own fused multiply-add into the running sum (one FP64
  // pipe operation per multiply-add; the grouped form h1 x - z h2 costs three).
  for (int c = 0; c < d; ++c) {
    const R h1 = Ha[c];
    const R h2 = M.H[(int64_t)c * d + b];
    const C x = wn[(int64_t)c * d + b];
    const C z = wn[(int64_t)a * d + c];
    re = fma(h1, x.x, re);
    im = fma(h1, x.y, im);
    re = fma(-z.x, h2, re);
    im = fma(-z.y, h2, im);
  }
  // -i [H, w]
  R ore = im, oim = -re;
  const R dec = (R)M.decay[n];
  const C self = wn[el];
  ore -= dec * self.x;
  oim -= dec * self.y;
  for (int s = 0; s < M.n_modes; ++s) {
    const int o0 = M.nb_off[n * M.n_modes + s], o1 = M.nb_off[n * M.n_modes + s + 1];
    if (o0 == o1) continue;
    const int ns = M.dims[s], st = M.stride[s];
    const int as = (a / st) % ns, bs = (b / st) % ns;
    const int abase = a - as * st, bbase = b - bs * st;
    const R *V = M.vloc + M.vloc_off[s];
    for (int q = o0; q < o1; ++q) {
      const C *wm = wb + (int64_t)M.nb_idx[q] * dd;
      R lx = 0, ly = 0, rx = 0, ry = 0;
      for (int k = 0; k < ns; ++k) {
        const R vl = V[as * ns + k];
        const C xl = wm[(int64_t)(abase + k * st) * d + b];
        lx += vl * xl.x;
        ly += vl * xl.y;
        const R vr = V[k * ns + bs];
        const C xr = wm[(int64_t)a * d + bbase + k * st];
        rx += xr.x * vr;
        ry += xr.y * vr;
      }
      const R cA = M.nb_cA[q], cB = M.nb_cB[q];
      ore += cA * (ly - ry) + cB * (lx + rx);
      oim += -cA * (lx - rx) + cB * (ly + ry);
    }
  }
  const C yv = y[e];
  C o;
  o.x = yv.x + alpha * ore;
  o.y = yv.y + alpha * oim;
  out[e] = o;
}

template <typename R>
__global__ void __launch_bounds__(256) stage_kernel(const typename CxT<R>::type *__restrict__ w,
                                                    const typename CxT<R>::type *y,
                                                    typename CxT<R>::type *out, R alpha,
                                                    DevModel<R> M, int64_t total) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    stage_element<R>(w, y, out, alpha, M, e);
}

// The same stage for several hierarchies (parameter sets, any basis size) in one
// launch: set k owns elements [begin_k, begin_k + total_k) of the flattened
// index space and has its own model and state pointers.
template <typename R>
struct SetStage {
  DevModel<R> M;
  const typename CxT<R>::type *w, *y;
  typename CxT<R>::type *out;
  int64_t begin, total;
};

template <typename R>
__global__ void __launch_bounds__(256) multi_stage_kernel(const SetStage<R> *__restrict__ sets, int n_sets,
                                                          R alpha, int64_t grand_total) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < grand_total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < n_sets && e >= sets[k + 1].begin) ++k;
    const SetStage<R> &S = sets[k];
    stage_element<R>(S.w, S.y, S.out, alpha, S.M, e - S.begin);
  }
}

// out = K w - w K for every ADO of every branch (dipole kick K^x).  K real d x d.
template <typename R>
__global__ void __launch_bounds__(256) kick_kernel(const typename CxT<R>::type *__restrict__ w,
                                                   typename CxT<R>::type *__restrict__ out,
                                                   const R *__restrict__ K, int d, int64_t total) {
  using C = typename CxT<R>::type;
  const int64_t dd = (int64_t)d * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t el = e % dd;
    const C *wn = w + (e - el);
    const int a = (int)(el / d), b = (int)(el % d);
    R re = 0, im = 0;
    for (int c = 0; c < d; ++c) {
      const R k1 = K[(int64_t)a * d + c], k2 = K[(int64_t)c * d + b];
      const C x = wn[(int64_t)c * d + b], z = wn[(int64_t)a * d + c];
      re += k1 * x.x - z.x * k2;
      im += k1 * x.y - z.y * k2;
    }
    C o;
    o.x = re;
    o.y = im;
    out[e] = o;
  }
}

// Second kick of both pathways from one t1 trunk sample (Sec. II.C procedure):
// the non-rephasing trunk equals -(rephasing trunk)^dagger ADO by ADO because the
// equilibrium ADOs are Hermitian and Eq. HEOM_DB commutes with the dagger.
//   outI  = K2I^x  T
//   outII = K2II^x (-T^dagger)
// T: one branch (n_ado x d x d); outI/outII: one branch each.
template <typename R>
__global__ void __launch_bounds__(256) kick2_pair_kernel(const typename CxT<R>::type *__restrict__ T,
                                                         typename CxT<R>::type *__restrict__ outI,
                                                         typename CxT<R>::type *__restrict__ outII,
                                                         const R *__restrict__ KI, const R *__restrict__ KII,
                                                         int d, int64_t total) {
  using C = typename CxT<R>::type;
  const int64_t dd = (int64_t)d * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t el = e % dd;
    const C *wn = T + (e - el);
    const int a = (int)(el / d), b = (int)(el % d);
    R re = 0, im = 0, re2 = 0, im2 = 0;
    for (int c = 0; c < d; ++c) {
      const C x = wn[(int64_t)c * d + b], z = wn[(int64_t)a * d + c];
      const R k1 = KI[(int64_t)a * d + c], k2 = KI[(int64_t)c * d + b];
      re += k1 * x.x - z.x * k2;
      im += k1 * x.y - z.y * k2;
      // U = -T^dagger: U[c][b] = -conj(T[b][c]), U[a][c] = -conj(T[c][a])
      const C xt = wn[(int64_t)b * d + c], zt = wn[(int64_t)c * d + a];
      const R l1 = KII[(int64_t)a * d + c], l2 = KII[(int64_t)c * d + b];
      re2 += l1 * (-xt.x) - (-zt.x) * l2;
      im2 += l1 * (xt.y) - (zt.y) * l2;
    }
    C o;
    o.x = re;
    o.y = im;
    outI[e] = o;
    o.x = re2;
    o.y = im2;
    outII[e] = o;
  }
}

// R[br * ostride] = i^order * tr{mu w_{br, ado 0}}, FP64 accumulation.  One block per branch.
template <typename R>
__global__ void __launch_bounds__(256) trace_kernel(const typename CxT<R>::type *__restrict__ w,
                                                    const double *__restrict__ mu, int d, int n_ado,
                                                    int order, double2 *__restrict__ R_out,
                                                    int64_t ostride) {
  using C = typename CxT<R>::type;
  const int64_t dd = (int64_t)d * d;
  const int br = blockIdx.x;
  const C *w0 = w + (int64_t)br * n_ado * dd;
  double re = 0, im = 0;
  for (int64_t el = threadIdx.x; el < dd; el += blockDim.x) {
    const int a = (int)(el / d), b = (int)(el % d);
    const double m = mu[(int64_t)b * d + a];
    const C x = w0[el];
    re += m * (double)x.x;
    im += m * (double)x.y;
  }
  __shared__ double sre[256], sim[256];
  sre[threadIdx.x] = re;
  sim[threadIdx.x] = im;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sre[threadIdx.x] += sre[threadIdx.x + s];
      sim[threadIdx.x] += sim[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double tr = sre[0], ti = sim[0];
    // multiply by i^order
    for (int k = 0; k < (order & 3); ++k) {
      double t = tr;
      tr = -ti;
      ti = t;
    }
    R_out[(int64_t)br * ostride] = make_double2(tr, ti);
  }
}

// Trapezoid 2D Fourier sum (Eqs. 2D-rephasing, 2D-nonrephasing) and the
// correlation spectrum (Eq. correlation-spectrum) for one t2:
//   S_X(q, p) = Im[dtau^2 sum_{j,k} w_j w_k exp(2 pi i (q j / n1 + p k / n3)) R_X[j][k]]
//   S_C(q, p) = S_R((n1 - q) mod n1, p) + S_NR(q, p)
// One thread per (q, p); FP64.
__global__ void dft2d_sc_kernel(const double2 *__restrict__ RI, const double2 *__restrict__ RII,
                                int n1, int n3, double dtau, double *__restrict__ SC);

// I(Omega_p) = Im[dtau sum_k w_k exp(2 pi i p k / n) R[k]] (linear absorption, Eq. R1 transform)
__global__ void dft1d_kernel(const double2 *__restrict__ R, int n, double dtau, double *__restrict__ I);

// y = (R) x : precision conversion of a state
__global__ void convert_f64_to_f32(const double2 *__restrict__ x, float2 *__restrict__ y, int64_t n);
__global__ void convert_f32_to_f64(const float2 *__restrict__ x, double2 *__restrict__ y, int64_t n);

// ---------------------------------------------------------------------------
// Coupling-eigenbasis representation (mixed-precision paths).  Every V_s is
// diagonal there, so V_s^x and V_s^o act elementwise with the factors
// lam_s[a_s] -+ lam_s[b_s]; H' = U^T H_S' U is dense.
// ---------------------------------------------------------------------------
struct VbModel {
  int d, n_ado, n_modes;
  const float *H;          // d x d, coupling basis
  const float *lam;        // [n_modes][d]: lam_s[digit_s(a)] for every product index a
  const double *decay;     // [n_ado]
  const int *nb_off, *nb_idx;
  const float *nb_cA, *nb_cB;
};

// Fused RK4 stage in the coupling basis on CUDA cores (FP32):
//   out = y + alpha * ( -i [H', w_n] - gamma_n w_n + sum_nb kappa_nb(a, b) w_nb )
// kappa = -i cA (lam_a - lam_b) + cB (lam_a + lam_b) for the coupling list of (n, s).
__global__ void __launch_bounds__(256) stage_kernel_vb(const float2 *__restrict__ w, const float2 *y, float2 *out,
                                                       float alpha, VbModel M, int64_t total);
// The same stage with the commutator tiled through shared memory (one block per
// 32 x 32 output tile of one item; grid = items x tiles^2, tiles = ceil(d / 32)).
// out may alias y but not w.
constexpr int kVbTiledMinD = 24;
__global__ void __launch_bounds__(256) stage_kernel_vb_tiled(const float2 *__restrict__ w, const float2 *y,
                                                             float2 *out, float alpha, VbModel M, int tiles);

// Similarity transform of every ADO: out_n = P^T x_n P (double accumulation).
// Two passes through tmp (double2, same element count as x).
template <typename Tin>
__global__ void __launch_bounds__(256) sim_left_kernel(const Tin *__restrict__ x, double2 *__restrict__ tmp,
                                                       const double *__restrict__ P, int d, int64_t total) {
  const int64_t dd = (int64_t)d * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t el = e % dd;
    const Tin *xn = x + (e - el);
    const int a = (int)(el / d), b = (int)(el % d);
    double re = 0, im = 0;
    for (int c = 0; c < d; ++c) {
      const double p = P[(int64_t)c * d + a];
      re += p * (double)xn[(int64_t)c * d + b].x;
      im += p * (double)xn[(int64_t)c * d + b].y;
    }
    tmp[e] = make_double2(re, im);
  }
}

template <typename Tout>
__global__ void __launch_bounds__(256) sim_right_kernel(const double2 *__restrict__ tmp, Tout *__restrict__ out,
                                                        const double *__restrict__ P, int d, int64_t total) {
  const int64_t dd = (int64_t)d * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t el = e % dd;
    const double2 *tn = tmp + (e - el);
    const int a = (int)(el / d), b = (int)(el % d);
    double re = 0, im = 0;
    for (int c = 0; c < d; ++c) {
      const double p = P[(int64_t)c * d + b];
      re += tn[(int64_t)a * d + c].x * p;
      im += tn[(int64_t)a * d + c].y * p;
    }
    Tout o;
    o.x = re;
    o.y = im;
    out[e] = o;
  }
}

// Per-ADO squared Frobenius norms of one branch: out[n] = ||w_n||_F^2
template <typename R>
__global__ void ado_norms_kernel(const typename CxT<R>::type *__restrict__ w, int64_t dd, int n_ado,
                                 double *__restrict__ out) {
  const int n = blockIdx.x;
  if (n >= n_ado) return;
  const typename CxT<R>::type *wn = w + (int64_t)n * dd;
  double s = 0;
  for (int64_t el = threadIdx.x; el < dd; el += blockDim.x) {
    double x = wn[el].x, yv = wn[el].y;
    s += x * x + yv * yv;
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = sh[0];
}

}  // namespace heom
