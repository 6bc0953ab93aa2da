// Kernels of the discrete adjoint of the FP64 propagation (reverse mode through
// the RK4 stages, kicks and traces of Sec. II.C), used by heom_response_2d_grad.
//
// Inner product: <x, y> = Re sum conj(x) y over every entry of every ADO and
// branch.  For a complex-linear map y = A x the adjoint is the conjugate
// transpose; the gradient of a real loss with respect to a real model entry M is
// Re <ybar, (dA/dM) x>.  The RHS adjoint L^H has the structure of L itself
// (H -> -H, each coupling entry n <- m with (cA, cB) becomes m <- n with
// (-cA, cB)), so it runs through stage_kernel<double> with a second DevModel;
// the kernels here only accumulate the model gradients and apply the trace and
// dagger adjoints.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "kernels.cuh"

namespace heom {

constexpr int kAdjMaxExp = 32;
constexpr int kAdjMaxVl = 4 * 16 * 16;   // sum_s n_s^2 (n_s <= 16)

// y += a x over n complex entries.
static __global__ void __launch_bounds__(256) axpy_kernel(double2 *__restrict__ y, const double2 *__restrict__ x, double a,
                                                   int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[e];
    y[e].x += a * v.x;
    y[e].y += a * v.y;
  }
}

// out_n = -(in_n)^dagger for every ADO matrix (the map that turns the R_I trunk
// into the R_II trunk; as a real-linear map it is its own adjoint).
static __global__ void __launch_bounds__(256) neg_dagger_kernel(const double2 *__restrict__ in, double2 *__restrict__ out,
                                                         int d, int64_t total) {
  const int64_t dd = (int64_t)d * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t el = e % dd, base = e - el;
    const int a = (int)(el / d), b = (int)(el % d);
    const double2 v = in[base + (int64_t)b * d + a];
    out[e] = make_double2(-v.x, v.y);
  }
}

// Commutator-type gradient: for every item (ADO matrix) i,
//   G[p][q] += alpha Re[ phase ( sum_b conj(g_i[p][b]) w_i[q][b] - sum_a w_i[a][p] conj(g_i[a][q]) ) ],
// the derivative of Re <g, phase^* ... > with respect to a matrix K in K^x w
// (phase = -i for the Hamiltonian term -i[H, w], 1 for a kick K^x w).  Only the
// component the phase selects is accumulated: the imaginary part for -i, the real
// part for 1 (half the arithmetic of the full complex product).
// Block = 16 x 16 entries of G, looping over a chunk of items with 16-wide
// slices of the contraction index staged in shared memory.
template <bool kImag>
__global__ void __launch_bounds__(256) comm_grad_kernel(const double2 *__restrict__ g, const double2 *__restrict__ w,
                                                        int64_t n_items, int d, double alpha, double *__restrict__ G) {
  __shared__ double2 sg1[16][17], sw1[16][17], sw2[16][17], sg2[16][17];
  const int tiles = (d + 15) / 16;
  const int tile = blockIdx.x % (tiles * tiles);
  const int chunk = blockIdx.x / (tiles * tiles);
  const int n_chunks = gridDim.x / (tiles * tiles);
  const int p0 = (tile / tiles) * 16, q0 = (tile % tiles) * 16;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  const int64_t dd = (int64_t)d * d;
  double acc = 0.0;
  for (int64_t i = chunk; i < n_items; i += n_chunks) {
    const double2 *gi = g + i * dd, *wi = w + i * dd;
    for (int k0 = 0; k0 < d; k0 += 16) {
      const int k = k0 + tx, kr = k0 + ty;
      const double2 z = make_double2(0.0, 0.0);
      sg1[ty][tx] = (p0 + ty < d && k < d) ? gi[(int64_t)(p0 + ty) * d + k] : z;
      sw1[ty][tx] = (q0 + ty < d && k < d) ? wi[(int64_t)(q0 + ty) * d + k] : z;
      sw2[ty][tx] = (kr < d && p0 + tx < d) ? wi[(int64_t)kr * d + p0 + tx] : z;
      sg2[ty][tx] = (kr < d && q0 + tx < d) ? gi[(int64_t)kr * d + q0 + tx] : z;
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        const double2 a1 = sg1[ty][kk], b1 = sw1[tx][kk];   // conj(g[p][k]) w[q][k]
        const double2 a2 = sw2[kk][ty], b2 = sg2[kk][tx];   // w[k][p] conj(g[k][q])
        if (kImag)
          acc += (a1.x * b1.y - a1.y * b1.x) - (a2.y * b2.x - a2.x * b2.y);
        else
          acc += (a1.x * b1.x + a1.y * b1.y) - (a2.x * b2.x + a2.y * b2.y);
      }
      __syncthreads();
    }
  }
  const int p = p0 + ty, q = q0 + tx;
  if (p < d && q < d) atomicAdd(G + (int64_t)p * d + q, alpha * acc);
}

// Gradients of the system-bath and decay terms of L (Eq. HEOM_DB) for one pair
// (g, w) of an adjoint and a forward state, summed over branches and ADOs:
//   Gv[s][p][r]  += alpha d/dv_s[p][r]   Re <g, V X^L - X^R V>,  X^L = sum (-i cA + cB) w_m,
//                                                                X^R = sum (-i cA - cB) w_m
//   Gre[j], Gim[j] += alpha n_j Re <g_n, -i [V_s, w_{n-e_j}]>,  alpha n_j Re <g_n, {V_s, w_{n-e_j}}>
//   Gnu[j]       -= alpha n_j Re <g_n, w_n>
// (cA = n_j Re c_j and cB = n_j Im c_j on down-neighbours; up-neighbours carry
// constants).  One block per item; warps walk rows for the V X^L part (mode
// digit of the row uniform per warp) and columns for the X^R V part.
// entry_exp[q] = exponential j of a down-neighbour entry, -1 for up entries.
static __global__ void __launch_bounds__(256) coupling_grad_kernel(const double2 *__restrict__ g,
                                                            const double2 *__restrict__ w, DevModel<double> M,
                                                            const int *__restrict__ ado, int n_exp,
                                                            const int *__restrict__ entry_exp, int64_t n_items,
                                                            double alpha, double *__restrict__ Gv,
                                                            double *__restrict__ Gre, double *__restrict__ Gim,
                                                            double *__restrict__ Gnu) {
  __shared__ double s_v[kAdjMaxVl];
  __shared__ double s_re[kAdjMaxExp], s_im[kAdjMaxExp];
  __shared__ double s_dot;
  const int d = M.d, S = M.n_modes;
  const int64_t dd = (int64_t)d * d;
  int nvl = 0;
  for (int s = 0; s < S; ++s) nvl += M.dims[s] * M.dims[s];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    for (int i = threadIdx.x; i < nvl; i += blockDim.x) s_v[i] = 0.0;
    for (int i = threadIdx.x; i < n_exp; i += blockDim.x) s_re[i] = s_im[i] = 0.0;
    if (threadIdx.x == 0) s_dot = 0.0;
    __syncthreads();
    const int n = (int)(item % M.n_ado);
    const double2 *gn = g + item * dd;
    const double2 *wb = w + (item - n) * dd;     // first ADO of this branch
    double dot = 0.0;
    // rows: V X^L part, decay, and the exponential gradients
    for (int a = warp; a < d; a += nwarps) {
      for (int c0 = 0; c0 < d; c0 += 32) {
        const int c = c0 + lane;
        const bool ok = c < d;
        const double2 gv = ok ? gn[(int64_t)a * d + c] : make_double2(0.0, 0.0);
        if (ok) {
          const double2 wv = wb[(int64_t)n * dd + (int64_t)a * d + c];
          dot += gv.x * wv.x + gv.y * wv.y;
        }
        for (int s = 0; s < S; ++s) {
          const int ns = M.dims[s], st = M.stride[s];
          const int as = (a / st) % ns, cs = ok ? (c / st) % ns : 0;
          const double *v = M.vloc + M.vloc_off[s];
          const int lo = M.nb_off[n * S + s], hi = M.nb_off[n * S + s + 1];
          for (int q = lo; q < hi; ++q) {
            const double2 *wm = wb + (int64_t)M.nb_idx[q] * dd;
            const double cA = M.nb_cA[q], cB = M.nb_cB[q];
            const int j = entry_exp[q];
            double vw_r = 0, vw_i = 0;
            for (int r = 0; r < ns; ++r) {
              const double2 x = ok ? wm[(int64_t)(a + (r - as) * st) * d + c] : make_double2(0.0, 0.0);
              // conj(g) (-i cA + cB) x, real part
              const double kr = cB, ki = -cA;
              const double xr = kr * x.x - ki * x.y, xi = kr * x.y + ki * x.x;
              double val = gv.x * xr + gv.y * xi;
              for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
              if (lane == 0) atomicAdd(&s_v[M.vloc_off[s] + as * ns + r], val);
              if (j >= 0) {
                const double vv = v[as * ns + r];
                vw_r += vv * x.x;
                vw_i += vv * x.y;
              }
            }
            if (j >= 0) {   // (V w_m)[a][c] and (w_m V)[a][c]
              double wv_r = 0, wv_i = 0;
              for (int r = 0; r < ns; ++r) {
                const double2 x = ok ? wm[(int64_t)a * d + c + (r - cs) * st] : make_double2(0.0, 0.0);
                const double vv = v[r * ns + cs];
                wv_r += x.x * vv;
                wv_i += x.y * vv;
              }
              const double nj = (double)ado[(int64_t)n * n_exp + j];
              const double cm_r = vw_r - wv_r, cm_i = vw_i - wv_i;   // [V, w]
              const double ac_r = vw_r + wv_r, ac_i = vw_i + wv_i;   // {V, w}
              // Re conj(g) (-i [V, w]) = g.x * cm_i - g.y * cm_r
              double vre = nj * (gv.x * cm_i - gv.y * cm_r);
              double vim = nj * (gv.x * ac_r + gv.y * ac_i);
              for (int o = 16; o > 0; o >>= 1) {
                vre += __shfl_xor_sync(0xffffffffu, vre, o);
                vim += __shfl_xor_sync(0xffffffffu, vim, o);
              }
              if (lane == 0) {
                atomicAdd(&s_re[j], vre);
                atomicAdd(&s_im[j], vim);
              }
            }
          }
        }
      }
    }
    // columns: - X^R V part
    for (int c = warp; c < d; c += nwarps) {
      for (int a0 = 0; a0 < d; a0 += 32) {
        const int a = a0 + lane;
        const bool ok = a < d;
        const double2 gv = ok ? gn[(int64_t)a * d + c] : make_double2(0.0, 0.0);
        for (int s = 0; s < S; ++s) {
          const int ns = M.dims[s], st = M.stride[s];
          const int cs = (c / st) % ns;
          const int lo = M.nb_off[n * S + s], hi = M.nb_off[n * S + s + 1];
          for (int q = lo; q < hi; ++q) {
            const double2 *wm = wb + (int64_t)M.nb_idx[q] * dd;
            const double cA = M.nb_cA[q], cB = M.nb_cB[q];
            for (int p = 0; p < ns; ++p) {
              const double2 x = ok ? wm[(int64_t)a * d + c + (p - cs) * st] : make_double2(0.0, 0.0);
              // conj(g) (-i cA - cB) x, real part, with a minus sign
              const double kr = -cB, ki = -cA;
              const double xr = kr * x.x - ki * x.y, xi = kr * x.y + ki * x.x;
              double val = -(gv.x * xr + gv.y * xi);
              for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
              if (lane == 0) atomicAdd(&s_v[M.vloc_off[s] + p * ns + cs], val);
            }
          }
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    if (lane == 0) atomicAdd(&s_dot, dot);
    __syncthreads();
    for (int i = threadIdx.x; i < nvl; i += blockDim.x)
      if (s_v[i] != 0.0) atomicAdd(Gv + i, alpha * s_v[i]);
    for (int j = threadIdx.x; j < n_exp; j += blockDim.x) {
      const double nj = (double)ado[(int64_t)n * n_exp + j];
      if (s_re[j] != 0.0) atomicAdd(Gre + j, alpha * s_re[j]);
      if (s_im[j] != 0.0) atomicAdd(Gim + j, alpha * s_im[j]);
      if (nj != 0.0) atomicAdd(Gnu + j, -alpha * nj * s_dot);
    }
    __syncthreads();
  }
}

// Trace adjoint: R_b = c tr{mu rho_{b,0}} for every branch b, c = i^order.
// lam_{b,0} += conj(c) Rbar_b mu^T, and Gmu[p][q] += Re(conj(Rbar_b) c rho_{b,0}[q][p]).
static __global__ void __launch_bounds__(256) trace_adjoint_kernel(double2 *__restrict__ lam, const double2 *__restrict__ rho,
                                                            const double2 *__restrict__ rbar, int64_t rbar_stride,
                                                            const double *__restrict__ mu, int d, int64_t per_branch,
                                                            int branches, double c_re, double c_im,
                                                            double *__restrict__ Gmu) {
  const int64_t dd = (int64_t)d * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < dd; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / d), b = (int)(e % d);
    const double m = mu[(int64_t)b * d + a];
    double gsum = 0.0;
    for (int br = 0; br < branches; ++br) {
      const double2 rb = rbar[(int64_t)br * rbar_stride];
      // conj(c) Rbar
      const double t_re = c_re * rb.x + c_im * rb.y, t_im = c_re * rb.y - c_im * rb.x;
      double2 &l = lam[(int64_t)br * per_branch + e];
      l.x += t_re * m;
      l.y += t_im * m;
      // Re(conj(Rbar) c rho[b][a]) for G[a][b]
      const double2 r = rho[(int64_t)br * per_branch + (int64_t)b * d + a];
      const double u_re = rb.x * c_re + rb.y * c_im, u_im = rb.x * c_im - rb.y * c_re;   // conj(Rbar) c
      gsum += u_re * r.x - u_im * r.y;
    }
    Gmu[e] += gsum;
  }
}

}  // namespace heom
