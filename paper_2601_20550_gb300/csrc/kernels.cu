// Non-template kernels: 2D Fourier sums / correlation spectrum and state conversion.
#include "kernels.cuh"

namespace heom {

__global__ void dft2d_sc_kernel(const double2 *__restrict__ RI, const double2 *__restrict__ RII,
                                int n1, int n3, double dtau, double *__restrict__ SC) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n1 * n3) return;
  const int q = idx / n3, p = idx % n3;
  const int qf = (n1 - q) % n1;   // -Omega1 for the rephasing part
  double sr = 0, snr = 0;         // imaginary parts only
  for (int j = 0; j < n1; ++j) {
    const double wj = j == 0 ? 0.5 : 1.0;
    double s1r, c1r, s1n, c1n;
    sincospi(2.0 * (double)((long long)qf * j % n1) / n1, &s1r, &c1r);
    sincospi(2.0 * (double)((long long)q * j % n1) / n1, &s1n, &c1n);
    for (int k = 0; k < n3; ++k) {
      const double w = wj * (k == 0 ? 0.5 : 1.0);
      double s3, c3;
      sincospi(2.0 * (double)((long long)p * k % n3) / n3, &s3, &c3);
      const double2 a = RI[(long long)j * n3 + k];
      const double2 b = RII[(long long)j * n3 + k];
      // Im[(cos + i sin)(x + i y)] = sin x + cos y, phase = phase1 + phase3
      const double cr = c1r * c3 - s1r * s3, sr_ = s1r * c3 + c1r * s3;
      const double cn = c1n * c3 - s1n * s3, sn = s1n * c3 + c1n * s3;
      sr += w * (sr_ * a.x + cr * a.y);
      snr += w * (sn * b.x + cn * b.y);
    }
  }
  SC[idx] = dtau * dtau * (sr + snr);
}

__global__ void dft1d_kernel(const double2 *__restrict__ R, int n, double dtau, double *__restrict__ I) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double s = 0;
  for (int k = 0; k < n; ++k) {
    double sn, cs;
    sincospi(2.0 * (double)((long long)p * k % n) / n, &sn, &cs);
    const double w = k == 0 ? 0.5 : 1.0;
    s += w * (sn * R[k].x + cs * R[k].y);
  }
  I[p] = dtau * s;
}

__global__ void __launch_bounds__(256) stage_kernel_vb(const float2 *__restrict__ w, const float2 *y, float2 *out,
                                                       float alpha, VbModel M, int64_t total) {
  const int d = M.d;
  const int64_t dd = (int64_t)d * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t el = e % dd;
    const int64_t bn = e / dd;
    const int n = (int)(bn % M.n_ado);
    const int64_t br = bn / M.n_ado;
    const int a = (int)(el / d), b = (int)(el % d);
    const float2 *wb = w + br * M.n_ado * dd;
    const float2 *wn = wb + (int64_t)n * dd;
    float re = 0.f, im = 0.f;
    const float *Ha = M.H + (int64_t)a * d;
    for (int c = 0; c < d; ++c) {
      const float h1 = Ha[c], h2 = M.H[(int64_t)c * d + b];
      const float2 x = wn[(int64_t)c * d + b], z = wn[(int64_t)a * d + c];
      re += h1 * x.x - z.x * h2;
      im += h1 * x.y - z.y * h2;
    }
    float ore = im, oim = -re;
    const float dec = (float)M.decay[n];
    const float2 self = wn[el];
    ore -= dec * self.x;
    oim -= dec * self.y;
    for (int s = 0; s < M.n_modes; ++s) {
      const int o0 = M.nb_off[n * M.n_modes + s], o1 = M.nb_off[n * M.n_modes + s + 1];
      if (o0 == o1) continue;
      const float la = M.lam[s * d + a], lb = M.lam[s * d + b];
      const float f = la - lb, g = la + lb;
      for (int q = o0; q < o1; ++q) {
        const float2 x = wb[(int64_t)M.nb_idx[q] * dd + el];
        const float p = M.nb_cB[q] * g, qq = M.nb_cA[q] * f;
        ore += p * x.x + qq * x.y;
        oim += p * x.y - qq * x.x;
      }
    }
    const float2 yv = y[e];
    out[e] = make_float2(yv.x + alpha * ore, yv.y + alpha * oim);
  }
}

// Tiled variant for larger bases: one block per 32 x 32 output tile of one item,
// 8 rows x 32 columns of threads with 4 rows each.  The commutator's contraction
// runs over 32-wide slices of H' and w_n staged in shared memory (each element
// reused 32 times instead of re-read per output); the decay and system-bath terms
// are the same elementwise code as stage_kernel_vb, in the same summation order.
__global__ void __launch_bounds__(256) stage_kernel_vb_tiled(const float2 *__restrict__ w, const float2 *y,
                                                             float2 *out, float alpha, VbModel M, int tiles) {
  __shared__ float sHa[32][33], sHb[32][33];
  __shared__ float2 sWa[32][33], sWb[32][33];
  const int d = M.d;
  const int64_t dd = (int64_t)d * d;
  const int64_t item = blockIdx.x / (tiles * tiles);
  const int tile = (int)(blockIdx.x - item * tiles * tiles);
  const int a0 = (tile / tiles) * 32, b0 = (tile % tiles) * 32;
  const int n = (int)(item % M.n_ado);
  const int64_t br = item / M.n_ado;
  const float2 *wb = w + br * M.n_ado * dd;
  const float2 *wn = wb + (int64_t)n * dd;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
  for (int c0 = 0; c0 < d; c0 += 32) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = ty + 8 * i;                       // tile row / slice index
      const bool ca = c0 + tx < d, cr = c0 + r < d;
      sHa[r][tx] = (a0 + r < d && ca) ? M.H[(int64_t)(a0 + r) * d + c0 + tx] : 0.f;
      sWa[r][tx] = (a0 + r < d && ca) ? wn[(int64_t)(a0 + r) * d + c0 + tx] : make_float2(0.f, 0.f);
      sHb[r][tx] = (cr && b0 + tx < d) ? M.H[(int64_t)(c0 + r) * d + b0 + tx] : 0.f;
      sWb[r][tx] = (cr && b0 + tx < d) ? wn[(int64_t)(c0 + r) * d + b0 + tx] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float2 x = sWb[k][tx];
      const float h2 = sHb[k][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = ty + 8 * i;
        const float h1 = sHa[r][k];
        const float2 z = sWa[r][k];
        re[i] += h1 * x.x - z.x * h2;
        im[i] += h1 * x.y - z.y * h2;
      }
    }
    __syncthreads();
  }
  const int b = b0 + tx;
  if (b >= d) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty + 8 * i;
    if (a >= d) continue;
    const int64_t el = (int64_t)a * d + b;
    float ore = im[i], oim = -re[i];
    const float dec = (float)M.decay[n];
    const float2 self = wn[el];
    ore -= dec * self.x;
    oim -= dec * self.y;
    for (int s = 0; s < M.n_modes; ++s) {
      const int o0 = M.nb_off[n * M.n_modes + s], o1 = M.nb_off[n * M.n_modes + s + 1];
      if (o0 == o1) continue;
      const float la = M.lam[s * d + a], lb = M.lam[s * d + b];
      const float f = la - lb, g = la + lb;
      for (int q = o0; q < o1; ++q) {
        const float2 xv = wb[(int64_t)M.nb_idx[q] * dd + el];
        const float p = M.nb_cB[q] * g, qq = M.nb_cA[q] * f;
        ore += p * xv.x + qq * xv.y;
        oim += p * xv.y - qq * xv.x;
      }
    }
    const int64_t e = item * dd + el;
    const float2 yv = y[e];
    out[e] = make_float2(yv.x + alpha * ore, yv.y + alpha * oim);
  }
}

__global__ void convert_f64_to_f32(const double2 *__restrict__ x, float2 *__restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = make_float2((float)x[i].x, (float)x[i].y);
}

__global__ void convert_f32_to_f64(const float2 *__restrict__ x, double2 *__restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = make_double2((double)x[i].x, (double)x[i].y);
}

}  // namespace heom
