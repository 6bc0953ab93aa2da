// Vector kernels of the restarted GMRES solve for the stationary hierarchy
// (heom_steady_state): block-partial inner products of one vector with several
// basis vectors, and a combination of basis vectors added to a vector.  The
// Arnoldi bookkeeping (Hessenberg matrix, Givens rotations) is host code.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace heom {

constexpr int kKrylovBlocks = 512;

// partial[blk * k + j] = sum over this block's slice of conj(V_j[e]) w[e], j < k.
static __global__ void __launch_bounds__(256) multi_dot_kernel(const double2 *__restrict__ V, int64_t n, int k,
                                                        const double2 *__restrict__ w, double2 *__restrict__ partial) {
  __shared__ double sre[256], sim[256];
  for (int j = 0; j < k; ++j) {
    const double2 *v = V + (int64_t)j * n;
    double re = 0.0, im = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
      const double2 a = v[e], b = w[e];
      re += a.x * b.x + a.y * b.y;
      im += a.x * b.y - a.y * b.x;
    }
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
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * k + j] = make_double2(sre[0], sim[0]);
    __syncthreads();
  }
}

// w += sum_{j < k} c_j V_j (complex coefficients c on the device).
static __global__ void __launch_bounds__(256) multi_axpy_kernel(double2 *__restrict__ w, const double2 *__restrict__ V,
                                                         int64_t n, int k, const double2 *__restrict__ c) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = w[e];
    for (int j = 0; j < k; ++j) {
      const double2 v = V[(int64_t)j * n + e], cj = c[j];
      acc.x += cj.x * v.x - cj.y * v.y;
      acc.y += cj.x * v.y + cj.y * v.x;
    }
    w[e] = acc;
  }
}

// x = a x (complex a).
static __global__ void __launch_bounds__(256) zscal_kernel(double2 *__restrict__ x, int64_t n, double ar, double ai) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[e];
    x[e] = make_double2(ar * v.x - ai * v.y, ar * v.y + ai * v.x);
  }
}

}  // namespace heom
