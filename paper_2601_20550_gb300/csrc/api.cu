// C-ABI entry points of libheom2dvs (declared in include/heom2dvs.h).
//
// The host code here only allocates, uploads the model built by model.cpp and
// sequences kernel launches; every step of the propagation, the kicks, the
// traces and the Fourier sums runs on the GPU.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <functional>
#include <future>
#include <memory>
#include <stdexcept>
#include <string>
#include <map>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "heom2dvs.h"
#include "internal.h"
#include "kernels.cuh"
#include "model.h"
#include "tc_stage.h"

namespace heom {

thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Allocation-failure injection: -1 = off; otherwise the number of device
// allocations that still succeed before every following one fails.
static std::atomic<int64_t> g_alloc_budget{-1};

cudaError_t device_malloc(void **p, size_t bytes) {
  int64_t b = g_alloc_budget.load();
  while (b >= 0) {
    if (b == 0) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
    if (g_alloc_budget.compare_exchange_weak(b, b - 1)) break;
  }
  return cudaMalloc(p, bytes);
}

}  // namespace heom

using namespace heom;

namespace heom {


// Necessary condition for RK4 stability: the largest Bohr frequency of H_S' and
// the largest ADO decay rate must each lie inside the RK4 region (|z| < 2.78 on
// the axes).  It does not bound the system-bath couplings.
void stability_check(heom_hier *h, double dt) {
  if (!(dt > 0) || !std::isfinite(dt)) throw Fail{HEOM_EINVAL, "dt must be > 0"};
  const Model &M = h->M;
  std::vector<double> A = M.H, w, Z;
  jacobi_eigh(A, M.d, w, Z);
  double spread = w.back() - w.front();
  double maxdecay = 0;
  for (double g : M.decay) maxdecay = std::max(maxdecay, g);
  if (dt * spread > 2.78 || dt * maxdecay > 2.78)
    throw Fail{HEOM_EUNSTABLE, "dt outside the RK4 stability region (dt*spread(H) = " +
                                   std::to_string(dt * spread) + ", dt*max decay = " +
                                   std::to_string(dt * maxdecay) + ")"};
}

// Launch-shape autotuner for the grid-stride stage kernels.  The first launch of
// a kernel kind at a given size times every candidate (block of 64, 128 or 256
// threads; 4, 16 or 64 blocks per SM, capped at one element per thread) on the
// real operands -- three timed launches each after one untimed -- and keeps the
// fastest for this hierarchy; a size whose default launch already takes over
// 50 ms keeps the default.  Candidate launches repeat the caller's first
// stage, whose output is scratch that the step overwrites next, so tuning
// changes no result.  Inside a stream capture, or when timing fails, the
// default shape (256 threads, grid_for) is used and nothing is cached.
enum TuneKind { kTuneStage64 = 0, kTuneStageVb = 1 };

static std::pair<int, int> tuned_shape(heom_hier *h, int kind, int64_t total, cudaStream_t st,
                                       const std::function<void(int, int)> &launch) {
  const std::pair<int, int> dflt(256, grid_for(total));
  auto it = h->tuned.find({kind, total});
  if (it != h->tuned.end()) return it->second;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return dflt;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return dflt;
  }
  std::pair<int, int> best = dflt;
  float best_ms = 1e30f;
  bool ok = true;
  {
    // one launch of the default shape first: launches longer than 50 ms are
    // saturated by their size and not worth 36 more, so the default is kept
    float ms = 0.f;
    cudaEventRecord(e0, st);
    launch(dflt.first, dflt.second);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ok = false;
    if (ok && ms > 50.f) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      LAUNCH_CHECK();
      h->tuned[{kind, total}] = dflt;
      return dflt;
    }
  }
  for (int block : {64, 128, 256})
    for (int per_sm : {4, 16, 64}) {
      const int64_t need = (total + block - 1) / block;
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, 152LL * per_sm * 256 / block));
      launch(block, grid);
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3; ++r) launch(block, grid);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        ok = false;
        break;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = {block, grid};
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  LAUNCH_CHECK();
  if (!ok) return dflt;
  h->tuned[{kind, total}] = best;
  return best;
}

// One RK4 step on branches [y] with scratch wa, wb, Horner form:
//   wa = y + dt/4 L(y); wb = y + dt/3 L(wa); wa = y + dt/2 L(wb); y = y + dt L(wa)
template <typename R>
void rk4_steps(heom_hier *h, typename CxT<R>::type *y, typename CxT<R>::type *wa,
                      typename CxT<R>::type *wb, int branches, double dt, int64_t nsteps,
                      cudaStream_t st, int precision) {
  const DevModel<R> &dm = dev_model<R>(h);
  const int64_t total = (int64_t)branches * dm.n_ado * dm.d * dm.d;
  if (total == 0 || nsteps <= 0) return;
  if (sizeof(R) == 4) {
    float2 *fy = (float2 *)y, *fa = (float2 *)wa, *fb = (float2 *)wb;
    if (precision == HEOM_TC) {
      if (!tc_supported(h->tc)) throw Fail{HEOM_EINVAL, "tensor-core path not prepared for this hierarchy"};
      tc_rk4_steps(h->tc, fy, fa, fb, branches, dt, nsteps, st);
    } else if (h->M.d >= kVbTiledMinD) {
      // larger bases: the commutator tiled through shared memory, one block per
      // 32 x 32 output tile of one item
      const int tiles = (h->M.d + 31) / 32;
      const int64_t nb = (int64_t)branches * h->M.n_ado * tiles * tiles;
      if (nb > 0x7fffffffLL) throw Fail{HEOM_EINVAL, "too many tiles for one launch"};
      for (int64_t s = 0; s < nsteps; ++s) {
        stage_kernel_vb_tiled<<<(unsigned)nb, 256, 0, st>>>(fy, fy, fa, (float)(dt / 4), h->vb, tiles);
        stage_kernel_vb_tiled<<<(unsigned)nb, 256, 0, st>>>(fa, fy, fb, (float)(dt / 3), h->vb, tiles);
        stage_kernel_vb_tiled<<<(unsigned)nb, 256, 0, st>>>(fb, fy, fa, (float)(dt / 2), h->vb, tiles);
        stage_kernel_vb_tiled<<<(unsigned)nb, 256, 0, st>>>(fa, fy, fy, (float)dt, h->vb, tiles);
        count_launch(4);
      }
    } else {
      const auto sh = tuned_shape(h, kTuneStageVb, total, st, [&](int block, int grid) {
        stage_kernel_vb<<<grid, block, 0, st>>>(fy, fy, fa, (float)(dt / 4), h->vb, total);
        count_launch(1);
      });
      const int grid = sh.second, block = sh.first;
      for (int64_t s = 0; s < nsteps; ++s) {
        stage_kernel_vb<<<grid, block, 0, st>>>(fy, fy, fa, (float)(dt / 4), h->vb, total);
        stage_kernel_vb<<<grid, block, 0, st>>>(fa, fy, fb, (float)(dt / 3), h->vb, total);
        stage_kernel_vb<<<grid, block, 0, st>>>(fb, fy, fa, (float)(dt / 2), h->vb, total);
        stage_kernel_vb<<<grid, block, 0, st>>>(fa, fy, fy, (float)dt, h->vb, total);
        count_launch(4);
      }
    }
    LAUNCH_CHECK();
    return;
  }
  const auto sh = tuned_shape(h, kTuneStage64, total, st, [&](int block, int grid) {
    stage_kernel<R><<<grid, block, 0, st>>>(y, y, wa, (R)(dt / 4), dm, total);
    count_launch(1);
  });
  const int grid = sh.second, block = sh.first;
  for (int64_t s = 0; s < nsteps; ++s) {
    stage_kernel<R><<<grid, block, 0, st>>>(y, y, wa, (R)(dt / 4), dm, total);
    stage_kernel<R><<<grid, block, 0, st>>>(wa, y, wb, (R)(dt / 3), dm, total);
    stage_kernel<R><<<grid, block, 0, st>>>(wb, y, wa, (R)(dt / 2), dm, total);
    stage_kernel<R><<<grid, block, 0, st>>>(wa, y, y, (R)dt, dm, total);
    count_launch(4);
  }
  LAUNCH_CHECK();
}

template <typename R>
void kick_into(heom_hier *h, const typename CxT<R>::type *in, typename CxT<R>::type *out,
                      int branches, int which, cudaStream_t st) {
  const Model &M = h->M;
  const int64_t total = (int64_t)branches * M.n_ado * M.d * M.d;
  kick_kernel<R><<<grid_for(total), 256, 0, st>>>(in, out, mu_of<R>(h, which), M.d, total);
  count_launch(1);
  LAUNCH_CHECK();
}

template <typename R>
void trace_into(heom_hier *h, const typename CxT<R>::type *w, int branches, int order,
                       double2 *out, int64_t ostride, cudaStream_t st) {
  const Model &M = h->M;
  const double *mu = sizeof(R) == 8 ? h->mu_trace : h->mu_vb64;
  trace_kernel<R><<<branches, 256, 0, st>>>(w, mu, M.d, M.n_ado, order, out, ostride);
  count_launch(1);
  LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// 2D response (Sec. II.C.2) in precision R.
// ---------------------------------------------------------------------------


// Original-basis complex128 ADOs -> coupling-basis complex64 (U^T x U), and back.
void to_coupling_basis(heom_hier *h, const double2 *x, float2 *out, int64_t elems, cudaStream_t st) {
  DeviceBuffer tmp(elems * 16);
  sim_left_kernel<double2><<<grid_for(elems), 256, 0, st>>>(x, (double2 *)tmp.p, h->U64, h->M.d, elems);
  sim_right_kernel<float2><<<grid_for(elems), 256, 0, st>>>((const double2 *)tmp.p, out, h->U64, h->M.d, elems);
  count_launch(2);
  LAUNCH_CHECK();
  CUDA_TRY(cudaStreamSynchronize(st));
}

static void from_coupling_basis(heom_hier *h, const float2 *x, double2 *out, int64_t elems, cudaStream_t st) {
  DeviceBuffer tmp(elems * 16);
  sim_left_kernel<float2><<<grid_for(elems), 256, 0, st>>>(x, (double2 *)tmp.p, h->UT64, h->M.d, elems);
  sim_right_kernel<double2><<<grid_for(elems), 256, 0, st>>>((const double2 *)tmp.p, out, h->UT64, h->M.d, elems);
  count_launch(2);
  LAUNCH_CHECK();
  CUDA_TRY(cudaStreamSynchronize(st));
}

void check_tc_error(heom_hier *h) {
  if (!h->tc.ready) return;
  int e = 0;
  CUDA_TRY(cudaMemcpy(&e, h->tc.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CUDA_TRY(cudaMemsetAsync(h->tc.err, 0, sizeof(int), h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    throw Fail{HEOM_ETIMEOUT, "a tensor-core stage wait ran out"};
  }
}

// Rows [jr0, jr1) of R_I and R_II into Rdev laid out [n_t2][2][jr1 - jr0][n3].
template <typename R>
void response_2d_rows_impl(heom_hier *h, const heom_state *eq, const heom_grid *g, int jr0, int jr1,
                                  double2 *Rdev) {
  using C = typename CxT<R>::type;
  const Model &M = h->M;
  cudaStream_t st = h->stream;
  const int n1 = jr1 - jr0, n3 = g->n3, m = g->steps_per_sample, nt2 = g->n_t2;
  const double dt = g->dt_fs;
  const int64_t per_branch = (int64_t)M.n_ado * M.d * M.d;
  const size_t cb = sizeof(C);
  // t2 in ascending order, as step counts
  std::vector<int> order(nt2);
  std::vector<int64_t> n2(nt2);
  for (int i = 0; i < nt2; ++i) {
    order[i] = i;
    double r = g->t2_fs[i] / dt;
    n2[i] = (int64_t)std::llround(r);
    if (g->t2_fs[i] < 0 || std::fabs(r - n2[i]) > 1e-6) throw Fail{HEOM_EINVAL, "t2 must be a non-negative multiple of dt"};
  }
  std::sort(order.begin(), order.end(), [&](int a, int b) { return n2[a] < n2[b]; });
  // single-branch buffers: equilibrium (precision R), trunk and its scratch
  DeviceBuffer eqR(per_branch * cb), T(per_branch * cb), ta(per_branch * cb), tb(per_branch * cb);
  if (sizeof(R) == 8) {
    CUDA_TRY(cudaMemcpyAsync(eqR.p, eq->buf.p, per_branch * cb, cudaMemcpyDeviceToDevice, st));
  } else {
    to_coupling_basis(h, (const double2 *)eq->buf.p, (float2 *)eqR.p, per_branch, st);
  }
  // branch chunk size: both pathways of jc t1 samples, 3 or 4 state sets
  const int nsets = nt2 > 1 ? 4 : 3;
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  const double budget = 0.85 * (double)free_b;
  int jc = n1;
  while (jc > 1 && (double)nsets * 2 * jc * per_branch * cb > budget) jc = (jc + 1) / 2;
  if ((double)nsets * 2 * jc * per_branch * cb > budget) throw Fail{HEOM_ENOMEM, "state does not fit in device memory"};
  const int64_t setb = 2LL * jc * per_branch * cb;
  DeviceBuffer P0(setb), P1(setb), P2(setb), P3(nsets == 4 ? setb : 16);
  for (int j0 = 0; j0 < n1; j0 += jc) {
    const int nj = std::min(jc, n1 - j0);
    const int B = 2 * nj;
    C *BR = (C *)P0.p;
    // trunk: rephasing first kick, propagated to t1 = j0 m dt.  On the tensor-core
    // path the single-branch trunk runs on the FP32 CUDA-core stage (same
    // coupling-basis complex64 state): its error would reach every t1 row, and one
    // branch is a small share of the scan's work.
    const int trunk_prec = M.precision == HEOM_TC ? HEOM_FP32 : M.precision;
    PhaseRange phase("heom: t1 trunk");
    kick_into<R>(h, (const C *)eqR.p, (C *)T.p, 1, 2, st);
    rk4_steps<R>(h, (C *)T.p, (C *)ta.p, (C *)tb.p, 1, dt, (int64_t)(jr0 + j0) * m, st, trunk_prec);
    for (int j = 0; j < nj; ++j) {
      if (j > 0) rk4_steps<R>(h, (C *)T.p, (C *)ta.p, (C *)tb.p, 1, dt, m, st, trunk_prec);
      kick2_pair_kernel<R><<<grid_for(per_branch), 256, 0, st>>>(
          (const C *)T.p, BR + (int64_t)j * per_branch, BR + (int64_t)(nj + j) * per_branch,
          mu_of<R>(h, 1), mu_of<R>(h, 2), M.d, per_branch);
      count_launch(1);
      LAUNCH_CHECK();
    }
    int64_t t_now = 0;
    if (sizeof(R) == 4 && M.precision == HEOM_TC) tc_reserve(h->tc, (int64_t)B * M.n_ado);
    for (int oi = 0; oi < nt2; ++oi) {
      const int it = order[oi];
      C *Y = (C *)P1.p, *WA = (C *)P2.p, *WB = (C *)(nsets == 4 ? P3.p : P0.p);
      phase.next("heom: t2 fork");
      rk4_steps<R>(h, BR, Y, WA, B, dt, n2[it] - t_now, st, M.precision);
      t_now = n2[it];
      kick_into<R>(h, BR, Y, B, 1, st);
      // the coupling kernel's shape is tuned (once per size) before the capture
      if (sizeof(R) == 4 && M.precision == HEOM_TC)
        tc_tune({TcRk4Set{&h->tc, (float2 *)Y, (float2 *)WA, (float2 *)WB, B}}, dt, st);
      // the t3 scan (n3 samples of m RK4 steps and two traces) is captured once
      // into a CUDA graph and replayed as a single launch
      phase.next("heom: t3 scan");
      GraphCapture cap(st);
      for (int k = 0; k < n3; ++k) {
        if (k > 0) rk4_steps<R>(h, Y, WA, WB, B, dt, m, st, M.precision);
        for (int pw = 0; pw < 2; ++pw) {
          double2 *base = Rdev + (int64_t)it * 2 * n1 * n3 + (int64_t)pw * n1 * n3 + (int64_t)j0 * n3 + k;
          trace_into<R>(h, Y + (int64_t)pw * nj * per_branch, nj, 3, base, n3, st);
        }
      }
      cap.replay();
    }
  }
}

// Instantiations used by the other translation units (batched.cu, grad.cu, steady.cu).
template void rk4_steps<double>(heom_hier *, double2 *, double2 *, double2 *, int, double, int64_t, cudaStream_t, int);
template void rk4_steps<float>(heom_hier *, float2 *, float2 *, float2 *, int, double, int64_t, cudaStream_t, int);
template void kick_into<double>(heom_hier *, const double2 *, double2 *, int, int, cudaStream_t);
template void kick_into<float>(heom_hier *, const float2 *, float2 *, int, int, cudaStream_t);
template void trace_into<double>(heom_hier *, const double2 *, int, int, double2 *, int64_t, cudaStream_t);
template void trace_into<float>(heom_hier *, const float2 *, int, int, double2 *, int64_t, cudaStream_t);
template void response_2d_rows_impl<double>(heom_hier *, const heom_state *, const heom_grid *, int, int, double2 *);
template void response_2d_rows_impl<float>(heom_hier *, const heom_state *, const heom_grid *, int, int, double2 *);

// Device set-up of a hierarchy: stream, operator and table uploads.  Runs at the
// first call that needs the GPU, so the host-side model can be built and
// inspected without one.
void ensure_device(heom_hier *h) {
  if (h->on_device) return;
  Model &M = h->M;
  // (a set-up that failed part-way is redone from the start by the next call;
  // what it allocated stays owned by the handle)
  // a blocking stream: ordered with work on the legacy default stream, so a state
  // zeroed or filled there before a call is seen by the call's kernels
  if (!h->stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamDefault));
  std::vector<double> vl;
  DevModel<double> d64{};
  d64.d = M.d;
  d64.n_ado = M.n_ado;
  d64.n_modes = M.n_modes;
  for (int s = 0; s < M.n_modes; ++s) {
    d64.dims[s] = M.dims[s];
    d64.stride[s] = M.stride[s];
    d64.vloc_off[s] = (int)vl.size();
    vl.insert(vl.end(), M.Vloc[s].begin(), M.Vloc[s].end());
  }
  DevModel<float> d32{};
  d32.d = d64.d;
  d32.n_ado = d64.n_ado;
  d32.n_modes = d64.n_modes;
  std::memcpy(d32.dims, d64.dims, sizeof(d64.dims));
  std::memcpy(d32.stride, d64.stride, sizeof(d64.stride));
  std::memcpy(d32.vloc_off, d64.vloc_off, sizeof(d64.vloc_off));
  d64.H = h->up(M.H);
  d32.H = h->up(cast_vec<float>(M.H));
  d64.vloc = h->up(vl);
  d32.vloc = h->up(cast_vec<float>(vl));
  d64.decay = d32.decay = h->up(M.decay);
  d64.nb_off = d32.nb_off = h->up(M.nb_off);
  d64.nb_idx = d32.nb_idx = h->up(M.nb_idx);
  d64.nb_cA = h->up(M.nb_cA);
  d64.nb_cB = h->up(M.nb_cB);
  d32.nb_cA = h->up(cast_vec<float>(M.nb_cA));
  d32.nb_cB = h->up(cast_vec<float>(M.nb_cB));
  h->dm64 = d64;
  h->dm32 = d32;
  std::vector<double> mum((size_t)M.d * M.d);
  for (int a = 0; a < M.d; ++a)
    for (int b = 0; b < M.d; ++b) mum[(size_t)a * M.d + b] = M.mu_plus[(size_t)b * M.d + a];
  h->mu64 = h->up(M.mu);
  h->mup64 = h->up(M.mu_plus);
  h->mum64 = h->up(mum);
  h->mu32 = h->up(cast_vec<float>(M.mu));
  h->mup32 = h->up(cast_vec<float>(M.mu_plus));
  h->mum32 = h->up(cast_vec<float>(mum));
  h->mu_trace = h->mu64;
  // coupling eigenbasis (FP32 and tensor-core paths)
  std::vector<double> UT((size_t)M.d * M.d), mumv((size_t)M.d * M.d);
  for (int a = 0; a < M.d; ++a)
    for (int b = 0; b < M.d; ++b) {
      UT[(size_t)a * M.d + b] = M.vb_U[(size_t)b * M.d + a];
      mumv[(size_t)a * M.d + b] = M.vb_mu_plus[(size_t)b * M.d + a];
    }
  h->U64 = h->up(M.vb_U);
  h->UT64 = h->up(UT);
  h->mu_vb64 = h->up(M.vb_mu);
  h->mu_vb32 = h->up(cast_vec<float>(M.vb_mu));
  h->mup_vb32 = h->up(cast_vec<float>(M.vb_mu_plus));
  h->mum_vb32 = h->up(cast_vec<float>(mumv));
  std::vector<float> lam((size_t)M.n_modes * M.d);
  for (int s = 0; s < M.n_modes; ++s)
    for (int a = 0; a < M.d; ++a) lam[(size_t)s * M.d + a] = (float)M.vb_lam[s][(a / M.stride[s]) % M.dims[s]];
  VbModel vb{};
  vb.d = M.d;
  vb.n_ado = M.n_ado;
  vb.n_modes = M.n_modes;
  vb.H = h->up(cast_vec<float>(M.vb_H));
  vb.lam = h->up(lam);
  vb.decay = d64.decay;
  vb.nb_off = d64.nb_off;
  vb.nb_idx = d64.nb_idx;
  vb.nb_cA = d32.nb_cA;
  vb.nb_cB = d32.nb_cB;
  h->vb = vb;
  if (M.precision == HEOM_TC) tc_build(h->tc, M, h->vb, h->allocs);
  // the table uploads above are complete before any launch on any stream
  CUDA_TRY(cudaDeviceSynchronize());
  h->on_device = true;
}

}  // namespace heom




// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *heom_last_error(void) { return g_last_error.c_str(); }
uint64_t heom_launch_count(void) { return g_launches.load(); }

heom_status heom_build_hierarchy(const heom_model *m, heom_hier **out) {
  if (!m || !out) return fail(HEOM_EINVAL, "null argument");
  *out = nullptr;
  return guarded([&]() -> heom_status {
    if (m->precision < 0 || m->precision > 2) throw Fail{HEOM_EINVAL, "precision must be 0, 1 or 2"};
    auto h = new heom_hier();
    try {
      h->desc = *m;
      h->desc_modes.assign(m->modes, m->modes + m->n_modes);
      if (m->n_pairs > 0 && m->pairs) h->desc_pairs.assign(m->pairs, m->pairs + m->n_pairs);
      h->desc.modes = h->desc_modes.data();
      h->desc.pairs = h->desc_pairs.empty() ? nullptr : h->desc_pairs.data();
      h->desc.n_pairs = (int)h->desc_pairs.size();
      h->M = build_model(*m);
      if (h->M.n_modes > kMaxModes) throw Fail{HEOM_EINVAL, "too many modes"};
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
    return HEOM_OK;
  });
}

heom_status heom_get_info(const heom_hier *h, heom_hier_info *info) {
  if (!h || !info) return fail(HEOM_EINVAL, "null argument");
  info->d = h->M.d;
  info->n_ado = h->M.n_ado;
  info->n_exp = h->M.n_exp;
  info->n_modes = h->M.n_modes;
  info->precision = h->M.precision;
  info->beta = h->M.beta;
  return HEOM_OK;
}

heom_status heom_get_operators(const heom_hier *h, double *H, double *mu, double *mu_plus, double *bath,
                               int32_t *ado) {
  if (!h) return fail(HEOM_EINVAL, "null handle");
  const Model &M = h->M;
  if (H) std::memcpy(H, M.H.data(), M.H.size() * sizeof(double));
  if (mu) std::memcpy(mu, M.mu.data(), M.mu.size() * sizeof(double));
  if (mu_plus) std::memcpy(mu_plus, M.mu_plus.data(), M.mu_plus.size() * sizeof(double));
  if (bath)
    for (int j = 0; j < M.n_exp; ++j) {
      bath[4 * j] = M.exp_mode[j];
      bath[4 * j + 1] = M.exp_nu[j];
      bath[4 * j + 2] = M.exp_re[j];
      bath[4 * j + 3] = M.exp_im[j];
    }
  if (ado) std::memcpy(ado, M.ado.data(), M.ado.size() * sizeof(int32_t));
  return HEOM_OK;
}

heom_status heom_get_mode(const heom_hier *h, int s, double *energies, double *qk) {
  if (!h || s < 0 || s >= h->M.n_modes) return fail(HEOM_EINVAL, "bad handle or mode index");
  const ModeBasis &mb = h->M.modes[s];
  if (energies) std::memcpy(energies, mb.E.data(), mb.n * sizeof(double));
  if (qk)
    for (int k = 1; k <= 4; ++k) std::memcpy(qk + (size_t)(k - 1) * mb.n * mb.n, mb.q[k].data(), (size_t)mb.n * mb.n * sizeof(double));
  return HEOM_OK;
}

heom_status heom_state_create(const heom_hier *h, int branches, int precision, heom_state **out) {
  if (!h || !out || branches < 1 || precision < 0 || precision > 2) return fail(HEOM_EINVAL, "bad state arguments");
  *out = nullptr;
  return guarded([&]() -> heom_status {
    ensure_device(const_cast<heom_hier *>(h));
    auto s = new heom_state();
    s->branches = branches;
    s->precision = precision;
    s->d = h->M.d;
    s->n_ado = h->M.n_ado;
    s->hier = const_cast<heom_hier *>(h);
    try {
      s->buf.alloc(s->elems() * s->elem_bytes());
      // zeroed on the hierarchy's stream and complete before the call returns, so
      // that work the caller issues next, on any stream, sees the zeros
      CUDA_TRY(cudaMemsetAsync(s->buf.p, 0, s->buf.bytes, h->stream));
      CUDA_TRY(cudaStreamSynchronize(h->stream));
    } catch (...) {
      delete s;
      throw;
    }
    *out = s;
    return HEOM_OK;
  });
}

int heom_state_branches(const heom_state *s) { return s ? s->branches : 0; }

heom_status heom_state_upload(heom_state *s, const double *host) {
  if (!s || !host) return fail(HEOM_EINVAL, "null argument");
  return guarded([&]() -> heom_status {
    const int64_t n = s->elems();
    cudaStream_t st = s->hier->stream;
    if (s->precision == HEOM_FP64) {
      CUDA_TRY(cudaMemcpyAsync(s->buf.p, host, n * 16, cudaMemcpyHostToDevice, st));
      CUDA_TRY(cudaStreamSynchronize(st));
    } else {
      DeviceBuffer tmp(n * 16);
      CUDA_TRY(cudaMemcpyAsync(tmp.p, host, n * 16, cudaMemcpyHostToDevice, st));
      to_coupling_basis(s->hier, (const double2 *)tmp.p, (float2 *)s->buf.p, n, st);
    }
    return HEOM_OK;
  });
}

heom_status heom_state_download(const heom_state *s, double *host) {
  if (!s || !host) return fail(HEOM_EINVAL, "null argument");
  return guarded([&]() -> heom_status {
    const int64_t n = s->elems();
    if (s->precision == HEOM_FP64) {
      CUDA_TRY(cudaMemcpy(host, s->buf.p, n * 16, cudaMemcpyDeviceToHost));
    } else {
      DeviceBuffer tmp(n * 16);
      from_coupling_basis(s->hier, (const float2 *)s->buf.p, (double2 *)tmp.p, n, s->hier->stream);
      CUDA_TRY(cudaMemcpy(host, tmp.p, n * 16, cudaMemcpyDeviceToHost));
    }
    return HEOM_OK;
  });
}

heom_status heom_state_copy_out(const heom_state *s, double *host) { return heom_state_download(s, host); }

heom_status heom_propagate(heom_hier *h, heom_state *rho, double dt_fs, int64_t n_steps) {
  if (!h || !rho || n_steps < 0) return fail(HEOM_EINVAL, "bad propagate arguments");
  if (rho->d != h->M.d || rho->n_ado != h->M.n_ado) return fail(HEOM_EINVAL, "state does not match hierarchy");
  PhaseRange phase("heom: propagate");
  return guarded([&]() -> heom_status {
    stability_check(h, dt_fs);
    ensure_device(h);
    const size_t bytes = rho->elems() * rho->elem_bytes();
    DeviceBuffer a(bytes), b(bytes);
    if (rho->precision == HEOM_FP64)
      rk4_steps<double>(h, (double2 *)rho->buf.p, (double2 *)a.p, (double2 *)b.p, rho->branches, dt_fs, n_steps, h->stream, HEOM_FP64);
    else
      rk4_steps<float>(h, (float2 *)rho->buf.p, (float2 *)a.p, (float2 *)b.p, rho->branches, dt_fs, n_steps, h->stream, rho->precision);
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    check_tc_error(h);
    return HEOM_OK;
  });
}

heom_status heom_propagate_dev(heom_hier *h, void *state, void *scratch_a, void *scratch_b, int branches,
                               int precision, double dt_fs, int64_t n_steps, void *stream) {
  if (!h || !state || !scratch_a || !scratch_b || branches < 1 || n_steps < 0 || precision < 0 || precision > 2)
    return fail(HEOM_EINVAL, "bad propagate_dev arguments");
  if ((((uintptr_t)state | (uintptr_t)scratch_a | (uintptr_t)scratch_b) & (precision == HEOM_FP64 ? 15u : 7u)))
    return fail(HEOM_EINVAL, "state buffers must be aligned to their complex element size");
  return guarded([&]() -> heom_status {
    stability_check(h, dt_fs);
    ensure_device(h);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == HEOM_FP64)
      rk4_steps<double>(h, (double2 *)state, (double2 *)scratch_a, (double2 *)scratch_b, branches, dt_fs, n_steps, st, precision);
    else
      rk4_steps<float>(h, (float2 *)state, (float2 *)scratch_a, (float2 *)scratch_b, branches, dt_fs, n_steps, st, precision);
    return HEOM_OK;
  });
}

heom_status heom_kick(heom_hier *h, heom_state *rho, int which) {
  if (!h || !rho || which < 0 || which > 2) return fail(HEOM_EINVAL, "bad kick arguments");
  return guarded([&]() -> heom_status {
    ensure_device(h);
    const size_t bytes = rho->elems() * rho->elem_bytes();
    DeviceBuffer tmp(bytes);
    if (rho->precision == HEOM_FP64)
      kick_into<double>(h, (const double2 *)rho->buf.p, (double2 *)tmp.p, rho->branches, which, h->stream);
    else
      kick_into<float>(h, (const float2 *)rho->buf.p, (float2 *)tmp.p, rho->branches, which, h->stream);
    CUDA_TRY(cudaMemcpyAsync(rho->buf.p, tmp.p, bytes, cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return HEOM_OK;
  });
}

heom_status heom_trace(heom_hier *h, const heom_state *rho, int order, double *out) {
  if (!h || !rho || !out) return fail(HEOM_EINVAL, "bad trace arguments");
  return guarded([&]() -> heom_status {
    ensure_device(h);
    DeviceBuffer o((size_t)rho->branches * 16);
    if (rho->precision == HEOM_FP64)
      trace_into<double>(h, (const double2 *)rho->buf.p, rho->branches, order, (double2 *)o.p, 1, h->stream);
    else
      trace_into<float>(h, (const float2 *)rho->buf.p, rho->branches, order, (double2 *)o.p, 1, h->stream);
    CUDA_TRY(cudaMemcpyAsync(out, o.p, (size_t)rho->branches * 16, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return HEOM_OK;
  });
}

heom_status heom_equilibrate(heom_hier *h, double dt_fs, double t_max_fs, double tol, heom_state **rho_eq) {
  if (!h || !rho_eq || !(t_max_fs >= 0)) return fail(HEOM_EINVAL, "bad equilibrate arguments");
  PhaseRange phase("heom: equilibrate");
  *rho_eq = nullptr;
  {
    heom_status e = guarded([&]() -> heom_status {
      stability_check(h, dt_fs);
      ensure_device(h);
      return HEOM_OK;
    });
    if (e != HEOM_OK) return e;
  }
  heom_state *s = nullptr;
  heom_status st0 = heom_state_create(h, 1, HEOM_FP64, &s);
  if (st0 != HEOM_OK) return st0;
  heom_status rc = guarded([&]() -> heom_status {
    stability_check(h, dt_fs);
    const Model &M = h->M;
    const int64_t per = (int64_t)M.n_ado * M.d * M.d;
    double one[2] = {1.0, 0.0};
    CUDA_TRY(cudaMemcpyAsync(s->buf.p, one, 16, cudaMemcpyHostToDevice, h->stream));   // rho_0 = |0><0|
    DeviceBuffer a(per * 16), b(per * 16);
    const int64_t nmax = (int64_t)std::llround(t_max_fs / dt_fs);
    s->eq_dt = dt_fs;
    if (tol <= 0) {
      rk4_steps<double>(h, (double2 *)s->buf.p, (double2 *)a.p, (double2 *)b.p, 1, dt_fs, nmax, h->stream, HEOM_FP64);
      CUDA_TRY(cudaStreamSynchronize(h->stream));
      s->eq_steps = nmax;
      return HEOM_OK;
    }
    DeviceBuffer norms((size_t)M.n_ado * 8), zero(per * 16);
    CUDA_TRY(cudaMemsetAsync(zero.p, 0, per * 16, h->stream));
    std::vector<double> hn(M.n_ado);
    int64_t done = 0;
    while (done < nmax) {
      int64_t chunk = std::min<int64_t>(100, nmax - done);
      rk4_steps<double>(h, (double2 *)s->buf.p, (double2 *)a.p, (double2 *)b.p, 1, dt_fs, chunk, h->stream, HEOM_FP64);
      done += chunk;
      s->eq_steps = done;
      // residual: a = 0 + 1 * L(rho)
      stage_kernel<double><<<grid_for(per), 256, 0, h->stream>>>((const double2 *)s->buf.p, (const double2 *)zero.p,
                                                                  (double2 *)a.p, 1.0, h->dm64, per);
      ado_norms_kernel<double><<<M.n_ado, 256, 0, h->stream>>>((const double2 *)a.p, (int64_t)M.d * M.d, M.n_ado, (double *)norms.p);
      count_launch(2);
      LAUNCH_CHECK();
      CUDA_TRY(cudaMemcpyAsync(hn.data(), norms.p, M.n_ado * 8, cudaMemcpyDeviceToHost, h->stream));
      CUDA_TRY(cudaStreamSynchronize(h->stream));
      double res = 0;
      for (double v : hn) res = std::max(res, v);
      ado_norms_kernel<double><<<1, 256, 0, h->stream>>>((const double2 *)s->buf.p, (int64_t)M.d * M.d, 1, (double *)norms.p);
      count_launch(1);
      double n0 = 0;
      CUDA_TRY(cudaMemcpyAsync(&n0, norms.p, 8, cudaMemcpyDeviceToHost, h->stream));
      CUDA_TRY(cudaStreamSynchronize(h->stream));
      if (!std::isfinite(res) || !std::isfinite(n0)) throw Fail{HEOM_ENONFINITE, "equilibrium residual is not finite"};
      if (std::sqrt(res) <= tol * std::sqrt(n0)) return HEOM_OK;
    }
    g_last_error = "equilibrium tolerance not reached by t_max";
    return HEOM_ENOTCONV;
  });
  if (rc == HEOM_OK || rc == HEOM_ENOTCONV) {
    *rho_eq = s;
  } else {
    heom_free_state(s);
  }
  return rc;
}


static void rows_dispatch(heom_hier *h, const heom_state *rho_eq, const heom_grid *g, int j0, int j1, double2 *Rdev) {
  if (h->M.precision == HEOM_FP64)
    response_2d_rows_impl<double>(h, rho_eq, g, j0, j1, Rdev);
  else
    response_2d_rows_impl<float>(h, rho_eq, g, j0, j1, Rdev);
}

heom_status heom_response_2d(heom_hier *h, const heom_state *rho_eq, const heom_grid *g, double *R_I,
                             double *R_II, double *S_C) {
  heom_status a = check_response_args(h, rho_eq, g);
  if (a != HEOM_OK) return a;
  return guarded([&]() -> heom_status {
    ensure_device(h);
    stability_check(h, g->dt_fs);
    const int n1 = g->n1, n3 = g->n3, nt2 = g->n_t2;
    DeviceBuffer Rdev((size_t)nt2 * 2 * n1 * n3 * 16), SCdev((size_t)nt2 * n1 * n3 * 8);
    CUDA_TRY(cudaMemsetAsync(Rdev.p, 0, Rdev.bytes, h->stream));
    rows_dispatch(h, rho_eq, g, 0, n1, (double2 *)Rdev.p);
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    check_tc_error(h);
    PhaseRange phase("heom: 2D DFT");
    const double dtau = g->dt_fs * g->steps_per_sample;
    for (int it = 0; it < nt2; ++it) {
      double2 *RI = (double2 *)Rdev.p + (int64_t)it * 2 * n1 * n3;
      dft2d_sc_kernel<<<(n1 * n3 + 255) / 256, 256, 0, h->stream>>>(RI, RI + (int64_t)n1 * n3, n1, n3, dtau,
                                                                     (double *)SCdev.p + (int64_t)it * n1 * n3);
      count_launch(1);
      LAUNCH_CHECK();
    }
    std::vector<double> Rh((size_t)nt2 * 2 * n1 * n3 * 2);
    CUDA_TRY(cudaMemcpyAsync(Rh.data(), Rdev.p, Rdev.bytes, cudaMemcpyDeviceToHost, h->stream));
    if (S_C) CUDA_TRY(cudaMemcpyAsync(S_C, SCdev.p, SCdev.bytes, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    const size_t blk = (size_t)n1 * n3 * 2;
    for (int it = 0; it < nt2; ++it) {
      if (R_I) std::memcpy(R_I + it * blk, Rh.data() + (size_t)it * 2 * blk, blk * 8);
      if (R_II) std::memcpy(R_II + it * blk, Rh.data() + (size_t)it * 2 * blk + blk, blk * 8);
    }
    for (double v : Rh)
      if (!std::isfinite(v)) throw Fail{HEOM_ENONFINITE, "response is not finite"};
    return HEOM_OK;
  });
}


heom_status heom_response_2d_rows(heom_hier *h, const heom_state *rho_eq, const heom_grid *g, int j0, int j1,
                                  double *R_I, double *R_II) {
  heom_status a = check_response_args(h, rho_eq, g);
  if (a != HEOM_OK) return a;
  if (j0 < 0 || j1 > g->n1 || j0 >= j1) return fail(HEOM_EINVAL, "bad row range");
  return guarded([&]() -> heom_status {
    ensure_device(h);
    stability_check(h, g->dt_fs);
    const int nr = j1 - j0, n3 = g->n3, nt2 = g->n_t2;
    DeviceBuffer Rdev((size_t)nt2 * 2 * nr * n3 * 16);
    CUDA_TRY(cudaMemsetAsync(Rdev.p, 0, Rdev.bytes, h->stream));
    rows_dispatch(h, rho_eq, g, j0, j1, (double2 *)Rdev.p);
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    check_tc_error(h);
    std::vector<double> Rh((size_t)nt2 * 2 * nr * n3 * 2);
    CUDA_TRY(cudaMemcpyAsync(Rh.data(), Rdev.p, Rdev.bytes, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    const size_t blk = (size_t)nr * n3 * 2;
    for (int it = 0; it < nt2; ++it) {
      if (R_I) std::memcpy(R_I + it * blk, Rh.data() + (size_t)it * 2 * blk, blk * 8);
      if (R_II) std::memcpy(R_II + it * blk, Rh.data() + (size_t)it * 2 * blk + blk, blk * 8);
    }
    for (double v : Rh)
      if (!std::isfinite(v)) throw Fail{HEOM_ENONFINITE, "response is not finite"};
    return HEOM_OK;
  });
}

heom_status heom_spectrum_2d(const double *R_I, const double *R_II, int n_t2, int n1, int n3, double dtau_fs,
                             double *S_C) {
  if (!R_I || !R_II || !S_C || n_t2 < 1 || n1 < 1 || n3 < 1 || !(dtau_fs > 0))
    return fail(HEOM_EINVAL, "bad spectrum arguments");
  return guarded([&]() -> heom_status {
    const size_t blk = (size_t)n1 * n3;
    DeviceBuffer R((size_t)n_t2 * 2 * blk * 16), S((size_t)n_t2 * blk * 8);
    for (int it = 0; it < n_t2; ++it) {
      CUDA_TRY(cudaMemcpy((char *)R.p + (size_t)it * 2 * blk * 16, R_I + it * blk * 2, blk * 16, cudaMemcpyHostToDevice));
      CUDA_TRY(cudaMemcpy((char *)R.p + ((size_t)it * 2 + 1) * blk * 16, R_II + it * blk * 2, blk * 16,
                          cudaMemcpyHostToDevice));
    }
    for (int it = 0; it < n_t2; ++it) {
      const double2 *RI = (const double2 *)R.p + (size_t)it * 2 * blk;
      dft2d_sc_kernel<<<(unsigned)((blk + 255) / 256), 256>>>(RI, RI + blk, n1, n3, dtau_fs, (double *)S.p + it * blk);
      count_launch(1);
      LAUNCH_CHECK();
    }
    CUDA_TRY(cudaMemcpy(S_C, S.p, S.bytes, cudaMemcpyDeviceToHost));
    return HEOM_OK;
  });
}

heom_status heom_state_broadcast(const heom_state *src, heom_state *dst) {
  if (!src || !dst || src->d != dst->d || src->n_ado != dst->n_ado) return fail(HEOM_EINVAL, "bad broadcast arguments");
  return guarded([&]() -> heom_status {
    const int64_t per = (int64_t)src->n_ado * src->d * src->d;
    // branch 0 (with the basis/precision conversion), then device copies
    char *out0 = (char *)dst->buf.p;
    if (src->precision == dst->precision || (src->precision != HEOM_FP64 && dst->precision != HEOM_FP64)) {
      CUDA_TRY(cudaMemcpy(out0, src->buf.p, per * src->elem_bytes(), cudaMemcpyDeviceToDevice));
    } else if (src->precision == HEOM_FP64) {
      to_coupling_basis(dst->hier, (const double2 *)src->buf.p, (float2 *)out0, per, dst->hier->stream);
    } else {
      from_coupling_basis(dst->hier, (const float2 *)src->buf.p, (double2 *)out0, per, dst->hier->stream);
    }
    for (int b = 1; b < dst->branches; ++b)
      CUDA_TRY(cudaMemcpy(out0 + (size_t)b * per * dst->elem_bytes(), out0, per * dst->elem_bytes(),
                          cudaMemcpyDeviceToDevice));
    CUDA_TRY(cudaDeviceSynchronize());
    return HEOM_OK;
  });
}

void *heom_state_device_ptr(heom_state *s) { return s ? s->buf.p : nullptr; }

heom_status heom_state_export_dev(const heom_state *s, void *dst, void *stream) {
  if (!s || !dst) return fail(HEOM_EINVAL, "null argument");
  return guarded([&]() -> heom_status {
    CUDA_TRY(cudaMemcpyAsync(dst, s->buf.p, s->elems() * s->elem_bytes(), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return HEOM_OK;
  });
}

heom_status heom_state_import_dev(heom_state *s, const void *src, void *stream) {
  if (!s || !src) return fail(HEOM_EINVAL, "null argument");
  return guarded([&]() -> heom_status {
    CUDA_TRY(cudaMemcpyAsync(s->buf.p, src, s->elems() * s->elem_bytes(), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return HEOM_OK;
  });
}

heom_status heom_kick_dev(heom_hier *h, const void *in, void *out, int branches, int precision, int which,
                          void *stream) {
  if (!h || !in || !out || in == out || branches < 1 || precision < 0 || precision > 2 || which < 0 || which > 2)
    return fail(HEOM_EINVAL, "bad kick_dev arguments");
  return guarded([&]() -> heom_status {
    ensure_device(h);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == HEOM_FP64)
      kick_into<double>(h, (const double2 *)in, (double2 *)out, branches, which, st);
    else
      kick_into<float>(h, (const float2 *)in, (float2 *)out, branches, which, st);
    return HEOM_OK;
  });
}

heom_status heom_trace_dev(heom_hier *h, const void *state, int branches, int precision, int order, void *out,
                           void *stream) {
  if (!h || !state || !out || branches < 1 || precision < 0 || precision > 2) return fail(HEOM_EINVAL, "bad trace_dev arguments");
  return guarded([&]() -> heom_status {
    ensure_device(h);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == HEOM_FP64)
      trace_into<double>(h, (const double2 *)state, branches, order, (double2 *)out, 1, st);
    else
      trace_into<float>(h, (const float2 *)state, branches, order, (double2 *)out, 1, st);
    return HEOM_OK;
  });
}

heom_status heom_response_1d(heom_hier *h, const heom_state *rho_eq, double dt_fs, int m, int n, double *R1,
                             double *I) {
  if (!h || !rho_eq || !R1 || m < 1 || n < 1) return fail(HEOM_EINVAL, "bad response_1d arguments");
  if (rho_eq->precision != HEOM_FP64 || rho_eq->branches != 1 || rho_eq->d != h->M.d)
    return fail(HEOM_EINVAL, "rho_eq must be a single-branch FP64 state of this hierarchy");
  return guarded([&]() -> heom_status {
    ensure_device(h);
    stability_check(h, dt_fs);
    const Model &M = h->M;
    const int64_t per = (int64_t)M.n_ado * M.d * M.d;
    DeviceBuffer y(per * 16), a(per * 16), b(per * 16), Rd((size_t)n * 16);
    kick_into<double>(h, (const double2 *)rho_eq->buf.p, (double2 *)y.p, 1, 0, h->stream);
    for (int k = 0; k < n; ++k) {
      if (k > 0) rk4_steps<double>(h, (double2 *)y.p, (double2 *)a.p, (double2 *)b.p, 1, dt_fs, m, h->stream, HEOM_FP64);
      trace_into<double>(h, (const double2 *)y.p, 1, 1, (double2 *)Rd.p + k, 1, h->stream);
    }
    CUDA_TRY(cudaMemcpyAsync(R1, Rd.p, (size_t)n * 16, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (I) {
      DeviceBuffer Id((size_t)n * 8);
      dft1d_kernel<<<(n + 127) / 128, 128, 0, h->stream>>>((const double2 *)Rd.p, n, dt_fs * m, (double *)Id.p);
      count_launch(1);
      LAUNCH_CHECK();
      CUDA_TRY(cudaMemcpyAsync(I, Id.p, (size_t)n * 8, cudaMemcpyDeviceToHost, h->stream));
      CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    return HEOM_OK;
  });
}

heom_status heom_set_wait_limit_ns(heom_hier *h, uint64_t ns) {
  if (!h || ns == 0) return fail(HEOM_EINVAL, "bad wait limit arguments");
  h->tc.wait_ns = ns;
  return HEOM_OK;
}

void heom_debug_fail_alloc(int64_t after) { g_alloc_budget.store(after < 0 ? -1 : after); }

heom_status heom_debug_force_tc_shape(int shape) { return tc_force_shape(shape) ? HEOM_OK : HEOM_EINVAL; }

int heom_tc_shape_count(void) { return tc_shape_count(); }

heom_status heom_tc_shape_params(int shape, int *rows_per_thread, int *row_groups, int *ados_per_block,
                                 int *flags) {
  return tc_shape_params(shape, rows_per_thread, row_groups, ados_per_block, flags) ? HEOM_OK : HEOM_EINVAL;
}

#ifndef HEOM_TC_STAGE_TAG
#define HEOM_TC_STAGE_TAG "unknown"
#endif
const char *heom_source_tag(void) { return HEOM_TC_STAGE_TAG; }

int heom_get_tc_shape(const heom_hier *h, int64_t elements, int *rows_per_thread, int *row_groups,
                      int *ados_per_block, int *flags) {
  if (!h) return 0;
  auto it = h->tc.vt_tuned.find(elements);
  if (it == h->tc.vt_tuned.end()) return 0;
  return tc_shape_params(it->second.shape, rows_per_thread, row_groups, ados_per_block, flags) ? 1 : 0;
}

void heom_free_hier(heom_hier *h) { delete h; }
void heom_free_state(heom_state *s) { delete s; }

}  // extern "C"

// Read-only views of a hierarchy for entry points defined in other files.
namespace heom {
bool hier_on_device(const heom_hier *h) { return h && h->on_device; }
const DevModel<double> &hier_dm64(const heom_hier *h) { return h->dm64; }
void hier_set_error(const char *msg) { g_last_error = msg; }
}  // namespace heom

extern "C" int heom_get_tuning(const heom_hier *h, int cap, int *kind, int64_t *elements, int *block, int *grid) {
  if (!h) return 0;
  int k = 0;
  for (const auto &e : h->tuned) {
    if (k < cap) {
      if (kind) kind[k] = e.first.first;
      if (elements) elements[k] = e.first.second;
      if (block) block[k] = e.second.first;
      if (grid) grid[k] = e.second.second;
    }
    ++k;
  }
  for (const auto &e : h->tc.vt_tuned) {
    if (k < cap) {
      if (kind) kind[k] = 2;
      if (elements) elements[k] = e.first;
      if (block) block[k] = e.second.block;
      if (grid) grid[k] = (int)e.second.grid;
    }
    ++k;
  }
  return k;
}

