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
#include "adjoint.cuh"
#include "kernels.cuh"
#include "krylov.cuh"
#include "model.h"
#include "tc_stage.h"

namespace heom {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

struct Fail {
  heom_status st;
  std::string msg;
};

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      throw Fail{HEOM_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)};       \
  } while (0)

#define LAUNCH_CHECK()                                                                   \
  do {                                                                                   \
    cudaError_t _e = cudaGetLastError();                                                 \
    if (_e != cudaSuccess) throw Fail{HEOM_ECUDA, std::string("launch: ") + cudaGetErrorString(_e)}; \
  } while (0)

template <typename T>
static T *dev_upload(const std::vector<T> &v) {
  T *p = nullptr;
  size_t bytes = std::max<size_t>(1, v.size() * sizeof(T));
  if (cudaMalloc(&p, bytes) != cudaSuccess) throw Fail{HEOM_ENOMEM, "cudaMalloc failed (model tables)"};
  if (!v.empty()) CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return p;
}

template <typename T>
static std::vector<T> cast_vec(const std::vector<double> &v) {
  return std::vector<T>(v.begin(), v.end());
}

struct DeviceBuffer {
  void *p = nullptr;
  size_t bytes = 0;
  DeviceBuffer() = default;
  explicit DeviceBuffer(size_t n) { alloc(n); }
  void alloc(size_t n) {
    release();
    if (n == 0) n = 16;
    if (cudaMalloc(&p, n) != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      throw Fail{HEOM_ENOMEM, "cudaMalloc of " + std::to_string(n) + " bytes failed"};
    }
    bytes = n;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  ~DeviceBuffer() { release(); }
  DeviceBuffer(const DeviceBuffer &) = delete;
  DeviceBuffer &operator=(const DeviceBuffer &) = delete;
};

static int grid_for(int64_t total) {
  int64_t blocks = (total + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, 152LL * 64));
}

}  // namespace heom

using namespace heom;

struct heom_hier {
  Model M;
  cudaStream_t stream = nullptr;
  // device copies
  std::vector<void *> allocs;
  DevModel<double> dm64{};
  DevModel<float> dm32{};
  double *mu64 = nullptr, *mup64 = nullptr, *mum64 = nullptr;
  float *mu32 = nullptr, *mup32 = nullptr, *mum32 = nullptr;
  double *mu_trace = nullptr;   // FP64 mu for traces
  TcOperators tc{};             // tensor-core operator tiles (HEOM_TC)
  VbModel vb{};                 // coupling-eigenbasis model (FP32 paths)
  double *U64 = nullptr, *UT64 = nullptr;        // coupling eigenbasis U and U^T
  float *mu_vb32 = nullptr, *mup_vb32 = nullptr, *mum_vb32 = nullptr;
  double *mu_vb64 = nullptr;                     // mu in the coupling basis (traces)
  bool on_device = false;
  // copy of the model description (for the parameter gradient)
  heom_model desc{};
  std::vector<heom_mode> desc_modes;
  std::vector<heom_pair> desc_pairs;
  // adjoint RHS tables (built on the first gradient call)
  // launch shapes picked by the autotuner: (kernel kind, elements) -> (block, grid)
  std::map<std::pair<int, int64_t>, std::pair<int, int>> tuned;
  bool adj_ready = false;
  DevModel<double> dm_adj{};
  int *adj_ado = nullptr, *adj_entry_exp = nullptr;
  ~heom_hier() {
    if (tc.maxbuf) cudaFree(tc.maxbuf);
    for (void *p : allocs) cudaFree(p);
    if (stream) cudaStreamDestroy(stream);
  }
  template <typename T>
  T *up(const std::vector<T> &v) {
    T *p = dev_upload(v);
    allocs.push_back(p);
    return p;
  }
};

struct heom_state {
  int branches = 0, precision = 0, d = 0, n_ado = 0;
  int64_t eq_steps = -1;         // RK4 steps from |0><0| when made by heom_equilibrate
  double eq_dt = 0.0;
  heom_hier *hier = nullptr;     // owner of the basis transforms (not owned)
  DeviceBuffer buf;
  int64_t elems() const { return (int64_t)branches * n_ado * d * d; }
  size_t elem_bytes() const { return precision == HEOM_FP64 ? 16 : 8; }
};

namespace heom {

static heom_status fail(heom_status st, const std::string &msg) {
  g_last_error = msg;
  return st;
}

template <typename F>
static heom_status guarded(F &&f) {
  try {
    return f();
  } catch (const Fail &e) {
    return fail(e.st, e.msg);
  } catch (const std::invalid_argument &e) {
    return fail(HEOM_EINVAL, e.what());
  } catch (const std::bad_alloc &) {
    return fail(HEOM_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(HEOM_EINVAL, e.what());
  }
}

template <typename R>
static DevModel<R> &dev_model(heom_hier *h);
template <>
DevModel<double> &dev_model<double>(heom_hier *h) { return h->dm64; }
template <>
DevModel<float> &dev_model<float>(heom_hier *h) { return h->dm32; }

template <typename R>
static const R *mu_of(heom_hier *h, int which);
template <>
const double *mu_of<double>(heom_hier *h, int which) { return which == 0 ? h->mu64 : which == 1 ? h->mup64 : h->mum64; }
template <>
const float *mu_of<float>(heom_hier *h, int which) {
  return which == 0 ? h->mu_vb32 : which == 1 ? h->mup_vb32 : h->mum_vb32;
}

// Necessary condition for RK4 stability: the largest Bohr frequency of H_S' and
// the largest ADO decay rate must each lie inside the RK4 region (|z| < 2.78 on
// the axes).  It does not bound the system-bath couplings.
static void stability_check(heom_hier *h, double dt) {
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
static void rk4_steps(heom_hier *h, typename CxT<R>::type *y, typename CxT<R>::type *wa,
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
static void kick_into(heom_hier *h, const typename CxT<R>::type *in, typename CxT<R>::type *out,
                      int branches, int which, cudaStream_t st) {
  const Model &M = h->M;
  const int64_t total = (int64_t)branches * M.n_ado * M.d * M.d;
  kick_kernel<R><<<grid_for(total), 256, 0, st>>>(in, out, mu_of<R>(h, which), M.d, total);
  count_launch(1);
  LAUNCH_CHECK();
}

template <typename R>
static void trace_into(heom_hier *h, const typename CxT<R>::type *w, int branches, int order,
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
// Stream capture of a launch sequence into a CUDA graph, replayed once by
// replay().  If an exception leaves the scope during capture, the capture is
// ended and discarded so the stream is usable again.
struct GraphCapture {
  cudaStream_t st;
  bool capturing = false;
  explicit GraphCapture(cudaStream_t s) : st(s) {
    CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    capturing = true;
  }
  void replay() {
    cudaGraph_t g = nullptr;
    capturing = false;
    CUDA_TRY(cudaStreamEndCapture(st, &g));
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ex, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (ex) cudaGraphExecDestroy(ex);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) throw Fail{HEOM_ECUDA, std::string("graph replay: ") + cudaGetErrorString(e)};
  }
  ~GraphCapture() {
    if (capturing) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    }
  }
};

// Original-basis complex128 ADOs -> coupling-basis complex64 (U^T x U), and back.
static void to_coupling_basis(heom_hier *h, const double2 *x, float2 *out, int64_t elems, cudaStream_t st) {
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

static void check_tc_error(heom_hier *h) {
  if (!h->tc.ready) return;
  int e = 0;
  CUDA_TRY(cudaMemcpy(&e, h->tc.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CUDA_TRY(cudaMemset(h->tc.err, 0, sizeof(int)));
    throw Fail{HEOM_ETIMEOUT, "a tensor-core stage wait ran out"};
  }
}

// Rows [jr0, jr1) of R_I and R_II into Rdev laid out [n_t2][2][jr1 - jr0][n3].
template <typename R>
static void response_2d_rows_impl(heom_hier *h, const heom_state *eq, const heom_grid *g, int jr0, int jr1,
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
    // trunk: rephasing first kick, propagated to t1 = j0 m dt
    kick_into<R>(h, (const C *)eqR.p, (C *)T.p, 1, 2, st);
    rk4_steps<R>(h, (C *)T.p, (C *)ta.p, (C *)tb.p, 1, dt, (int64_t)(jr0 + j0) * m, st, M.precision);
    for (int j = 0; j < nj; ++j) {
      if (j > 0) rk4_steps<R>(h, (C *)T.p, (C *)ta.p, (C *)tb.p, 1, dt, m, st, M.precision);
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
      rk4_steps<R>(h, BR, Y, WA, B, dt, n2[it] - t_now, st, M.precision);
      t_now = n2[it];
      kick_into<R>(h, BR, Y, B, 1, st);
      // the t3 scan (n3 samples of m RK4 steps and two traces) is captured once
      // into a CUDA graph and replayed as a single launch
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

// Device set-up of a hierarchy: stream, operator and table uploads.  Runs at the
// first call that needs the GPU, so the host-side model can be built and
// inspected without one.
static void ensure_device(heom_hier *h) {
  if (h->on_device) return;
  Model &M = h->M;
  CUDA_TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
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
  h->on_device = true;
}

}  // namespace heom

namespace heom {

// Several FP64 parameter sets (hierarchies of any basis size) on one grid, with
// every RK4 stage of all sets in one launch of multi_stage_kernel.  The branch
// schedule is that of response_2d_rows_impl (one t1 trunk per set, both
// pathways from it, t2 forks in ascending order, the t3 scan captured once into
// a CUDA graph); kicks and traces stay per set (they are cheap).  Rdev[k] gets
// set k's R in the layout [n_t2][2][n1][n3].
struct MultiSet {
  heom_hier *h;
  const heom_state *eq;
  int64_t per;                                     // n_ado d^2
  std::unique_ptr<DeviceBuffer> T, ta, tb, P[4];   // trunk and its scratch; branch sets
};

// Descriptor arrays (device) for the four Horner stages of one RK4 step on the
// buffers (y, wa, wb) of every set.
struct MultiStep {
  DeviceBuffer desc[4];
  int64_t grand = 0;
};

static void multi_step_setup(std::vector<MultiSet> &S, MultiStep &ms, int which_y, int which_a, int which_b,
                             int branches, cudaStream_t st) {
  const int n = (int)S.size();
  std::vector<SetStage<double>> d4[4];
  int64_t begin = 0;
  for (int k = 0; k < n; ++k) {
    auto buf = [&](int w) -> double2 * {
      if (w == -1) return (double2 *)S[k].T->p;
      if (w == -2) return (double2 *)S[k].ta->p;
      if (w == -3) return (double2 *)S[k].tb->p;
      return (double2 *)S[k].P[w]->p;
    };
    double2 *y = buf(which_y), *wa = buf(which_a), *wb = buf(which_b);
    const int64_t tot = (int64_t)branches * S[k].per;
    const double2 *ws[4] = {y, wa, wb, wa};
    double2 *outs[4] = {wa, wb, wa, y};
    for (int q = 0; q < 4; ++q) {
      SetStage<double> x{};
      x.M = S[k].h->dm64;
      x.w = ws[q];
      x.y = y;
      x.out = outs[q];
      x.begin = begin;
      x.total = tot;
      d4[q].push_back(x);
    }
    begin += tot;
  }
  ms.grand = begin;
  for (int q = 0; q < 4; ++q) {
    ms.desc[q].alloc(sizeof(SetStage<double>) * n);
    CUDA_TRY(cudaMemcpyAsync(ms.desc[q].p, d4[q].data(), sizeof(SetStage<double>) * n, cudaMemcpyHostToDevice, st));
  }
  CUDA_TRY(cudaStreamSynchronize(st));
}

static void multi_rk4(const MultiStep &ms, int n_sets, double dt, int64_t nsteps, cudaStream_t st) {
  if (ms.grand == 0 || nsteps <= 0) return;
  const double al[4] = {dt / 4, dt / 3, dt / 2, dt};
  const int grid = grid_for(ms.grand);
  for (int64_t s = 0; s < nsteps; ++s) {
    for (int q = 0; q < 4; ++q)
      multi_stage_kernel<double><<<grid, 256, 0, st>>>((const SetStage<double> *)ms.desc[q].p, n_sets, al[q],
                                                       ms.grand);
    count_launch(4);
  }
  LAUNCH_CHECK();
}

}  // namespace heom

namespace heom {

static void response_2d_multi(heom_hier *const *hs, const heom_state *const *eqs, int n_sets, const heom_grid *g,
                              const std::vector<double2 *> &Rdev) {
  cudaStream_t st = hs[0]->stream;
  const int n1 = g->n1, n3 = g->n3, m = g->steps_per_sample, nt2 = g->n_t2;
  const double dt = g->dt_fs;
  std::vector<int> order(nt2);
  std::vector<int64_t> n2(nt2);
  for (int i = 0; i < nt2; ++i) {
    order[i] = i;
    const double r = g->t2_fs[i] / dt;
    n2[i] = (int64_t)std::llround(r);
    if (g->t2_fs[i] < 0 || std::fabs(r - n2[i]) > 1e-6) throw Fail{HEOM_EINVAL, "t2 must be a non-negative multiple of dt"};
  }
  std::sort(order.begin(), order.end(), [&](int a, int b) { return n2[a] < n2[b]; });
  std::vector<MultiSet> S(n_sets);
  int64_t sum_per = 0;
  for (int k = 0; k < n_sets; ++k) {
    const Model &M = hs[k]->M;
    S[k].h = hs[k];
    S[k].eq = eqs[k];
    S[k].per = (int64_t)M.n_ado * M.d * M.d;
    sum_per += S[k].per;
    S[k].T.reset(new DeviceBuffer(S[k].per * 16));
    S[k].ta.reset(new DeviceBuffer(S[k].per * 16));
    S[k].tb.reset(new DeviceBuffer(S[k].per * 16));
  }
  // t1 rows per chunk: both pathways of J rows, 3 or 4 branch sets per parameter set
  const int nbuf = nt2 > 1 ? 4 : 3;
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  const double budget = 0.85 * (double)free_b;
  int J = n1;
  while (J > 1 && (double)nbuf * 2 * J * sum_per * 16 > budget) J = (J + 1) / 2;
  if ((double)nbuf * 2 * J * sum_per * 16 > budget) throw Fail{HEOM_ENOMEM, "states do not fit in device memory"};
  for (int k = 0; k < n_sets; ++k)
    for (int q = 0; q < 4; ++q)
      S[k].P[q].reset(new DeviceBuffer(q < nbuf ? (size_t)2 * J * S[k].per * 16 : 16));
  MultiStep trunk;
  multi_step_setup(S, trunk, -1, -2, -3, 1, st);
  for (int j0 = 0; j0 < n1; j0 += J) {
    const int nj = std::min(J, n1 - j0), B = 2 * nj;
    MultiStep fork, scan;
    multi_step_setup(S, fork, 0, 1, 2, B, st);                       // y = BR, scratch Y, WA
    multi_step_setup(S, scan, 1, 2, nbuf == 4 ? 3 : 0, B, st);       // y = Y, scratch WA, WB
    for (int k = 0; k < n_sets; ++k)
      kick_into<double>(S[k].h, (const double2 *)S[k].eq->buf.p, (double2 *)S[k].T->p, 1, 2, st);
    multi_rk4(trunk, n_sets, dt, (int64_t)j0 * m, st);
    for (int j = 0; j < nj; ++j) {
      if (j > 0) multi_rk4(trunk, n_sets, dt, m, st);
      for (int k = 0; k < n_sets; ++k) {
        const int64_t per = S[k].per;
        double2 *br = (double2 *)S[k].P[0]->p;
        kick2_pair_kernel<double><<<grid_for(per), 256, 0, st>>>((const double2 *)S[k].T->p, br + (int64_t)j * per,
                                                                br + (int64_t)(nj + j) * per, S[k].h->mup64,
                                                                S[k].h->mum64, S[k].h->M.d, per);
        count_launch(1);
        LAUNCH_CHECK();
      }
    }
    int64_t t_now = 0;
    for (int oi = 0; oi < nt2; ++oi) {
      const int it = order[oi];
      multi_rk4(fork, n_sets, dt, n2[it] - t_now, st);
      t_now = n2[it];
      for (int k = 0; k < n_sets; ++k)
        kick_into<double>(S[k].h, (const double2 *)S[k].P[0]->p, (double2 *)S[k].P[1]->p, B, 1, st);
      GraphCapture cap(st);
      for (int kk = 0; kk < n3; ++kk) {
        if (kk > 0) multi_rk4(scan, n_sets, dt, m, st);
        for (int k = 0; k < n_sets; ++k)
          for (int pw = 0; pw < 2; ++pw) {
            double2 *base = Rdev[k] + (int64_t)it * 2 * n1 * n3 + (int64_t)pw * n1 * n3 + (int64_t)j0 * n3 + kk;
            trace_into<double>(S[k].h, (const double2 *)S[k].P[1]->p + (int64_t)pw * nj * S[k].per, nj, 3, base, n3, st);
          }
      }
      cap.replay();
    }
  }
  CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace heom

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
      CUDA_TRY(cudaMemset(s->buf.p, 0, s->buf.bytes));
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
    if (s->precision == HEOM_FP64) {
      CUDA_TRY(cudaMemcpy(s->buf.p, host, n * 16, cudaMemcpyHostToDevice));
    } else {
      DeviceBuffer tmp(n * 16);
      CUDA_TRY(cudaMemcpy(tmp.p, host, n * 16, cudaMemcpyHostToDevice));
      to_coupling_basis(s->hier, (const double2 *)tmp.p, (float2 *)s->buf.p, n, s->hier->stream);
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

heom_status heom_propagate(heom_hier *h, heom_state *rho, double dt_fs, int64_t n_steps) {
  if (!h || !rho || n_steps < 0) return fail(HEOM_EINVAL, "bad propagate arguments");
  if (rho->d != h->M.d || rho->n_ado != h->M.n_ado) return fail(HEOM_EINVAL, "state does not match hierarchy");
  return guarded([&]() -> heom_status {
    ensure_device(h);
    stability_check(h, dt_fs);
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
    ensure_device(h);
    stability_check(h, dt_fs);
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
  heom_status rc = guarded([&]() -> heom_status {
    stability_check(h, dt_fs);
    const Model &M = h->M;
    const int64_t per = (int64_t)M.n_ado * M.d * M.d;
    double one[2] = {1.0, 0.0};
    CUDA_TRY(cudaMemcpy(s->buf.p, one, 16, cudaMemcpyHostToDevice));   // rho_0 = |0><0|
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
    CUDA_TRY(cudaMemset(zero.p, 0, per * 16));
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

static heom_status check_response_args(heom_hier *h, const heom_state *rho_eq, const heom_grid *g) {
  if (!h || !rho_eq || !g) return fail(HEOM_EINVAL, "null argument");
  if (g->n1 < 1 || g->n3 < 1 || g->n_t2 < 1 || !g->t2_fs || g->steps_per_sample < 1)
    return fail(HEOM_EINVAL, "bad grid");
  if (rho_eq->precision != HEOM_FP64 || rho_eq->branches != 1 || rho_eq->d != h->M.d || rho_eq->n_ado != h->M.n_ado)
    return fail(HEOM_EINVAL, "rho_eq must be a single-branch FP64 state of this hierarchy");
  return HEOM_OK;
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

heom_status heom_response_2d_batched(heom_hier *const *hs, const heom_state *const *eqs, int n_sets,
                                     const heom_grid *g, double *R_I, double *R_II, double *S_C) {
  if (!hs || !eqs || !g || n_sets < 1) return fail(HEOM_EINVAL, "bad batched arguments");
  const size_t blk = (size_t)g->n_t2 * g->n1 * g->n3;
  bool one_launch = n_sets > 1;
  for (int i = 0; i < n_sets; ++i) {
    heom_status a = check_response_args(hs[i], eqs[i], g);
    if (a != HEOM_OK) return a;
    one_launch = one_launch && hs[i]->M.precision == HEOM_FP64;
  }
  if (!one_launch) {
    for (int i = 0; i < n_sets; ++i) {
      heom_status st = heom_response_2d(hs[i], eqs[i], g, R_I ? R_I + i * blk * 2 : nullptr,
                                        R_II ? R_II + i * blk * 2 : nullptr, S_C ? S_C + i * blk : nullptr);
      if (st != HEOM_OK) return st;
    }
    return HEOM_OK;
  }
  return guarded([&]() -> heom_status {
    for (int i = 0; i < n_sets; ++i) {
      ensure_device(hs[i]);
      stability_check(hs[i], g->dt_fs);
    }
    cudaStream_t st = hs[0]->stream;
    const int n1 = g->n1, n3 = g->n3, nt2 = g->n_t2;
    const size_t one = (size_t)n1 * n3;
    DeviceBuffer Rall((size_t)n_sets * nt2 * 2 * one * 16), SCall((size_t)n_sets * blk * 8);
    CUDA_TRY(cudaMemsetAsync(Rall.p, 0, Rall.bytes, st));
    std::vector<double2 *> Rdev(n_sets);
    for (int i = 0; i < n_sets; ++i) Rdev[i] = (double2 *)Rall.p + (size_t)i * nt2 * 2 * one;
    response_2d_multi(hs, eqs, n_sets, g, Rdev);
    const double dtau = g->dt_fs * g->steps_per_sample;
    for (int i = 0; i < n_sets; ++i)
      for (int it = 0; it < nt2; ++it) {
        double2 *RI = Rdev[i] + (int64_t)it * 2 * one;
        dft2d_sc_kernel<<<(unsigned)((one + 255) / 256), 256, 0, st>>>(RI, RI + one, n1, n3, dtau,
                                                                       (double *)SCall.p + (size_t)i * blk + it * one);
        count_launch(1);
        LAUNCH_CHECK();
      }
    std::vector<double> Rh(Rall.bytes / 8);
    CUDA_TRY(cudaMemcpyAsync(Rh.data(), Rall.p, Rall.bytes, cudaMemcpyDeviceToHost, st));
    if (S_C) CUDA_TRY(cudaMemcpyAsync(S_C, SCall.p, SCall.bytes, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < n_sets; ++i)
      for (int it = 0; it < nt2; ++it) {
        const double *src = Rh.data() + ((size_t)i * nt2 * 2 + (size_t)it * 2) * one * 2;
        if (R_I) std::memcpy(R_I + ((size_t)i * blk + it * one) * 2, src, one * 16);
        if (R_II) std::memcpy(R_II + ((size_t)i * blk + it * one) * 2, src + one * 2, one * 16);
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

void heom_free_hier(heom_hier *h) { delete h; }
void heom_free_state(heom_state *s) { delete s; }

}  // extern "C"

// Read-only views of a hierarchy for entry points defined in other files.
namespace heom {
bool hier_on_device(const heom_hier *h) { return h && h->on_device; }
const DevModel<double> &hier_dm64(const heom_hier *h) { return h->dm64; }
void hier_set_error(const char *msg) { g_last_error = msg; }
}  // namespace heom

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
  return k;
}

extern "C" heom_status heom_steady_state(heom_hier *h, double tol, int restart, int max_iter, double dt_fs,
                                         int steps_per_matvec, heom_state **rho_eq, int *iterations) {
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
    CUDA_TRY(cudaMemcpy(x, one, 16, cudaMemcpyHostToDevice));   // x = |0><0|, tr x_0 = 1
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
