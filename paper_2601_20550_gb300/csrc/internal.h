// Internal declarations shared by the translation units of libheom2dvs: error
// handling, device buffers, the hierarchy and state handles, and the launch
// sequences (RK4 steps, kicks, traces, the 2D branch schedule) that the C ABI,
// the batched, gradient and steady-state entry points build on.  Not installed.
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define HEOM_NVTX_PUSH(name) nvtxRangePushA(name)
#define HEOM_NVTX_POP() nvtxRangePop()
#else  // a toolkit without the NVTX headers: phase ranges compile to nothing
#define HEOM_NVTX_PUSH(name) ((void)(name))
#define HEOM_NVTX_POP() ((void)0)
#endif

#include "heom2dvs.h"
#include "kernels.cuh"
#include "model.h"
#include "tc_stage.h"

namespace heom {

extern thread_local std::string g_last_error;
void count_launch(uint64_t n);

// NVTX range over a phase of a call (equilibrate, t1 trunk, t2 fork, t3 scan, DFT,
// ...); no-ops unless a profiler is attached.  next() closes the current phase and
// opens the following one; the destructor closes the last (also on an exception).
class PhaseRange {
 public:
  explicit PhaseRange(const char *name) { HEOM_NVTX_PUSH(name); }
  ~PhaseRange() { HEOM_NVTX_POP(); }
  void next(const char *name) {
    HEOM_NVTX_POP();
    HEOM_NVTX_PUSH(name);
  }
  PhaseRange(const PhaseRange &) = delete;
  PhaseRange &operator=(const PhaseRange &) = delete;
};

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
T *dev_upload(const std::vector<T> &v) {
  T *p = nullptr;
  size_t bytes = std::max<size_t>(1, v.size() * sizeof(T));
  if (device_malloc((void **)&p, bytes) != cudaSuccess) throw Fail{HEOM_ENOMEM, "device allocation failed (model tables)"};
  if (!v.empty()) CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return p;
}

template <typename T>
std::vector<T> cast_vec(const std::vector<double> &v) {
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
    if (device_malloc(&p, n) != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      throw Fail{HEOM_ENOMEM, "device allocation of " + std::to_string(n) + " bytes failed"};
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

inline int grid_for(int64_t total) {
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

inline heom_status fail(heom_status st, const std::string &msg) {
  g_last_error = msg;
  return st;
}

template <typename F>
heom_status guarded(F &&f) {
  try {
    return f();
  } catch (const Fail &e) {
    return fail(e.st, e.msg);
  } catch (const std::invalid_argument &e) {
    return fail(HEOM_EINVAL, e.what());
  } catch (const DeviceOom &e) {
    return fail(HEOM_ENOMEM, e.what());
  } catch (const std::bad_alloc &) {
    return fail(HEOM_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(HEOM_EINVAL, e.what());
  }
}

template <typename R>
DevModel<R> &dev_model(heom_hier *h);
template <>
inline DevModel<double> &dev_model<double>(heom_hier *h) { return h->dm64; }
template <>
inline DevModel<float> &dev_model<float>(heom_hier *h) { return h->dm32; }

template <typename R>
const R *mu_of(heom_hier *h, int which);
template <>
inline const double *mu_of<double>(heom_hier *h, int which) { return which == 0 ? h->mu64 : which == 1 ? h->mup64 : h->mum64; }
template <>
inline const float *mu_of<float>(heom_hier *h, int which) {
  return which == 0 ? h->mu_vb32 : which == 1 ? h->mup_vb32 : h->mum_vb32;
}

// Necessary condition for RK4 stability (Bohr spread and decay rates x dt inside
// the RK4 region); throws HEOM_EUNSTABLE.
void stability_check(heom_hier *h, double dt);

// nsteps RK4 steps (Horner form) of every branch in y, scratch wa and wb.
template <typename R>
void rk4_steps(heom_hier *h, typename CxT<R>::type *y, typename CxT<R>::type *wa, typename CxT<R>::type *wb,
               int branches, double dt, int64_t nsteps, cudaStream_t st, int precision);
// out = K^x in for K = mu (which 0), mu+ (1), mu- (2).
template <typename R>
void kick_into(heom_hier *h, const typename CxT<R>::type *in, typename CxT<R>::type *out, int branches, int which,
               cudaStream_t st);
// i^order tr{mu rho_0} of each branch into out[branch * ostride].
template <typename R>
void trace_into(heom_hier *h, const typename CxT<R>::type *w, int branches, int order, double2 *out,
                int64_t ostride, cudaStream_t st);

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

// Raises HEOM_ETIMEOUT if a tensor-core stage wait ran out.
void check_tc_error(heom_hier *h);
// Product-basis complex128 ADOs -> coupling-basis complex64 (U^T x U U); synchronises st.
void to_coupling_basis(heom_hier *h, const double2 *x, float2 *out, int64_t elems, cudaStream_t st);
// Rows [jr0, jr1) of R_I and R_II into Rdev laid out [n_t2][2][jr1 - jr0][n3].
template <typename R>
void response_2d_rows_impl(heom_hier *h, const heom_state *eq, const heom_grid *g, int jr0, int jr1,
                           double2 *Rdev);
// Device set-up of a hierarchy at its first GPU use.
void ensure_device(heom_hier *h);

inline heom_status check_response_args(heom_hier *h, const heom_state *rho_eq, const heom_grid *g) {
  if (!h || !rho_eq || !g) return fail(HEOM_EINVAL, "null argument");
  if (g->n1 < 1 || g->n3 < 1 || g->n_t2 < 1 || !g->t2_fs || g->steps_per_sample < 1)
    return fail(HEOM_EINVAL, "bad grid");
  if (rho_eq->precision != HEOM_FP64 || rho_eq->branches != 1 || rho_eq->d != h->M.d || rho_eq->n_ado != h->M.n_ado)
    return fail(HEOM_EINVAL, "rho_eq must be a single-branch FP64 state of this hierarchy");
  return HEOM_OK;
}

}  // namespace heom
