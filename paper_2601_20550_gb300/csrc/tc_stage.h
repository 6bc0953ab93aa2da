// Tensor-core (tcgen05) RK4 stage for the mixed-precision path (HEOM_TC).
//
// The state is held in the coupling eigenbasis (see kernels.cuh, VbModel): the
// dense commutator [H', w_n] runs on the 5th-generation tensor cores with
// split-FP16 operands (per-ADO power-of-two scaling, FP32 accumulation in
// tensor memory) and the system-bath terms are elementwise in the epilogue.
#pragma once

#include <cstdint>
#include <map>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.cuh"
#include "model.h"

namespace heom {

// Every device allocation of the library goes through device_malloc, which
// honours the host-side allocation-failure injection (heom_debug_fail_alloc).
cudaError_t device_malloc(void **p, size_t bytes);
// A device allocation failed (reported as HEOM_ENOMEM).
struct DeviceOom : std::bad_alloc {
  const char *what() const noexcept override { return "device allocation failed"; }
};

// Coupling-kernel shape chosen by the autotuner for one launch size: index into
// the kernel's candidate list, threads per block, blocks per launch, and the
// time of three first-stage launches (tensor-core and coupling kernel) in ms.
struct TcTuned {
  int shape;
  int block;
  int64_t grid;
  float ms;
};

struct TcOperators {
  bool ready = false;
  int d = 0, n_ado = 0, n_modes = 0, n_hpieces = 3;
  float inv_sh = 1.f;             // 1 / (power-of-two scale applied to H')
  const uint4 *himg = nullptr;    // n_hpieces shared-memory images of H' pieces (32 KB each)
  const float *lam = nullptr;     // [n_modes][128] lam_s[digit_s(a)]
  // coupling-kernel tables for groups of 1, 2, 4, 8 consecutive ADOs (index log2 of
  // the group size): union offsets and members, and one term per (member, ADO)
  const int *vt_uoff[4] = {nullptr, nullptr, nullptr, nullptr};
  const int *vt_uidx[4] = {nullptr, nullptr, nullptr, nullptr};
  const float4 *vt_desc[4] = {nullptr, nullptr, nullptr, nullptr};
  int *err = nullptr;             // device error word (bounded waits)
  uint64_t wait_ns = 2000000000ull;  // time limit of each device-side wait
  int sms = 0;
  unsigned *maxbuf = nullptr;     // workspace: per-item max |w| of y, wa, wb (grown on demand)
  int64_t max_items = 0;
  std::map<int64_t, TcTuned> vt_tuned;  // by total state elements of the launch
};

// Prepare the tensor-core operator images of M (device allocations are appended
// to allocs).  vb supplies the device coupling tables.  Throws std::invalid_argument
// if the model does not fit the kernel (d > 128 or more than 4 modes).
void tc_build(TcOperators &tc, const Model &M, const VbModel &vb, std::vector<void *> &allocs);
bool tc_supported(const TcOperators &tc);
// n RK4 steps (Horner form) on complex64 coupling-basis branches y with scratch wa, wb.
// The hierarchy keeps a workspace of three per-item maxima (12 bytes per ADO
// per branch), grown on the first call with a larger batch.
void tc_rk4_steps(TcOperators &tc, float2 *y, float2 *wa, float2 *wb, int branches, double dt,
                  int64_t nsteps, cudaStream_t st);
// Grow the per-item maxima workspace to n_items (outside any stream capture).
void tc_reserve(TcOperators &tc, int64_t n_items);
// Buffers of one parameter set for tc_rk4_sets: the state y and two scratch
// states, each [branches][n_ado][d][d] complex64 in the coupling basis.
struct TcRk4Set {
  TcOperators *tc;
  float2 *y, *wa, *wb;
  int branches;
};
// n RK4 steps (Horner form) of several parameter sets (up to 16, hierarchies built
// with HEOM_TC, any basis size up to 128) together: every stage of all sets is one
// tensor-core launch and one coupling-kernel launch.  Each stage writes
// tpart = alpha (-i [H', w]) (the tensor-core kernel), then out = y + tpart +
// alpha (-gamma w + sum kappa w_nb) (the coupling kernel).  Per item the
// arithmetic does not depend on the other sets, so results equal per-set calls.
void tc_rk4_sets(const std::vector<TcRk4Set> &sets, double dt, int64_t nsteps, cudaStream_t st);

// Tune the coupling kernel's shape for a launch over these sets (outside any
// stream capture; a size tuned before is not re-timed).  The sets' y must hold
// the state the launches will see; wa receives scratch.  tc_rk4_sets tunes an
// untuned size itself when it is not being captured.
void tc_tune(const std::vector<TcRk4Set> &sets, double dt, cudaStream_t st);
// Use coupling-kernel shape `shape` (0-16) for every launch instead of the tuned
// one, or tune again (-1).  Process-wide; false if shape is out of range.
bool tc_force_shape(int shape);
// Number of coupling-kernel shapes (valid shapes are 0 .. count - 1).
int tc_shape_count();
// Rows per thread, row groups of 128 threads, consecutive ADOs per block and the
// flags (bit 0: L2 prefetch, bit 1: two sources in flight) of coupling-kernel
// shape `shape`; false if out of range.
bool tc_shape_params(int shape, int *rpt, int *groups, int *ados, int *flags);

}  // namespace heom
