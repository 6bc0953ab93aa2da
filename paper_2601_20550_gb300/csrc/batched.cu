// Several parameter sets on one grid (heom_response_2d_batched): FP64 sets
// advance together, one launch per RK4 stage across all sets and branches;
// tensor-core sets likewise, one launch pair per stage.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <future>
#include <memory>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"

using namespace heom;

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
    PhaseRange phase("heom: t1 trunk (sets)");
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
      phase.next("heom: t2 fork (sets)");
      multi_rk4(fork, n_sets, dt, n2[it] - t_now, st);
      t_now = n2[it];
      for (int k = 0; k < n_sets; ++k)
        kick_into<double>(S[k].h, (const double2 *)S[k].P[0]->p, (double2 *)S[k].P[1]->p, B, 1, st);
      phase.next("heom: t3 scan (sets)");
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

// The same schedule for parameter sets built with HEOM_TC (up to 16): the t2
// forks and the t3 scan of all sets advance together, every RK4 stage one
// tensor-core launch and one coupling-kernel launch for all sets
// (tc_rk4_sets); the single-branch t1 trunk of each set runs on the FP32
// CUDA-core stage, as in response_2d_rows_impl.  Per item the arithmetic is that
// of the per-set path, so results equal heom_response_2d per set.
static void response_2d_multi_tc(heom_hier *const *hs, const heom_state *const *eqs, int n_sets, const heom_grid *g,
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
  struct TcSetBufs {
    heom_hier *h;
    int64_t per;
    std::unique_ptr<DeviceBuffer> eqR, T, ta, tb, P[4];
  };
  std::vector<TcSetBufs> S(n_sets);
  int64_t sum_per = 0;
  for (int k = 0; k < n_sets; ++k) {
    const Model &M = hs[k]->M;
    S[k].h = hs[k];
    S[k].per = (int64_t)M.n_ado * M.d * M.d;
    sum_per += S[k].per;
    for (auto *b : {&S[k].eqR, &S[k].T, &S[k].ta, &S[k].tb}) b->reset(new DeviceBuffer(S[k].per * 8));
    to_coupling_basis(hs[k], (const double2 *)eqs[k]->buf.p, (float2 *)S[k].eqR->p, S[k].per, st);
  }
  const int nbuf = nt2 > 1 ? 4 : 3;
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  const double budget = 0.85 * (double)free_b;
  int J = n1;
  while (J > 1 && (double)nbuf * 2 * J * sum_per * 8 > budget) J = (J + 1) / 2;
  if ((double)nbuf * 2 * J * sum_per * 8 > budget) throw Fail{HEOM_ENOMEM, "states do not fit in device memory"};
  for (int k = 0; k < n_sets; ++k) {
    for (int q = 0; q < 4; ++q)
      S[k].P[q].reset(new DeviceBuffer(q < nbuf ? (size_t)2 * J * S[k].per * 8 : 16));
    tc_reserve(hs[k]->tc, (int64_t)2 * J * hs[k]->M.n_ado);
  }
  auto bufs = [&](int yq, int aq, int bq, int B) {
    std::vector<TcRk4Set> v;
    for (int k = 0; k < n_sets; ++k)
      v.push_back(TcRk4Set{&hs[k]->tc, (float2 *)S[k].P[yq]->p, (float2 *)S[k].P[aq]->p, (float2 *)S[k].P[bq]->p, B});
    return v;
  };
  for (int j0 = 0; j0 < n1; j0 += J) {
    const int nj = std::min(J, n1 - j0), B = 2 * nj;
    const std::vector<TcRk4Set> fork = bufs(0, 1, 2, B), scan = bufs(1, 2, nbuf == 4 ? 3 : 0, B);
    PhaseRange phase("heom: t1 trunk (tensor-core sets)");
    for (int k = 0; k < n_sets; ++k) {
      // trunk on the FP32 CUDA-core stage, then the second kick of both pathways
      heom_hier *h = hs[k];
      const int64_t per = S[k].per;
      float2 *T = (float2 *)S[k].T->p;
      kick_into<float>(h, (const float2 *)S[k].eqR->p, T, 1, 2, st);
      rk4_steps<float>(h, T, (float2 *)S[k].ta->p, (float2 *)S[k].tb->p, 1, dt, (int64_t)j0 * m, st, HEOM_FP32);
      float2 *br = (float2 *)S[k].P[0]->p;
      for (int j = 0; j < nj; ++j) {
        if (j > 0) rk4_steps<float>(h, T, (float2 *)S[k].ta->p, (float2 *)S[k].tb->p, 1, dt, m, st, HEOM_FP32);
        kick2_pair_kernel<float><<<grid_for(per), 256, 0, st>>>(T, br + (int64_t)j * per, br + (int64_t)(nj + j) * per,
                                                               h->mup_vb32, h->mum_vb32, h->M.d, per);
        count_launch(1);
        LAUNCH_CHECK();
      }
    }
    int64_t t_now = 0;
    for (int oi = 0; oi < nt2; ++oi) {
      const int it = order[oi];
      phase.next("heom: t2 fork (tensor-core sets)");
      tc_rk4_sets(fork, dt, n2[it] - t_now, st);
      t_now = n2[it];
      for (int k = 0; k < n_sets; ++k)
        kick_into<float>(hs[k], (const float2 *)S[k].P[0]->p, (float2 *)S[k].P[1]->p, B, 1, st);
      tc_tune(scan, dt, st);   // coupling-kernel shape, once per size, before the capture
      phase.next("heom: t3 scan (tensor-core sets)");
      GraphCapture cap(st);
      for (int kk = 0; kk < n3; ++kk) {
        if (kk > 0) tc_rk4_sets(scan, dt, m, st);
        for (int k = 0; k < n_sets; ++k)
          for (int pw = 0; pw < 2; ++pw) {
            double2 *base = Rdev[k] + (int64_t)it * 2 * n1 * n3 + (int64_t)pw * n1 * n3 + (int64_t)j0 * n3 + kk;
            trace_into<float>(hs[k], (const float2 *)S[k].P[1]->p + (int64_t)pw * nj * S[k].per, nj, 3, base, n3, st);
          }
      }
      cap.replay();
    }
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  for (int k = 0; k < n_sets; ++k) check_tc_error(hs[k]);
}

}  // namespace heom

extern "C" {

heom_status heom_response_2d_batched(heom_hier *const *hs, const heom_state *const *eqs, int n_sets,
                                     const heom_grid *g, double *R_I, double *R_II, double *S_C) {
  if (!hs || !eqs || !g || n_sets < 1) return fail(HEOM_EINVAL, "bad batched arguments");
  const size_t blk = (size_t)g->n_t2 * g->n1 * g->n3;
  bool all64 = n_sets > 1, alltc = n_sets > 1 && n_sets <= 16;
  for (int i = 0; i < n_sets; ++i) {
    heom_status a = check_response_args(hs[i], eqs[i], g);
    if (a != HEOM_OK) return a;
    all64 = all64 && hs[i]->M.precision == HEOM_FP64;
    alltc = alltc && hs[i]->M.precision == HEOM_TC;
    // a tensor-core hierarchy keeps per-item scale workspace for one set at a
    // time: a batch that names one twice runs set by set
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) alltc = false;
  }
  if (!all64 && !alltc) {
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
    if (alltc) {
      for (int i = 0; i < n_sets; ++i)
        if (!tc_supported(hs[i]->tc)) throw Fail{HEOM_EINVAL, "tensor-core path not prepared for this hierarchy"};
      response_2d_multi_tc(hs, eqs, n_sets, g, Rdev);
    } else {
      response_2d_multi(hs, eqs, n_sets, g, Rdev);
    }
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

}  // extern "C"
