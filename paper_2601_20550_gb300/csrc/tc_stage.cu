// Tensor-core (tcgen05) RK4 stage of the HEOM right-hand side (Eq. HEOM_DB) for
// the mixed-precision path, sm_103a.  A stage out = y + alpha L(w) runs as two
// kernels.
//
// tc_stage_kernel: one persistent CTA per SM walks the work items (branch, ADO):
//   1. producer warps 0-11 load w_n (complex64, d x d), scale it by the power of
//      two taken from its largest component (tracked by the previous stage) into
//      FP16 range and split every component into hi + lo FP16 parts, written to
//      shared memory in the 128-byte-swizzled UMMA layout (re rows 0..127, im
//      rows 128..255; hi tiles ZZ1, lo tiles ZZ2);
//   2. one thread of warp 16 issues tcgen05.mma: D = Z^T H' - H' Z^T = [H', Z]^T
//      with the H' pieces (hi, mid, lo) resident in shared memory and FP32
//      accumulation in tensor memory (256 columns: Re D | Im D, double-buffered),
//      the small split products first and the hi x hi product last (see the
//      issue loop for why), the tiles released when all have completed;
//   3. epilogue warps 12-15 read D from tensor memory (lane = column b of w_n,
//      column = row a) and store tpart = alpha (-i C) with coalesced accesses.
// vterm_kernel then adds y, tpart and the elementwise decay and system-bath
// terms (out = y + tpart + alpha (-gamma_n w_n + sum kappa w_nb)) as a streaming
// kernel at high occupancy, so that enough neighbour loads are in flight.
// (Moving y and the decay into the epilogue took 35 ns per item off this
// kernel but added 80 to the tensor-core kernel, whose four epilogue warps
// cannot hide the latency of two more loads per element.)
// All waits are bounded: on expiry the kernel sets the error word, frees its
// tensor memory and returns.
#include "tc_stage.h"

#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>
#include <map>
#include <stdexcept>

#include <cuda_fp16.h>

namespace heom {

void count_launch(uint64_t n);

namespace {

constexpr int kThreads = 544;
constexpr int kTcMaxModes = 4;
constexpr int kTcMaxSets = 16;
constexpr uint32_t kHTile = 32768;               // 128 x 128 FP16
constexpr uint32_t kZZ = 65536;                  // 256 x 128 FP16 (re | im rows)
constexpr uint32_t kTiles = 2 * kZZ + 3 * kHTile;
constexpr uint32_t kSmemDyn = kTiles + 1024;     // + alignment slack
constexpr uint32_t kTmemCols = 512;             // two accumulator buffers of 256 columns
constexpr int kProducers = 384;                  // warps 0-11
constexpr int kEpilogue = 128;                   // warps 12-15
constexpr int kMmaWarp = 16;                     // warp 16: tensor-core issue
// Rows of w_n per producer thread: 24 (6 row groups x 24 = 144 >= 128 rows), loaded
// in 3 batches of 8 (with the hi parts of all 24 held until the tiles are free, a
// batch of 12 exceeds the 96-register budget of a 17-warp CTA and spills).
constexpr int kProdSlots = 24;
static_assert(kProducers + kEpilogue + 32 == kThreads, "warp roles");
// Bounded waits: a wait gives up after the hierarchy's time limit (globaltimer,
// checked at the second poll and then every 256 polls) or after kWaitPolls
// polls, whichever comes first.
constexpr long kWaitPolls = 1L << 30;
// Drain of the MMAs already committed when a block aborts: bounded by its own
// limit, independent of the (possibly shortened) wait limit.
constexpr uint64_t kDrainNs = 2000000000ull;

// One parameter set of a stage launch: its operators and this stage's buffers.
// A launch covers up to kTcMaxSets sets (hierarchies of any basis size up to
// 128); their work items are concatenated, set after set.
struct TcSet {
  const uint4 *himg;          // shared-memory images of the H' pieces
  const float *lam;           // [n_modes][128] lam_s[digit_s(a)]
  // coupling kernel tables for groups of 1, 2, 4 and 8 consecutive ADOs: per group
  // the union of its ADOs and their neighbours (offsets, ascending ADO indices) and
  // per (member, ADO of the group) the term: (cA or the decay, cB, term, 0) with
  // term = -2 none, -1 the decay, s >= 0 a coupling of mode s
  const int *vt_uoff[4], *vt_uidx[4];
  const float4 *vt_desc[4];
  const float2 *w, *y;        // stage input and step-start state
  float2 *out, *tpart;        // stage output; tensor-core part (may equal out, not w or y)
  const unsigned *max_in;     // per item: largest |component| of w (float bits)
  unsigned *max_out;          // per item: running max |component| of out
  int64_t item_begin;         // first work item of the set in the launch
  int64_t vt_begin;           // first block of the set in the coupling kernel's grid
  float inv_sh;               // 1 / (power-of-two scale applied to H')
  int d, n_ado, n_modes, bands;
};

struct TcArgs {
  TcSet sets[kTcMaxSets];
  int n_sets, n_hpieces;
  int64_t n_items;            // work items of all sets
  float alpha;
  int *err;                   // device error word (bounded waits)
  uint64_t wait_ns;           // time limit of each wait
};

// Set of a work item (items are concatenated set after set).
__device__ __forceinline__ int set_of_item(const TcArgs &P, int64_t item) {
  int k = 0;
  while (k + 1 < P.n_sets && item >= P.sets[k + 1].item_begin) ++k;
  return k;
}

__host__ __device__ inline uint32_t sw128_offset(int r, int c, uint32_t colblock_stride) {
  const int j = c >> 6, cc = c & 63;
  const uint32_t logical = (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u + (uint32_t)cc * 2u;
  const uint32_t chunk = (logical >> 4) & 7u, row8 = (logical >> 7) & 7u;
  return (uint32_t)j * colblock_stride + ((logical & ~(7u << 4)) | ((chunk ^ row8) << 4));
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// UMMA shared-memory descriptor, 128-byte swizzle, sm_100 version bits.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: kind::f16, FP16 A and B, FP32 accumulator.
__host__ __device__ constexpr uint32_t idesc(int M, int N, int a_mn, int b_mn, int neg_a) {
  return (1u << 4) | ((uint32_t)neg_a << 13) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ uint32_t mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}\n"
      : "=r"(done)
      : "r"(addr), "r"(parity));
  return done;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// TMA bulk prefetch of [p, p + bytes) into L2, restricted to its 16-byte-aligned
// interior (a prefetch need not cover every byte).
__device__ __forceinline__ void l2_prefetch_bulk(const void *p, int64_t bytes) {
  uint64_t lo = ((uint64_t)p + 15u) & ~(uint64_t)15u;
  const uint64_t hi = ((uint64_t)p + (uint64_t)bytes) & ~(uint64_t)15u;
  while (lo < hi) {
    const uint32_t n = (uint32_t)((hi - lo) < (1u << 16) ? (hi - lo) : (1u << 16));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"(n) : "memory");
    lo += n;
  }
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)));
}

// Bounded wait on an mbarrier phase; returns false (and raises the error word)
// when the iteration limit runs out.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// A wait also returns false, without raising the error word, as soon as another
// role of the block has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, int *abort_flag,
                                          uint64_t limit_ns) {
  const uint32_t addr = smem_u32(bar);
  if (mbar_try(addr, parity)) return true;
  const uint64_t t0 = global_ns();
  for (long it = 1; it < kWaitPolls; ++it) {
    if (mbar_try(addr, parity)) return true;
    if (it == 1 || (it & 255) == 0) {
      if (*(volatile int *)abort_flag) return false;
      if (global_ns() - t0 > limit_ns) break;
    }
  }
  atomicExch(err, 1);
  *(volatile int *)abort_flag = 1;
  return false;
}

// Wait for the completion of MMAs that were committed before an abort; the
// abort flag does not end this wait (the tensor memory and the tiles they use
// must outlive them).  Bounded by kDrainNs.
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity, int *err) {
  const uint32_t addr = smem_u32(bar);
  const uint64_t t0 = global_ns();
  for (long it = 0; it < kWaitPolls; ++it) {
    if (mbar_try(addr, parity)) return;
    if ((it & 255) == 255 && global_ns() - t0 > kDrainNs) break;
  }
  atomicExch(err, 1);
}

// Barrier of the producer warps that also ORs a flag over them, so that every
// producer takes the same decision (a plain re-read of the shared abort flag
// after the barrier could differ between threads if another role sets it
// meanwhile, and the threads that continued would wait at the next barrier for
// the ones that left).
__device__ __forceinline__ bool producer_sync_any(bool flag) {
  uint32_t any;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(any)
      : "r"((uint32_t)flag), "n"(kProducers));
  return any != 0;
}

// Power-of-two scale that brings an item's largest component (float bits m)
// below 2^14; producers and epilogue derive it from the same word.
__device__ __forceinline__ float item_scale(unsigned mbits) {
  const float m = __uint_as_float(mbits);
  float scale = 1.f;
  if (m > 0.f && isfinite(m)) {
    int e;
    frexpf(m, &e);
    scale = ldexpf(1.f, 14 - e);
  }
  return scale;
}

// Warp-specialised persistent stage kernel.
//   warps 0-11 (producers): per item, load the first half of w_n, wait until the
//              previous item's MMAs have released the hi tiles, split w_n (hi
//              parts to the tiles, signalled at once; lo parts held in registers),
//              wait for the previous item's MMAs to release the lo tiles, write the
//              lo parts and signal them.
//   warp 16    (MMA issue): per item, wait for the hi tiles and for the
//              tensor-memory buffer of the item's parity, issue the products with
//              the hi tiles that do not involve H1, wait for the lo tiles, issue
//              H1 Z2 and H1 Z1.  Issue blocks while the tensor cores drain the
//              queue, so it runs in its own warp and the producers convert the
//              next item meanwhile.
//   warps 12-15 (epilogue): per item, wait for the MMAs, read the accumulator,
//              store tpart and release the buffer.
// The epilogue of item k overlaps the MMAs of item k + 1 and the loads of k + 2.
template <bool kMulti>
__global__ void __launch_bounds__(kThreads, 1) tc_stage_kernel(const __grid_constant__ TcArgs P) {
  constexpr int kProdRows = 8;                             // rows per producer batch
  constexpr int kProdBatches = kProdSlots / kProdRows;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_mma[2], bar_lo[2], bar_full[2], bar_epi[2], bar_ready_hi[2], bar_ready_lo[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint8_t *ZZ1 = base, *ZZ2 = base + kZZ, *HT = base + 2 * kZZ;

  // tiles zeroed (rows and columns past d stay zero) and the H' pieces of the set
  // of this CTA's first item
  const int first_set = kMulti && (int64_t)blockIdx.x < P.n_items ? set_of_item(P, blockIdx.x) : 0;
  for (uint32_t i = tid; i < 2 * kZZ / 16; i += kThreads) reinterpret_cast<uint4 *>(base)[i] = make_uint4(0, 0, 0, 0);
  for (uint32_t i = tid; i < (uint32_t)P.n_hpieces * kHTile / 16; i += kThreads)
    reinterpret_cast<uint4 *>(HT)[i] = P.sets[first_set].himg[i];
  if (tid == 0) {
    s_abort = 0;
    for (int t = 0; t < 2; ++t) {
      mbar_init(&bar_mma[t], 1);
      mbar_init(&bar_lo[t], 1);
      mbar_init(&bar_full[t], 1);
      mbar_init(&bar_epi[t], kEpilogue / 32);
      mbar_init(&bar_ready_hi[t], kProducers / 32);
      mbar_init(&bar_ready_lo[t], kProducers / 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  const int64_t n_mine = P.n_items > blockIdx.x ? (P.n_items - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (tid < kProducers) {
    // ------------------------------------------------------------ producers
    const int cp = tid & 63;           // column pair: columns 2cp, 2cp + 1
    const int r0 = tid >> 6;           // first row; rows r0, r0 + 6, ...
    const int c = 2 * cp;
    // byte offsets of this thread's __half2 in the 128B-swizzled tiles: row a of a
    // 64-column block sits at 128 a, its 16-byte chunk (c mod 64) / 8 is XORed with
    // a mod 8.  Rows a = r0 + 6 g repeat a mod 8 every 4 steps of g (6 * 4 = 24),
    // so four offsets plus a multiple of 4 * 6 * 128 = 3072 bytes cover all rows
    // (the imaginary half, rows a + 128, adds 16384).
    uint32_t row_ofs[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int a = r0 + 6 * u, cc = c & 63;
      row_ofs[u] = (uint32_t)(c >> 6) * (kZZ / 2) + (uint32_t)a * 128u +
                   ((uint32_t)((cc >> 3) ^ (a & 7)) << 4) + (uint32_t)((cc * 2) & 15);
    }
    int prev_set = first_set;
    for (int64_t k = 0; k < n_mine; ++k) {
      const int64_t item = blockIdx.x + k * gridDim.x;
      const int t = (int)(k & 1);
      const int ks = kMulti ? set_of_item(P, item) : 0;
      const TcSet &S = P.sets[ks];
      const int d = S.d;
      const int64_t dd = (int64_t)d * d, li = item - S.item_begin;
      const bool active = c < d;
      const float2 *wn = S.w + li * dd;
      // warm L2 with the next item's w_n while this one is converted (one bulk prefetch)
      if (k + 1 < n_mine && tid == 0) {
        const int64_t nx = item + gridDim.x;
        const TcSet &SN = P.sets[kMulti ? set_of_item(P, nx) : 0];
        const int64_t ddn = (int64_t)SN.d * SN.d;
        l2_prefetch_bulk(SN.w + (nx - SN.item_begin) * ddn, ddn * 8);
      }
      // The first batch of w_n is loaded before the wait, so its latency overlaps
      // the previous item's first MMA group.
      float2 v[2 * kProdRows];   // one batch: kProdRows rows x 2 columns
      auto load_batch = [&](int bt) {
        const int ab = r0 + 6 * kProdRows * bt;
#pragma unroll
        for (int i = 0; i < kProdRows; ++i) {
          const int a = min(ab + 6 * i, d - 1);
          v[2 * i] = active ? wn[(int64_t)a * d + c] : make_float2(0.f, 0.f);
          v[2 * i + 1] = (active && c + 1 < d) ? wn[(int64_t)a * d + c + 1] : make_float2(0.f, 0.f);
        }
      };
      load_batch(0);
      // power-of-two scale from the item's largest component (kept by the previous stage)
      const float scale = item_scale(S.max_in[li]);
      // The lo tiles are free once the previous item's first MMA (H1 Z2) has
      // completed; every producer takes the same decision to go on or to leave.
      // An item of another parameter set than the previous one waits for all of
      // the previous item's MMAs (they read H'), then the producers load the new
      // set's H' pieces and clear the tiles (its basis may be smaller).
      const bool new_set = kMulti && ks != prev_set;
      prev_set = ks;
      if (k >= 1) {
        if (new_set)
          mbar_wait(&bar_mma[(k - 1) & 1], (uint32_t)(((k - 1) >> 1) & 1), P.err, &s_abort, P.wait_ns);
        else
          mbar_wait(&bar_lo[(k - 1) & 1], (uint32_t)(((k - 1) >> 1) & 1), P.err, &s_abort, P.wait_ns);
      }
      if (producer_sync_any(*(volatile int *)&s_abort != 0)) break;
      if (new_set) {
        for (uint32_t i = tid; i < 2 * kZZ / 16; i += kProducers)
          reinterpret_cast<uint4 *>(base)[i] = make_uint4(0, 0, 0, 0);
        for (uint32_t i = tid; i < (uint32_t)P.n_hpieces * kHTile / 16; i += kProducers)
          reinterpret_cast<uint4 *>(HT)[i] = S.himg[i];
        producer_sync_any(false);   // cleared before any producer writes its tile parts
      }
      // scale and split into FP16 hi + lo; lo goes to the tiles now (the MMA warp
      // starts this item with H1 Z2 as soon as they are all written), hi is kept in
      // registers until the previous item's MMAs have all completed
      __half2 hre[kProdSlots], him[kProdSlots];
#pragma unroll
      for (int bt = 0; bt < kProdBatches; ++bt) {
        if (bt > 0) load_batch(bt);
#pragma unroll
        for (int i = 0; i < kProdRows; ++i) {
          const int g = kProdRows * bt + i;                  // row a = r0 + 6 g
          const float2 xr = make_float2(v[2 * i].x * scale, v[2 * i + 1].x * scale);
          const float2 xi = make_float2(v[2 * i].y * scale, v[2 * i + 1].y * scale);
          hre[g] = __float22half2_rn(xr);
          him[g] = __float22half2_rn(xi);
          const float2 fr = __half22float2(hre[g]), fi = __half22float2(him[g]);
          const __half2 lr = __float22half2_rn(make_float2(xr.x - fr.x, xr.y - fr.y));
          const __half2 lim = __float22half2_rn(make_float2(xi.x - fi.x, xi.y - fi.y));
          if (active && r0 + 6 * g < d) {
            const uint32_t o = row_ofs[g & 3] + 3072u * (uint32_t)(g >> 2);
            *reinterpret_cast<__half2 *>(ZZ2 + o) = lr;
            *reinterpret_cast<__half2 *>(ZZ2 + o + 16384u) = lim;
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_ready_lo[t]);
      // the hi tiles are free once the previous item's MMAs have all completed
      if (k >= 1) mbar_wait(&bar_mma[(k - 1) & 1], (uint32_t)(((k - 1) >> 1) & 1), P.err, &s_abort, P.wait_ns);
      if (active) {
#pragma unroll
        for (int g = 0; g < kProdSlots; ++g)
          if (r0 + 6 * g < d) {
            const uint32_t o = row_ofs[g & 3] + 3072u * (uint32_t)(g >> 2);
            *reinterpret_cast<__half2 *>(ZZ1 + o) = hre[g];
            *reinterpret_cast<__half2 *>(ZZ1 + o + 16384u) = him[g];
          }
      }
      asm volatile("fence.proxy.async.shared::cta;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_ready_hi[t]);
    }
  } else if (warp < kMmaWarp) {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - kProducers / 32;          // 0..3: TMEM lane quadrant
    const int b = 32 * ew + lane;                   // TMEM lane = column b of w_n
    const uint32_t lane_field = (uint32_t)(32 * ew) << 16;
    for (int64_t k = 0; k < n_mine; ++k) {
      const int64_t item = blockIdx.x + k * gridDim.x;
      const int t = (int)(k & 1);
      const uint32_t par = (uint32_t)((k >> 1) & 1);
      bool ok = mbar_wait(&bar_full[t], par, P.err, &s_abort, P.wait_ns);
      ok = ok && mbar_wait(&bar_mma[t], par, P.err, &s_abort, P.wait_ns);
      if (!__all_sync(0xffffffffu, ok)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      // tpart = alpha (-i C); the streaming kernel adds y and the rest next
      const TcSet &S = P.sets[kMulti ? set_of_item(P, item) : 0];
      const int d = S.d;
      const int64_t dd = (int64_t)d * d, li = item - S.item_begin;
      if (tid == kProducers) S.max_out[li] = 0u;
      const float sc = P.alpha * S.inv_sh / item_scale(S.max_in[li]);
      float2 *ob = S.tpart + li * dd;
      const uint32_t tcol = tmem + lane_field + (uint32_t)t * 256u;
      for (int a0 = 0; a0 < d; a0 += 16) {
        uint32_t rr[16], ri[16];
        tmem_ld16(tcol + (uint32_t)a0, rr);
        tmem_ld16(tcol + 128u + (uint32_t)a0, ri);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (b < d) {
          const int64_t e0 = (int64_t)a0 * d + b;
#pragma unroll
          for (int jj = 0; jj < 16; ++jj)
            if (a0 + jj < d)
              __stcg(ob + e0 + (int64_t)jj * d,
                     make_float2(sc * __uint_as_float(ri[jj]), -sc * __uint_as_float(rr[jj])));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_epi[t]);
    }
  } else {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t zz[2] = {smem_u32(ZZ1), smem_u32(ZZ2)};
      const uint32_t hh = smem_u32(HT);
      const uint32_t id_neg = idesc(128, 256, 0, 0, 1);
      const uint32_t id_mn = idesc(128, 128, 1, 0, 0);
      const int nh = P.n_hpieces;
      // the mbarrier phase of the most recent commit (bar_lo[t] as 2 t, bar_mma[t]
      // as 2 t + 1; -1 none): every MMA issued before it has completed once that
      // phase completes
      int last_bar = -1;
      uint32_t last_par = 0;
      for (int64_t k = 0; k < n_mine; ++k) {
        const int t = (int)(k & 1);
        // the tiles of item k are written; its accumulator buffer is free once
        // the epilogue of item k - 2 released it
        bool ok = mbar_wait(&bar_ready_lo[t], (uint32_t)((k >> 1) & 1), P.err, &s_abort, P.wait_ns);
        ok = ok && (k < 2 || mbar_wait(&bar_epi[t], (uint32_t)(((k - 2) >> 1) & 1), P.err, &s_abort, P.wait_ns));
        if (!ok) break;
        // Products kept by the split, the small ones first: H1 Z2 (lo tiles, group
        // 0, committed on its own so the producers can refill the lo tiles), then
        // H2 Z1 and H3 Z1, and the largest, H1 Z1, last (group 1, hi tiles).  The
        // accumulator holds only small partial sums until the largest product
        // arrives, and the two halves of each commutator (Z^T H' and -H' Z^T) are
        // interleaved along the contraction, so the partial sums follow the
        // commutator rather than either product.  (Each MMA step's FP32 rounding
        // error scales with the partial sum; on c3 this order cut the error of
        // 1016 RK4 steps 5x.)
        const uint32_t dcol = tmem + (uint32_t)t * 256u;
        for (int grp = 0; grp < 2; ++grp) {
          if (grp == 1) {
            if (!mbar_wait(&bar_ready_hi[t], (uint32_t)((k >> 1) & 1), P.err, &s_abort, P.wait_ns)) break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int np = grp == 0 ? 1 : nh;
          for (int i = 0; i < np; ++i) {
            const int j = grp == 0 ? 0 : (i + 1) % nh;    // H piece: group 1 takes H2, H3, then H1
            const int zk = grp == 0 ? 1 : 0;              // Z piece: 0 hi, 1 lo
            const uint32_t ha = hh + (uint32_t)j * kHTile, zb = zz[zk];
            for (int kk = 0; kk < 8; ++kk) {
              const uint64_t hd = sdesc(ha + (kk >> 2) * 16384u + (kk & 3) * 32u, 16, 1024);
              const uint64_t zd = sdesc(zb + (kk >> 2) * (kZZ / 2) + (kk & 3) * 32u, 16, 1024);
              umma(dcol, hd, zd, id_neg, (grp == 0 && kk == 0) ? 0u : 1u);
              for (int part = 0; part < 2; ++part) {
                const uint64_t za = sdesc(zb + (uint32_t)part * 16384u + (uint32_t)kk * 2048u, kZZ / 2, 1024);
                umma(dcol + (uint32_t)part * 128u, za, hd, id_mn, 1);
              }
            }
          }
          last_bar = 2 * t + grp;
          last_par = (uint32_t)((k >> 1) & 1);
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(grp == 0 ? &bar_lo[t] : &bar_mma[t])));
        }
        if (*(volatile int *)&s_abort) break;
        mbar_arrive(&bar_full[t]);
      }
      // drain, on the normal and on the abort path: every committed MMA must
      // complete before the tiles and the tensor memory go away
      if (last_bar >= 0)
        mbar_drain((last_bar & 1) ? &bar_mma[last_bar >> 1] : &bar_lo[last_bar >> 1], last_par, P.err);
    }
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// Elementwise terms in the coupling eigenbasis (CUDA cores): decay and system-bath
//   out[a][b] = y[a][b] + tpart[a][b]
//             + alpha * (-gamma_n w_n[a][b] + sum_q kappa_q(a, b) w_{nb_q}[a][b]),
//   kappa_q = -i cA_q (lam_s[a_s] - lam_s[b_s]) + cB_q (lam_s[a_s] + lam_s[b_s]),
// over the coupling list of the ADO (up- and down-neighbours of every mode).
// One block per (group of kAdos consecutive ADOs of one branch, band of
// kRows = kRpt x kGroups rows); thread = (column b, row group), kRpt rows per
// thread (rows a0, a0 + kGroups, ...) and kAdos accumulators per row held in
// registers.  The block walks the union of the group's ADOs and their
// neighbours in ascending ADO order (a host-built table of that union and, per
// (member, ADO of the group), the term it contributes: none, the decay, or a
// coupling of mode s with cA, cB), so each neighbour state is read once for the
// whole group (lam through L1: no shared-memory staging or barrier before the
// first gather).  Every element accumulates its own terms in ascending neighbour
// index with explicit fused operations, so all shapes round identically.  The
// block raises each item's running maximum |out|, which the tensor-core kernel
// cleared, with one atomic per warp.  The shape is chosen per size by the
// autotuner (tc_tune).
constexpr int kMaxNb = 32;

template <int kRpt, int kGroups, int kAdos, bool kPf, bool kTwo>
__global__ void __launch_bounds__(128 * kGroups) vterm_kernel(const __grid_constant__ TcArgs P) {
  constexpr int kRows = kRpt * kGroups;
  constexpr int kLog = kAdos == 1 ? 0 : kAdos == 2 ? 1 : kAdos == 4 ? 2 : 3;
  int ks = 0;   // the parameter set of this block (blocks are concatenated set after set)
  while (ks + 1 < P.n_sets && (int64_t)blockIdx.x >= P.sets[ks + 1].vt_begin) ++ks;
  const TcSet &S = P.sets[ks];
  const int d = S.d, nm = S.n_modes, bands = S.bands;
  const int64_t dd = (int64_t)d * d;
  const int gpb = (S.n_ado + kAdos - 1) / kAdos;   // ADO groups per branch
  const int64_t lb = (int64_t)blockIdx.x - S.vt_begin;
  const int64_t gi = lb / bands;                   // group within the set (branch-major)
  const int band = (int)(lb - gi * bands);
  const int64_t br = gi / gpb;
  const int g = (int)(gi - br * gpb);
  const int n0 = g * kAdos;
  const float2 *wb = S.w + br * S.n_ado * dd;
  const float alpha = P.alpha;
  const float *__restrict__ lam = S.lam;   // [n_modes][128], read through L1
  const int b = threadIdx.x & 127, par = threadIdx.x >> 7;
  const int a0 = band * kRows + par;
  // lanes past the last column keep running (no loads or stores) so that the
  // warp-wide maxima below see every lane
  const int nrow = b < d ? max(0, min(kRpt, (d - a0 + kGroups - 1) / kGroups)) : 0;
  const int64_t e0 = (int64_t)a0 * d + b, es = (int64_t)kGroups * d;
  float re[kAdos][kRpt], im[kAdos][kRpt];
#pragma unroll
  for (int k = 0; k < kAdos; ++k)
#pragma unroll
    for (int j = 0; j < kRpt; ++j) re[k][j] = im[k][j] = 0.f;
  int arow[kRpt];
#pragma unroll
  for (int j = 0; j < kRpt; ++j) arow[j] = min(a0 + kGroups * j, d - 1);
  const int *uoff = S.vt_uoff[kLog];
  const int *uidx = S.vt_uidx[kLog];
  const float4 *desc = S.vt_desc[kLog];
  const int u0 = uoff[g], u1 = uoff[g + 1];
  if (kPf && threadIdx.x < 32) {
    // request the band of every source state (the union members, then y and tpart
    // of each ADO of the group) into L2 up front, one bulk prefetch per lane, so
    // that the gather rounds below find them there
    const int r0 = band * kRows, nr = min(kRows, d - r0);
    if (nr > 0) {
      const int64_t off = (int64_t)r0 * d, bytes = (int64_t)nr * d * (int64_t)sizeof(float2);
      const int nu = u1 - u0, nk = min(kAdos, S.n_ado - n0);
      for (int i = threadIdx.x; i < nu + 2 * nk; i += 32) {
        const float2 *src;
        if (i < nu) {
          src = wb + (int64_t)uidx[u0 + i] * dd + off;
        } else {
          const int64_t item = br * S.n_ado + n0 + ((i - nu) >> 1);
          src = (((i - nu) & 1) ? S.tpart : S.y) + item * dd + off;
        }
        l2_prefetch_bulk(src, bytes);
      }
    }
  }
  // the terms of union member u (states x of its rows) added to every ADO of the group
  auto add_member = [&](int u, const float2 (&x)[kRpt]) {
#pragma unroll
    for (int k = 0; k < kAdos; ++k) {
      const float4 t = desc[(int64_t)u * kAdos + k];   // (cA or decay, cB, term, -)
      const int term = __float_as_int(t.z);
      if (term == -1) {   // decay of the ADO itself: - gamma_n w_n
#pragma unroll
        for (int j = 0; j < kRpt; ++j) {
          re[k][j] = __fmaf_rn(-t.x, x[j].x, re[k][j]);
          im[k][j] = __fmaf_rn(-t.x, x[j].y, im[k][j]);
        }
      } else if (term >= 0) {   // coupling of mode `term`
        const float lbv = __ldg(lam + term * 128 + b);
#pragma unroll
        for (int j = 0; j < kRpt; ++j) {
          const float la = __ldg(lam + term * 128 + arow[j]);
          const float pc = t.y * (la + lbv), qc = t.x * (la - lbv);
          re[k][j] = __fmaf_rn(qc, x[j].y, __fmaf_rn(pc, x[j].x, re[k][j]));
          im[k][j] = __fmaf_rn(-qc, x[j].x, __fmaf_rn(pc, x[j].y, im[k][j]));
        }
      }
    }
  };
  int u = u0;
  if (kTwo) {
    // two members' loads in flight per thread (same per-element order: u, then u + 1)
    for (; u + 1 < u1; u += 2) {
      const float2 *wm0 = wb + (int64_t)uidx[u] * dd + e0;
      const float2 *wm1 = wb + (int64_t)uidx[u + 1] * dd + e0;
      float2 x0[kRpt], x1[kRpt];
#pragma unroll
      for (int j = 0; j < kRpt; ++j) {
        x0[j] = j < nrow ? wm0[j * es] : make_float2(0.f, 0.f);
        x1[j] = j < nrow ? wm1[j * es] : make_float2(0.f, 0.f);
      }
      add_member(u, x0);
      add_member(u + 1, x1);
    }
  }
  for (; u < u1; ++u) {
    const float2 *wm = wb + (int64_t)uidx[u] * dd + e0;
    float2 x[kRpt];
#pragma unroll
    for (int j = 0; j < kRpt; ++j) x[j] = j < nrow ? wm[j * es] : make_float2(0.f, 0.f);
    add_member(u, x);
  }
#pragma unroll
  for (int k = 0; k < kAdos; ++k) {
    if (n0 + k >= S.n_ado) break;   // ragged last group (uniform across the block)
    const int64_t item = br * S.n_ado + n0 + k;
    const float2 *yb = S.y + item * dd + e0;
    const float2 *tb = S.tpart + item * dd + e0;
    float2 *ob = S.out + item * dd + e0;
    float omax = 0.f;
#pragma unroll
    for (int j = 0; j < kRpt; ++j)
      if (j < nrow) {
        const float2 yv = __ldcs(yb + j * es), tv = __ldcs(tb + j * es);
        const float2 v = make_float2(__fmaf_rn(alpha, re[k][j], __fadd_rn(yv.x, tv.x)),
                                     __fmaf_rn(alpha, im[k][j], __fadd_rn(yv.y, tv.y)));
        omax = fmaxf(omax, fmaxf(fabsf(v.x), fabsf(v.y)));
        __stcs(ob + j * es, v);
      }
    // running max |out| of the item (the tensor-core kernel cleared it)
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) omax = fmaxf(omax, __shfl_xor_sync(0xffffffffu, omax, o2));
    if ((threadIdx.x & 31) == 0 && S.max_out) atomicMax(S.max_out + item, __float_as_uint(omax));
  }
}

// Largest component magnitude of every item of a state (bit pattern of a
// non-negative float, so integer max orders them).
__global__ void __launch_bounds__(256) item_max_kernel(const float2 *__restrict__ x, int64_t dd, unsigned *max_out) {
  const float2 *xi = x + (int64_t)blockIdx.x * dd;
  float m = 0.f;
  for (int64_t e = threadIdx.x; e < dd; e += blockDim.x) m = fmaxf(m, fmaxf(fabsf(xi[e].x), fabsf(xi[e].y)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red[i]);
    max_out[blockIdx.x] = __float_as_uint(red[0] > m ? red[0] : m);
  }
}

}  // namespace

static float bits_as_float(int v) {
  float f;
  std::memcpy(&f, &v, 4);
  return f;
}

static uint16_t half_bits(double x) {
  __half h = __double2half(x);
  uint16_t u;
  std::memcpy(&u, &h, 2);
  return u;
}

static double half_value(uint16_t u) {
  __half h;
  std::memcpy(&h, &u, 2);
  return (double)__half2float(h);
}

void tc_build(TcOperators &tc, const Model &M, const VbModel &vb, std::vector<void *> &allocs) {
  const int d = M.d;
  if (d > 128 || M.n_modes > kTcMaxModes)
    throw std::invalid_argument("tensor-core path supports d <= 128 and at most 4 modes");
  tc.d = d;
  tc.n_ado = M.n_ado;
  tc.n_modes = M.n_modes;
  tc.n_hpieces = 3;
  // H' shifted by a multiple of the identity (the commutator is unchanged), scaled
  // by a power of two so the largest entry is below 2^14, split into 3 FP16 pieces.
  // The shift is the energy of the product ground state, <0|H_S'|0>: the states
  // the response carries most weight on (the equilibrium populations and the
  // coherences with the ground state) then have small products (H' - c) w and
  // w (H' - c), and the tensor cores' FP32 accumulation, whose rounding error
  // scales with the partial sums, stays close to the size of the commutator.
  const double shift = M.H[0];
  double amax = 0.0;
  for (int a = 0; a < d; ++a)
    for (int b2 = 0; b2 < d; ++b2) amax = std::max(amax, std::fabs(M.vb_H[(size_t)a * d + b2] - (a == b2 ? shift : 0.0)));
  int e = 0;
  std::frexp(amax > 0 ? amax : 1.0, &e);
  const double sh = std::ldexp(1.0, 13 - e);
  tc.inv_sh = (float)(1.0 / sh);
  std::vector<uint16_t> img((size_t)3 * kHTile / 2, 0);
  for (int a = 0; a < d; ++a)
    for (int b2 = 0; b2 < d; ++b2) {
      double x = (M.vb_H[(size_t)a * d + b2] - (a == b2 ? shift : 0.0)) * sh;
      const uint32_t off = sw128_offset(a, b2, 16384) / 2;
      for (int piece = 0; piece < 3; ++piece) {
        const uint16_t u = half_bits(x);
        img[(size_t)piece * kHTile / 2 + off] = u;
        x -= half_value(u);
      }
    }
  void *p = nullptr;
  if (device_malloc(&p, img.size() * 2) != cudaSuccess) throw DeviceOom();
  allocs.push_back(p);
  cudaMemcpy(p, img.data(), img.size() * 2, cudaMemcpyHostToDevice);
  tc.himg = (const uint4 *)p;
  std::vector<float> lam((size_t)M.n_modes * 128, 0.f);
  for (int s = 0; s < M.n_modes; ++s)
    for (int a = 0; a < d; ++a) lam[(size_t)s * 128 + a] = (float)M.vb_lam[s][(a / M.stride[s]) % M.dims[s]];
  if (device_malloc(&p, lam.size() * 4) != cudaSuccess) throw DeviceOom();
  allocs.push_back(p);
  cudaMemcpy(p, lam.data(), lam.size() * 4, cudaMemcpyHostToDevice);
  tc.lam = (const float *)p;
  if (device_malloc(&p, 16) != cudaSuccess) throw DeviceOom();
  allocs.push_back(p);
  cudaMemset(p, 0, 16);
  tc.err = (int *)p;
  for (int n = 0; n < M.n_ado; ++n)
    if (M.nb_off[(size_t)n * M.n_modes + M.n_modes] - M.nb_off[(size_t)n * M.n_modes] > kMaxNb)
      throw std::invalid_argument("tensor-core path supports at most 32 coupling entries per ADO");
  // coupling-kernel tables for groups of G = 1, 2, 4, 8 consecutive ADOs: the union
  // of the group's ADOs and their neighbours in ascending order, and the term each
  // member contributes to each ADO of the group (same float values as the FP32
  // coupling lists: (float) of the FP64 model entries)
  for (int q = 0; q < 4; ++q) {
    const int G = 1 << q;
    const int ngroups = (M.n_ado + G - 1) / G;
    std::vector<int> uoff(1, 0), uidx;
    std::vector<float4> desc;
    for (int g = 0; g < ngroups; ++g) {
      std::map<int, std::vector<float4>> terms;   // member -> term per ADO of the group
      const float4 none = make_float4(0.f, 0.f, bits_as_float(-2), 0.f);
      for (int k = 0; k < G && g * G + k < M.n_ado; ++k) {
        const int n = g * G + k;
        auto slot = [&](int m) -> float4 & {
          auto &v = terms[m];
          if (v.empty()) v.assign(G, none);
          return v[k];
        };
        slot(n) = make_float4((float)M.decay[n], 0.f, bits_as_float(-1), 0.f);
        for (int sm = 0; sm < M.n_modes; ++sm)
          for (int e = M.nb_off[(size_t)n * M.n_modes + sm]; e < M.nb_off[(size_t)n * M.n_modes + sm + 1]; ++e)
            slot(M.nb_idx[e]) = make_float4((float)M.nb_cA[e], (float)M.nb_cB[e], bits_as_float(sm), 0.f);
      }
      for (auto &kv : terms) {
        uidx.push_back(kv.first);
        desc.insert(desc.end(), kv.second.begin(), kv.second.end());
      }
      uoff.push_back((int)uidx.size());
    }
    void *pu = nullptr, *pi = nullptr, *pd = nullptr;
    if (device_malloc(&pu, uoff.size() * 4) != cudaSuccess) throw DeviceOom();
    allocs.push_back(pu);
    if (device_malloc(&pi, std::max<size_t>(uidx.size(), 1) * 4) != cudaSuccess) throw DeviceOom();
    allocs.push_back(pi);
    if (device_malloc(&pd, std::max<size_t>(desc.size(), 1) * sizeof(float4)) != cudaSuccess) throw DeviceOom();
    allocs.push_back(pd);
    cudaMemcpy(pu, uoff.data(), uoff.size() * 4, cudaMemcpyHostToDevice);
    if (!uidx.empty()) cudaMemcpy(pi, uidx.data(), uidx.size() * 4, cudaMemcpyHostToDevice);
    if (!desc.empty()) cudaMemcpy(pd, desc.data(), desc.size() * sizeof(float4), cudaMemcpyHostToDevice);
    tc.vt_uoff[q] = (const int *)pu;
    tc.vt_uidx[q] = (const int *)pi;
    tc.vt_desc[q] = (const float4 *)pd;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&tc.sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaFuncSetAttribute(tc_stage_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDyn) !=
          cudaSuccess ||
      cudaFuncSetAttribute(tc_stage_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemDyn) != cudaSuccess)
    throw std::invalid_argument("cannot reserve shared memory for the tensor-core stage");
  tc.ready = true;
}

bool tc_supported(const TcOperators &tc) { return tc.ready; }

// Shapes of the coupling kernel the autotuner chooses from: rows per thread x
// row groups (128 threads each) per block x consecutive ADOs per block.
struct VtShape {
  int rpt, groups, ados;
  bool pf;    // bulk L2 prefetch of the block's source bands at its start
  bool two;   // two union members' loads in flight per thread
};
constexpr VtShape kVtShapes[] = {
    {8, 2, 1, false, false}, {4, 2, 1, false, false}, {8, 1, 1, false, false}, {4, 2, 2, false, false},
    {4, 2, 4, false, false}, {4, 1, 4, false, false}, {2, 2, 8, false, false}, {4, 1, 8, false, false},
    {8, 1, 1, true, false},  {4, 2, 1, true, false},  {8, 2, 1, true, false},  {4, 2, 4, true, false},
    {16, 1, 1, true, false}, {4, 1, 1, true, false},  {8, 1, 1, true, true},   {4, 1, 1, true, true},
    {4, 2, 1, true, true}};
constexpr int kVtShapeCount = (int)(sizeof(kVtShapes) / sizeof(kVtShapes[0]));

static void launch_vterm(int shape, int64_t blocks, const TcArgs &a, cudaStream_t st) {
  const unsigned g = (unsigned)blocks;
  switch (shape) {
    case 1: vterm_kernel<4, 2, 1, false, false><<<g, 256, 0, st>>>(a); break;
    case 2: vterm_kernel<8, 1, 1, false, false><<<g, 128, 0, st>>>(a); break;
    case 3: vterm_kernel<4, 2, 2, false, false><<<g, 256, 0, st>>>(a); break;
    case 4: vterm_kernel<4, 2, 4, false, false><<<g, 256, 0, st>>>(a); break;
    case 5: vterm_kernel<4, 1, 4, false, false><<<g, 128, 0, st>>>(a); break;
    case 6: vterm_kernel<2, 2, 8, false, false><<<g, 256, 0, st>>>(a); break;
    case 7: vterm_kernel<4, 1, 8, false, false><<<g, 128, 0, st>>>(a); break;
    case 8: vterm_kernel<8, 1, 1, true, false><<<g, 128, 0, st>>>(a); break;
    case 9: vterm_kernel<4, 2, 1, true, false><<<g, 256, 0, st>>>(a); break;
    case 10: vterm_kernel<8, 2, 1, true, false><<<g, 256, 0, st>>>(a); break;
    case 11: vterm_kernel<4, 2, 4, true, false><<<g, 256, 0, st>>>(a); break;
    case 12: vterm_kernel<16, 1, 1, true, false><<<g, 128, 0, st>>>(a); break;
    case 13: vterm_kernel<4, 1, 1, true, false><<<g, 128, 0, st>>>(a); break;
    case 14: vterm_kernel<8, 1, 1, true, true><<<g, 128, 0, st>>>(a); break;
    case 15: vterm_kernel<4, 1, 1, true, true><<<g, 128, 0, st>>>(a); break;
    case 16: vterm_kernel<4, 2, 1, true, true><<<g, 256, 0, st>>>(a); break;
    default: vterm_kernel<8, 2, 1, false, false><<<g, 256, 0, st>>>(a); break;
  }
}

// One RK4 stage, out = y + alpha L(w), of every set: one tensor-core launch and
// one coupling-kernel launch (of the given shape) for all of them.  which = 0..3
// selects the Horner stage's buffers (w, out, tpart, max_in, max_out) of each
// set.  Returns the coupling kernel's block count.
static int64_t tc_stage_sets(const std::vector<TcRk4Set> &sets, int which, float alpha, int shape, cudaStream_t st) {
  const int rows = kVtShapes[shape].rpt * kVtShapes[shape].groups, ados = kVtShapes[shape].ados;
  TcArgs a;
  std::memset(&a, 0, sizeof a);
  a.n_sets = (int)sets.size();
  a.alpha = alpha;
  a.n_hpieces = sets[0].tc->n_hpieces;
  a.err = sets[0].tc->err;
  a.wait_ns = sets[0].tc->wait_ns;
  int64_t items = 0, blocks = 0;
  for (int k = 0; k < a.n_sets; ++k) {
    const TcRk4Set &R = sets[k];
    const TcOperators &tc = *R.tc;
    TcSet &S = a.sets[k];
    unsigned *my = tc.maxbuf, *ma = tc.maxbuf + tc.max_items, *mb = tc.maxbuf + 2 * tc.max_items;
    // stage buffers of the nested (Horner) form; the tensor-core part goes to a
    // buffer that is neither y nor w: out itself in stages 1-3, the free scratch wb
    // in stage 4 (out = y there)
    const float2 *w[4] = {R.y, R.wa, R.wb, R.wa};
    float2 *out[4] = {R.wa, R.wb, R.wa, R.y};
    float2 *tp[4] = {R.wa, R.wb, R.wa, R.wb};
    const unsigned *mi[4] = {my, ma, mb, ma};
    unsigned *mo[4] = {ma, mb, ma, my};
    S.himg = tc.himg;
    S.lam = tc.lam;
    for (int q = 0; q < 4; ++q) {
      S.vt_uoff[q] = tc.vt_uoff[q];
      S.vt_uidx[q] = tc.vt_uidx[q];
      S.vt_desc[q] = tc.vt_desc[q];
    }
    S.w = w[which];
    S.y = R.y;
    S.out = out[which];
    S.tpart = tp[which];
    S.max_in = mi[which];
    S.max_out = mo[which];
    S.inv_sh = tc.inv_sh;
    S.d = tc.d;
    S.n_ado = tc.n_ado;
    S.n_modes = tc.n_modes;
    S.bands = (tc.d + rows - 1) / rows;
    S.item_begin = items;
    S.vt_begin = blocks;
    const int64_t n = (int64_t)R.branches * tc.n_ado;
    items += n;
    blocks += (int64_t)R.branches * ((tc.n_ado + ados - 1) / ados) * S.bands;
  }
  a.n_items = items;
  if (items == 0) return 0;
  if (blocks > 0x7fffffffLL) throw std::invalid_argument("too many work items for one stage launch");
  const int grid = (int)std::min<int64_t>(items, sets[0].tc->sms);
  if (a.n_sets > 1)
    tc_stage_kernel<true><<<grid, kThreads, kSmemDyn, st>>>(a);
  else
    tc_stage_kernel<false><<<grid, kThreads, kSmemDyn, st>>>(a);
  launch_vterm(shape, blocks, a, st);
  count_launch(2);
  return blocks;
}

static int64_t total_elements(const std::vector<TcRk4Set> &sets) {
  int64_t e = 0;
  for (const TcRk4Set &R : sets) e += (int64_t)R.branches * R.tc->n_ado * R.tc->d * R.tc->d;
  return e;
}

// Coupling-kernel shape for a launch over these sets: the tuned one for their
// total size (kept by the first set's hierarchy), else the default.  Outside a
// stream capture, an untuned size is tuned first: every candidate shape times
// three first-stage launches after one untimed one.  The first stage reads only
// y and its item maxima and writes scratch (wa and its maxima) that the RK4
// step overwrites, so tuning changes no result.  Needs the item maxima of y.
static std::atomic<int> g_forced_shape{-1};

bool tc_shape_params(int shape, int *rpt, int *groups, int *ados, int *flags) {
  if (shape < 0 || shape >= kVtShapeCount) return false;
  if (rpt) *rpt = kVtShapes[shape].rpt;
  if (groups) *groups = kVtShapes[shape].groups;
  if (ados) *ados = kVtShapes[shape].ados;
  if (flags) *flags = (kVtShapes[shape].pf ? 1 : 0) | (kVtShapes[shape].two ? 2 : 0);
  return true;
}

int tc_shape_count() { return kVtShapeCount; }

bool tc_force_shape(int shape) {
  if (shape < -1 || shape >= kVtShapeCount) return false;
  g_forced_shape.store(shape);
  return true;
}

static int vterm_shape(const std::vector<TcRk4Set> &sets, double dt, cudaStream_t st) {
  const int forced = g_forced_shape.load();
  if (forced >= 0) return forced;
  TcOperators &t0 = *sets[0].tc;
  const int64_t key = total_elements(sets);
  auto it = t0.vt_tuned.find(key);
  if (it != t0.vt_tuned.end()) return it->second.shape;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    (void)cudaGetLastError();
    return 0;
  }
  TcTuned best{0, 0, 0, 1e30f};
  bool ok = true;
  for (int c = 0; c < kVtShapeCount && ok; ++c) {
    const int64_t blocks = tc_stage_sets(sets, 0, (float)(dt / 4), c, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) tc_stage_sets(sets, 0, (float)(dt / 4), c, st);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ok = false;
    if (ok && ms < best.ms) best = TcTuned{c, 128 * kVtShapes[c].groups, blocks, ms};
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return 0;
  t0.vt_tuned[key] = best;
  return best.shape;
}

void tc_reserve(TcOperators &tc, int64_t n_items) {
  if (n_items <= tc.max_items) return;
  if (tc.maxbuf) cudaFree(tc.maxbuf);
  tc.maxbuf = nullptr;
  tc.max_items = 0;
  if (device_malloc((void **)&tc.maxbuf, (size_t)n_items * 3 * sizeof(unsigned)) != cudaSuccess) throw DeviceOom();
  tc.max_items = n_items;
}

// Item maxima of every set's y (the first stage's input scaling); false if the
// sets hold no work item.
static bool tc_prologue(const std::vector<TcRk4Set> &sets, cudaStream_t st) {
  if ((int)sets.size() > kTcMaxSets) throw std::invalid_argument("too many parameter sets for one stage launch");
  bool any = false;
  for (const TcRk4Set &R : sets) {
    const int64_t n_items = (int64_t)R.branches * R.tc->n_ado;
    if (n_items <= 0) continue;
    any = true;
    tc_reserve(*R.tc, n_items);
    item_max_kernel<<<(unsigned)n_items, 256, 0, st>>>(R.y, (int64_t)R.tc->d * R.tc->d, R.tc->maxbuf);
    count_launch(1);
  }
  return any;
}

void tc_tune(const std::vector<TcRk4Set> &sets, double dt, cudaStream_t st) {
  if (sets.empty() || !tc_prologue(sets, st)) return;
  vterm_shape(sets, dt, st);
}

void tc_rk4_sets(const std::vector<TcRk4Set> &sets, double dt, int64_t nsteps, cudaStream_t st) {
  if (sets.empty() || nsteps <= 0) return;
  if (!tc_prologue(sets, st)) return;
  const int shape = vterm_shape(sets, dt, st);
  for (int64_t s = 0; s < nsteps; ++s) {
    tc_stage_sets(sets, 0, (float)(dt / 4), shape, st);
    tc_stage_sets(sets, 1, (float)(dt / 3), shape, st);
    tc_stage_sets(sets, 2, (float)(dt / 2), shape, st);
    tc_stage_sets(sets, 3, (float)dt, shape, st);
  }
}

void tc_rk4_steps(TcOperators &tc, float2 *y, float2 *wa, float2 *wb, int branches, double dt, int64_t nsteps,
                  cudaStream_t st) {
  tc_rk4_sets({TcRk4Set{&tc, y, wa, wb, branches}}, dt, nsteps, st);
}

}  // namespace heom
