// pt_batch.cu -- the batched path: one persistent kernel advances many independent PT
// problems of uneven L and R.
//
// Work items are whole problems (n sweeps each, exchange every m). Items are sorted by work
// and split in two queues:
//   joint  -- one problem spread over the G CTAs of a thread-block cluster (rows split
//             between the CTAs); half sweeps are separated by hardware cluster barriers
//             (barrier.cluster with release/acquire), so no CTA ever spins on memory;
//   single -- one problem owned by one CTA (__syncthreads between half sweeps).
// Each cluster drains the joint queue first (its leader CTA takes the next item and shares
// the index through distributed shared memory), then every CTA drains the single queue on
// its own. The lattices stay in global memory (L2-resident for the batched workloads);
// lattice words are read with ld.global.cg so that rows written by another CTA of the
// cluster are never served stale from L1.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "pt_batch.h"
#include "pt_debug.cuh"
#include "pt_device.cuh"
#include "pt_internal.h"
#include "pt_launch.h"

namespace cg = cooperative_groups;

namespace ptb {

namespace {

constexpr int kBatchThreads = 384;

struct BatchItem {
  DevProblem p;
  uint64_t t0, e0;  // counters when the batch starts
  int64_t n;        // sweeps
  int m;            // exchange every m sweeps (0 = never)
  int pad;
};

struct BatchQueues {
  int next_joint;
  int next_single;
  int n_joint;
  int n_single;
};

__device__ __forceinline__ uint32_t ldcg(const uint32_t* p) { return __ldcg(p); }

// A group of CTAs working on one problem: the whole cluster (joint) or one CTA (single).
template <bool JOINT>
struct Gang {
  int rank, size;
  __device__ __forceinline__ void sync() const {
    if (JOINT)
      cg::this_cluster().sync();
    else
      __syncthreads();
  }
};

__device__ __forceinline__ int plane_slots(int R, int w) { return min(32, R - 32 * w); }

// Per-thread view of the threshold registers of the plane a warp works on.
struct FerroRegs {
  uint32_t T0[32], T1[32];
  uint32_t alw0, alw1, used;

  __device__ __forceinline__ void load(const PlaneFerro* pl) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(pl);
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      T0[b] = ldcg(src + b);
      T1[b] = ldcg(src + 32 + b);
    }
    alw0 = ldcg(src + 64);
    alw1 = ldcg(src + 65);
    used = ldcg(src + 66);
  }
};

// Warps are dealt to planes round-robin: warp v works on plane v % W (and on v % W + nwarps,
// ... when W > nwarps). Inside a plane, the words of rows [y0, y1) of one colour are dealt
// to the plane's warps lane by lane.
struct PlaneDeal {
  int w_first, w_step;   // planes of this warp: w_first, w_first + w_step, ...
  int rank, nranks;      // this warp's rank among the warps of its plane
  __device__ __forceinline__ PlaneDeal(int W) {
    const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5;
    w_first = warp % W;
    w_step = nwarps;
    if (W <= nwarps) {
      rank = warp / W;
      nranks = (nwarps - w_first + W - 1) / W;
    } else {
      rank = 0;
      nranks = 1;
    }
  }
};

// Walks this warp's words of rows [y0, y1) of one colour: q = rank * 32 + lane, stepping by
// nranks * 32, with (row, i) kept up to date by additions only.
struct WordWalk {
  int q, step, yy, i, dyy, di, half;
  __device__ __forceinline__ WordWalk(int q0, int step_, int half_)
      : q(q0), step(step_), half(half_) {
    yy = q0 / half_;
    i = q0 - yy * half_;
    dyy = step_ / half_;
    di = step_ - dyy * half_;
  }
  __device__ __forceinline__ void next() {
    q += step;
    i += di;
    yy += dyy;
    if (i >= half) {
      i -= half;
      yy += 1;
    }
  }
};

// The five words one update reads: the centre and its four neighbours (other colour).
struct Nb5 {
  uint32_t s, n0, n1, n2, n3;
};

// Rows inside [y0, y1) were last written by this CTA, so L1 may serve them; the two halo
// rows just outside belong to another CTA of the cluster and are read from L2 (.cg), never
// from a possibly stale L1 line. A single-CTA gang owns every row.
__device__ __forceinline__ uint32_t ld_row(const uint32_t* p, bool own) {
  return own ? *p : __ldcg(p);
}

__device__ __forceinline__ Nb5 load_nb(const DevProblem& p, const uint32_t* own,
                                       const uint32_t* oth, int L, int half, int y, int i,
                                       int colour, int y0, int y1) {
  const int par = (y + colour) & 1;
  const int ym = (y == 0) ? L - 1 : y - 1;
  const int yp = (y == L - 1) ? 0 : y + 1;
  const int ih = par ? ((i + 1 == half) ? 0 : i + 1) : ((i == 0) ? half - 1 : i - 1);
  const size_t idx = (size_t)y * half + i;
  const int nw = L * half;  // words of one colour (the debug checks' range)
  (void)p;
  (void)nw;
  Nb5 v;
  v.s = own[PT_DBG_IDX(p, idx, nw, kDbgSpinLoad)];
  v.n0 = ld_row(oth + PT_DBG_IDX(p, (size_t)ym * half + i, nw, kDbgSpinLoad), ym >= y0 && ym < y1);
  v.n1 = ld_row(oth + PT_DBG_IDX(p, (size_t)yp * half + i, nw, kDbgSpinLoad), yp >= y0 && yp < y1);
  v.n2 = oth[PT_DBG_IDX(p, idx, nw, kDbgSpinLoad)];
  v.n3 = oth[PT_DBG_IDX(p, (size_t)y * half + ih, nw, kDbgSpinLoad)];
  return v;
}

template <int MODE>
__device__ __forceinline__ void half_sweep_plane(const DevProblem& p, int w, int colour,
                                                 uint64_t t, const SweepCtr& cx, int y0, int y1,
                                                 int nwords,
                                                 const PlaneDeal& deal, const FerroRegs& th,
                                                 const PlaneGeneric* gen_smem) {
  const int L = p.L, half = L >> 1;
  const int lane = threadIdx.x & 31;
  const int nblk = (plane_slots(p.R, w) + 3) >> 2;
  const size_t own_base = word_index(L, w, colour, 0, 0);
  uint32_t* own = p.spins + own_base;
  const uint32_t* oth = p.spins + word_index(L, w, colour ^ 1, 0, 0);
  (void)own_base;
  PT_DBG_CHECK(p, w, p.W, kDbgSpinLoad);
  WordWalk ww(deal.rank * 32 + lane, deal.nranks * 32, half);
  if (ww.q >= nwords) return;
  // software pipeline: the next word's loads are in flight while this word is updated
  Nb5 cur = load_nb(p, own, oth, L, half, y0 + ww.yy, ww.i, colour, y0, y1);
  for (;;) {
    const int y = y0 + ww.yy, i = ww.i;
    WordWalk nx = ww;
    nx.next();
    Nb5 nxt = cur;
    if (nx.q < nwords) nxt = load_nb(p, own, oth, L, half, y0 + nx.yy, nx.i, colour, y0, y1);
    const int par = (y + colour) & 1;
    const uint32_t site = (uint32_t)(y * L + 2 * i + par);
    const size_t idx = (size_t)y * half + i;
    uint32_t ns;
    if (MODE == kModeFerro)
      ns = update_word_ferro(cur.s, cur.n0, cur.n1, cur.n2, cur.n3, site, (uint32_t)(8 * w),
                             nblk, th.T0, th.T1, th.alw0, th.alw1, th.used, cx);
    else
      ns = update_word_generic(cur.s, cur.n0, cur.n1, cur.n2, cur.n3, site, (uint32_t)(8 * w),
                               nblk, gen_smem[w], cx);
    if (PT_DBG_STORE(p, idx, L * half, own_base, t, colour)) own[idx] = ns;
    if (nx.q >= nwords) break;
    ww = nx;
    cur = nxt;
  }
}

// One half sweep of rows [y0, y1). `th` holds the thresholds of this warp's plane when the
// warp owns a single plane (W <= warps per CTA); otherwise they are loaded plane by plane.
template <int MODE>
__device__ void half_sweep_rows(const DevProblem& p, int colour, uint64_t t, int y0, int y1,
                                FerroRegs& th, bool th_loaded, const PlaneGeneric* gen_smem) {
  const SweepCtr cx = make_sweep_ctr(t, p.key0, p.key1);
  const PlaneDeal deal(p.W);
  const int nwords = (y1 - y0) * (p.L >> 1);
  for (int w = deal.w_first; w < p.W; w += deal.w_step) {
    if (MODE == kModeFerro && !th_loaded) th.load(reinterpret_cast<const PlaneFerro*>(p.planes) + w);
    half_sweep_plane<MODE>(p, w, colour, t, cx, y0, y1, nwords, deal, th, gen_smem);
  }
}

// Unsatisfied bonds and up spins of rows [y0, y1), added into p.cnt (see k_energy).
__device__ void count_rows(const DevProblem& p, int y0, int y1, uint32_t* acc_smem /*[2][W*32]*/) {
  const int L = p.L, half = L >> 1;
  const PlaneDeal deal(p.W);
  const int lane = threadIdx.x & 31;
  const int nwords = (y1 - y0) * half;
  for (int w = deal.w_first; w < p.W; w += deal.w_step) {
    const uint32_t* c0 = p.spins + word_index(L, w, 0, 0, 0);
    const uint32_t* c1 = p.spins + word_index(L, w, 1, 0, 0);
    BitCounter<20, 14> U, N;
    U.zero();
    N.zero();
    for (WordWalk ww(deal.rank * 32 + lane, deal.nranks * 32, half); ww.q < nwords; ww.next()) {
      const int y = y0 + ww.yy, i = ww.i;
      const int par = y & 1;
      const int ym = (y == 0) ? L - 1 : y - 1;
      const int yp = (y == L - 1) ? 0 : y + 1;
      const int ih = par ? ((i + 1 == half) ? 0 : i + 1) : ((i == 0) ? half - 1 : i - 1);
      const size_t idx = (size_t)y * half + i;
      const int nw = L * half;
      (void)nw;
      const uint32_t s = c0[PT_DBG_IDX(p, idx, nw, kDbgSpinLoad)];
      const uint32_t o = c1[PT_DBG_IDX(p, idx, nw, kDbgSpinLoad)];
      const NbCount k = count4(
          s ^ ld_row(c1 + PT_DBG_IDX(p, (size_t)ym * half + i, nw, kDbgSpinLoad), ym >= y0 && ym < y1),
          s ^ ld_row(c1 + PT_DBG_IDX(p, (size_t)yp * half + i, nw, kDbgSpinLoad), yp >= y0 && yp < y1),
          s ^ o, s ^ c1[PT_DBG_IDX(p, (size_t)y * half + ih, nw, kDbgSpinLoad)]);
      U.add3(k.b0, k.b1, k.b2);
      N.add2(s ^ o, s & o);
    }
    const uint32_t u = U.warp_total_for_lane();
    const uint32_t nn = N.warp_total_for_lane();
    if (u) atomicAdd(&acc_smem[w * 32 + lane], u);
    if (nn) atomicAdd(&acc_smem[p.W * 32 + w * 32 + lane], nn);
  }
}

// Exchange step of one problem by one CTA (same three parts as k_exchange).
__device__ void exchange_step(const DevProblem& p, uint64_t e) {
  const int R = p.R, W = p.W;
  const int64_t L2 = (int64_t)p.L * p.L;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const int64_t U = __ldcg(p.cnt + r);
    const int64_t ones = __ldcg(p.cnt + W * 32 + r);
    const int64_t bonds = 2 * L2 - 2 * U;
    const int64_t M = 2 * ones - L2;
    p.E_slot[r] = -p.J_int * bonds + p.h_int * M;
    p.M_slot[r] = M;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * W * 32; q += blockDim.x) p.cnt[q] = 0;
  const int parity = (int)(e & 1);
  const uint32_t c3 = kTagExch | ((uint32_t)(e >> 32) << 8);
  for (int k = parity + 2 * threadIdx.x; k + 1 < R; k += 2 * blockDim.x) {
    const int a = p.slot_of_temp[k], b = p.slot_of_temp[k + 1];
    const int64_t n = p.E_slot[a] - p.E_slot[b];
    const SwapPair sp = p.pairs[k];
    const uint64_t S = pair_threshold(sp, p.swap_table, p.table_shift, n);
    const Philox4 rnd = philox4x32_10((uint32_t)k, (uint32_t)e, 0u, c3, p.key0, p.key1);
    const bool accept = (uint64_t)rnd.x < S;
    count_swap(p.attempted, p.accepted, k, accept);
    if (accept) {
      p.slot_of_temp[k] = b;
      p.slot_of_temp[k + 1] = a;
      p.temp_of_slot[a] = k + 1;
      p.temp_of_slot[b] = k;
    }
  }
  __syncthreads();
  // refresh the plane thresholds for the new slot -> temperature map
  constexpr uint64_t kTwo32 = 1ull << 32;
  for (int r = threadIdx.x; r < W * 32; r += blockDim.x) {
    const int w = r >> 5, b = r & 31;
    const bool in_use = r < R;
    const int temp = in_use ? p.temp_of_slot[r] : 0;
    if (p.mode == kModeFerro) {
      PlaneFerro* pl = reinterpret_cast<PlaneFerro*>(p.planes) + w;
      const uint64_t t0 = in_use ? p.T_temp[(size_t)temp * kClasses + 1] : 0;
      const uint64_t t1 = in_use ? p.T_temp[(size_t)temp * kClasses + 3] : 0;
      pl->T0[b] = (uint32_t)min(t0, kTwo32 - 1);
      pl->T1[b] = (uint32_t)min(t1, kTwo32 - 1);
      const uint32_t a0 = __ballot_sync(0xffffffffu, in_use && t0 >= kTwo32);
      const uint32_t a1 = __ballot_sync(0xffffffffu, in_use && t1 >= kTwo32);
      if (b == 0) {
        pl->alw0 = a0;
        pl->alw1 = a1;
      }
    } else {
      PlaneGeneric* pl = reinterpret_cast<PlaneGeneric*>(p.planes) + w;
#pragma unroll
      for (int c = 0; c < kClasses; ++c) {
        const uint64_t tc = in_use ? p.T_temp[(size_t)temp * kClasses + c] : 0;
        pl->T[c][b] = (uint32_t)min(tc, kTwo32 - 1);
        const uint32_t a = __ballot_sync(0xffffffffu, in_use && tc >= kTwo32);
        if (b == 0) pl->alw[c] = a;
      }
    }
  }
}

__device__ void load_generic_planes(const DevProblem& p, PlaneGeneric* smem) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(p.planes);
  uint32_t* dst = reinterpret_cast<uint32_t*>(smem);
  const int nw = p.W * (int)(sizeof(PlaneGeneric) / 4);
  for (int q = threadIdx.x; q < nw; q += blockDim.x) dst[q] = __ldcg(src + q);
}

template <bool JOINT>
__device__ void run_item(const BatchItem& it, const Gang<JOINT>& gang, uint32_t* smem_words) {
  const DevProblem& p = it.p;
  const int L = p.L;
  const int y0 = (int)((int64_t)L * gang.rank / gang.size);
  const int y1 = (int)((int64_t)L * (gang.rank + 1) / gang.size);
  PlaneGeneric* gen = reinterpret_cast<PlaneGeneric*>(smem_words);
  uint32_t* acc = smem_words;  // [2][W*32] counters (generic tables are reloaded after use)
  const bool one_plane = p.W <= (int)(blockDim.x >> 5);
  FerroRegs th;
  if (p.mode == kModeFerro) {
    if (one_plane) th.load(reinterpret_cast<const PlaneFerro*>(p.planes) + PlaneDeal(p.W).w_first);
  } else {
    load_generic_planes(p, gen);
    __syncthreads();
  }
  uint64_t e = it.e0;
  for (int64_t j = 0; j < it.n; ++j) {
    const uint64_t t = it.t0 + (uint64_t)j;
    if (p.mode == kModeFerro) {
      half_sweep_rows<kModeFerro>(p, 0, t, y0, y1, th, one_plane, gen);
      gang.sync();
      half_sweep_rows<kModeFerro>(p, 1, t, y0, y1, th, one_plane, gen);
    } else {
      half_sweep_rows<kModeGeneric>(p, 0, t, y0, y1, th, false, gen);
      gang.sync();
      half_sweep_rows<kModeGeneric>(p, 1, t, y0, y1, th, false, gen);
    }
    gang.sync();
    if (it.m > 0 && (t + 1) % (uint64_t)it.m == 0) {
      // count this CTA's rows into shared counters, then into the problem's counters
      for (int q = threadIdx.x; q < 2 * p.W * 32; q += blockDim.x) acc[q] = 0;
      __syncthreads();
      count_rows(p, y0, y1, acc);
      __syncthreads();
      for (int q = threadIdx.x; q < 2 * p.W * 32; q += blockDim.x)
        if (acc[q]) atomicAdd(&p.cnt[PT_DBG_IDX(p, q, 2 * p.W * 32, kDbgCount)], acc[q]);
      gang.sync();
      if (gang.rank == 0) exchange_step(p, e);
      e += 1;
      gang.sync();
      if (p.mode == kModeFerro) {
        if (one_plane)
          th.load(reinterpret_cast<const PlaneFerro*>(p.planes) + PlaneDeal(p.W).w_first);
      } else {
        load_generic_planes(p, gen);
        __syncthreads();
      }
    }
  }
}

__device__ __forceinline__ void stage_item(const BatchItem* src, BatchItem* dst) {
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int q = threadIdx.x; q < (int)(sizeof(BatchItem) / 4); q += blockDim.x) d[q] = s[q];
  __syncthreads();
}

__global__ void __launch_bounds__(kBatchThreads, 1)
    k_batch(const BatchItem* __restrict__ items, BatchQueues* queues, int single_only) {
  extern __shared__ uint32_t smem_words[];
  __shared__ int item_s;
  __shared__ __align__(16) BatchItem cur;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int G = (int)cluster.num_blocks();
  const int n_joint = queues->n_joint;
  // joint items: one problem per cluster
  if (!single_only && G > 1 && n_joint > 0) {
    for (;;) {
      if (rank == 0 && threadIdx.x == 0) item_s = atomicAdd(&queues->next_joint, 1);
      cluster.sync();
      int* leader = cluster.map_shared_rank(&item_s, 0);
      const int item = *leader;
      cluster.sync();  // everyone has read the index before the leader takes the next
      if (item >= n_joint) break;
      Gang<true> gang{rank, G};
      stage_item(items + item, &cur);
      run_item<true>(cur, gang, smem_words);
      cluster.sync();
    }
  }
  // single items: one problem per CTA (with G == 1 the joint items are single ones too)
  const int n_single = queues->n_single;
  const bool split = single_only || G > 1;
  const int base = split ? n_joint : 0;
  const int total = split ? n_single : n_joint + n_single;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) item_s = atomicAdd(&queues->next_single, 1);
    __syncthreads();
    const int item = item_s;
    if (item >= total) break;
    Gang<false> gang{0, 1};
    stage_item(items + base + item, &cur);
    run_item<false>(cur, gang, smem_words);
  }
}

// A second stream per device for the helper launch (fork / join through events, so the
// pair also records into a CUDA graph when the caller's stream is being captured).
struct HelperStream {
  bool ok = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

HelperStream& helper_stream(int device) {
  static std::mutex mu;
  static std::map<int, HelperStream> streams;
  std::lock_guard<std::mutex> lk(mu);
  HelperStream& hs = streams[device];
  if (!hs.ok) {
    hs.ok = cudaStreamCreateWithFlags(&hs.stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&hs.fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&hs.join, cudaEventDisableTiming) == cudaSuccess;
  }
  return hs;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
BatchTuning g_batch_tuning;  // set through pt_set_batch_tuning (the autotuner)

// Host mirrors of the sweep and swap-iteration counters after a batch.
static void advance_counters(pt_problem* const* ps, int count, const int64_t* n,
                             const int* every) {
  for (int j = 0; j < count; ++j) {
    pt_problem* p = ps[j];
    const int m = every[j];
    if (m > 0) p->e += (p->t + (uint64_t)n[j]) / (uint64_t)m - p->t / (uint64_t)m;
    p->t += (uint64_t)n[j];
  }
}

// Checks of the allocation-free entry point: valid problems, counts, one stream, one device,
// no problem twice, and a stream that is not being captured. Nothing here allocates: the
// duplicate check compares pairs (count is at most kStaticMaxBatch). Returns the stream
// through *st.
static int check_batch_static(pt_problem* const* ps, int count, const int64_t* n,
                              const int* every, cudaStream_t* st_out) {
  if (count > kStaticMaxBatch)
    return fail(PT_EINVAL, "pt_sweep_batch_static: %d problems, more than %d", count,
                kStaticMaxBatch);
  cudaStream_t st = ps[0] ? ps[0]->stream : 0;
  int dev = -1;
  for (int j = 0; j < count; ++j) {
    pt_problem* p = ps[j];
    int rc = problem_check(p);
    if (rc) return rc;
    if (n[j] < 0 || every[j] < 0)
      return fail(PT_EINVAL, "problem %d: n = %lld, exchange_every = %d", j, (long long)n[j],
                  every[j]);
    if (p->stream != st) return fail(PT_EINVAL, "problems of one batch must share a stream");
    if (dev < 0) dev = p->dev_info.device;
    if (p->dev_info.device != dev) return fail(PT_EINVAL, "problems on different devices");
  }
  for (int a = 1; a < count; ++a)
    for (int b = 0; b < a; ++b)
      if (ps[a] == ps[b]) return fail(PT_EINVAL, "a problem appears twice in one batch");
  int rc = problem_device_guard(ps[0]);
  if (rc) return rc;
  // The call copies its work lists from host arrays that the next call overwrites, and it
  // waits for those copies: neither can be recorded into a graph. Refused before anything
  // is queued, so no problem is touched.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t err = cudaStreamIsCapturing(st, &cap);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return fail(PT_EINVAL, "pt_sweep_batch_static: the stream's capture state cannot be read "
                "(%s)", cudaGetErrorString(err));
  }
  if (cap != cudaStreamCaptureStatusNone)
    return fail(PT_EINVAL, "pt_sweep_batch_static: the problems' stream is being captured; "
                "this entry point cannot be captured into a CUDA graph");
  *st_out = st;
  return PT_OK;
}

int sweep_batch_static_entry(pt_problem* const* ps, int count, const int64_t* n,
                             const int* every) {
  cudaStream_t st = 0;
  int rc = check_batch_static(ps, count, n, every, &st);
  if (rc) return rc;
  const BatchTuning tune = batch_tuning();
  rc = sweep_batch_static(ps, count, n, every, st, ps[0]->dev_info, tune.tile_words,
                          tune.strategy == PT_BATCH_QUEUE);
  if (rc) return rc;
  advance_counters(ps, count, n, every);
  return PT_OK;
}

int sweep_batch(pt_problem* const* ps, int count, const int64_t* n, const int* every) {
  // checks
  cudaStream_t st = ps[0] ? ps[0]->stream : 0;
  int dev = -1;
  for (int j = 0; j < count; ++j) {
    pt_problem* p = ps[j];
    int rc = problem_check(p);
    if (rc) return rc;
    if (n[j] < 0 || every[j] < 0)
      return fail(PT_EINVAL, "problem %d: n = %lld, exchange_every = %d", j, (long long)n[j],
                  every[j]);
    if (p->stream != st) return fail(PT_EINVAL, "problems of one batch must share a stream");
    if (dev < 0) dev = p->dev_info.device;
    if (p->dev_info.device != dev) return fail(PT_EINVAL, "problems on different devices");
  }
  {
    std::vector<pt_problem*> sorted(ps, ps + count);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(PT_EINVAL, "a problem appears twice in one batch");
  }
  int rc = problem_device_guard(ps[0]);
  if (rc) return rc;
  const DeviceInfo& di = ps[0]->dev_info;
  BatchTuning tune = batch_tuning();
  for (int j = 0; j < count; ++j)  // trace rows are written by the lock-step exchange launch
    if (ps[j]->dev.trace_E != nullptr && tune.strategy != PT_BATCH_QUEUE)
      tune.strategy = PT_BATCH_FLAT;
  if (tune.strategy == PT_BATCH_FLAT || tune.strategy == PT_BATCH_QUEUE ||
      tune.strategy == PT_BATCH_FLOW) {
    rc = tune.strategy == PT_BATCH_FLOW
             ? sweep_batch_flow(ps, count, n, every, st, di, tune.tile_words)
             : sweep_batch_flat(ps, count, n, every, st, di, tune.tile_words,
                                tune.strategy == PT_BATCH_QUEUE, tune.streams,
                                tune.graphs != 0);
    if (rc) return rc;
    advance_counters(ps, count, n, every);
    return PT_OK;
  }

  // items, heaviest first; joint = large enough to share a cluster
  struct Order {
    double work;
    int j;
  };
  std::vector<Order> order;
  for (int j = 0; j < count; ++j)
    if (n[j] > 0)
      order.push_back({(double)ps[j]->L * ps[j]->L * ps[j]->W * (double)n[j], j});
  if (order.empty()) return PT_OK;
  std::stable_sort(order.begin(), order.end(),
                   [](const Order& a, const Order& b) { return a.work > b.work; });
  std::vector<BatchItem> joint, single;
  size_t smem = 0;
  for (const Order& o : order) {
    pt_problem* p = ps[o.j];
    BatchItem it{};
    it.p = p->dev;
    it.t0 = p->t;
    it.e0 = p->e;
    it.n = n[o.j];
    it.m = every[o.j];
    const size_t need = std::max<size_t>(
        (size_t)2 * p->W * 32 * 4, p->mode == kModeFerro ? 0 : (size_t)p->W * sizeof(PlaneGeneric));
    smem = std::max(smem, need);
    if (tune.cluster > 1 && p->L >= tune.joint_min_L && p->L >= 2 * tune.cluster)
      joint.push_back(it);
    else
      single.push_back(it);
  }
  if (smem > di.smem_optin - 1024) return fail(PT_EINVAL, "too many replicas for one CTA");
  std::vector<BatchItem> all(joint);
  all.insert(all.end(), single.begin(), single.end());
  BatchQueues q{0, 0, (int)joint.size(), (int)single.size()};

  // stream-ordered scratch for the item list and the queue heads
  const size_t items_bytes = all.size() * sizeof(BatchItem);
  const size_t total = ((items_bytes + 255) & ~size_t(255)) + sizeof(BatchQueues);
  void* scratch = nullptr;
  cudaError_t err = cudaMallocAsync(&scratch, total, st);
  if (err != cudaSuccess) return fail(PT_ENOMEM, "batch scratch: %s", cudaGetErrorString(err));
  BatchItem* d_items = (BatchItem*)scratch;
  BatchQueues* d_q = (BatchQueues*)((char*)scratch + ((items_bytes + 255) & ~size_t(255)));
  err = cudaMemcpyAsync(d_items, all.data(), items_bytes, cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(d_q, &q, sizeof q, cudaMemcpyHostToDevice, st);

  // one persistent launch: as many clusters as fit; with clusters, a second launch of
  // plain CTAs on a forked stream drains the single queue on the SMs the clusters leave idle
  const int G = std::max(1, tune.cluster);
  // the limit belongs to the kernel, not to this batch: all the device allows, so that a
  // concurrent smaller batch never lowers it under this one's launch
  cudaFuncAttributes fa;
  if (err == cudaSuccess) err = cudaFuncGetAttributes(&fa, k_batch);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(di.smem_optin - fa.sharedSizeBytes));
  if (err == cudaSuccess && G > 8)
    err = cudaFuncSetAttribute(k_batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kBatchThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (err == cudaSuccess) {
    cfg.gridDim = dim3(G * di.sms);
    err = cudaOccupancyMaxActiveClusters(&clusters, (void*)k_batch, &cfg);
  }
  if (err == cudaSuccess) {
    if (clusters < 1) clusters = 1;
    cfg.gridDim = dim3(G * clusters);
    err = cudaLaunchKernelEx(&cfg, k_batch, (const BatchItem*)d_items, d_q, 0);
  }
  const int helpers = G > 1 && !single.empty() ? di.sms - G * clusters : 0;
  if (err == cudaSuccess && helpers > 0) {
    HelperStream& hs = helper_stream(di.device);
    if (!hs.ok) err = cudaErrorNotReady;
    if (err == cudaSuccess) err = cudaEventRecord(hs.fork, st);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(hs.stream, hs.fork, 0);
    if (err == cudaSuccess) {
      k_batch<<<helpers, kBatchThreads, smem, hs.stream>>>(d_items, d_q, 1);
      err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaEventRecord(hs.join, hs.stream);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(st, hs.join, 0);
  }
  cudaError_t err2 = cudaFreeAsync(scratch, st);
  if (err == cudaSuccess) err = err2;
  if (err != cudaSuccess) {
    for (int j = 0; j < count; ++j) ps[j]->poisoned = PT_ECUDA;
    return fail(PT_ECUDA, "batch launch: %s", cudaGetErrorString(err));
  }
  advance_counters(ps, count, n, every);
  return PT_OK;
}

}  // namespace ptb
