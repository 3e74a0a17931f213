// pt_flat.cu -- the lock-step batched path: all problems of a batch advance sweep by sweep
// together. Each half sweep is one launch over a list of equal-sized word tiles drawn from
// every problem and plane, so the work is balanced across the SMs however uneven L and R
// are; the exchange step of every problem due for one is one more launch. Kernel
// boundaries order the steps: nothing waits on a flag.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <queue>
#include <utility>
#include <vector>

#include "pt_batch.h"
#include "pt_device.cuh"
#include "pt_flat.cuh"
#include "pt_internal.h"
#include "pt_launch.h"

namespace ptb {

namespace {

// ---------------------------------------------------------------------------------------
// Two ways to hand a launch's tiles to its warps (the host sorts a mode's tiles by their
// Philox work, largest first, for both):
//  * dealt (PT_BATCH_FLAT): the host deals the sorted tiles to the warps longest-processing-
//    time first, warp g taking tiles [first[g], first[g + 1]);
//  * queued (PT_BATCH_QUEUE): the first G tiles (G = the launch's warps) are dealt one per
//    warp, round robin over the CTAs (warp i of CTA c takes tile i * gridDim.x + c), so the
//    largest tiles spread evenly over the SMs; after that a warp that finishes a tile takes
//    the next one from a device counter, so the rest go greedily to whichever warp is free
//    (list scheduling) and the warps finish together whatever their SM's load. A warp takes
//    a counter value only when it is free: taking one a tile ahead would let the warps that
//    start first claim two tiles each while others still have none.
// The queue counter runs on across the launches of a batch: a launch takes ntiles - G
// values from it when ntiles > G (one per queued tile and one that ends each warp's loop)
// and ntiles when ntiles <= G (one per warp with a tile) -- ntiles either way -- so launch
// number k of the mode starts at base = k ntiles, which the host passes in.
// ---------------------------------------------------------------------------------------
struct TileQueue {
  unsigned long long* ctr;  // values taken so far by this mode's launches in the batch
  unsigned long long base;  // the counter's value when this launch starts
  int ntiles;
};

// Half sweep over all tiles of the launch (QUEUED: handed out by the queue; else dealt,
// `first` the per-warp offsets). With COUNT (colour 1 only) warps whose problem is due for
// an exchange after this sweep also count bonds (and up spins) for it.
template <int MODE, bool COUNT, bool QUEUED>
__global__ void __launch_bounds__(kFlatThreads, 2) k_flat_half(const FlatProblem* __restrict__ probs,
                                                             const Tile* __restrict__ tiles,
                                                             const int* __restrict__ first,
                                                             const TileQueue q, int colour,
                                                             int64_t j) {
  __shared__ __align__(16) PlaneGeneric gen[kFlatThreads / 32];  // 16-byte rows (uint4 reads)
  __shared__ uint4 thr_s[kFlatThreads / 32][16];  // ferro thresholds of each warp's tile
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto run = [&](long long tix) {
    const Tile tl = tiles[tix];
    const FlatProblem& fp = probs[tl.prob];
    if (j >= fp.n) return;  // warp-uniform
    const bool count = COUNT && counts_after(fp, j);
    tile_half<MODE, COUNT, false>(fp, tl, colour, j, count, thr_s[wib], &gen[wib]);
  };
  if (!QUEUED) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int tend = first[g + 1];
    for (int tix = first[g]; tix < tend; ++tix) run(tix);
    return;
  }
  const long long G = (long long)gridDim.x * (kFlatThreads / 32);
  long long tix = (long long)wib * gridDim.x + blockIdx.x;  // the dealt first tile
  while (tix < q.ntiles) {
    run(tix);
    unsigned long long v = 0;
    if (lane == 0) v = atomicAdd(q.ctr, 1ull) - q.base;
    tix = G + (long long)__shfl_sync(0xffffffffu, v, 0);
  }
}

// ---------------------------------------------------------------------------------------
// End of sweep j for every problem counted after it (a swap iteration or a trace row
// follows), one block per problem: energies from the counts (then cleared), the swap
// iteration of Sec. 3, the plane thresholds of the new map, the trace row. What the step
// reads that does not depend on its own results -- the counts, both maps, the thread's
// first pair and the threshold row of every temperature -- is loaded at once, into shared
// memory; after that only the pairs' table lookups and the stores touch global memory.
// Shared memory: flat_exchange_smem(R, mode) bytes.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kFlatThreads) k_flat_exchange(const FlatProblem* __restrict__ probs,
                                                                 int nprobs, int64_t j) {
  extern __shared__ __align__(16) unsigned char xs[];
  constexpr uint64_t kTwo32 = 1ull << 32;
  for (int pi = blockIdx.x; pi < nprobs; pi += gridDim.x) {
    const FlatProblem& fp = probs[pi];
    if (!counts_after(fp, j)) continue;
    const DevProblem& p = fp.p;
    const bool ex = exchanges_after(fp, j);
    const uint64_t e = ex ? exchange_index(fp, j) : 0;
    const int R = p.R, W = p.W;
    const int64_t L2 = (int64_t)p.L * p.L;
    const bool ferro = p.mode == kModeFerro;
    const int ncls = ferro ? 2 : kClasses;  // threshold row entries per temperature
    int64_t* const E_s = reinterpret_cast<int64_t*>(xs);  // [R] by slot
    int64_t* const M_s = E_s + R;                          // [R] by slot
    uint64_t* const T_s = reinterpret_cast<uint64_t*>(M_s + R);  // [R][ncls] by temperature
    int32_t* const sot = reinterpret_cast<int32_t*>(T_s + (size_t)ncls * R);
    int32_t* const tos = sot + R;
    const int parity = (int)(e & 1);
    const int k0 = parity + 2 * (int)threadIdx.x;  // this thread's first pair
    __syncthreads();  // the previous problem's readers are done
    SwapPair sp0{};
    if (ex && k0 + 1 < R) sp0 = p.pairs[k0];
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      const int64_t U = p.cnt[r];
      const int64_t ones = p.cnt[W * 32 + r];
      sot[r] = p.slot_of_temp[r];
      tos[r] = p.temp_of_slot[r];
      if (ex) {
        if (ferro) {
          T_s[2 * r] = p.T_temp[(size_t)r * kClasses + 1];
          T_s[2 * r + 1] = p.T_temp[(size_t)r * kClasses + 3];
        } else {
#pragma unroll
          for (int c = 0; c < kClasses; ++c)
            T_s[(size_t)r * kClasses + c] = p.T_temp[(size_t)r * kClasses + c];
        }
      }
      p.cnt[r] = 0;
      p.cnt[W * 32 + r] = 0;
      const int64_t bonds = 2 * L2 - 2 * U;
      const int64_t M = 2 * ones - L2;
      const int64_t E = -p.J_int * bonds + p.h_int * M;
      E_s[r] = E;
      M_s[r] = M;
      p.E_slot[r] = E;
      p.M_slot[r] = M;
    }
    __syncthreads();
    if (ex) {
      const uint32_t c3 = kTagExch | ((uint32_t)(e >> 32) << 8);
      for (int k = k0; k + 1 < R; k += 2 * blockDim.x) {
        const int a = sot[k], b = sot[k + 1];
        const int64_t n = E_s[a] - E_s[b];
        const SwapPair sp = k == k0 ? sp0 : p.pairs[k];
        const uint64_t S = pair_threshold(sp, p.swap_table, p.table_shift, n);
        const Philox4 rnd = philox4x32_10((uint32_t)k, (uint32_t)e, 0u, c3, p.key0, p.key1);
        const bool accept = (uint64_t)rnd.x < S;
        count_swap(p.attempted, p.accepted, k, accept);
        if (accept) {  // pairs of one parity are disjoint
          sot[k] = b;
          sot[k + 1] = a;
          tos[a] = k + 1;
          tos[b] = k;
        }
      }
      __syncthreads();
      for (int r = threadIdx.x; r < R; r += blockDim.x) {
        p.slot_of_temp[r] = sot[r];
        p.temp_of_slot[r] = tos[r];
      }
      for (int r = threadIdx.x; r < W * 32; r += blockDim.x) {  // whole warps
        const int w = r >> 5, b = r & 31;
        const bool in_use = r < R;
        const int temp = in_use ? tos[r] : 0;
        if (ferro) {
          PlaneFerro* pl = reinterpret_cast<PlaneFerro*>(p.planes) + w;
          const uint64_t t0 = in_use ? T_s[2 * temp] : 0;
          const uint64_t t1 = in_use ? T_s[2 * temp + 1] : 0;
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
            const uint64_t tc = in_use ? T_s[(size_t)temp * kClasses + c] : 0;
            pl->T[c][b] = (uint32_t)min(tc, kTwo32 - 1);
            const uint32_t a = __ballot_sync(0xffffffffu, in_use && tc >= kTwo32);
            if (b == 0) pl->alw[c] = a;
          }
        }
      }
    }
    if (p.trace_E != nullptr) {
      // the trace row of this sweep, by temperature index after its swap iteration
      const uint64_t t = fp.t0 + (uint64_t)j;
      const int64_t row = (int64_t)((t - p.trace_t0) % (uint64_t)p.trace_cap);
      for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const int k = tos[r];
        const int64_t at = PT_DBG_IDX(p, row * R + k, p.trace_cap * R, kDbgTrace);
        p.trace_E[at] = E_s[r];
        p.trace_M[at] = M_s[r];
      }
    }
  }
}

size_t flat_exchange_smem(int R, int mode) {
  return (size_t)R * (2 * sizeof(int64_t) + 2 * sizeof(int32_t) +
                      (mode == kModeFerro ? 2 : kClasses) * sizeof(uint64_t));
}

// Threads of an exchange block: one per slot of the batch's widest problem (whole warps, at
// most kFlatThreads), so that the block barriers of small ladders span few warps.
int flat_exchange_threads(int W) { return std::min(kFlatThreads, 32 * std::max(1, W)); }

// The exchange launch of sweep j with `smem` bytes of shared memory (the largest problem's
// need, flat_exchange_smem) and `threads` threads per block (flat_exchange_threads).
cudaError_t launch_flat_exchange(const FlatProblem* d_probs, int np, int64_t j, size_t smem,
                                 int threads, int sms, cudaStream_t st) {
  k_flat_exchange<<<std::min(np, sms * 8), threads, smem, st>>>(d_probs, np, j);
  return cudaGetLastError();
}

// One mode's tiles on the device and the state of its queue in a batch.
struct ModeTiles {
  int grid = 0;  // CTAs of each launch (0: the mode has no tiles)
  const Tile* tiles = nullptr;
  int ntiles = 0;
  const int* first = nullptr;         // dealt: per-warp offsets; queued: nullptr
  unsigned long long* ctr = nullptr;  // queued: zeroed before the batch's first launch
  unsigned long long base = 0;
};

// Half sweep `colour` of sweep j over one mode's tiles.
template <int MODE, bool COUNT>
cudaError_t launch_flat_half(ModeTiles& mt, const FlatProblem* d_probs, int colour, int64_t j,
                             cudaStream_t st) {
  if (mt.grid == 0) return cudaSuccess;
  const TileQueue q{mt.ctr, mt.base, mt.ntiles};
  if (mt.first != nullptr) {
    k_flat_half<MODE, COUNT, false><<<mt.grid, kFlatThreads, 0, st>>>(d_probs, mt.tiles,
                                                                      mt.first, q, colour, j);
  } else {
    k_flat_half<MODE, COUNT, true><<<mt.grid, kFlatThreads, 0, st>>>(d_probs, mt.tiles, nullptr,
                                                                     q, colour, j);
    mt.base += (unsigned long long)mt.ntiles;
  }
  return cudaGetLastError();
}

// The launches of sweep j: half sweep 0, half sweep 1 (counting when `counted`: some
// problem's swap iteration or trace row follows), then the exchange step when counted.
cudaError_t launch_flat_sweep(ModeTiles mt[2], const FlatProblem* d_probs, int np, int64_t j,
                              bool counted, size_t xsmem, int xthreads, int sms,
                              cudaStream_t st) {
  cudaError_t err = launch_flat_half<kModeFerro, false>(mt[0], d_probs, 0, j, st);
  if (err == cudaSuccess) err = launch_flat_half<kModeGeneric, false>(mt[1], d_probs, 0, j, st);
  if (counted) {
    if (err == cudaSuccess) err = launch_flat_half<kModeFerro, true>(mt[0], d_probs, 1, j, st);
    if (err == cudaSuccess) err = launch_flat_half<kModeGeneric, true>(mt[1], d_probs, 1, j, st);
    if (err == cudaSuccess) err = launch_flat_exchange(d_probs, np, j, xsmem, xthreads, sms, st);
  } else {
    if (err == cudaSuccess) err = launch_flat_half<kModeFerro, false>(mt[0], d_probs, 1, j, st);
    if (err == cudaSuccess) err = launch_flat_half<kModeGeneric, false>(mt[1], d_probs, 1, j, st);
  }
  return err;
}

// Shared memory of the batch's exchange launches: when a problem needs more than the
// default 48 KB, the kernel's limit is raised to what the largest problem can need
// (R = 2048, generic: 208 KB). The limit belongs to the kernel, so it is never lowered under
// another batch's launch.
cudaError_t flat_exchange_prepare(size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k_flat_exchange, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)flat_exchange_smem(PT_MAX_R, kModeGeneric));
}

}  // namespace

// ---------------------------------------------------------------------------------------
// host: one batch = per sweep j, half sweep 0 and 1 over all tiles of both modes, then the
// exchange launch when any problem is due for an exchange after sweep j
// ---------------------------------------------------------------------------------------
// The queued schedule's tail (refine_tail): the cheapest share of a launch's work whose
// tiles are cut, and into how many parts. Measured on batched-256 with 1024-word tiles,
// per sweep with / without exchanges: none 158 / 143 us; (0.25, 4) 145.8 / 131.7;
// (0.25, 2) 142.0 / 131.3; (0.15, 4) 143.8 / 131.4; (0.4, 4) 149.1 / 135.2.
constexpr double kTailShare = 0.25;
constexpr int kTailPieces = 2;

// Work of a tile in Philox blocks (the dominant cost of a word).
int64_t tile_cost(const Tile& t, int R) {
  const int slots = std::min(32, R - 32 * t.w);
  return (int64_t)((slots + 3) / 4 + 1) * (t.q1 - t.q0);
}

void deal_tiles(const std::vector<Tile>& in, const std::vector<FlatProblem>& probs,
                int nwarps, std::vector<Tile>* out, std::vector<int>* first) {
  std::vector<int> order(in.size());
  for (size_t k = 0; k < in.size(); ++k) order[k] = (int)k;
  std::vector<int64_t> cost(in.size());
  for (size_t k = 0; k < in.size(); ++k) cost[k] = tile_cost(in[k], probs[in[k].prob].p.R);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  typedef std::pair<int64_t, int> Load;  // (work so far, warp)
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int w = 0; w < nwarps; ++w) heap.push(Load(0, w));
  std::vector<std::vector<int>> per(nwarps);
  for (int k : order) {
    Load l = heap.top();
    heap.pop();
    per[l.second].push_back(k);
    l.first += cost[k];
    heap.push(l);
  }
  out->clear();
  first->assign((size_t)nwarps + 1, 0);
  for (int w = 0; w < nwarps; ++w) {
    (*first)[w] = (int)out->size();
    for (int k : per[w]) out->push_back(in[k]);
  }
  (*first)[nwarps] = (int)out->size();
}

// Splits the tiles that make up the cheapest kTailShare of a mode's Philox work into
// kTailPieces equal parts (tiles of fewer than 64 words per part are kept whole). The
// queue hands out large tiles first, so a launch then ends on small tiles: the warps finish
// closer together, and the extra tile starts fall only on that last share. (The host's
// longest-processing-time dealing was measured slower with the split tiles: its cost model
// cannot see what the queue measures, how fast each warp really runs.) Each problem's tile
// count (FlatProblem::ntiles) follows.
void refine_tail(std::vector<Tile>* tiles, std::vector<FlatProblem>* probs) {
  const size_t nt = tiles->size();
  if (nt == 0) return;
  std::vector<int64_t> cost(nt);
  int64_t total = 0;
  for (size_t k = 0; k < nt; ++k) {
    cost[k] = tile_cost((*tiles)[k], (*probs)[(*tiles)[k].prob].p.R);
    total += cost[k];
  }
  std::vector<int> order(nt);
  for (size_t k = 0; k < nt; ++k) order[k] = (int)k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] < cost[b]; });
  const int64_t budget = (int64_t)(kTailShare * (double)total);
  int64_t acc = 0;
  tiles->reserve(nt + nt * (kTailPieces - 1));
  for (int k : order) {
    if (acc >= budget) break;
    acc += cost[k];
    const Tile whole = (*tiles)[(size_t)k];  // a copy: push_back below may move the vector
    const int words = whole.q1 - whole.q0;
    if (words < 64 * kTailPieces) continue;
    for (int piece = 0; piece < kTailPieces; ++piece) {
      Tile s = whole;
      s.q0 = whole.q0 + (int)((int64_t)words * piece / kTailPieces);
      s.q1 = whole.q0 + (int)((int64_t)words * (piece + 1) / kTailPieces);
      if (piece == 0)
        (*tiles)[(size_t)k] = s;  // the first part stays in place
      else
        tiles->push_back(s);
    }
    (*probs)[(size_t)whole.prob].ntiles += kTailPieces - 1;
  }
}

// Every tile inside its problem's plane and word range; checked on the host before any
// list is uploaded (a bad list must never reach a kernel).
bool tiles_valid(const std::vector<Tile>& tiles, const std::vector<FlatProblem>& probs) {
  for (const Tile& t : tiles) {
    if (t.prob < 0 || (size_t)t.prob >= probs.size()) return false;
    const DevProblem& p = probs[(size_t)t.prob].p;
    const int words = p.L * (p.L / 2);
    if (t.w < 0 || t.w >= p.W || t.q0 < 0 || t.q0 >= t.q1 || t.q1 > words) return false;
  }
  return true;
}

// A mode's tiles sorted by tile_cost, largest first (ties keep their order).
void sort_tiles(std::vector<Tile>* tiles, const std::vector<FlatProblem>& probs) {
  std::stable_sort(tiles->begin(), tiles->end(), [&](const Tile& a, const Tile& b) {
    return tile_cost(a, probs[a.prob].p.R) > tile_cost(b, probs[b.prob].p.R);
  });
}

// The descriptor of problem p in a batch that runs it n sweeps with exchange interval m.
FlatProblem flat_problem(pt_problem* p, int64_t n, int m, int tile_words) {
  FlatProblem fp{};
  fp.p = p->dev;
  fp.t0 = p->t;
  fp.e0 = p->e;
  fp.n = n;
  fp.m = m;
  fp.wait_ns = p->wait_limit_ns;
  fp.stall = p->stall;
  const int words = p->L * (p->L / 2);
  fp.ntiles = std::max(1, (words + tile_words / 2) / tile_words) * p->W;
  return fp;
}

int64_t build_flat_lists(pt_problem* const* ps, int count, const int64_t* n, const int* every,
                         int tile_words, bool refine, std::vector<FlatProblem>* probs,
                         std::vector<Tile> tiles[2]) {
  int64_t n_max = 0;
  for (int j = 0; j < count; ++j) {
    if (n[j] <= 0) continue;
    pt_problem* p = ps[j];
    const FlatProblem fp = flat_problem(p, n[j], every[j], tile_words);
    const int pi = (int)probs->size();
    const int words = p->L * (p->L / 2);
    const int ntile = std::max(1, (words + tile_words / 2) / tile_words);
    probs->push_back(fp);
    n_max = std::max(n_max, n[j]);
    for (int w = 0; w < p->W; ++w)
      for (int k = 0; k < ntile; ++k) {
        Tile t;
        t.prob = pi;
        t.w = w;
        t.q0 = (int)((int64_t)words * k / ntile);
        t.q1 = (int)((int64_t)words * (k + 1) / ntile);
        tiles[p->mode == kModeFerro ? 0 : 1].push_back(t);
      }
  }
  for (int md = 0; md < 2; ++md) {
    if (refine) refine_tail(&tiles[md], probs);
    if (!tiles_valid(tiles[md], *probs)) return -1;
  }
  return n_max;
}

// One lock-step batch on one stream, in three steps: prepare (work lists built, uploaded to
// stream-ordered scratch), the launches of one sweep at a time, and finish (scratch freed).
struct FlatRun {
  cudaStream_t st = 0;
  std::vector<FlatProblem> probs;
  std::vector<Tile> tiles[2];  // by mode
  std::vector<int> first[2];   // dealt: per-warp offsets
  std::vector<char> counted;   // per sweep: a swap iteration or trace row follows for some problem
  ModeTiles mt[2];
  const FlatProblem* d_probs = nullptr;
  void* scratch = nullptr;
  int np = 0;
  int64_t n_max = 0;
  size_t xsmem = 0;
  int xthreads = 32;
  int sms = 0;
  // persistent: the lists live in memory the caller owns after prepare (a replayed graph's),
  // allocated with cudaMalloc and filled with blocking copies; finish() leaves them alone
  bool persistent = false;
  unsigned long long* d_ctr = nullptr;

  int prepare(pt_problem* const* ps, int count, const int64_t* n, const int* every,
              cudaStream_t stream, const DeviceInfo& di, int tile_words, bool queued);
  cudaError_t launch_sweep(int64_t j) {
    if (j >= n_max) return cudaSuccess;
    return launch_flat_sweep(mt, d_probs, np, j, counted[(size_t)j] != 0, xsmem, xthreads, sms,
                             st);
  }
  cudaError_t finish() {
    if (!scratch || persistent) return cudaSuccess;
    const cudaError_t err = cudaFreeAsync(scratch, st);
    scratch = nullptr;
    return err;
  }
};

int FlatRun::prepare(pt_problem* const* ps, int count, const int64_t* n, const int* every,
                     cudaStream_t stream, const DeviceInfo& di, int tile_words, bool queued) {
  st = stream;
  sms = di.sms;
  n_max = build_flat_lists(ps, count, n, every, tile_words, queued, &probs, tiles);
  if (n_max < 0) return fail(PT_EINTERNAL, "batch work tiles outside their planes");
  if (probs.empty()) {
    n_max = 0;
    return PT_OK;
  }
  // one wave per launch: as many CTAs as are resident at once, their warps taking the
  // tiles from the mode's queue
  int per_sm[2] = {1, 1};
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm[0], k_flat_half<kModeFerro, true, false>, kFlatThreads, 0);
  if (err == cudaSuccess)
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm[1], k_flat_half<kModeGeneric, true, false>, kFlatThreads, 0);
  if (err != cudaSuccess) return fail(PT_ECUDA, "occupancy: %s", cudaGetErrorString(err));
  const int wpb = kFlatThreads / 32;
  for (int md = 0; md < 2; ++md) {
    if (tiles[md].empty()) continue;
    const int blocks = std::max(1, per_sm[md]) * di.sms;
    const int needed = (int)((tiles[md].size() + wpb - 1) / wpb);
    mt[md].grid = std::max(1, std::min(blocks, needed));
    mt[md].ntiles = (int)tiles[md].size();
    if (queued) {
      sort_tiles(&tiles[md], probs);
    } else {
      std::vector<Tile> dealt;
      deal_tiles(tiles[md], probs, mt[md].grid * wpb, &dealt, &first[md]);
      tiles[md].swap(dealt);
    }
  }
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t pb = probs.size() * sizeof(FlatProblem);
  const size_t tb[2] = {tiles[0].size() * sizeof(Tile), tiles[1].size() * sizeof(Tile)};
  const size_t fb[2] = {first[0].size() * sizeof(int), first[1].size() * sizeof(int)};
  const size_t qb = 2 * sizeof(unsigned long long);  // the two modes' queue counters
  const size_t total = al(pb) + al(tb[0]) + al(tb[1]) + al(fb[0]) + al(fb[1]) + al(qb) + 256;
  err = persistent ? cudaMalloc(&scratch, total) : cudaMallocAsync(&scratch, total, st);
  if (err != cudaSuccess) {
    scratch = nullptr;
    return fail(PT_ENOMEM, "batch scratch: %s", cudaGetErrorString(err));
  }
  char* cur = (char*)scratch;
  d_probs = (const FlatProblem*)cur;
  cur += al(pb);
  for (int md = 0; md < 2; ++md) {
    mt[md].tiles = (const Tile*)cur;
    cur += al(tb[md]);
  }
  for (int md = 0; md < 2; ++md) {
    if (fb[md]) mt[md].first = (const int*)cur;
    cur += al(fb[md]);
  }
  d_ctr = (unsigned long long*)cur;
  mt[0].ctr = d_ctr;
  mt[1].ctr = d_ctr + 1;
  // (persistent: the memory is new and used by no queued work, so blocking copies are safe)
  const auto copy = [&](void* dst, const void* src, size_t bytes) {
    return persistent ? cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice)
                      : cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  err = copy((void*)d_probs, probs.data(), pb);
  for (int md = 0; md < 2 && err == cudaSuccess; ++md) {
    if (!tb[md]) continue;
    err = copy((void*)mt[md].tiles, tiles[md].data(), tb[md]);
    if (err == cudaSuccess && fb[md]) err = copy((void*)mt[md].first, first[md].data(), fb[md]);
  }
  if (err == cudaSuccess)
    err = persistent ? cudaMemset(d_ctr, 0, qb) : cudaMemsetAsync(d_ctr, 0, qb, st);
  // which sweeps are counted for at least one problem (a swap iteration or a trace row)
  counted.assign((size_t)n_max, 0);
  for (const FlatProblem& fp : probs)
    for (int64_t j = 0; j < fp.n; ++j)
      if (fp.p.trace_E != nullptr ||
          (fp.m > 0 && (fp.t0 + (uint64_t)j + 1) % (uint64_t)fp.m == 0))
        counted[(size_t)j] = 1;
  np = (int)probs.size();
  for (const FlatProblem& fp : probs) {
    xsmem = std::max(xsmem, flat_exchange_smem(fp.p.R, fp.p.mode));
    xthreads = std::max(xthreads, flat_exchange_threads(fp.p.W));
  }
  if (err == cudaSuccess) err = flat_exchange_prepare(xsmem);
  if (err != cudaSuccess) return fail(PT_ECUDA, "flat batch set-up: %s", cudaGetErrorString(err));
  return PT_OK;
}

// Side streams per device for the multi-stream lock-step batch (fork / join through
// events); the mutex keeps two host threads from using one set of streams and events at once.
constexpr int kMaxBatchStreams = PT_BATCH_STREAMS_MAX;
struct SideStreams {
  bool ok = false;
  cudaStream_t stream[kMaxBatchStreams - 1] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kMaxBatchStreams - 1] = {};
  std::mutex mu;
};

SideStreams& side_streams(int device) {
  static std::mutex mu;
  static SideStreams streams[64];
  std::lock_guard<std::mutex> lk(mu);
  SideStreams& s = streams[device & 63];
  if (!s.ok) {
    bool ok = cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < kMaxBatchStreams - 1; ++k)
      ok = cudaStreamCreateWithFlags(&s.stream[k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&s.join[k], cudaEventDisableTiming) == cudaSuccess;
    s.ok = ok;
  }
  return s;
}

// ---------------------------------------------------------------------------------------
// Replay of repeated batches from captured CUDA graphs (pt_set_batch_graphs). The launches
// of a lock-step batch call depend only on the batch's shape: per problem, in call order,
// L, R, the mode, the sweeps n and interval m, the phase of its exchange schedule (t mod m)
// and whether a trace is on, plus the tile size, the schedule, the parts and the stream.
// Everything else a kernel reads -- the sweep and swap counters, the problem's device arrays
// -- comes from the problem descriptors, which every call copies to the device before its
// launches. So a call whose shape was seen before copies its descriptors, clears its queue
// counters and launches the graph captured the first time: one graph launch instead of about
// three launches per part and sweep. The first call of a shape builds the work lists in
// memory of their own, captures the launches (forks and joins of the parts included) and
// instantiates the graph. A few shapes are kept per device, the least recently used dropped.
// ---------------------------------------------------------------------------------------
struct GraphEntry {
  std::vector<int64_t> key;
  cudaGraphExec_t exec = nullptr;
  FlatRun run[kMaxBatchStreams];  // each part's lists, in the entry's own device memory
  int parts = 0;
  uint64_t used = 0;
  // the descriptors of a call go up from page-locked host memory, two buffers used in turn;
  // copied[b] marks when the copy that read buffer b is done (before b is written again).
  // `launched` follows the entry's last graph launch: the next call's copies wait for it, so
  // a call on another stream cannot overwrite descriptors a running replay still reads.
  FlatProblem* host[2] = {nullptr, nullptr};
  size_t host_count = 0;
  cudaEvent_t copied[2] = {nullptr, nullptr};
  cudaEvent_t launched = nullptr;
  bool pending[2] = {false, false};
  bool ever_launched = false;
  int next = 0;
};
constexpr size_t kGraphCacheEntries = 4;
std::mutex g_graph_mu;
std::vector<GraphEntry*> g_graph_cache[64];  // per device
uint64_t g_graph_clock = 0;

void free_graph_entry(GraphEntry* e) {
  if (e->exec) cudaGraphExecDestroy(e->exec);
  for (int g = 0; g < e->parts; ++g)
    if (e->run[g].scratch) cudaFree(e->run[g].scratch);  // waits for work that reads it
  for (int b = 0; b < 2; ++b) {
    if (e->host[b]) cudaFreeHost(e->host[b]);
    if (e->copied[b]) cudaEventDestroy(e->copied[b]);
  }
  if (e->launched) cudaEventDestroy(e->launched);
  delete e;
}

std::vector<int64_t> graph_key(std::vector<pt_problem*> gp[], std::vector<int64_t> gn[],
                               std::vector<int> ge[], int parts, cudaStream_t st,
                               int tile_words, bool queued) {
  std::vector<int64_t> key = {(int64_t)(intptr_t)st, queued ? 1 : 0, tile_words, parts};
  for (int g = 0; g < parts; ++g) {
    key.push_back(-1 - g);
    for (size_t i = 0; i < gp[g].size(); ++i) {
      const pt_problem* p = gp[g][i];
      const int m = ge[g][i];
      key.insert(key.end(), {(int64_t)p->L, (int64_t)p->R, (int64_t)p->mode, gn[g][i],
                             (int64_t)m, m > 0 ? (int64_t)(p->t % (uint64_t)m) : 0,
                             p->dev.trace_E != nullptr ? 1 : 0});
    }
  }
  return key;
}

// The batch through a cached or newly captured graph. Returns 1 (nothing done) when the
// problems' stream cannot be captured (the legacy default stream) or is being captured by
// the caller: the caller then launches as usual.
int sweep_batch_graph(std::vector<pt_problem*> gp[], std::vector<int64_t> gn[],
                      std::vector<int> ge[], int parts, cudaStream_t st, const DeviceInfo& di,
                      int tile_words, bool queued, SideStreams* ss) {
  // the legacy default stream cannot be captured: launch as without replay
  if (st == nullptr || st == cudaStreamLegacy) return 1;
  std::lock_guard<std::mutex> glk(g_graph_mu);
  std::vector<GraphEntry*>& cache = g_graph_cache[di.device & 63];
  const std::vector<int64_t> key = graph_key(gp, gn, ge, parts, st, tile_words, queued);
  GraphEntry* e = nullptr;
  for (GraphEntry* c : cache)
    if (c->key == key) e = c;
  cudaError_t err = cudaSuccess;
  if (!e) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    err = cudaStreamIsCapturing(st, &cs);
    if (err != cudaSuccess) return fail(PT_ECUDA, "batch graph: %s", cudaGetErrorString(err));
    if (cs != cudaStreamCaptureStatusNone) return 1;
    e = new GraphEntry;
    e->key = key;
    e->parts = parts;
    int64_t n_max = 0;
    int rc = PT_OK;
    for (int g = 0; g < parts && !rc; ++g) {
      e->run[g].persistent = true;
      rc = e->run[g].prepare(gp[g].data(), (int)gp[g].size(), gn[g].data(), ge[g].data(),
                             g == 0 ? st : ss->stream[g - 1], di, tile_words, queued);
      n_max = std::max(n_max, e->run[g].n_max);
    }
    if (rc) {
      free_graph_entry(e);
      return rc;
    }
    for (int g = 0; g < parts; ++g) e->host_count += e->run[g].probs.size();
    for (int b = 0; b < 2 && err == cudaSuccess; ++b) {
      err = cudaMallocHost(&e->host[b], std::max<size_t>(1, e->host_count) * sizeof(FlatProblem));
      if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->copied[b], cudaEventDisableTiming);
    }
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->launched, cudaEventDisableTiming);
    if (err != cudaSuccess) {
      free_graph_entry(e);
      return fail(PT_ECUDA, "batch graph buffers: %s", cudaGetErrorString(err));
    }
    // relaxed: a kernel's first launch in the process may load its code during the capture
    err = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
    if (err == cudaSuccess) {
      cudaError_t cap = cudaSuccess;
      if (parts > 1) {
        cap = cudaEventRecord(ss->fork, st);
        for (int k = 0; k + 1 < parts && cap == cudaSuccess; ++k)
          cap = cudaStreamWaitEvent(ss->stream[k], ss->fork, 0);
      }
      for (int64_t j = 0; j < n_max && cap == cudaSuccess; ++j)
        for (int g = 0; g < parts && cap == cudaSuccess; ++g) cap = e->run[g].launch_sweep(j);
      for (int k = 0; k + 1 < parts && cap == cudaSuccess; ++k) {
        cap = cudaEventRecord(ss->join[k], ss->stream[k]);
        if (cap == cudaSuccess) cap = cudaStreamWaitEvent(st, ss->join[k], 0);
      }
      cudaGraph_t graph = nullptr;
      err = cudaStreamEndCapture(st, &graph);  // always ends the capture, also after an error
      if (err == cudaSuccess) err = cap;
      if (err == cudaSuccess) err = cudaGraphInstantiate(&e->exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
    }
    if (err != cudaSuccess) {
      free_graph_entry(e);
      return fail(PT_ECUDA, "batch graph capture: %s", cudaGetErrorString(err));
    }
    if (cache.size() >= kGraphCacheEntries) {
      auto lru = std::min_element(cache.begin(), cache.end(), [](GraphEntry* a, GraphEntry* b) {
        return a->used < b->used;
      });
      free_graph_entry(*lru);
      cache.erase(lru);
    }
    cache.push_back(e);
  }
  e->used = ++g_graph_clock;
  // this call's descriptors (counters, device arrays) into the next host buffer, up to the
  // device after the entry's last replay, queue counters cleared, then the graph
  const int b = e->next;
  e->next ^= 1;
  if (e->pending[b]) err = cudaEventSynchronize(e->copied[b]);  // its last copy is done
  size_t at = 0;
  for (int g = 0; g < parts; ++g)
    for (size_t i = 0; i < gp[g].size(); ++i)
      if (gn[g][i] > 0)
        e->host[b][at++] = flat_problem(gp[g][i], gn[g][i], ge[g][i], tile_words);
  if (err == cudaSuccess && e->ever_launched) err = cudaStreamWaitEvent(st, e->launched, 0);
  at = 0;
  for (int g = 0; g < parts && err == cudaSuccess; ++g) {
    const size_t k = e->run[g].probs.size();
    if (k == 0) continue;
    err = cudaMemcpyAsync((void*)e->run[g].d_probs, e->host[b] + at, k * sizeof(FlatProblem),
                          cudaMemcpyHostToDevice, st);
    at += k;
    if (err == cudaSuccess && queued)
      err = cudaMemsetAsync(e->run[g].d_ctr, 0, 2 * sizeof(unsigned long long), st);
  }
  if (err == cudaSuccess) err = cudaEventRecord(e->copied[b], st);
  if (err == cudaSuccess) e->pending[b] = true;
  if (err == cudaSuccess) err = cudaGraphLaunch(e->exec, st);
  if (err == cudaSuccess) err = cudaEventRecord(e->launched, st);
  if (err == cudaSuccess) e->ever_launched = true;
  if (err != cudaSuccess) return fail(PT_ECUDA, "batch graph launch: %s", cudaGetErrorString(err));
  return PT_OK;
}

// The lock-step batch as `parts` parts of about equal work (L^2 W n each, heaviest first onto
// the lightest part), each on its own stream: sweep j of one part runs beside sweep j of the
// others, so one part's exchange launch, launch gaps and last tiles overlap the others' half
// sweeps. Part 0 runs on the problems' stream, the others on side streams that start after
// everything queued on it so far and that it waits for at the end.
int sweep_batch_flat_parts(pt_problem* const* ps, int count, const int64_t* n, const int* every,
                           cudaStream_t st, const DeviceInfo& di, int tile_words, bool queued,
                           int parts, bool graphs) {
  std::vector<int> order;
  for (int j = 0; j < count; ++j)
    if (n[j] > 0) order.push_back(j);
  auto work = [&](int j) { return (double)ps[j]->L * ps[j]->L * ps[j]->W * (double)n[j]; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
  parts = std::max(1, std::min(parts, std::min(kMaxBatchStreams, (int)order.size())));
  std::vector<pt_problem*> gp[kMaxBatchStreams];
  std::vector<int64_t> gn[kMaxBatchStreams];
  std::vector<int> ge[kMaxBatchStreams];
  double load[kMaxBatchStreams] = {};
  for (int j : order) {
    int g = 0;
    for (int k = 1; k < parts; ++k)
      if (load[k] < load[g]) g = k;
    gp[g].push_back(ps[j]);
    gn[g].push_back(n[j]);
    ge[g].push_back(every[j]);
    load[g] += work(j);
  }
  SideStreams* ss = parts > 1 ? &side_streams(di.device) : nullptr;
  std::unique_lock<std::mutex> lk;
  if (ss) {
    lk = std::unique_lock<std::mutex>(ss->mu);
    if (!ss->ok) return fail(PT_ECUDA, "batch side streams could not be created");
  }
  if (graphs && !order.empty()) {
    const int grc = sweep_batch_graph(gp, gn, ge, parts, st, di, tile_words, queued, ss);
    if (grc <= 0) {
      if (grc == PT_ECUDA)
        for (int j = 0; j < count; ++j) ps[j]->poisoned = PT_ECUDA;
      return grc;
    }
  }
  cudaError_t err = cudaSuccess;
  if (parts > 1) {
    err = cudaEventRecord(ss->fork, st);
    for (int k = 0; k + 1 < parts && err == cudaSuccess; ++k)
      err = cudaStreamWaitEvent(ss->stream[k], ss->fork, 0);
    if (err != cudaSuccess) return fail(PT_ECUDA, "batch fork: %s", cudaGetErrorString(err));
  }
  FlatRun run[kMaxBatchStreams];
  int rc = PT_OK;
  int64_t n_max = 0;
  for (int g = 0; g < parts && !rc; ++g) {
    rc = run[g].prepare(gp[g].data(), (int)gp[g].size(), gn[g].data(), ge[g].data(),
                        g == 0 ? st : ss->stream[g - 1], di, tile_words, queued);
    n_max = std::max(n_max, run[g].n_max);
  }
  err = rc ? cudaErrorUnknown : cudaSuccess;
  for (int64_t j = 0; j < n_max && err == cudaSuccess; ++j)
    for (int g = 0; g < parts && err == cudaSuccess; ++g) err = run[g].launch_sweep(j);
  cudaError_t err2 = cudaSuccess;
  for (int g = 0; g < parts; ++g) {
    const cudaError_t e = run[g].finish();
    if (err2 == cudaSuccess) err2 = e;
  }
  // the problems' stream waits for the side streams' work
  for (int k = 0; k + 1 < parts; ++k) {
    if (err2 == cudaSuccess) err2 = cudaEventRecord(ss->join[k], ss->stream[k]);
    if (err2 == cudaSuccess) err2 = cudaStreamWaitEvent(st, ss->join[k], 0);
  }
  if (rc == PT_ECUDA || (!rc && (err != cudaSuccess || err2 != cudaSuccess)))
    for (int j = 0; j < count; ++j) ps[j]->poisoned = PT_ECUDA;
  if (rc) return rc;
  if (err == cudaSuccess) err = err2;
  if (err != cudaSuccess) return fail(PT_ECUDA, "flat batch launch: %s", cudaGetErrorString(err));
  return PT_OK;
}

int sweep_batch_flat(pt_problem* const* ps, int count, const int64_t* n, const int* every,
                     cudaStream_t st, const DeviceInfo& di, int tile_words, bool queued,
                     int streams, bool graphs) {
  return sweep_batch_flat_parts(ps, count, n, every, st, di, tile_words, queued, streams,
                                graphs);
}

// =======================================================================================
// Allocation-free variant of the lock-step batch.
//
// Some callers must not allocate device memory while they run: code that works inside a
// memory budget it has already fixed, that runs under a custom allocator which this
// library cannot see, or that must not let an allocation synchronise the device or fail
// part-way. For them pt_sweep_batch_static does the work of pt_sweep_batch (lock-step
// strategy) with its per-call work lists -- the problem descriptors, the warp tiles and
// the per-warp tile offsets -- in one fixed array of device memory that the library
// defines at file scope, instead of memory it allocates per call. The host side builds
// the lists in fixed host arrays as well, so no call allocates on the heap either.
// =======================================================================================
namespace {

constexpr size_t kStaticScratchBytes = size_t(1) << 20;  // 1 MiB on every device
constexpr int kStaticMaxProblems = kStaticMaxBatch;
constexpr int kStaticMaxTiles = 65536;
constexpr int kStaticMaxWarps = 16384;

// The device array. Every GPU that loads the library holds it until the process exits.
// Host code must not use its name as an address: it gets the device address through
// cudaGetSymbolAddress once per device.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct StaticDevice {
  bool ready = false;
  void* ptr = nullptr;
};

std::mutex g_static_mu;  // the host arrays below are shared by all calls
StaticDevice g_static_dev[64];
FlatProblem g_sp_probs[kStaticMaxProblems];
Tile g_sp_tiles[kStaticMaxTiles];
Tile g_sp_dealt[kStaticMaxTiles];
int64_t g_sp_cost[kStaticMaxTiles];
int g_sp_order[kStaticMaxTiles];
int g_sp_owner[kStaticMaxTiles];
int g_sp_first[2][kStaticMaxWarps + 1];
int64_t g_sp_heap_load[kStaticMaxWarps];
int g_sp_heap_warp[kStaticMaxWarps];

// Tiles [lo, hi) of g_sp_tiles sorted by tile_cost, largest first (ties keep their order),
// written to g_sp_dealt[lo..hi).
// (std::sort with the index as tie-break: the order std::stable_sort would give, without the
// temporary buffer it may take from the heap.)
void static_sort(int lo, int hi) {
  const int nt = hi - lo;
  for (int k = 0; k < nt; ++k) {
    g_sp_order[k] = lo + k;
    g_sp_cost[lo + k] = tile_cost(g_sp_tiles[lo + k], g_sp_probs[g_sp_tiles[lo + k].prob].p.R);
  }
  std::sort(g_sp_order, g_sp_order + nt, [](int a, int b) {
    return g_sp_cost[a] > g_sp_cost[b] || (g_sp_cost[a] == g_sp_cost[b] && a < b);
  });
  for (int k = 0; k < nt; ++k) g_sp_dealt[lo + k] = g_sp_tiles[g_sp_order[k]];
}

// refine_tail on tiles [lo, hi) of g_sp_tiles, in the fixed arrays: the first part of a
// split tile stays in place, the others go after hi. Returns the new end, or -1 when the
// array would overflow.
int static_refine(int lo, int hi) {
  const int nt = hi - lo;
  int64_t total = 0;
  for (int k = 0; k < nt; ++k) {
    g_sp_order[k] = lo + k;
    g_sp_cost[lo + k] = tile_cost(g_sp_tiles[lo + k], g_sp_probs[g_sp_tiles[lo + k].prob].p.R);
    total += g_sp_cost[lo + k];
  }
  std::sort(g_sp_order, g_sp_order + nt, [](int a, int b) {
    return g_sp_cost[a] < g_sp_cost[b] || (g_sp_cost[a] == g_sp_cost[b] && a < b);
  });
  const int64_t budget = (int64_t)(kTailShare * (double)total);
  int64_t acc = 0;
  int end = hi;
  for (int i = 0; i < nt && acc < budget; ++i) {
    const int k = g_sp_order[i];
    acc += g_sp_cost[k];
    const Tile whole = g_sp_tiles[k];
    const int words = whole.q1 - whole.q0;
    if (words < 64 * kTailPieces) continue;
    if (end + kTailPieces - 1 > kStaticMaxTiles) return -1;
    for (int piece = 0; piece < kTailPieces; ++piece) {
      Tile s = whole;
      s.q0 = whole.q0 + (int)((int64_t)words * piece / kTailPieces);
      s.q1 = whole.q0 + (int)((int64_t)words * (piece + 1) / kTailPieces);
      if (piece == 0)
        g_sp_tiles[k] = s;
      else
        g_sp_tiles[end++] = s;
    }
    g_sp_probs[whole.prob].ntiles += kTailPieces - 1;
  }
  return end;
}

// Longest-processing-time-first dealing of tiles [lo, hi) of g_sp_tiles to `nwarps` warps,
// written to g_sp_dealt[lo..hi) warp by warp with offsets first[0..nwarps] (relative to lo).
void static_deal(int lo, int hi, int nwarps, int* first) {
  const int nt = hi - lo;
  for (int k = 0; k < nt; ++k) {
    g_sp_order[k] = lo + k;
    g_sp_cost[lo + k] = tile_cost(g_sp_tiles[lo + k], g_sp_probs[g_sp_tiles[lo + k].prob].p.R);
  }
  std::sort(g_sp_order, g_sp_order + nt, [](int a, int b) {
    return g_sp_cost[a] > g_sp_cost[b] || (g_sp_cost[a] == g_sp_cost[b] && a < b);
  });
  // binary min-heap of (load, warp) in two fixed arrays
  for (int w = 0; w < nwarps; ++w) {
    g_sp_heap_load[w] = 0;
    g_sp_heap_warp[w] = w;
  }
  auto less = [](int a, int b) {
    return g_sp_heap_load[a] < g_sp_heap_load[b] ||
           (g_sp_heap_load[a] == g_sp_heap_load[b] && g_sp_heap_warp[a] < g_sp_heap_warp[b]);
  };
  auto swap_at = [](int a, int b) {
    std::swap(g_sp_heap_load[a], g_sp_heap_load[b]);
    std::swap(g_sp_heap_warp[a], g_sp_heap_warp[b]);
  };
  for (int k = 0; k < nt; ++k) {
    const int t = g_sp_order[k];
    g_sp_owner[t] = g_sp_heap_warp[0];
    g_sp_heap_load[0] += g_sp_cost[t];
    int i = 0;  // sift down
    for (;;) {
      const int l = 2 * i + 1, r = l + 1;
      int m = i;
      if (l < nwarps && less(l, m)) m = l;
      if (r < nwarps && less(r, m)) m = r;
      if (m == i) break;
      swap_at(i, m);
      i = m;
    }
  }
  // counting sort of the tiles by owner
  for (int w = 0; w <= nwarps; ++w) first[w] = 0;
  for (int k = 0; k < nt; ++k) first[g_sp_owner[lo + k] + 1] += 1;
  for (int w = 0; w < nwarps; ++w) first[w + 1] += first[w];
  for (int k = 0; k < nt; ++k) {
    const int t = g_sp_order[k];
    g_sp_dealt[lo + first[g_sp_owner[t]]++] = g_sp_tiles[t];
  }
  for (int w = nwarps; w > 0; --w) first[w] = first[w - 1];
  first[0] = 0;
}

}  // namespace

int sweep_batch_static(pt_problem* const* ps, int count, const int64_t* n, const int* every,
                       cudaStream_t st, const DeviceInfo& di, int tile_words, bool queued) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (di.device < 0 || di.device >= 64) return fail(PT_ENODEV, "device index %d", di.device);
  // set-up, once per device, with that device current: the device address of the array
  StaticDevice& sd = g_static_dev[di.device];
  if (!sd.ready) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess)
      return fail(PT_ECUDA, "cudaGetSymbolAddress of the static scratch: %s",
                  cudaGetErrorString(e));
    sd.ptr = ptr;
    sd.ready = true;
  }
  // problems and tiles, ferro-mode tiles first, then generic-mode ones
  int np = 0, nt = 0, split = 0;  // split = number of ferro-mode tiles (they come first)
  int64_t n_max = 0;
  for (int mode_pass = 0; mode_pass < 2; ++mode_pass) {
    for (int j = 0; j < count; ++j) {
      if (n[j] <= 0) continue;
      pt_problem* p = ps[j];
      const int md = p->mode == kModeFerro ? 0 : 1;
      if (md != mode_pass) continue;
      if (np >= kStaticMaxProblems)
        return fail(PT_EINVAL, "pt_sweep_batch_static: more than %d problems", kStaticMaxProblems);
      FlatProblem& fp = g_sp_probs[np];
      fp = FlatProblem{};
      fp.p = p->dev;
      fp.t0 = p->t;
      fp.e0 = p->e;
      fp.n = n[j];
      fp.m = every[j];
      n_max = std::max(n_max, n[j]);
      const int words = p->L * (p->L / 2);
      const int ntile = std::max(1, (words + tile_words / 2) / tile_words);
      fp.ntiles = ntile * p->W;
      if ((int64_t)nt + (int64_t)ntile * p->W > kStaticMaxTiles)
        return fail(PT_EINVAL, "pt_sweep_batch_static: more than %d work tiles (the batch is "
                    "too large for the %zu-byte static work area)", kStaticMaxTiles,
                    kStaticScratchBytes);
      for (int w = 0; w < p->W; ++w)
        for (int k = 0; k < ntile; ++k) {
          Tile& t = g_sp_tiles[nt++];
          t.prob = np;
          t.w = w;
          t.q0 = (int)((int64_t)words * k / ntile);
          t.q1 = (int)((int64_t)words * (k + 1) / ntile);
        }
      ++np;
    }
    if (queued) {  // the queued schedule ends each launch on split tiles (refine_tail)
      const int end = static_refine(mode_pass == 0 ? 0 : split, nt);
      if (end < 0)
        return fail(PT_EINVAL, "pt_sweep_batch_static: more than %d work tiles (the batch is "
                    "too large for the %zu-byte static work area)", kStaticMaxTiles,
                    kStaticScratchBytes);
      nt = end;
    }
    if (mode_pass == 0) split = nt;
  }
  for (int k = 0; k < nt; ++k) {  // every tile inside its plane before anything is uploaded
    const Tile& t = g_sp_tiles[k];
    if (t.prob < 0 || t.prob >= np)
      return fail(PT_EINTERNAL, "pt_sweep_batch_static: work tile of no problem");
    const DevProblem& dp = g_sp_probs[t.prob].p;
    if (t.w < 0 || t.w >= dp.W || t.q0 < 0 || t.q0 >= t.q1 || t.q1 > dp.L * (dp.L / 2))
      return fail(PT_EINTERNAL, "pt_sweep_batch_static: work tile outside its plane");
  }
  if (np == 0) return PT_OK;
  int per_sm[2] = {1, 1};
  cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm[0], k_flat_half<kModeFerro, true, false>, kFlatThreads, 0);
  if (err == cudaSuccess)
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm[1], k_flat_half<kModeGeneric, true, false>, kFlatThreads, 0);
  if (err != cudaSuccess) return fail(PT_ECUDA, "occupancy: %s", cudaGetErrorString(err));
  const int wpb = kFlatThreads / 32;
  const int lo[2] = {0, split}, hi[2] = {split, nt};
  int grid[2] = {0, 0}, nwarps[2] = {0, 0};
  for (int md = 0; md < 2; ++md) {
    const int cnt = hi[md] - lo[md];
    if (cnt == 0) continue;
    const int blocks = std::max(1, per_sm[md]) * di.sms;
    grid[md] = std::max(1, std::min(blocks, (cnt + wpb - 1) / wpb));
    nwarps[md] = grid[md] * wpb;
  }
  if (nwarps[0] > kStaticMaxWarps || nwarps[1] > kStaticMaxWarps)
    return fail(PT_EINTERNAL, "pt_sweep_batch_static: warp table too small");
  // layout inside the static array: problems | tiles (mode 0, then mode 1) | per-warp
  // offsets (mode 0) | per-warp offsets (mode 1) | queue counters
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t off_tiles = al((size_t)np * sizeof(FlatProblem));
  const size_t off_first0 = off_tiles + al((size_t)nt * sizeof(Tile));
  const size_t off_first1 = off_first0 + al((size_t)(nwarps[0] + 1) * sizeof(int));
  const size_t off_ctr = off_first1 + al((size_t)(nwarps[1] + 1) * sizeof(int));
  const size_t need = off_ctr + al(2 * sizeof(unsigned long long));
  if (need > kStaticScratchBytes)
    return fail(PT_EINVAL, "pt_sweep_batch_static: the batch needs %zu bytes of work lists, "
                "more than the %zu-byte static work area", need, kStaticScratchBytes);
  char* base = (char*)sd.ptr;
  const size_t off_first[2] = {off_first0, off_first1};
  ModeTiles mt[2];
  for (int md = 0; md < 2; ++md) {
    if (grid[md] == 0) continue;
    mt[md].grid = grid[md];
    mt[md].ntiles = hi[md] - lo[md];
    mt[md].tiles = (const Tile*)(base + off_tiles) + lo[md];
    mt[md].ctr = (unsigned long long*)(base + off_ctr) + md;
    if (queued) {
      static_sort(lo[md], hi[md]);
    } else {
      static_deal(lo[md], hi[md], nwarps[md], g_sp_first[md]);
      mt[md].first = (const int*)(base + off_first[md]);
    }
  }
  err = cudaMemcpyAsync(base, g_sp_probs, (size_t)np * sizeof(FlatProblem),
                        cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(base + off_tiles, g_sp_dealt, (size_t)nt * sizeof(Tile),
                          cudaMemcpyHostToDevice, st);
  for (int md = 0; md < 2 && err == cudaSuccess; ++md)
    if (mt[md].first != nullptr)
      err = cudaMemcpyAsync(base + off_first[md], g_sp_first[md],
                            (size_t)(nwarps[md] + 1) * sizeof(int), cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess)
    err = cudaMemsetAsync(base + off_ctr, 0, 2 * sizeof(unsigned long long), st);
  // the host arrays are reused by the next call: wait until the copies have read them
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  const FlatProblem* d_probs = (const FlatProblem*)base;
  size_t xsmem = 0;
  int xthreads = 32;
  for (int k = 0; k < np; ++k) {
    xsmem = std::max(xsmem, flat_exchange_smem(g_sp_probs[k].p.R, g_sp_probs[k].p.mode));
    xthreads = std::max(xthreads, flat_exchange_threads(g_sp_probs[k].p.W));
  }
  if (err == cudaSuccess) err = flat_exchange_prepare(xsmem);
  for (int64_t j = 0; j < n_max && err == cudaSuccess; ++j) {
    bool ex = false;  // counted for at least one problem (a swap iteration or a trace row)
    for (int k = 0; k < np && !ex; ++k) {
      const FlatProblem& fp = g_sp_probs[k];
      ex = j < fp.n && (fp.p.trace_E != nullptr ||
                        (fp.m > 0 && (fp.t0 + (uint64_t)j + 1) % (uint64_t)fp.m == 0));
    }
    err = launch_flat_sweep(mt, d_probs, np, j, ex, xsmem, xthreads, di.sms, st);
  }
  if (err != cudaSuccess) {
    for (int j = 0; j < count; ++j) ps[j]->poisoned = PT_ECUDA;
    return fail(PT_ECUDA, "static batch launch: %s", cudaGetErrorString(err));
  }
  return PT_OK;
}

}  // namespace ptb
