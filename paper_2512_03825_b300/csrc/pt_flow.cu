// pt_flow.cu -- the dataflow batched path: one cooperative launch per batch call and mode.
//
// The word tiles of the lock-step path, dealt to warps the same way, but every warp runs all
// sweeps of the batch inside one launch. Per-problem counters take the place of kernel
// boundaries and order the steps of each problem (Sec. 3: the two colours of a sweep
// alternate and the swap iteration follows its sweep):
//   colour 0 of sweep j   waits for colour 1 of sweep j-1 (done1 = j x tiles) or, when a swap
//                         iteration followed sweep j-1, for that iteration (xdone);
//   colour 1 of sweep j   waits for colour 0 of sweep j (done0 = (j+1) x tiles);
//   the swap iteration    is run by the warp that completes the problem's last colour-1 tile
//   after sweep j         of sweep j (its ticket on done1), which then bumps xdone.
// Each wait is for work of an earlier step, and every warp is resident (cooperative
// launch), so the waits end; each still has a time limit, after which the warp marks every
// problem of the batch PT_ETIMEOUT and all warps leave. Problems never wait for each other:
// a warp whose next tile is not ready waits for that tile's problem only.
//
// Completions are released by lane 0 after the warp barrier (a release-ordered add) and
// acquired by lane 0 of the waiting warp (an acquire fence after its polling) before its
// warp barrier. Every word a tile or a swap iteration
// reads from another warp (the other colour, the thresholds, the maps) was written before
// a release it has so acquired, directly or through a chain of them, so plain loads,
// L1 included, see it under the PTX memory model, as after a grid-wide barrier. The
// neighbour words and the swap iteration's maps are still read through L2: with L1 loads,
// sweeps followed by a swap iteration ran about 35 us slower on the 256-problem workload
// (measured; not explained).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "pt.h"
#include "pt_batch.h"
#include "pt_device.cuh"
#include "pt_flat.cuh"
#include "pt_internal.h"

namespace ptb {

namespace {

struct FlowSync {  // per problem, zeroed before each launch
  unsigned done0;  // colour-0 tiles completed (all sweeps of this launch)
  unsigned done1;  // colour-1 tiles completed
  unsigned xdone;  // swap iterations completed
  unsigned pad;
};

struct FlowArgs {
  const FlatProblem* probs;
  const Tile* tiles;
  const int* first;  // warp g: tiles [first[g], first[g + 1])
  FlowSync* sync;
  int* abort;        // set by the first wait that runs out
  int nprobs;
  int64_t n_max;
};

// Lane 0 waits until *ctr reaches target (wrap-safe), then the warp continues. The counter
// is polled with relaxed loads; one acquire after the wait orders the warp's reads after the
// releases it observed (an acquire also drops the SM's L1 lines, so it is never polled).
// False when the wait ran out or another warp's did.
__device__ bool warp_wait(const unsigned* ctr, unsigned target, const FlowArgs& a,
                          uint64_t limit_ns) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    if ((int)(ld_relaxed_u32(ctr) - target) < 0) {
      const uint64_t t0 = global_ns();
      for (;;) {
        __nanosleep(64);
        if ((int)(ld_relaxed_u32(ctr) - target) >= 0) break;
        if (*(volatile int*)a.abort != 0) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > limit_ns) {
          if (atomicExch(a.abort, 1) == 0)
            for (int pi = 0; pi < a.nprobs; ++pi) atomicCAS(a.probs[pi].p.status, 0, PT_ETIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    fence_acq_rel_gpu();
  }
  __syncwarp();
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Lane 0 publishes the warp's completed work (the warp barrier orders every lane's writes
// before its release).
__device__ __forceinline__ void warp_release_add(unsigned* ctr) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) red_release_add_u32(ctr, 1u);
}

template <int MODE>
__global__ void __launch_bounds__(kFlatThreads, 2) k_flow(const __grid_constant__ FlowArgs a) {
  __shared__ __align__(16) PlaneGeneric gen[kFlatThreads / 32];  // 16-byte rows (uint4 reads)
  __shared__ uint4 thr_s[kFlatThreads / 32][16];  // ferro thresholds of each warp's tile
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int tbeg = a.first[g], tend = a.first[g + 1];
  for (int64_t j = 0; j < a.n_max; ++j) {
    for (int colour = 0; colour < 2; ++colour) {
      for (int tix = tbeg; tix < tend; ++tix) {
        const Tile tl = a.tiles[tix];
        const FlatProblem& fp = a.probs[tl.prob];
        if (j >= fp.n) continue;  // warp-uniform
        FlowSync& sy = a.sync[tl.prob];
        const unsigned nt = (unsigned)fp.ntiles;
        const unsigned* ctr = nullptr;
        unsigned target = 0;
        if (colour == 1) {
          ctr = &sy.done0;
          target = (unsigned)(j + 1) * nt + (j == 0 ? (unsigned)fp.stall : 0u);
        } else if (j > 0 && exchanges_after(fp, j - 1)) {
          ctr = &sy.xdone;
          target = (unsigned)exchanges_through(fp, j - 1);
        } else if (j > 0) {
          ctr = &sy.done1;
          target = (unsigned)j * nt;
        }
        if (ctr && !warp_wait(ctr, target, a, fp.wait_ns)) return;
        const bool count = colour == 1 && exchanges_after(fp, j);
        if (!count) {
          tile_half<MODE, false, true>(fp, tl, colour, j, false, thr_s[wib], &gen[wib]);
          warp_release_add(colour == 0 ? &sy.done0 : &sy.done1);
          continue;
        }
        tile_half<MODE, true, true>(fp, tl, 1, j, true, thr_s[wib], &gen[wib]);
        // the ticket releases this warp's tile and counts; the warp that draws the last one
        // of the sweep acquires every other warp's and runs the swap iteration
        __syncwarp();
        unsigned ticket = 0;
        if (lane == 0) {
          ticket = atom_release_add_u32(&sy.done1, 1u);
          if (ticket + 1u == (unsigned)(j + 1) * nt) fence_acq_rel_gpu();
        }
        ticket = __shfl_sync(0xffffffffu, ticket, 0);
        if (ticket + 1u == (unsigned)(j + 1) * nt) {
          __syncwarp();
          exchange_warp(fp.p, exchange_index(fp, j));
          warp_release_add(&sy.xdone);
        }
      }
    }
  }
}

const void* flow_fn(int md) {
  return md == 0 ? (const void*)k_flow<kModeFerro> : (const void*)k_flow<kModeGeneric>;
}

}  // namespace

int sweep_batch_flow(pt_problem* const* ps, int count, const int64_t* n, const int* every,
                     cudaStream_t st, const DeviceInfo& di, int tile_words) {
  std::vector<FlatProblem> probs;
  std::vector<Tile> tiles[2];  // by mode
  const int64_t n_max = build_flat_lists(ps, count, n, every, tile_words, false, &probs, tiles);
  if (n_max < 0) return fail(PT_EINTERNAL, "batch work tiles outside their planes");
  for (int j = 0; j < count; ++j) ps[j]->stall = 0;  // test support applies to one call
  if (probs.empty()) return PT_OK;
  // one resident wave per mode (the cooperative launch needs every CTA resident)
  const int wpb = kFlatThreads / 32;
  std::vector<Tile> dealt[2];
  std::vector<int> first[2];
  int grid[2] = {0, 0};
  for (int md = 0; md < 2; ++md) {
    if (tiles[md].empty()) continue;
    int per_sm = 0;
    const cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, flow_fn(md), kFlatThreads, 0);
    if (e != cudaSuccess) return fail(PT_ECUDA, "occupancy: %s", cudaGetErrorString(e));
    if (per_sm < 1) return fail(PT_EINTERNAL, "dataflow kernel does not fit an SM");
    const int needed = (int)((tiles[md].size() + wpb - 1) / wpb);
    grid[md] = std::max(1, std::min(per_sm * di.sms, needed));
    deal_tiles(tiles[md], probs, grid[md] * wpb, &dealt[md], &first[md]);
  }
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t pb = probs.size() * sizeof(FlatProblem);
  const size_t tb[2] = {dealt[0].size() * sizeof(Tile), dealt[1].size() * sizeof(Tile)};
  const size_t fb[2] = {first[0].size() * sizeof(int), first[1].size() * sizeof(int)};
  const size_t sb = probs.size() * sizeof(FlowSync) + sizeof(int);  // counters, then abort
  const size_t total = al(pb) + al(tb[0]) + al(tb[1]) + al(fb[0]) + al(fb[1]) + al(sb);
  void* scratch = nullptr;
  cudaError_t err = cudaMallocAsync(&scratch, total, st);
  if (err != cudaSuccess) return fail(PT_ENOMEM, "batch scratch: %s", cudaGetErrorString(err));
  char* cur = (char*)scratch;
  FlatProblem* d_probs = (FlatProblem*)cur;
  cur += al(pb);
  Tile* d_tiles[2];
  int* d_first[2];
  for (int md = 0; md < 2; ++md) {
    d_tiles[md] = (Tile*)cur;
    cur += al(tb[md]);
  }
  for (int md = 0; md < 2; ++md) {
    d_first[md] = (int*)cur;
    cur += al(fb[md]);
  }
  FlowSync* d_sync = (FlowSync*)cur;
  int* d_abort = (int*)(d_sync + probs.size());
  err = cudaMemsetAsync(d_sync, 0, sb, st);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(d_probs, probs.data(), pb, cudaMemcpyHostToDevice, st);
  for (int md = 0; md < 2 && err == cudaSuccess; ++md) {
    if (!tb[md]) continue;
    err = cudaMemcpyAsync(d_tiles[md], dealt[md].data(), tb[md], cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(d_first[md], first[md].data(), fb[md], cudaMemcpyHostToDevice, st);
  }
  // the two modes' problems are disjoint: one launch after the other
  for (int md = 0; md < 2 && err == cudaSuccess; ++md) {
    if (!grid[md]) continue;
    FlowArgs fa;
    fa.probs = d_probs;
    fa.tiles = d_tiles[md];
    fa.first = d_first[md];
    fa.sync = d_sync;
    fa.abort = d_abort;
    fa.nprobs = (int)probs.size();
    fa.n_max = n_max;
    void* args[] = {&fa};
    err = cudaLaunchCooperativeKernel(flow_fn(md), dim3(grid[md]), dim3(kFlatThreads), args, 0,
                                      st);
  }
  const cudaError_t err2 = cudaFreeAsync(scratch, st);
  if (err == cudaSuccess) err = err2;
  if (err != cudaSuccess) {
    for (int j = 0; j < count; ++j) ps[j]->poisoned = PT_ECUDA;
    return fail(PT_ECUDA, "dataflow batch launch: %s", cudaGetErrorString(err));
  }
  return PT_OK;
}

}  // namespace ptb
