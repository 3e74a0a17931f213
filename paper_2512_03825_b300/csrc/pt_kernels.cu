// pt_kernels.cu -- the per-problem ("plain") kernels: initial spins, one checkerboard half
// sweep per launch, bit-sliced energy/magnetisation count, and the exchange step.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pt_debug.cuh"
#include "pt_device.cuh"
#include "pt_launch.h"

namespace ptb {

namespace {

constexpr int kThreads = 256;

// Walks the words (y, i) of one colour of one plane with a grid-stride loop, keeping y and i
// up to date without a division per step.
struct RowWalker {
  int y, i, dy, di, half;
  __device__ __forceinline__ RowWalker(int start, int stride, int half_) : half(half_) {
    y = start / half_;
    i = start - y * half_;
    dy = stride / half_;
    di = stride - dy * half_;
  }
  __device__ __forceinline__ void step() {
    i += di;
    y += dy;
    if (i >= half) {
      i -= half;
      y += 1;
    }
  }
};

__device__ __forceinline__ int nslots_of_plane(int R, int w) { return min(32, R - 32 * w); }

__device__ __forceinline__ uint32_t used_mask(int nslots) {
  return nslots >= 32 ? 0xffffffffu : ((1u << nslots) - 1u);
}

// ---------------------------------------------------------------------------------------
// Initial state (Sec. 3 initialisation phase): sigma = +1 iff bit 31 of the TAG_INIT draw.
// grid = (X, W, 2 colours)
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_init(DevProblem p) {
  const int w = blockIdx.y, c = blockIdx.z;
  const int L = p.L, half = L >> 1;
  const int nslots = nslots_of_plane(p.R, w);
  const int nblk = (nslots + 3) >> 2;
  const uint32_t used = used_mask(nslots);
  uint32_t* out = p.spins + word_index(L, w, c, 0, 0);
  const int nwords = L * half;
  PT_DBG_CHECK(p, w, p.W, kDbgSpinStore);
  const int start = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  if (start >= nwords) return;
  RowWalker rw(start, stride, half);
  for (int idx = start; idx < nwords; idx += stride, rw.step()) {
    const int x = 2 * rw.i + ((rw.y + c) & 1);
    const uint32_t site = (uint32_t)(rw.y * L + x);
    uint32_t word = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (j < nblk) {
        const Philox4 r = philox4x32_10(site, 0u, (uint32_t)(8 * w + j), kTagInit, p.key0, p.key1);
        word |= ((r.x >> 31) << (4 * j)) | ((r.y >> 31) << (4 * j + 1)) |
                ((r.z >> 31) << (4 * j + 2)) | ((r.w >> 31) << (4 * j + 3));
      }
    }
    out[PT_DBG_IDX(p, idx, nwords, kDbgSpinStore)] = word & used;
  }
}

// ---------------------------------------------------------------------------------------
// One half sweep: every word of colour `colour` of plane blockIdx.y gets its Metropolis
// update. grid = (X, W)
// ---------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_half_sweep(DevProblem p, int colour, uint64_t t) {
  const int w = blockIdx.y;
  const int L = p.L, half = L >> 1;
  const int nslots = nslots_of_plane(p.R, w);
  const int nblk = (nslots + 3) >> 2;
  const SweepCtr cx = make_sweep_ctr(t, p.key0, p.key1);
  const size_t own_base = word_index(L, w, colour, 0, 0);
  uint32_t* own = p.spins + own_base;
  const uint32_t* oth = p.spins + word_index(L, w, colour ^ 1, 0, 0);
  const int nwords = L * half;
  const int start = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  // test hook of the debug build: one planted mistake in this launch (thread 0 only), which
  // the checks must catch: 1 stores its first word a second time (unchanged), 2 asks for a
  // neighbour one past the colour's words
  const int inject = (PT_DBG_ON && start == 0) ? p.dbg_inject : 0;

  if (MODE == kModeFerro) {
    const PlaneFerro* pl = reinterpret_cast<const PlaneFerro*>(p.planes) + w;
    uint32_t T0[32], T1[32];
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      T0[b] = pl->T0[b];
      T1[b] = pl->T1[b];
    }
    const uint32_t alw0 = pl->alw0, alw1 = pl->alw1, used = pl->used;
    if (start >= nwords) return;
    RowWalker rw(start, stride, half);
    for (int idx = start; idx < nwords; idx += stride, rw.step()) {
      const int y = rw.y, i = rw.i;
      const int par = (y + colour) & 1;
      const int ym = (y == 0) ? L - 1 : y - 1;
      const int yp = (y == L - 1) ? 0 : y + 1;
      const int ih = par ? ((i + 1 == half) ? 0 : i + 1) : ((i == 0) ? half - 1 : i - 1);
      const uint32_t s = own[PT_DBG_IDX(p, idx, nwords, kDbgSpinLoad)];
      const uint32_t n0 = oth[PT_DBG_IDX(p, ym * half + i, nwords, kDbgSpinLoad)];
      const uint32_t n1 = oth[PT_DBG_IDX(p, yp * half + i, nwords, kDbgSpinLoad)];
      const uint32_t n2 = oth[PT_DBG_IDX(p, y * half + i, nwords, kDbgSpinLoad)];
      const uint32_t n3 = oth[PT_DBG_IDX(p, (inject == 2 ? nwords : y * half + ih), nwords,
                                         kDbgSpinLoad)];
      const uint32_t site = (uint32_t)(y * L + 2 * i + par);
      const uint32_t ns = update_word_ferro(s, n0, n1, n2, n3, site, (uint32_t)(8 * w), nblk,
                                            T0, T1, alw0, alw1, used, cx);
      if (PT_DBG_STORE(p, idx, nwords, own_base, t, colour)) own[idx] = ns;
      if (inject == 1 && idx == start && PT_DBG_STORE(p, idx, nwords, own_base, t, colour))
        own[idx] = ns;
    }
  } else {
    __shared__ PlaneGeneric pl;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(
        reinterpret_cast<const PlaneGeneric*>(p.planes) + w);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&pl);
    for (int q = threadIdx.x; q < (int)(sizeof(PlaneGeneric) / 4); q += blockDim.x) dst[q] = src[q];
    __syncthreads();
    if (start >= nwords) return;
    RowWalker rw(start, stride, half);
    for (int idx = start; idx < nwords; idx += stride, rw.step()) {
      const int y = rw.y, i = rw.i;
      const int par = (y + colour) & 1;
      const int ym = (y == 0) ? L - 1 : y - 1;
      const int yp = (y == L - 1) ? 0 : y + 1;
      const int ih = par ? ((i + 1 == half) ? 0 : i + 1) : ((i == 0) ? half - 1 : i - 1);
      const uint32_t s = own[PT_DBG_IDX(p, idx, nwords, kDbgSpinLoad)];
      const uint32_t n0 = oth[PT_DBG_IDX(p, ym * half + i, nwords, kDbgSpinLoad)];
      const uint32_t n1 = oth[PT_DBG_IDX(p, yp * half + i, nwords, kDbgSpinLoad)];
      const uint32_t n2 = oth[PT_DBG_IDX(p, y * half + i, nwords, kDbgSpinLoad)];
      const uint32_t n3 = oth[PT_DBG_IDX(p, y * half + ih, nwords, kDbgSpinLoad)];
      const uint32_t site = (uint32_t)(y * L + 2 * i + par);
      const uint32_t ns =
          update_word_generic(s, n0, n1, n2, n3, site, (uint32_t)(8 * w), nblk, pl, cx);
      if (PT_DBG_STORE(p, idx, nwords, own_base, t, colour)) own[idx] = ns;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Energy / magnetisation count (per slot): every bond joins a colour-0 and a colour-1 site,
// so the unsatisfied bonds are the anti-aligned neighbours of the colour-0 sites; the up
// spins are counted on both colours. Accumulated into p.cnt (which must start at zero).
// grid = (X, W); each thread handles at most kMaxWordsPerThread colour-0 words.
// ---------------------------------------------------------------------------------------
constexpr int kMaxWordsPerThread = 4000;  // 4 * 4000 < 2^14 (per-thread counter depth)

// The counts of colour-0 words start, start + stride, ... below end of plane w, added to
// cnt (one call per block).
__device__ __forceinline__ void energy_count(const uint32_t* spins, uint32_t* cnt, int L, int W,
                                             int w, int start, int stride, int end,
                                             DbgSink dbg) {
  (void)dbg;
  const int half = L >> 1;
  const int nwords = L * half;
  (void)nwords;
  PT_DBG_CHECK(dbg, w, W, kDbgSpinLoad);
  PT_DBG_CHECK(dbg, end - 1, nwords, kDbgSpinLoad);
  const uint32_t* c0 = spins + word_index(L, w, 0, 0, 0);
  const uint32_t* c1 = spins + word_index(L, w, 1, 0, 0);
  BitCounter<20, 14> U, N;
  U.zero();
  N.zero();
  if (start < end) {
    RowWalker rw(start, stride, half);
    for (int idx = start; idx < end; idx += stride, rw.step()) {
      const int y = rw.y, i = rw.i;
      const int par = y & 1;
      const int ym = (y == 0) ? L - 1 : y - 1;
      const int yp = (y == L - 1) ? 0 : y + 1;
      const int ih = par ? ((i + 1 == half) ? 0 : i + 1) : ((i == 0) ? half - 1 : i - 1);
      const uint32_t s = c0[PT_DBG_IDX(dbg, idx, nwords, kDbgSpinLoad)];
      const uint32_t o = c1[PT_DBG_IDX(dbg, idx, nwords, kDbgSpinLoad)];
      const NbCount k = count4(s ^ c1[PT_DBG_IDX(dbg, ym * half + i, nwords, kDbgSpinLoad)],
                               s ^ c1[PT_DBG_IDX(dbg, yp * half + i, nwords, kDbgSpinLoad)],
                               s ^ o,
                               s ^ c1[PT_DBG_IDX(dbg, y * half + ih, nwords, kDbgSpinLoad)]);
      U.add3(k.b0, k.b1, k.b2);
      N.add2(s ^ o, s & o);
    }
  }
  const uint32_t u = U.warp_total_for_lane();
  const uint32_t n = N.warp_total_for_lane();
  __shared__ uint32_t acc[2][32];
  if (threadIdx.x < 64) (&acc[0][0])[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  atomicAdd(&acc[0][lane], u);
  atomicAdd(&acc[1][lane], n);
  __syncthreads();
  if (threadIdx.x < 32) {
    if (acc[0][threadIdx.x])
      atomicAdd(&cnt[PT_DBG_IDX(dbg, w * 32 + threadIdx.x, 2 * W * 32, kDbgCount)],
                acc[0][threadIdx.x]);
    if (acc[1][threadIdx.x])
      atomicAdd(&cnt[PT_DBG_IDX(dbg, W * 32 + w * 32 + threadIdx.x, 2 * W * 32, kDbgCount)],
                acc[1][threadIdx.x]);
  }
}

__global__ void __launch_bounds__(kThreads) k_energy(DevProblem p) {
  energy_count(p.spins, p.cnt, p.L, p.W, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x,
               gridDim.x * blockDim.x, p.L * (p.L >> 1), DbgSink{p.dbg, p.status});
}

// One chunk per block: kEnergyChunkWords / kThreads = 8 words per thread.
__global__ void __launch_bounds__(kThreads) k_energy_batch(const EnergyChunk* __restrict__ chunks) {
  const EnergyChunk c = chunks[blockIdx.x];
  energy_count(c.spins, c.cnt, c.L, c.W, c.w, c.first + (int)threadIdx.x, blockDim.x,
               c.first + c.count, DbgSink{c.dbg, c.status});
}

// ---------------------------------------------------------------------------------------
// Exchange step (Sec. 3), one block:
//   kEnergy:   E_slot / M_slot from the counts (then clears the counts)
//   kExchange: swap iteration e on pairs (k, k+1), k = e & 1 (mod 2); swaps temperature
//              indices of accepted pairs and counts attempts / acceptances
//   kRebuild:  rewrites the per-plane thresholds for the current slot -> temperature map
//   kTrace:    writes E_int / M of every slot at its (new) temperature index into the trace
//              row of sweep t
// ---------------------------------------------------------------------------------------
__device__ void rebuild_planes(const DevProblem& p) {
  const int R = p.R, W = p.W;
  constexpr uint64_t kTwo32 = 1ull << 32;
  for (int r = threadIdx.x; r < W * 32; r += blockDim.x) {  // whole warps: W * 32 % 32 == 0
    const int w = r >> 5, b = r & 31;
    const bool in_use = r < R;
    const int temp = in_use ? p.temp_of_slot[r] : 0;
    const uint32_t used = __ballot_sync(0xffffffffu, in_use);
    if (p.mode == kModeFerro) {
      PlaneFerro* pl = reinterpret_cast<PlaneFerro*>(p.planes) + w;
      // class index 2 k + 1 (sigma = +1; with h = 0 both signs share the threshold)
      const uint64_t t0 = in_use ? p.T_temp[(size_t)temp * kClasses + 1] : 0;
      const uint64_t t1 = in_use ? p.T_temp[(size_t)temp * kClasses + 3] : 0;
      pl->T0[b] = (uint32_t)min(t0, kTwo32 - 1);
      pl->T1[b] = (uint32_t)min(t1, kTwo32 - 1);
      const uint32_t a0 = __ballot_sync(0xffffffffu, in_use && t0 >= kTwo32);
      const uint32_t a1 = __ballot_sync(0xffffffffu, in_use && t1 >= kTwo32);
      if (b == 0) {
        pl->alw0 = a0;
        pl->alw1 = a1;
        pl->used = used;
        pl->pad = 0;
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
      if (b == 0) {
        pl->used = used;
        pl->pad = 0;
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_exchange(DevProblem p, uint64_t e, int flags,
                                                       uint64_t t) {
  const int R = p.R, W = p.W;
  const int64_t L2 = (int64_t)p.L * p.L;
  if (flags & kStepEnergy) {
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      const int64_t U = p.cnt[r];
      const int64_t ones = p.cnt[W * 32 + r];
      const int64_t bonds = 2 * L2 - 2 * U;  // sum over bonds of sigma_i sigma_j
      const int64_t M = 2 * ones - L2;
      p.E_slot[r] = -p.J_int * bonds + p.h_int * M;
      p.M_slot[r] = M;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * W * 32; q += blockDim.x) p.cnt[q] = 0;
  }
  if (flags & kStepExchange) {
    __syncthreads();
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
  }
  if (flags & kStepRebuild) {
    __syncthreads();
    rebuild_planes(p);
  }
  if (flags & kStepTrace) {
    __syncthreads();
    const int64_t row = (int64_t)((t - p.trace_t0) % (uint64_t)p.trace_cap);
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      const int k = p.temp_of_slot[r];
      const int64_t at = PT_DBG_IDX(p, row * R + k, p.trace_cap * R, kDbgTrace);
      p.trace_E[at] = p.E_slot[r];
      p.trace_M[at] = p.M_slot[r];
    }
  }
}

int grid_x_for(int nwords, int W, int sms, int per_sm) {
  int want = (nwords + kThreads - 1) / kThreads;
  int cap = (sms * per_sm + W - 1) / W;
  if (cap < 1) cap = 1;
  return want < cap ? (want > 0 ? want : 1) : cap;
}

// ---------------------------------------------------------------------------------------
// Results of many problems packed into one buffer (one block per problem record): status,
// E_int and M by slot, slot_of_temp, and the pair counters, each as an 8-byte word.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_gather(const GatherItem* __restrict__ items, int n,
                                                     uint64_t* __restrict__ out) {
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    const GatherItem it = items[j];
    uint64_t* const o = out + it.out;
    const int R = it.R, P = it.npairs;
    const int total = 1 + 3 * R + 2 * P;
    // the energy step: E_int and M per slot from the counts, then the counts cleared
    const int64_t L2 = (int64_t)it.L * it.L;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      const int64_t U = it.cnt[r];
      const int64_t ones = it.cnt[it.W * 32 + r];
      const int64_t bonds = 2 * L2 - 2 * U;  // sum over bonds of sigma_i sigma_j
      const int64_t M = 2 * ones - L2;
      it.E_slot[r] = -it.J_int * bonds + it.h_int * M;
      it.M_slot[r] = M;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * it.W * 32; q += blockDim.x) it.cnt[q] = 0;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
      uint64_t v;
      if (q == 0)
        v = (uint64_t)(int64_t)*it.status;
      else if (q <= R)
        v = (uint64_t)it.E_slot[q - 1];
      else if (q <= 2 * R)
        v = (uint64_t)it.M_slot[q - 1 - R];
      else if (q <= 3 * R)
        v = (uint64_t)(int64_t)it.slot_of_temp[q - 1 - 2 * R];
      else if (q <= 3 * R + P)
        v = it.attempted[q - 1 - 3 * R];
      else
        v = it.accepted[q - 1 - 3 * R - P];
      o[q] = v;
    }
    __syncthreads();  // the next record's energy step reuses the block
  }
}

}  // namespace

cudaError_t launch_gather(const GatherItem* items, int n, uint64_t* out, int sms,
                          cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<n < 8 * sms ? n : 8 * sms, kThreads, 0, st>>>(items, n, out);
  return cudaGetLastError();
}

cudaError_t launch_energy_batch(const EnergyChunk* chunks, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_energy_batch<<<n, kThreads, 0, st>>>(chunks);
  return cudaGetLastError();
}

cudaError_t launch_init(const DevProblem& p, const DeviceInfo& dev, cudaStream_t st) {
  const int nwords = p.L * (p.L >> 1);
  dim3 grid(grid_x_for(nwords, p.W, dev.sms, 8), p.W, 2);
  k_init<<<grid, kThreads, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_half_sweep(const DevProblem& p, const DeviceInfo& dev, int colour,
                              uint64_t t, cudaStream_t st) {
  const int nwords = p.L * (p.L >> 1);
  dim3 grid(grid_x_for(nwords, p.W, dev.sms, 4), p.W);
  if (p.mode == kModeFerro)
    k_half_sweep<kModeFerro><<<grid, kThreads, 0, st>>>(p, colour, t);
  else
    k_half_sweep<kModeGeneric><<<grid, kThreads, 0, st>>>(p, colour, t);
  return cudaGetLastError();
}

cudaError_t launch_energy(const DevProblem& p, const DeviceInfo& dev, cudaStream_t st) {
  const int nwords = p.L * (p.L >> 1);
  int gx = grid_x_for(nwords, p.W, dev.sms, 8);
  const int min_gx = (nwords + kThreads * kMaxWordsPerThread - 1) / (kThreads * kMaxWordsPerThread);
  if (gx < min_gx) gx = min_gx;
  dim3 grid(gx, p.W);
  k_energy<<<grid, kThreads, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_exchange(const DevProblem& p, uint64_t e, int flags, cudaStream_t st,
                            uint64_t t) {
  k_exchange<<<1, kThreads, 0, st>>>(p, e, flags, t);
  return cudaGetLastError();
}

}  // namespace ptb
