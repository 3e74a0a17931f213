// pt_persist.cu -- the single-problem path as one persistent launch per pt_sweep call.
//
// A cooperative launch keeps every CTA resident, so the CTAs can meet at a grid barrier
// between the two half sweeps of a sweep instead of ending the kernel (Sec. 3: all sites of
// one colour are independent given the other colour; the two colours alternate). Each CTA
// owns a fixed share of the words of one plane for the whole launch:
//   plane w = blockIdx.x % W, words q = q0, q0 + step, ... of each colour,
//   q0 = (blockIdx.x / W) * 256 + threadIdx.x, step = (gridDim.x / W) * 256,
// so the plane's thresholds stay in shared memory (read as 16-byte broadcasts) and the
// words the thread itself wrote come back through L1; the other colour, written by other
// CTAs, is read through L2 (ld.global.cg).
//
// Replica exchange (Sec. 3, Eq. 5): after the colour-1 half sweep of an exchange sweep each
// CTA adds its plane's bond (and up-spin) counts of the new state into a count buffer; after
// the barrier EVERY CTA computes the same swap iteration from the complete counts, on its own
// shared-memory copy of the temperature map, and rebuilds its plane's thresholds. Only block 0
// writes the swap statistics; the maps and the plane tables go back to global memory at the
// end of the launch. When an observable trace is on, every sweep counts, and block 0 writes
// the sweep's row. Three count buffers take turns between counted sweeps: after the barrier
// of one, block 0 clears the buffer of the counted sweep after next, which every CTA has
// finished reading and none writes before another grid barrier.
//
// The barrier counter and the count buffers are cleared by the host before each launch.
// A barrier wait that exceeds its time limit stores PT_ETIMEOUT in the status word; every
// waiting CTA that sees a non-zero status (or runs out of time itself) leaves the kernel.
//
// A grid of at most 16 CTAs can instead run as one thread-block cluster (CLUSTER): its CTAs
// are resident together by construction and meet at the hardware cluster barrier
// (barrier.cluster, release on arrival and acquire on the wait, at cluster scope), with no
// counter in memory and no waiting on one.
//
// When each plane has a single CTA (LOCAL: small lattices), no other CTA ever reads that
// CTA's words: the plane (both colours) is copied into shared memory at the start of the
// launch, every half sweep reads and writes it there, and it is copied back at the end. The
// half sweeps then meet at the block barrier alone; only the swap iterations, which need
// every plane's counts, still meet at the grid barrier.
#include <algorithm>
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pt.h"
#include "pt_debug.cuh"
#include "pt_device.cuh"
#include "pt_grid.cuh"
#include "pt_persist.h"

namespace ptb {

namespace {

constexpr uint64_t kTwo32 = 1ull << 32;

struct PersistArgs {
  DevProblem p;
  uint64_t t0, e0;
  int n;         // sweeps in this launch
  int m;         // exchange after every m-th sweep (0: never)
  int stall;     // extra arrivals the first barrier waits for (test of the bounded wait)
  uint64_t limit_ns;
  RoundKeys rk;  // Philox round keys of the seed (constant-bank operands)
};

// The plane's thresholds under the temperature map tos, staged in shared memory by warp 0
// (same rule as the plane rebuild of the exchange kernel). Ferro: from Tf[temp] = the
// thresholds of k = 0 and k = 1 at every temperature, which the kernel keeps in shared
// memory, so a swap iteration's restaging reads no global memory.
template <int MODE>
__device__ void stage_plane(const DevProblem& p, const int32_t* tos, int w, PlaneFerro& fer,
                            PlaneGeneric& gen, const ulonglong2* Tf) {
  if (threadIdx.x < 32) {
    const int b = threadIdx.x, r = 32 * w + b;
    const bool in_use = r < p.R;
    const int temp = in_use ? tos[r] : 0;
    const uint32_t used = __ballot_sync(0xffffffffu, in_use);
    if (MODE == kModeFerro) {
      const ulonglong2 tt = Tf[temp];
      const uint64_t t0 = in_use ? tt.x : 0;
      const uint64_t t1 = in_use ? tt.y : 0;
      fer.T0[b] = (uint32_t)min(t0, kTwo32 - 1);
      fer.T1[b] = (uint32_t)min(t1, kTwo32 - 1);
      const uint32_t a0 = __ballot_sync(0xffffffffu, in_use && t0 >= kTwo32);
      const uint32_t a1 = __ballot_sync(0xffffffffu, in_use && t1 >= kTwo32);
      if (b == 0) {
        fer.alw0 = a0;
        fer.alw1 = a1;
        fer.used = used;
        fer.pad = 0;
      }
    } else {
#pragma unroll
      for (int c = 0; c < kClasses; ++c) {
        const uint64_t tc = in_use ? p.T_temp[(size_t)temp * kClasses + c] : 0;
        gen.T[c][b] = (uint32_t)min(tc, kTwo32 - 1);
        const uint32_t a = __ballot_sync(0xffffffffu, in_use && tc >= kTwo32);
        if (b == 0) gen.alw[c] = a;
      }
      if (b == 0) {
        gen.used = used;
        gen.pad = 0;
      }
    }
  }
  __syncthreads();
}

// E_int of a slot from its counts: U unsatisfied bonds, `ones` up spins (zero in the
// ferromagnetic zero-field case, where h_int = 0 and they are not counted).
__device__ __forceinline__ int64_t slot_energy(const DevProblem& p, int64_t L2, int64_t U,
                                               int64_t ones) {
  return -p.J_int * (2 * L2 - 2 * U) + p.h_int * (2 * ones - L2);
}

// Swap iteration e on this CTA's copy of the maps (every CTA draws the same numbers and so
// reaches the same maps); `owner` also counts attempts and acceptances. cb: the counts, in
// global memory (read through L2) or, with SHARED_COUNTS, in this CTA's shared memory.
template <bool SHARED_COUNTS>
__device__ void exchange_local(const DevProblem& p, uint64_t e, const uint32_t* cb,
                               int32_t* sot, int32_t* tos, bool owner) {
  const int R = p.R, W = p.W;
  const int64_t L2 = (int64_t)p.L * p.L;
  const int parity = (int)(e & 1);
  const uint32_t c3 = kTagExch | ((uint32_t)(e >> 32) << 8);
  for (int k = parity + 2 * (int)threadIdx.x; k + 1 < R; k += 2 * (int)blockDim.x) {
    const int a = sot[k], b = sot[k + 1];
    const auto count = [&](int i) { return SHARED_COUNTS ? cb[i] : __ldcg(cb + i); };
    const int64_t Ea = slot_energy(p, L2, count(a), count(W * 32 + a));
    const int64_t Eb = slot_energy(p, L2, count(b), count(W * 32 + b));
    const int64_t n = Ea - Eb;
    const SwapPair sp = p.pairs[k];
    const uint64_t S = pair_threshold(sp, p.swap_table, p.table_shift, n);
    const Philox4 rnd = philox4x32_10((uint32_t)k, (uint32_t)e, 0u, c3, p.key0, p.key1);
    const bool accept = (uint64_t)rnd.x < S;
    if (owner) count_swap(p.attempted, p.accepted, k, accept);
    if (accept) {
      sot[k] = b;
      sot[k + 1] = a;
      tos[a] = k + 1;
      tos[b] = k;
    }
  }
  __syncthreads();
}

// One half sweep over this thread's words of colour `colour` of plane w. With COUNT, the
// new colour-1 words' anti-aligned neighbours (every bond has exactly one colour-1 end) and,
// with `ones` (always in the generic case), the up spins of the colour-1 word and of the
// colour-0 word one row up (a one-to-one pairing of the colours) are added to U / N.
// plane: the first word of plane w (colour 0, then colour 1), in global memory or (LOCAL)
// in this CTA's shared memory.
template <int MODE, bool COUNT, bool LOCAL>
__device__ __forceinline__ void half_pass(const DevProblem& p, uint32_t* plane, int w,
                                          int colour, uint64_t t, const RoundKeys& rk,
                                          const BlockTerms& bt, int q0, int step, int y0, int i0,
                                          int dy, int di, const uint4* thr, uint32_t alw0,
                                          uint32_t alw1, uint32_t used, const PlaneGeneric& gen,
                                          bool five, const int (&cls5)[5], bool ones,
                                          BitCounter<15, 10>& U, BitCounter<15, 10>& N) {
  const uint32_t c3 = kTagSpin | ((uint32_t)(t >> 32) << 8);
  const int L = p.L, half = L >> 1;
  const int nwords = L * half;
  const int nblk = (min(32, p.R - 32 * w) + 3) >> 2;
  uint32_t* own = plane + (size_t)colour * nwords;
  const uint32_t* oth = plane + (size_t)(colour ^ 1) * nwords;
  const size_t own_base = word_index(L, w, colour, 0, 0);  // own's first word in p.spins
  (void)own_base;
  const auto nb = [&](const uint32_t* q) { return LOCAL ? *q : __ldcg(q); };
  int y = y0, i = i0;
  for (int q = q0; q < nwords; q += step) {
    const int par = (y + colour) & 1;
    const int ym = (y == 0) ? L - 1 : y - 1;
    const int yp = (y == L - 1) ? 0 : y + 1;
    const int ih = par ? ((i + 1 == half) ? 0 : i + 1) : ((i == 0) ? half - 1 : i - 1);
    const uint32_t s = own[PT_DBG_IDX(p, q, nwords, kDbgSpinLoad)];
    const uint32_t n0 = nb(oth + PT_DBG_IDX(p, ym * half + i, nwords, kDbgSpinLoad));
    const uint32_t n1 = nb(oth + PT_DBG_IDX(p, yp * half + i, nwords, kDbgSpinLoad));
    const uint32_t n2 = nb(oth + PT_DBG_IDX(p, q, nwords, kDbgSpinLoad));
    const uint32_t n3 = nb(oth + PT_DBG_IDX(p, y * half + ih, nwords, kDbgSpinLoad));
    const uint32_t site = (uint32_t)(y * L + 2 * i + par);
    const SiteTerms st = site_terms(site, c3, rk);
    const auto draw = [&](int j) { return philox_site_block(st, bt, j, rk); };
    uint32_t ns;
    if (MODE == kModeFerro)
      ns = update_word_ferro_smem(s, n0, n1, n2, n3, nblk, thr, alw0, alw1, used, draw);
    else if (five)
      ns = update_word_generic_cmp<5>(s, n0, n1, n2, n3, nblk, gen, cls5, draw);
    else
      ns = update_word_generic_with(s, n0, n1, n2, n3, nblk, gen, draw);
    if (PT_DBG_STORE(p, q, nwords, own_base, t, colour)) own[q] = ns;
    if (COUNT) {
      const NbCount k = count4(ns ^ n0, ns ^ n1, ns ^ n2, ns ^ n3);
      U.add3(k.b0, k.b1, k.b2);
      if (MODE != kModeFerro || ones) N.add2(ns ^ n0, ns & n0);
    }
    i += di;
    y += dy;
    if (i >= half) {
      i -= half;
      y += 1;
    }
  }
}

// The band form of the persistent sweep (FORM == kFormBand). CTA b of a plane's G CTAs owns
// the rows [y0, y0 + H) of the plane, y0 = b L / G, and keeps them in shared memory: C0
// holds colour 0 of rows y0 - 1 .. y0 + H (its band and one halo row on either side), C1
// colour 1 of its band. Colour 0 is updated on all H + 2 rows of C0: the band's own rows are
// also stored to global memory, the two halo rows belong to the neighbouring bands and are
// computed here a second time from the same inputs (the same colour-1 neighbours, the same
// Philox draws), so they equal the owners' words bit for bit and stay in shared memory. Colour
// 1 of the band then reads all its colour-0 neighbours from C0, after a block barrier only:
// a sweep needs one grid barrier (before the next sweep's colour 0 reads the neighbouring
// bands' colour-1 rows) instead of two.
// With no grid barrier between the colours, a band may store its new colour 1 while a slower
// neighbour still reads the old one for its halo rows. So colour 1 lives in two global copies,
// the spin array and p.band_c1, and the sweeps of a launch alternate: sweep j stores colour 1
// in one copy (c1_dst) while colour 0 reads the other bands' colour 1 of sweep j - 1 from the
// other (c1_src). A copy is stored again only in sweep j + 2, after the grid barrier that
// ends sweep j + 1, when every band has finished reading it. The launch leaves colour 1 in
// the spin array (c1_to_spins: c1_dst is the spin array).
template <int MODE, int COLOUR, bool COUNT>
__device__ __forceinline__ void band_pass(const DevProblem& p, int w, uint64_t t,
                                          const RoundKeys& rk, const BlockTerms& bt, int y0,
                                          int H, uint32_t* C0, uint32_t* C1,
                                          const uint32_t* c1_src, uint32_t* c1_dst,
                                          bool c1_to_spins, const uint4* thr,
                                          uint32_t alw0, uint32_t alw1, uint32_t used,
                                          const PlaneGeneric& gen, bool five,
                                          const int (&cls5)[5], bool ones,
                                          BitCounter<15, 10>& U, BitCounter<15, 10>& N) {
  const uint32_t c3 = kTagSpin | ((uint32_t)(t >> 32) << 8);
  const int L = p.L, half = L >> 1;
  const int nwords = L * half;
  const int nblk = (min(32, p.R - 32 * w) + 3) >> 2;
  const size_t own_base = word_index(L, w, COLOUR, 0, 0);
  uint32_t* const g_own = COLOUR == 0 ? p.spins + own_base : c1_dst;
  (void)nwords;
  (void)c1_to_spins;
  // a colour-1 word as a neighbour of colour 0: the band's rows from C1, the others from
  // the copy the last sweep stored (before the last grid barrier; read through L2)
  const auto c1_word = [&](int yy, int ii) -> uint32_t {
    int d = yy - y0;
    if (d < 0) d += L;
    return d < H ? C1[d * half + ii]
                 : __ldcg(c1_src + PT_DBG_IDX(p, yy * half + ii, nwords, kDbgSpinLoad));
  };
  const int n = (COLOUR == 0 ? H + 2 : H) * half;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int r = k / half, i = k - r * half;
    int y = COLOUR == 0 ? y0 - 1 + r : y0 + r;
    if (y < 0) y += L;
    if (y >= L) y -= L;
    const int par = (y + COLOUR) & 1;
    const int ih = par ? ((i + 1 == half) ? 0 : i + 1) : ((i == 0) ? half - 1 : i - 1);
    uint32_t s, n0, n1, n2, n3;
    if (COLOUR == 0) {
      const int ym = (y == 0) ? L - 1 : y - 1;
      const int yp = (y == L - 1) ? 0 : y + 1;
      s = C0[k];
      n0 = c1_word(ym, i);
      n1 = c1_word(yp, i);
      n2 = c1_word(y, i);
      n3 = c1_word(y, ih);
    } else {
      s = C1[k];
      n0 = C0[r * half + i];        // row y - 1
      n1 = C0[(r + 2) * half + i];  // row y + 1
      n2 = C0[(r + 1) * half + i];  // row y
      n3 = C0[(r + 1) * half + ih];
    }
    const uint32_t site = (uint32_t)(y * L + 2 * i + par);
    const SiteTerms st = site_terms(site, c3, rk);
    const auto draw = [&](int j) { return philox_site_block(st, bt, j, rk); };
    uint32_t ns;
    if (MODE == kModeFerro)
      ns = update_word_ferro_smem(s, n0, n1, n2, n3, nblk, thr, alw0, alw1, used, draw);
    else if (five)
      ns = update_word_generic_cmp<5>(s, n0, n1, n2, n3, nblk, gen, cls5, draw);
    else
      ns = update_word_generic_with(s, n0, n1, n2, n3, nblk, gen, draw);
    const int q = y * half + i;
    if (COLOUR == 0) {
      C0[k] = ns;
      if (r >= 1 && r <= H && PT_DBG_STORE(p, q, nwords, own_base, t, COLOUR)) g_own[q] = ns;
    } else {
      C1[k] = ns;
      if (c1_to_spins ? PT_DBG_STORE(p, q, nwords, own_base, t, COLOUR)
                      : (PT_DBG_CHECK(p, q, nwords, kDbgSpinStore), true))
        g_own[q] = ns;
    }
    if (COUNT) {
      const NbCount kk = count4(ns ^ n0, ns ^ n1, ns ^ n2, ns ^ n3);
      U.add3(kk.b0, kk.b1, kk.b2);
      if (MODE != kModeFerro || ones) N.add2(ns ^ n0, ns & n0);
    }
  }
}

template <int MODE, bool CLUSTER, int FORM>
__global__ void __launch_bounds__(kPersistThreads, 2) k_persist(const __grid_constant__ PersistArgs a) {
  constexpr bool LOCAL = FORM == kFormLocal;
  constexpr bool BAND = FORM == kFormBand;
  // [R] ferro thresholds (k = 0, k = 1) by temperature, then [R] slot_of_temp and [R]
  // temp_of_slot; persist_smem(R, mode) bytes; then (LOCAL) the plane's L * L words or
  // (BAND) the band's C0 and C1 words
  extern __shared__ __align__(16) int32_t map_s[];
  __shared__ PlaneFerro fer;
  __shared__ uint4 thr[16];  // ferro thresholds, interleaved for 16-byte broadcast loads
  __shared__ __align__(16) PlaneGeneric gen;  // rows read four slots at a time
  __shared__ uint32_t acc[2][32];
  __shared__ int ok_s;
  const DevProblem& p = a.p;
  const int R = p.R, W = p.W;
  ulonglong2* const Tf = reinterpret_cast<ulonglong2*>(map_s);
  int32_t* sot = map_s + (MODE == kModeFerro ? 4 * R : 0);
  int32_t* tos = sot + R;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    sot[r] = p.slot_of_temp[r];
    tos[r] = p.temp_of_slot[r];
    if (MODE == kModeFerro)
      Tf[r] = make_ulonglong2(p.T_temp[(size_t)r * kClasses + 1], p.T_temp[(size_t)r * kClasses + 3]);
  }
  __syncthreads();

  const int w = blockIdx.x % W;
  const int plane_words = p.L * p.L;
  uint32_t* const plane_g = p.spins + word_index(p.L, w, 0, 0, 0);
  // after the persist_smem(R, MODE) bytes of thresholds and maps, 16-byte aligned
  const size_t maps_bytes = (size_t)2 * R * 4 + (MODE == kModeFerro ? (size_t)R * 16 : 0);
  uint32_t* const plane_s = reinterpret_cast<uint32_t*>(
      reinterpret_cast<unsigned char*>(map_s) + ((maps_bytes + 15) & ~size_t(15)));
  uint32_t* const plane = LOCAL ? plane_s : plane_g;
  PT_DBG_CHECK(p, w, W, kDbgSpinLoad);
  if (LOCAL) {
    for (int q = threadIdx.x; q < plane_words; q += blockDim.x) plane_s[q] = plane_g[q];
    __syncthreads();
  }
  const int q0 = (blockIdx.x / W) * kPersistThreads + threadIdx.x;
  const int step = (gridDim.x / W) * kPersistThreads;
  const int half = p.L >> 1;
  // BAND: this CTA's rows [by0, by0 + bH) of the plane and their shared copies
  const int nbands = gridDim.x / W, band = blockIdx.x / W;
  const int by0 = (int)((int64_t)band * p.L / nbands);
  const int bH = (int)((int64_t)(band + 1) * p.L / nbands) - by0;
  const int bHmax = (p.L + nbands - 1) / nbands;
  uint32_t* const C0 = plane_s;                          // [(bHmax + 2) * half]
  uint32_t* const C1 = plane_s + (size_t)(bHmax + 2) * half;  // [bHmax * half]
  if (BAND) {
    const uint32_t* g0 = plane_g;
    const uint32_t* g1 = plane_g + (size_t)p.L * half;
    for (int k = threadIdx.x; k < (bH + 2) * half; k += blockDim.x) {
      const int r = k / half, i = k - r * half;
      int y = by0 - 1 + r;
      if (y < 0) y += p.L;
      if (y >= p.L) y -= p.L;
      C0[k] = g0[PT_DBG_IDX(p, y * half + i, p.L * half, kDbgSpinLoad)];
    }
    for (int k = threadIdx.x; k < bH * half; k += blockDim.x)
      C1[k] = g1[PT_DBG_IDX(p, by0 * half + k, p.L * half, kDbgSpinLoad)];
    __syncthreads();
  }
  // BAND: the sweep (within this launch) whose colour 1 was stored last
  int band_last = -1;
  // LOCAL: the plane goes back to global memory at every exit of the kernel; BAND: colour 1
  // of the band goes to the spin array if the last sweep stored it in the other copy
  const auto flush = [&]() {
    if (LOCAL) {
      __syncthreads();
      for (int q = threadIdx.x; q < plane_words; q += blockDim.x) plane_g[q] = plane_s[q];
    }
    if (BAND && band_last >= 0 && (band_last & 1) == 0) {
      uint32_t* const a1 = plane_g + (size_t)p.L * half;
      const uint64_t tl = a.t0 + (uint64_t)band_last;
      (void)tl;
      __syncthreads();
      for (int k = threadIdx.x; k < bH * half; k += blockDim.x)
        if (PT_DBG_STORE(p, by0 * half + k, p.L * half, word_index(p.L, w, 1, 0, 0), tl, 1))
          a1[by0 * half + k] = C1[k];
    }
  };
  const int y0 = q0 / half, i0 = q0 - y0 * half;
  const int dy = step / half, di = step - dy * half;
  uint32_t* const cnt_base = p.cnt + 2 * W * 32;  // three buffers of [2][W * 32]
  unsigned* const bar = p.cnt + 8 * W * 32;

  uint32_t alw0 = 0, alw1 = 0, used = 0;
  // generic: the classes with dE > 0, when there are exactly five of them (each trial is
  // then compared with all five; update_word_generic_cmp)
  const bool five = MODE != kModeFerro && __popc((uint32_t)p.cmp_classes) == 5;
  int cls5[5] = {0, 0, 0, 0, 0};
  if (five) {
    uint32_t rest = (uint32_t)p.cmp_classes;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      cls5[c] = __ffs(rest) - 1;
      rest &= rest - 1;
    }
  }
  auto load_plane = [&]() {
    stage_plane<MODE>(p, tos, w, fer, gen, Tf);
    if (MODE == kModeFerro) {
      if (threadIdx.x < 16) {
        const int b = 2 * threadIdx.x;
        thr[threadIdx.x] = make_uint4(fer.T0[b], fer.T1[b], fer.T0[b + 1], fer.T1[b + 1]);
      }
      alw0 = fer.alw0;
      alw1 = fer.alw1;
      used = fer.used;
      __syncthreads();
    }
  };
  load_plane();

  const bool trace = p.trace_E != nullptr;
  const bool solo = gridDim.x == 1;  // then W == 1: one CTA holds every count
  unsigned counted = 0;  // sweeps counted so far in this launch
  unsigned target = 0;
  uint64_t e = a.e0;
  bool exchanged = false;
  // every CTA meets every other; false when a bounded wait gave up (the kernel then ends)
  auto sync_all = [&](unsigned extra) -> bool {
    if (CLUSTER) {
      cooperative_groups::this_cluster().sync();
      return true;
    }
    target += gridDim.x + extra;
    return grid_barrier(bar, target, p.status, a.limit_ns, &ok_s, a.stall != 0);
  };
  // between half sweeps: LOCAL planes are read by their own CTA only
  const auto sync_half = [&](unsigned extra) -> bool {
    if (LOCAL && extra == 0) {
      __syncthreads();
      return true;
    }
    return sync_all(extra);
  };
  bool tail_met = false;  // the CTAs met at a grid barrier after the last sweep done
  uint32_t* const band_a1 = plane_g + (size_t)p.L * half;  // colour 1 in the spin array
  uint32_t* const band_b1 = BAND ? p.band_c1 + (size_t)w * p.L * half : nullptr;
  // sweeps left before the next one that a swap iteration follows (0: this one): one 64-bit
  // remainder per launch instead of one per sweep (measured: L = 16, R = 8 1.41 -> 1.27 us
  // per sweep, L = 128, R = 32 5.90 -> 5.75 us)
  int until_ex = a.m > 0 ? (int)((uint64_t)(a.m - 1) - a.t0 % (uint64_t)a.m) : -1;
  for (int j = 0; j < a.n; ++j) {
    const uint64_t t = a.t0 + (uint64_t)j;
    // BAND: sweep j stores colour 1 in the spin array when j is odd, in the other copy when
    // j is even, and reads the other bands' colour 1 of sweep j - 1 from the other one
    uint32_t* const c1_dst = (j & 1) ? band_a1 : band_b1;
    const uint32_t* const c1_src = (j & 1) ? band_b1 : band_a1;
    BlockTerms bt;
    block_terms((uint32_t)(8 * w), (uint32_t)t, a.rk, bt);
    BitCounter<15, 10> U, N;
    // the stall test hook applies to the launch's first grid barrier: after colour 0, or in
    // the band form (no grid barrier between the colours) after colour 1
    const unsigned stall0 = j == 0 ? (unsigned)a.stall : 0u;
    if (BAND) {
      band_pass<MODE, 0, false>(p, w, t, a.rk, bt, by0, bH, C0, C1, c1_src, c1_dst, (j & 1) != 0,
                                thr, alw0, alw1, used, gen,
                                five, cls5, false, U, N);
      __syncthreads();
    } else {
      half_pass<MODE, false, LOCAL>(p, plane, w, 0, t, a.rk, bt, q0, step, y0, i0, dy, di, thr,
                                    alw0, alw1, used, gen, five, cls5, false, U, N);
      if (!sync_half(stall0)) return flush();
    }
    const bool ex = until_ex == 0;  // (t + 1) % m == 0
    if (a.m > 0) until_ex = ex ? a.m - 1 : until_ex - 1;
    if (!ex && !trace) {
      if (BAND)
        band_pass<MODE, 1, false>(p, w, t, a.rk, bt, by0, bH, C0, C1, c1_src, c1_dst,
                                  (j & 1) != 0, thr, alw0, alw1, used,
                                  gen, five, cls5, false, U, N);
      else
        half_pass<MODE, false, LOCAL>(p, plane, w, 1, t, a.rk, bt, q0, step, y0, i0, dy, di,
                                      thr, alw0, alw1, used, gen, five, cls5, false, U, N);
      band_last = j;
      tail_met = false;
      if (j + 1 == a.n) break;  // the kernel's end orders this half sweep before what follows
      if (!sync_half(BAND ? stall0 : 0u)) return flush();
      continue;
    }
    // a swap iteration or a trace row follows: count this sweep into buffer `counted % 3`
    // (the three buffers take turns between counted sweeps)
    uint32_t* const cb = cnt_base + (counted % 3) * 2 * W * 32;
    U.zero();
    N.zero();
    if (BAND)
      band_pass<MODE, 1, true>(p, w, t, a.rk, bt, by0, bH, C0, C1, c1_src, c1_dst, (j & 1) != 0,
                               thr, alw0, alw1, used, gen,
                               five, cls5, trace, U, N);
    else
      half_pass<MODE, true, LOCAL>(p, plane, w, 1, t, a.rk, bt, q0, step, y0, i0, dy, di, thr,
                                   alw0, alw1, used, gen, five, cls5, trace, U, N);
    band_last = j;
    const uint32_t u = U.warp_total_for_lane();
    const uint32_t nn = (MODE == kModeFerro && !trace) ? 0u : N.warp_total_for_lane();
    if (threadIdx.x < 64) (&acc[0][0])[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    if (u) atomicAdd(&acc[0][lane], u);
    if (nn) atomicAdd(&acc[1][lane], nn);
    __syncthreads();
    // a grid of one CTA (one plane) keeps its counts in shared memory: acc has the layout
    // of a count buffer with W = 1, and no other CTA needs them
    if (!solo && threadIdx.x < 32) {
      if (acc[0][threadIdx.x])
        atomicAdd(&cb[PT_DBG_IDX(p, w * 32 + threadIdx.x, 2 * W * 32, kDbgCount)],
                  acc[0][threadIdx.x]);
      if (acc[1][threadIdx.x])
        atomicAdd(&cb[PT_DBG_IDX(p, W * 32 + w * 32 + threadIdx.x, 2 * W * 32, kDbgCount)],
                  acc[1][threadIdx.x]);
    }
    if (!sync_all(BAND ? stall0 : 0u)) return flush();
    tail_met = true;  // every CTA is done with sweep j
    if (ex) {
      if (solo)
        exchange_local<true>(p, e, &acc[0][0], sot, tos, true);
      else
        exchange_local<false>(p, e, cb, sot, tos, blockIdx.x == 0);
    }
    if (blockIdx.x == 0) {
      if (trace) {
        // the trace row of sweep t, by temperature index after its swap iteration
        const int64_t L2 = (int64_t)p.L * p.L;
        const int64_t row = (int64_t)((t - p.trace_t0) % (uint64_t)p.trace_cap);
        for (int r = threadIdx.x; r < R; r += blockDim.x) {
          const int64_t U_r = solo ? acc[0][r] : __ldcg(cb + r);
          const int64_t ones = solo ? acc[1][r] : __ldcg(cb + W * 32 + r);
          const int64_t at = PT_DBG_IDX(p, row * R + tos[r], p.trace_cap * R, kDbgTrace);
          p.trace_E[at] = slot_energy(p, L2, U_r, ones);
          p.trace_M[at] = 2 * ones - L2;
        }
      }
      // buffer (counted + 2) % 3 was last read after counted sweep counted - 1, which every
      // CTA finished before it arrived at this sweep's barrier, and is next written in
      // counted sweep counted + 2, after at least one more grid barrier. (With two buffers
      // the band form, whose only barrier ends the sweep, could count the next sweep into
      // the buffer before block 0 cleared it.)
      if (!solo) {
        uint32_t* const nb = cnt_base + ((counted + 2) % 3) * 2 * W * 32;
        for (int q = threadIdx.x; q < 2 * W * 32; q += blockDim.x) nb[q] = 0;
      }
    }
    ++counted;
    if (ex) {
      load_plane();
      e += 1;
      exchanged = true;
    }
  }

  // BAND: when the last sweep's index is even, it stored colour 1 in the other copy, and the
  // spin array still holds the colour 1 that the other bands read for their halo rows in that
  // sweep (its c1_src). Only after every CTA is done with the sweep may a band copy its new
  // colour 1 back into the spin array. (A launch whose last sweep ends with a swap iteration
  // or a trace row has met at that sweep's barrier already; one that ends without must meet
  // here.)
  if (BAND && band_last >= 0 && (band_last & 1) == 0 && !tail_met)
    if (!sync_all(0u)) return flush();
  flush();
  if (exchanged) {
    if (blockIdx.x == 0)
      for (int r = threadIdx.x; r < R; r += blockDim.x) {
        p.slot_of_temp[r] = sot[r];
        p.temp_of_slot[r] = tos[r];
      }
    if (blockIdx.x < W) {  // one CTA per plane writes the plane's table back
      if (MODE == kModeFerro) {
        PlaneFerro* dst = reinterpret_cast<PlaneFerro*>(p.planes) + w;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&fer);
        for (int q = threadIdx.x; q < (int)(sizeof(PlaneFerro) / 4); q += blockDim.x)
          reinterpret_cast<uint32_t*>(dst)[q] = src[q];
      } else {
        PlaneGeneric* dst = reinterpret_cast<PlaneGeneric*>(p.planes) + w;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&gen);
        for (int q = threadIdx.x; q < (int)(sizeof(PlaneGeneric) / 4); q += blockDim.x)
          reinterpret_cast<uint32_t*>(dst)[q] = src[q];
      }
    }
  }
}

const void* persist_fn(int mode, bool cluster = false, int form = kFormStrided) {
  const bool f = mode == kModeFerro;
  if (cluster) {
    if (form == kFormBand)
      return f ? (const void*)k_persist<kModeFerro, true, kFormBand>
               : (const void*)k_persist<kModeGeneric, true, kFormBand>;
    return f ? (const void*)k_persist<kModeFerro, true, kFormStrided>
             : (const void*)k_persist<kModeGeneric, true, kFormStrided>;
  }
  if (form == kFormLocal)
    return f ? (const void*)k_persist<kModeFerro, false, kFormLocal>
             : (const void*)k_persist<kModeGeneric, false, kFormLocal>;
  if (form == kFormBand)
    return f ? (const void*)k_persist<kModeFerro, false, kFormBand>
             : (const void*)k_persist<kModeGeneric, false, kFormBand>;
  return f ? (const void*)k_persist<kModeFerro, false, kFormStrided>
           : (const void*)k_persist<kModeGeneric, false, kFormStrided>;
}

}  // namespace

size_t persist_smem(int R, int mode) {
  return (size_t)2 * R * sizeof(int32_t) + (mode == kModeFerro ? (size_t)R * 16 : 0);
}

// Shared words of a band-form CTA: C0 (its rows and two halo rows of colour 0) and C1 (its
// rows of colour 1), for the largest band of `bands` bands of L rows.
static size_t band_bytes(int L, int bands) {
  const size_t hmax = (size_t)((L + bands - 1) / bands);
  return (2 * hmax + 2) * (size_t)(L / 2) * sizeof(uint32_t);
}

size_t persist_launch_smem(int L, int R, int mode, int form, int bands) {
  const size_t base = persist_smem(R, mode);
  const size_t at = (base + 15) & ~size_t(15);
  if (form == kFormLocal) return at + (size_t)L * L * sizeof(uint32_t);
  if (form == kFormBand) return at + band_bytes(L, bands);
  return base;
}

cudaError_t persist_plan(const DevProblem& p, const DeviceInfo& dev, int words_per_thread,
                         int band, PersistPlan* plan) {
  plan->grid = 0;
  plan->words_per_thread = 0;
  plan->cluster = false;
  plan->local = false;
  plan->band = false;
  int per_sm = 0;
  // the maps and (ferro) the thresholds by temperature can pass the default 48 KB per block.
  // The limit belongs to the kernel, not to a problem: it is set to what the largest
  // problem needs, so that planning a smaller one never lowers it under a larger one's launch
  cudaError_t err = cudaSuccess;
  for (int c = 0; c < 2 && err == cudaSuccess; ++c)
    err = cudaFuncSetAttribute(persist_fn(p.mode, c == 1),
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)persist_smem(PT_MAX_R, p.mode));
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(persist_fn(p.mode, false, kFormLocal),
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(((persist_smem(PT_MAX_R, p.mode) + 15) & ~size_t(15)) +
                                     kPersistMaxLocalBytes));
  for (int c = 0; c < 2 && err == cudaSuccess; ++c)
    err = cudaFuncSetAttribute(persist_fn(p.mode, c == 1, kFormBand),
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(((persist_smem(PT_MAX_R, p.mode) + 15) & ~size_t(15)) +
                                     kPersistMaxBandBytes));
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(persist_fn(p.mode, true, kFormBand),
                               cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(persist_fn(p.mode, true),
                               cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err != cudaSuccess) return err;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_fn(p.mode),
                                                      kPersistThreads,
                                                      persist_smem(p.R, p.mode));
  if (err != cudaSuccess) return err;
  const int64_t planes_fit = (int64_t)per_sm * dev.sms / p.W;  // CTAs per plane at most
  if (planes_fit < 1) return cudaSuccess;
  const int64_t words = (int64_t)p.L * (p.L / 2);  // per colour and plane
  const int64_t per_cta = (int64_t)words_per_thread * kPersistThreads;
  int64_t g = (words + per_cta - 1) / per_cta;
  if (g > planes_fit) g = planes_fit;
  if (g < 1) g = 1;
  const int64_t wpt = (words + g * kPersistThreads - 1) / (g * kPersistThreads);
  if (wpt > kPersistMaxWordsPerThread) return cudaSuccess;
  plan->grid = (int)(g * p.W);
  plan->words_per_thread = (int)wpt;
  if (band != kBandNever) {
    // the band form: gb bands of rows per plane. A band of H rows updates H + 2 rows of
    // colour 0 and H of colour 1; with the default of one word per thread, H is the largest
    // height whose colour-0 rows a CTA takes in one pass (at least one row), so that a sweep
    // is one pass of each colour and one grid barrier. gb >= 2 (a band and its two halo rows
    // never wrap onto themselves when L >= 4); the shared copies must fit and every CTA stay
    // resident.
    const int64_t half_w = p.L / 2;
    int64_t H = words_per_thread <= 1
                    ? std::max<int64_t>(1, kPersistThreads / half_w - 2)
                    : std::max<int64_t>(1, (int64_t)words_per_thread * kPersistThreads / half_w);
    int64_t gb = std::max<int64_t>(2, (p.L + H - 1) / H);
    if (gb > planes_fit) {  // taller bands, so that every CTA stays resident
      H = (p.L + planes_fit - 1) / planes_fit;
      gb = (p.L + H - 1) / H;
    }
    int per_sm_band = 0;
    bool fits = gb >= 2 && gb <= planes_fit;
    if (fits) fits = band_bytes(p.L, (int)gb) <= (size_t)kPersistMaxBandBytes;
    if (fits) {
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm_band, persist_fn(p.mode, false, kFormBand), kPersistThreads,
          persist_launch_smem(p.L, p.R, p.mode, kFormBand, (int)gb));
      if (err != cudaSuccess) return err;
      fits = (int64_t)per_sm_band * dev.sms >= gb * p.W;
    }
    const bool coop = g * p.W > kPersistMaxCluster;  // the strided form's grid
    plan->band = fits && (band == kBandForce ||
                          (coop && words_per_thread <= 1 && half_w <= kBandAutoMaxHalf));
    if (plan->band) {
      plan->grid = (int)(gb * p.W);
      plan->words_per_thread = (int)(((H + 2) * half_w + kPersistThreads - 1) / kPersistThreads);
    } else if (band == kBandForce) {
      plan->grid = 0;
      return cudaSuccess;
    }
  }
  if (!plan->band && g == 1 && (int64_t)p.L * p.L * 4 <= kPersistMaxLocalBytes) {
    // one CTA per plane: its plane in shared memory, if every plane's CTA stays resident
    int per_sm_local = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm_local, persist_fn(p.mode, false, kFormLocal), kPersistThreads,
        persist_launch_smem(p.L, p.R, p.mode, kFormLocal, 1));
    if (err != cudaSuccess) return err;
    if ((int64_t)per_sm_local * dev.sms >= plan->grid) {
      plan->local = true;
      return cudaSuccess;
    }
  }
  if (plan->grid >= 2 && plan->grid <= kPersistMaxCluster) {
    // one cluster of the whole grid, if the device can place one (a single CTA keeps the
    // cooperative launch, whose barrier is then the block barrier)
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)plan->grid;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    const int form = plan->band ? kFormBand : kFormStrided;
    cfg.gridDim = dim3((unsigned)plan->grid);
    cfg.blockDim = dim3(kPersistThreads);
    cfg.dynamicSmemBytes = persist_launch_smem(p.L, p.R, p.mode, form, plan->grid / p.W);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    err = cudaOccupancyMaxActiveClusters(&clusters, persist_fn(p.mode, true, form), &cfg);
    if (err != cudaSuccess) {
      cudaGetLastError();  // not placeable: keep the cooperative launch
      return cudaSuccess;
    }
    plan->cluster = clusters >= 1;
  }
  return cudaSuccess;
}

cudaError_t launch_persist(const DevProblem& p, const PersistPlan& plan, uint64_t t0,
                           uint64_t e0, int n, int m, int stall, uint64_t limit_ns,
                           cudaStream_t st) {
  // the two count buffers and the barrier counter follow the per-launch kernels' counts
  cudaError_t err = cudaMemsetAsync(p.cnt + 2 * p.W * 32, 0, persist_clear_bytes(p.W), st);
  if (err != cudaSuccess) return err;
  PersistArgs a;
  a.p = p;
  a.t0 = t0;
  a.e0 = e0;
  a.n = n;
  a.m = m;
  a.stall = stall;
  a.limit_ns = limit_ns;
  for (int r = 0; r < 10; ++r) {
    a.rk.k0[r] = p.key0 + (uint32_t)r * kPhiloxW0;
    a.rk.k1[r] = p.key1 + (uint32_t)r * kPhiloxW1;
  }
  void* args[] = {&a};
  const int form = plan.band ? kFormBand : (plan.local ? kFormLocal : kFormStrided);
  if (plan.cluster && stall == 0) {
    // the test hook (stall) needs the counting barrier: it waits for a CTA that never comes
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)plan.grid;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)plan.grid);
    cfg.blockDim = dim3(kPersistThreads);
    cfg.dynamicSmemBytes = persist_launch_smem(p.L, p.R, p.mode, form, plan.grid / p.W);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, persist_fn(p.mode, true, form), args);
  }
  return cudaLaunchCooperativeKernel(persist_fn(p.mode, false, form), dim3(plan.grid),
                                     dim3(kPersistThreads), args,
                                     persist_launch_smem(p.L, p.R, p.mode, form,
                                                         plan.grid / p.W), st);
}

}  // namespace ptb
