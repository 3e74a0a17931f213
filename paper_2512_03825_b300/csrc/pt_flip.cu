// pt_flip.cu -- the single-spin-flip variant: the paper's "iteration" read as one Metropolis
// trial at one uniformly chosen site of each replica (Sec. 2.1: the trial state flips one
// spin; Eq. 1 accepts it), the scheme of the paper's own CUDA program, where one thread runs
// one replica.
//
// One cooperative launch per pt_flip call; thread r runs the replica in slot r. Iteration i
// draws one Philox block with the counters {lo32(i), r, 0, TAG_FLIP | hi32(i) << 8}: word 0
// picks the site floor(u0 * L^2 / 2^32) (row-major), word 1 is compared with the threshold
// of the trial's class (anti-aligned neighbours k, sign of the spin) at the slot's current
// temperature -- the same integer thresholds as a sweep's trials. The 32 replicas of a
// plane share each spin word, so a flip is an atomic XOR of the replica's bit, and every
// spin word is read through L2. Each thread keeps its replica's E_int and M, updated by the
// exact integer Delta E of every accepted flip.
//
// After every iteration that leaves the iteration count a multiple of m, all threads store
// their energies, meet at a bounded grid barrier, and every CTA computes the same swap
// iteration (Sec. 3) on its own copy of the temperature map; block 0 keeps the statistics.
// The energies alternate between two buffers, so a fast CTA storing the next ones never
// overwrites those another CTA still reads.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pt.h"
#include "pt_debug.cuh"
#include "pt_device.cuh"
#include "pt_flip.h"
#include "pt_grid.cuh"

namespace ptb {

namespace {

constexpr int kFlipThreads = 64;

struct FlipArgs {
  DevProblem p;
  uint64_t it0, e0;
  int64_t n;  // iterations in this launch
  int m;      // swap iteration after every m-th iteration (0: never)
  int stall;  // test support: the first barrier waits for this many CTAs more
  uint64_t limit_ns;
  RoundKeys rk;
};

// Swap iteration e from the slots' energies eb[R], on this CTA's copy of the maps; `owner`
// also counts attempts and acceptances. All decisions first (their loads independent of one
// another), then the swaps: a thread takes at most 32 pairs (R <= 2048, 32 threads).
__device__ void exchange_energies(const DevProblem& p, uint64_t e, const int64_t* eb,
                                  int32_t* sot, int32_t* tos, bool owner) {
  const int R = p.R;
  const int parity = (int)(e & 1);
  const uint32_t c3 = kTagExch | ((uint32_t)(e >> 32) << 8);
  const int stride = 2 * (int)blockDim.x;
  uint32_t accepted = 0;  // bit q: pair parity + 2 * threadIdx.x + q * stride accepted
#pragma unroll 4
  for (int q = 0; q < 32; ++q) {
    const int k = parity + 2 * (int)threadIdx.x + q * stride;
    if (k + 1 < R) {
      const int64_t n = __ldcg(eb + sot[k]) - __ldcg(eb + sot[k + 1]);
      const SwapPair sp = p.pairs[k];
      const uint64_t S = pair_threshold(sp, p.swap_table, p.table_shift, n);
      const Philox4 rnd = philox4x32_10((uint32_t)k, (uint32_t)e, 0u, c3, p.key0, p.key1);
      if ((uint64_t)rnd.x < S) accepted |= 1u << q;
    }
  }
  __syncthreads();
  for (int q = 0; q < 32; ++q) {
    const int k = parity + 2 * (int)threadIdx.x + q * stride;
    if (k + 1 >= R) break;
    const bool accept = (accepted >> q) & 1u;
    if (owner) count_swap(p.attempted, p.accepted, k, accept);
    if (accept) {
      const int a = sot[k], b = sot[k + 1];
      sot[k] = b;
      sot[k + 1] = a;
      tos[a] = k + 1;
      tos[b] = k;
    }
  }
  __syncthreads();
}

// The energy-independent part of one thread's pairs of swap iteration e -- each pair's
// table bounds and its draw -- for a block of 256 threads: pairs of one parity lie 512 apart,
// so a thread has at most 4 (R <= 2048). Read before the swap's grid barrier, so that after
// it only the energies and the table entries remain to be fetched.
constexpr int kSwapPerThread = 4;
struct SwapPrefetch {
  SwapPair sp[kSwapPerThread];
  uint32_t u[kSwapPerThread];
};

__device__ __forceinline__ void prefetch_swaps(const DevProblem& p, uint64_t e, SwapPrefetch& pf) {
  const int parity = (int)(e & 1);
  const uint32_t c3 = kTagExch | ((uint32_t)(e >> 32) << 8);
#pragma unroll
  for (int q = 0; q < kSwapPerThread; ++q) {
    const int k = parity + 2 * (int)threadIdx.x + q * 2 * (int)blockDim.x;
    if (k + 1 < p.R) {
      pf.sp[q] = p.pairs[k];
      pf.u[q] = philox4x32_10((uint32_t)k, (uint32_t)e, 0u, c3, p.key0, p.key1).x;
    }
  }
}

// exchange_energies from prefetched pair data (blockDim.x = 256).
__device__ void exchange_prefetched(const DevProblem& p, uint64_t e, const int64_t* eb,
                                    int32_t* sot, int32_t* tos, bool owner,
                                    const SwapPrefetch& pf) {
  const int R = p.R;
  const int parity = (int)(e & 1);
  const int stride = 2 * (int)blockDim.x;
  uint32_t accepted = 0;  // bit q: pair parity + 2 * threadIdx.x + q * stride accepted
#pragma unroll
  for (int q = 0; q < kSwapPerThread; ++q) {
    const int k = parity + 2 * (int)threadIdx.x + q * stride;
    if (k + 1 < R) {
      const int64_t n = __ldcg(eb + sot[k]) - __ldcg(eb + sot[k + 1]);
      const SwapPair& sp = pf.sp[q];
      const uint64_t S = pair_threshold(sp, p.swap_table, p.table_shift, n);
      if ((uint64_t)pf.u[q] < S) accepted |= 1u << q;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kSwapPerThread; ++q) {
    const int k = parity + 2 * (int)threadIdx.x + q * stride;
    if (k + 1 >= R) break;
    const bool accept = (accepted >> q) & 1u;
    if (owner) count_swap(p.attempted, p.accepted, k, accept);
    if (accept) {
      const int a = sot[k], b = sot[k + 1];
      sot[k] = b;
      sot[k + 1] = a;
      tos[a] = k + 1;
      tos[b] = k;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kFlipThreads) k_flip(const __grid_constant__ FlipArgs a) {
  extern __shared__ int32_t map_s[];  // [R] slot_of_temp, then [R] temp_of_slot
  __shared__ int ok_s;
  const DevProblem& p = a.p;
  const int R = p.R, L = p.L, half = L >> 1;
  int32_t* sot = map_s;
  int32_t* tos = map_s + R;
  for (int q = threadIdx.x; q < R; q += blockDim.x) {
    sot[q] = p.slot_of_temp[q];
    tos[q] = p.temp_of_slot[q];
  }
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = r < R;
  int64_t E = active ? p.E_slot[r] : 0, M = active ? p.M_slot[r] : 0;
  const uint32_t bit = 1u << (r & 31);
  uint32_t* const plane = p.spins + word_index(L, active ? (r >> 5) : 0, 0, 0, 0);
  const uint64_t L2 = (uint64_t)L * (uint64_t)L;
  int64_t* const ebuf = reinterpret_cast<int64_t*>(p.cnt + 2 * p.W * 32);  // [2][R]
  unsigned* const bar = p.cnt + 6 * p.W * 32;
  unsigned target = 0;
  unsigned swaps = 0;
  uint64_t e = a.e0;
  // iterations until the next swap iteration (after every m-th iteration count)
  int64_t left = a.m > 0 ? (int64_t)a.m - (int64_t)(a.it0 % (uint64_t)a.m) : 0;
  for (int64_t j = 0; j < a.n; ++j) {
    if (active) {
      const uint64_t i = a.it0 + (uint64_t)j;
      const Philox4 u = philox4x32_10_rk((uint32_t)i, (uint32_t)r, 0u,
                                         kTagFlip | ((uint32_t)(i >> 32) << 8), a.rk);
      const uint64_t site = ((uint64_t)u.x * L2) >> 32;
      // floor(site / L) = floor(u0 L^2 / (2^32 L)) = floor(u0 L / 2^32): one high product
      const int y = (int)__umulhi(u.x, (uint32_t)L), x = (int)(site - (uint64_t)y * L);
      const int c = (x + y) & 1;
      const int xm = x == 0 ? L - 1 : x - 1, xp = x == L - 1 ? 0 : x + 1;
      const int ym = y == 0 ? L - 1 : y - 1, yp = y == L - 1 ? 0 : y + 1;
      const int pw = L * L;  // words of one plane, both colours (the debug checks' range)
      (void)pw;
      uint32_t* const sw = plane + PT_DBG_IDX(p, ((size_t)c * L + y) * half + (x >> 1), pw, kDbgFlip);
      const size_t ob = (size_t)(c ^ 1) * L * half;  // the other colour's first word
      const uint32_t s0 = __ldcg(sw) & bit;
      const int k =
          (((__ldcg(plane + PT_DBG_IDX(p, ob + (size_t)y * half + (xm >> 1), pw, kDbgFlip)) & bit) ^ s0) != 0) +
          (((__ldcg(plane + PT_DBG_IDX(p, ob + (size_t)y * half + (xp >> 1), pw, kDbgFlip)) & bit) ^ s0) != 0) +
          (((__ldcg(plane + PT_DBG_IDX(p, ob + (size_t)ym * half + (x >> 1), pw, kDbgFlip)) & bit) ^ s0) != 0) +
          (((__ldcg(plane + PT_DBG_IDX(p, ob + (size_t)yp * half + (x >> 1), pw, kDbgFlip)) & bit) ^ s0) != 0);
      const int up = s0 != 0;
      const uint64_t T = p.T_temp[(size_t)tos[r] * kClasses + 2 * k + up];
      if ((uint64_t)u.y < T) {
        atomicXor(sw, bit);
        const int64_t sigma = up ? 1 : -1;
        // Delta E_int = 2 sigma (J_int sum_nb - h_int), sigma sum_nb = 4 - 2k
        E += 2 * (p.J_int * (4 - 2 * k) - p.h_int * sigma);
        M -= 2 * sigma;
      }
    }
    if (a.m > 0 && --left == 0) {
      left = a.m;
      int64_t* const eb = ebuf + (size_t)(swaps & 1) * R;
      if (active) eb[r] = E;
      target += gridDim.x + (swaps == 0 ? (unsigned)a.stall : 0u);
      if (!grid_barrier(bar, target, p.status, a.limit_ns, &ok_s, a.stall != 0)) return;
      exchange_energies(p, e, eb, sot, tos, blockIdx.x == 0);
      e += 1;
      swaps += 1;
    }
  }
  if (active) {
    p.E_slot[r] = E;
    p.M_slot[r] = M;
  }
  if (swaps > 0 && blockIdx.x == 0) {
    for (int q = threadIdx.x; q < R; q += blockDim.x) {
      p.slot_of_temp[q] = sot[q];
      p.temp_of_slot[q] = tos[q];
    }
  }
}

// The same iterations with each replica's lattice in shared memory. A block of 256 threads
// holds k replicas of one plane (k a power of two, so 32 / k blocks share a plane's words):
// every replica is a row-major bit array of L^2 bits (bit y*L + x) that lane l < k of warp 0
// reads and flips without atomics. All 256 threads load the arrays at the start, decide the
// swap iterations and merge the arrays back into the plane words at the end (an XOR of
// exactly the bits that changed, so the blocks sharing a word never interfere).
//
// The draws do not depend on the lattice, so warp 0 does not form them: the iterations are
// cut into chunks of at most kFlipChunk that end at every swap iteration, and while warp 0
// runs chunk q the other seven warps turn the draws of chunk q + 1 into what warp 0 needs
// -- the bit positions of the site and of its four neighbours, and the accept number u1 --
// in the other half of a two-chunk ring in shared memory; one block barrier per chunk
// hands the halves over. Warp 0 is left with the chain that really is serial (read five
// bits, count, compare, flip) and as few instructions as it can have: for h = 0 and J > 0
// the two thresholds that can decide (k = 0 and k = 1 anti-aligned neighbours) sit in
// registers, and accepted flips are tallied in 32-bit counters that are folded into E_int
// and M once per chunk.
constexpr int kFlipSmemThreads = 256;
constexpr int kFlipChunk = 32;
static_assert(2 * kFlipSmemThreads * kSwapPerThread >= PT_MAX_R,
              "each thread of k_flip_smem takes at most kSwapPerThread pairs of one parity");

// Shared-memory layout of k_flip_smem: [R] slot_of_temp, [R] temp_of_slot, [k][words] bit
// arrays, then (16-byte aligned) two rings of [2][kFlipChunk][k] entries: uint4 {bit
// positions of the site, left, right and upper neighbours} and uint2 {bit position of the
// lower neighbour, u1}.
__host__ __device__ inline size_t flip_ring_offset(int R, int k, int words) {
  return (((size_t)2 * R + (size_t)k * words) * 4 + 15) & ~size_t(15);
}
__host__ __device__ inline size_t flip_smem_bytes(int R, int k, int words) {
  return flip_ring_offset(R, k, words) + (size_t)2 * kFlipChunk * k * (16 + 8);
}

// bit b of a replica's row-major bit array (b >> 5 selects the word; the funnel shift takes
// b mod 32)
__device__ __forceinline__ uint32_t bit_at(const uint32_t* bits, uint32_t b) {
  const uint32_t w = bits[b >> 5];
  return __funnelshift_r(w, w, b) & 1u;
}

template <int MODE>
__global__ void __launch_bounds__(kFlipSmemThreads) k_flip_smem(const __grid_constant__ FlipArgs a,
                                                                int k_per_block,
                                                                int words_per_rep) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int ok_s;
  __shared__ uint64_t thr_s[kClasses][32];  // generic: lane l's thresholds at its temperature
  const DevProblem& p = a.p;
  const int R = p.R, L = p.L, half = L >> 1;
  int32_t* sot = reinterpret_cast<int32_t*>(smem);
  int32_t* tos = sot + R;
  uint32_t* const bits = smem + 2 * R;
  const size_t ring_n = (size_t)2 * kFlipChunk * k_per_block;  // entries of each ring
  uint4* const ring4 = reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(smem) +
                                                flip_ring_offset(R, k_per_block, words_per_rep));
  uint2* const ring2 = reinterpret_cast<uint2*>(ring4 + ring_n);
  const int tid = threadIdx.x;
  for (int q = tid; q < R; q += blockDim.x) {
    sot[q] = p.slot_of_temp[q];
    tos[q] = p.temp_of_slot[q];
  }
  const int r0 = blockIdx.x * k_per_block;  // first slot of this block
  const int kb = min(k_per_block, R - r0);  // replicas of this block
  const int b0 = r0 & 31;                   // their first bit in the plane words
  uint32_t* const plane = p.spins + word_index(L, r0 >> 5, 0, 0, 0);
  const int nsites = L * L;
  auto word_of = [&](int site) {
    const int y = site / L, x = site - y * L;
    return plane + PT_DBG_IDX(p, ((size_t)((x + y) & 1) * L + y) * half + (x >> 1), L * L,
                              kDbgFlip);
  };
  // bit-array word w of every replica: 32 sites, one plane word each
  for (int w = tid; w < words_per_rep; w += blockDim.x) {
    uint32_t pw[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) pw[j] = w * 32 + j < nsites ? *word_of(w * 32 + j) : 0u;
    for (int l = 0; l < kb; ++l) {
      uint32_t acc = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) acc |= ((pw[j] >> (b0 + l)) & 1u) << j;
      bits[(size_t)l * words_per_rep + w] = acc;
    }
  }
  int64_t* const ebuf = reinterpret_cast<int64_t*>(p.cnt + 2 * p.W * 32);  // [2][R]
  unsigned* const bar = p.cnt + 6 * p.W * 32;
  unsigned target = 0;
  unsigned swaps = 0;
  uint64_t e = a.e0;
  const bool active = tid < kb;  // lanes of warp 0 that own a replica
  const int r = r0 + tid;
  int64_t E = active ? p.E_slot[r] : 0, M = active ? p.M_slot[r] : 0;
  const uint32_t* const mine_c = bits + (size_t)(active ? tid : 0) * words_per_rep;
  uint32_t* const mine = bits + (size_t)(active ? tid : 0) * words_per_rep;
  const uint64_t L2 = (uint64_t)nsites;
  // thresholds of the lane's temperature (it changes only at swap iterations). Ferro:
  // accept u1 < T iff T > 0 and u1 <= T - 1, with T - 1 < 2^32. A swap moves a replica by
  // one temperature at most, so the lane also holds the two threshold pairs of the
  // temperatures next to its own (read one swap ahead, off the swap's critical path).
  uint32_t tm0 = 0, tm1 = 0;
  bool ok0 = false, ok1 = false;
  int cur_t = 0;
  uint64_t nb_lo0 = 0, nb_lo1 = 0, nb_mid0 = 0, nb_mid1 = 0, nb_hi0 = 0, nb_hi1 = 0;
  auto ferro_pair = [&](int t, uint64_t& t0, uint64_t& t1) {
    if (t >= 0 && t < R) {
      t0 = p.T_temp[(size_t)t * kClasses + 1];  // k = 0 (either spin)
      t1 = p.T_temp[(size_t)t * kClasses + 3];  // k = 1
    }
  };
  auto use_mid = [&]() {
    ok0 = nb_mid0 > 0;
    ok1 = nb_mid1 > 0;
    tm0 = (uint32_t)(nb_mid0 - 1);
    tm1 = (uint32_t)(nb_mid1 - 1);
  };
  auto stage_thresholds = [&](bool first) {
    if (!active) return;
    const int t = tos[r];
    if (MODE == kModeFerro) {
      if (first || (t != cur_t - 1 && t != cur_t && t != cur_t + 1)) {
        ferro_pair(t, nb_mid0, nb_mid1);
        ferro_pair(t - 1, nb_lo0, nb_lo1);
        ferro_pair(t + 1, nb_hi0, nb_hi1);
      } else if (t == cur_t - 1) {
        nb_hi0 = nb_mid0;
        nb_hi1 = nb_mid1;
        nb_mid0 = nb_lo0;
        nb_mid1 = nb_lo1;
        ferro_pair(t - 1, nb_lo0, nb_lo1);
      } else if (t == cur_t + 1) {
        nb_lo0 = nb_mid0;
        nb_lo1 = nb_mid1;
        nb_mid0 = nb_hi0;
        nb_mid1 = nb_hi1;
        ferro_pair(t + 1, nb_hi0, nb_hi1);
      }
      cur_t = t;
      use_mid();
    } else {
      const uint64_t* const src = p.T_temp + (size_t)t * kClasses;
#pragma unroll
      for (int c = 0; c < kClasses; ++c) thr_s[c][tid] = src[c];
    }
  };
  // iterations [j0, j1) into ring half h, by threads first, first + stride, ...
  auto produce = [&](int h, int64_t j0, int64_t j1, int first, int stride) {
    const int items = (int)(j1 - j0) * kb;
    for (int it = first; it < items; it += stride) {
      const int jj = it / kb, l = it - jj * kb;
      const uint64_t i = a.it0 + (uint64_t)(j0 + jj);
      const Philox4 u = philox4x32_10_rk((uint32_t)i, (uint32_t)(r0 + l), 0u,
                                         kTagFlip | ((uint32_t)(i >> 32) << 8), a.rk);
      const uint32_t site = (uint32_t)(((uint64_t)u.x * L2) >> 32);
      // floor(site / L) = floor(u0 L / 2^32): one high product instead of a division
      const uint32_t y = __umulhi(u.x, (uint32_t)L), x = site - y * (uint32_t)L;
      const uint32_t row = site - x;
      const uint32_t left = x == 0 ? site + (uint32_t)L - 1u : site - 1u;
      const uint32_t right = x == (uint32_t)L - 1u ? row : site + 1u;
      const uint32_t up = y == 0 ? site + (uint32_t)(nsites - L) : site - (uint32_t)L;
      const uint32_t down = y == (uint32_t)L - 1u ? x : site + (uint32_t)L;
      const size_t at = ((size_t)h * kFlipChunk + jj) * k_per_block + l;
      ring4[at] = make_uint4(site, left, right, up);
      ring2[at] = make_uint2(down, u.y);
    }
  };
  // the end of the chunk that starts at iteration j: kFlipChunk on, the end of the call, or
  // the next swap iteration, whichever comes first
  auto chunk_end = [&](int64_t j) {
    int64_t end = min(j + (int64_t)kFlipChunk, a.n);
    if (a.m > 0) end = min(end, j + (int64_t)a.m - (int64_t)((a.it0 + (uint64_t)j) % a.m));
    return end;
  };
  auto swap_point = [&]() -> bool {
    int64_t* const eb = ebuf + (size_t)(swaps & 1) * R;
    if (active) eb[r] = E;
    SwapPrefetch pf;
    prefetch_swaps(p, e, pf);
    target += gridDim.x + (swaps == 0 ? (unsigned)a.stall : 0u);
    if (!grid_barrier(bar, target, p.status, a.limit_ns, &ok_s, a.stall != 0)) return false;
    exchange_prefetched(p, e, eb, sot, tos, blockIdx.x == 0, pf);
    stage_thresholds(false);
    e += 1;
    swaps += 1;
    return true;
  };
  __syncthreads();  // maps and bit arrays in place
  stage_thresholds(true);
  int64_t j0 = 0, j1 = a.n > 0 ? chunk_end(0) : 0;
  produce(0, 0, j1, tid, blockDim.x);
  __syncthreads();
  for (int q = 0; j0 < a.n; ++q) {
    const int64_t j2 = j1 < a.n ? chunk_end(j1) : j1;  // the next chunk is [j1, j2)
    if (tid < 32) {
      if (active) {
        const size_t base = (size_t)(q & 1) * kFlipChunk * k_per_block + tid;
        // accepted flips of this chunk: their number, sum of k, sum of the flipped spins
        int nacc = 0, sumk = 0, sums = 0;
        const int len = (int)(j1 - j0);
        // the next item is read before this iteration's flip is stored (the compiler may not
        // move a shared-memory load above a shared-memory store on its own)
        uint4 na = ring4[base];
        uint2 nb = ring2[base];
        for (int jj = 0; jj < len; ++jj) {
          const uint4 pa = na;
          const uint2 pb = nb;
          if (jj + 1 < len) {
            na = ring4[base + (size_t)(jj + 1) * k_per_block];
            nb = ring2[base + (size_t)(jj + 1) * k_per_block];
          }
          const uint32_t s0 = bit_at(mine_c, pa.x);
          const int k = (int)((bit_at(mine_c, pa.y) ^ s0) + (bit_at(mine_c, pa.z) ^ s0) +
                              (bit_at(mine_c, pa.w) ^ s0) + (bit_at(mine_c, pb.x) ^ s0));
          bool accept;
          if (MODE == kModeFerro) {
            // dE <= 0 for k >= 2; the compares do not wait for the lattice
            const bool a0 = ok0 && pb.y <= tm0, a1 = ok1 && pb.y <= tm1;
            accept = k >= 2 || (k == 1 ? a1 : a0);
          } else {
            accept = (uint64_t)pb.y < thr_s[2 * k + (int)s0][tid];
          }
          if (accept) {
            mine[pa.x >> 5] ^= 1u << (pa.x & 31u);
            nacc += 1;
            sumk += k;
            sums += 2 * (int)s0 - 1;
          }
        }
        // Delta E_int = 2 sigma (J_int sum_nb - h_int) per flip, sigma sum_nb = 4 - 2k
        E += 2 * (p.J_int * (int64_t)(4 * nacc - 2 * sumk) - p.h_int * (int64_t)sums);
        M -= 2 * (int64_t)sums;
      }
    } else if (j1 < a.n) {
      produce((q + 1) & 1, j1, j2, tid - 32, blockDim.x - 32);
    }
    __syncthreads();  // chunk q done, chunk q + 1's items in place
    if (a.m > 0 && (a.it0 + (uint64_t)j1) % (uint64_t)a.m == 0)
      if (!swap_point()) return;
    j0 = j1;
    j1 = j2;
  }
  __syncthreads();
  // merge: site s gets this block's bits, changed ones XORed into the plane word (only this
  // block changes them, and not before this point)
  const unsigned lanes = k_per_block >= 32 ? 0xffffffffu : ((1u << k_per_block) - 1u);
  const uint32_t mask = lanes << b0;
  for (int site = tid; site < nsites; site += blockDim.x) {
    uint32_t now = 0;
    for (int l = 0; l < kb; ++l)
      now |= ((bits[(size_t)l * words_per_rep + (site >> 5)] >> (site & 31)) & 1u) << (b0 + l);
    uint32_t* const wp = word_of(site);
    const uint32_t delta = (__ldcg(wp) ^ now) & mask;
    if (delta) atomicXor(wp, delta);
  }
  if (active) {
    p.E_slot[r] = E;
    p.M_slot[r] = M;
  }
  if (swaps > 0 && blockIdx.x == 0) {
    for (int q = tid; q < R; q += blockDim.x) {
      p.slot_of_temp[q] = sot[q];
      p.temp_of_slot[q] = tos[q];
    }
  }
}

const void* flip_smem_fn(int mode) {
  return mode == kModeFerro ? (const void*)k_flip_smem<kModeFerro>
                            : (const void*)k_flip_smem<kModeGeneric>;
}

}  // namespace

int flip_smem_plan(const DevProblem& p, int sms, size_t smem_optin, int* k_out, size_t* bytes_out) {
  *k_out = 0;
  *bytes_out = 0;
  if (p.L > 65535) return PT_OK;  // the draw ring packs row and column in 16 bits each
  const int words = (p.L * p.L + 31) / 32;
  const void* fn = flip_smem_fn(p.mode);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return PT_ECUDA;
  if (fa.sharedSizeBytes >= smem_optin) return PT_OK;
  // the limit belongs to the kernel, not to a problem: set to all the device allows, so that
  // planning one problem never lowers it under another problem's launch
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(smem_optin - fa.sharedSizeBytes)) != cudaSuccess)
    return PT_ECUDA;
  for (int k = 32; k >= 1; k >>= 1) {
    const size_t bytes = flip_smem_bytes(p.R, k, words);
    if (bytes + fa.sharedSizeBytes > smem_optin) continue;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFlipSmemThreads, bytes) !=
        cudaSuccess)
      return PT_ECUDA;
    const int blocks = (p.R + k - 1) / k;
    if (per_sm >= 1 && blocks <= per_sm * sms) {
      *k_out = k;
      *bytes_out = bytes;
      return PT_OK;
    }
  }
  return PT_OK;
}

cudaError_t launch_flip_smem(const DevProblem& p, int k, size_t bytes, uint64_t it0,
                             uint64_t e0, int64_t n, int m, int stall, uint64_t limit_ns,
                             cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(p.cnt + 6 * p.W * 32, 0, sizeof(unsigned), st);
  if (err != cudaSuccess) return err;
  FlipArgs a;
  a.p = p;
  a.it0 = it0;
  a.e0 = e0;
  a.n = n;
  a.m = m;
  a.stall = stall;
  a.limit_ns = limit_ns;
  for (int r = 0; r < 10; ++r) {
    a.rk.k0[r] = p.key0 + (uint32_t)r * kPhiloxW0;
    a.rk.k1[r] = p.key1 + (uint32_t)r * kPhiloxW1;
  }
  int words = (p.L * p.L + 31) / 32;
  void* args[] = {&a, &k, &words};
  const int grid = (p.R + k - 1) / k;
  return cudaLaunchCooperativeKernel(flip_smem_fn(p.mode), dim3(grid), dim3(kFlipSmemThreads),
                                     args, bytes, st);
}

cudaError_t launch_flip(const DevProblem& p, uint64_t it0, uint64_t e0, int64_t n, int m,
                        int stall, uint64_t limit_ns, cudaStream_t st) {
  // the barrier counter, after the energy buffers
  cudaError_t err = cudaMemsetAsync(p.cnt + 6 * p.W * 32, 0, sizeof(unsigned), st);
  if (err != cudaSuccess) return err;
  FlipArgs a;
  a.p = p;
  a.it0 = it0;
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
  const int grid = (p.R + kFlipThreads - 1) / kFlipThreads;
  return cudaLaunchCooperativeKernel((const void*)k_flip, dim3(grid), dim3(kFlipThreads), args,
                                     (size_t)2 * p.R * sizeof(int32_t), st);
}

}  // namespace ptb
