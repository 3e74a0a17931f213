// pt_flat.cuh -- the parts shared by the two batched paths that work on word tiles: the
// lock-step launches (pt_flat.cu) and the dataflow persistent launch (pt_flow.cu). A batch
// is a list of problems and a list of equal-sized word tiles drawn from every problem and
// plane; the host deals the tiles to warps, longest first.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <vector>

#include "pt_debug.cuh"
#include "pt_device.cuh"
#include "pt_internal.h"

namespace ptb {

constexpr int kFlatThreads = 256;

struct FlatProblem {
  DevProblem p;
  uint64_t t0, e0;   // counters when the batch starts
  int64_t n;         // sweeps in this batch
  int m;             // exchange every m sweeps (0 = never)
  int ntiles;        // work tiles of this problem
  uint64_t wait_ns;  // dataflow path: time limit of each wait
  int stall;         // dataflow path, test support: tiles the first colour-1 wait adds
  int pad;
};

// A warp's unit of work: words [q0, q1) of one colour of plane w of one problem
// (q = y * L/2 + i). Tiles never straddle planes, so a warp's thresholds are uniform.
struct Tile {
  int prob;
  int w;
  int q0, q1;
};

// Does an exchange follow sweep j of this batch for problem fp?
__device__ __forceinline__ bool exchanges_after(const FlatProblem& fp, int64_t j) {
  return j < fp.n && fp.m > 0 && (fp.t0 + (uint64_t)j + 1) % (uint64_t)fp.m == 0;
}
// Is sweep j of this batch counted for problem fp (a swap iteration or a trace row follows)?
__device__ __forceinline__ bool counts_after(const FlatProblem& fp, int64_t j) {
  return exchanges_after(fp, j) || (j < fp.n && fp.p.trace_E != nullptr);
}
// Swap iterations of this batch up to and including the one after sweep j.
__device__ __forceinline__ uint64_t exchanges_through(const FlatProblem& fp, int64_t j) {
  const uint64_t m = (uint64_t)fp.m;
  return (fp.t0 + (uint64_t)j + 1) / m - fp.t0 / m;
}
// swap iteration index used after sweep j (valid when exchanges_after)
__device__ __forceinline__ uint64_t exchange_index(const FlatProblem& fp, int64_t j) {
  return fp.e0 + exchanges_through(fp, j) - 1;
}

// A neighbour word: through L1 (plain load) or, with NB_L2, through L2 only. Both are
// correct wherever the caller has acquired the writers' releases; the dataflow path takes
// L2, where measured exchange sweeps ran faster.
template <bool NB_L2>
__device__ __forceinline__ uint32_t ld_nb(const uint32_t* p) {
  if (NB_L2) return __ldcg(p);
  return *p;
}

// ---------------------------------------------------------------------------------------
// Exchange step of one problem by one warp (the three parts of the exchange kernel):
// energies from the counts (then cleared), the swap iteration of Sec. 3, and the plane
// thresholds for the new slot -> temperature map. Every word it reads was written before
// the launch, or before a release that the caller has acquired; the maps and energies,
// which the previous swap iteration may have written from another SM, are read through L2.
// ---------------------------------------------------------------------------------------
__device__ inline void exchange_warp(const DevProblem& p, uint64_t e) {
  const int lane = threadIdx.x & 31;
  const int R = p.R, W = p.W;
  const int64_t L2 = (int64_t)p.L * p.L;
  for (int r = lane; r < R; r += 32) {
    const int64_t U = __ldcg(p.cnt + r);
    const int64_t ones = __ldcg(p.cnt + W * 32 + r);
    const int64_t bonds = 2 * L2 - 2 * U;
    const int64_t M = 2 * ones - L2;
    p.E_slot[r] = -p.J_int * bonds + p.h_int * M;
    p.M_slot[r] = M;
  }
  __syncwarp();
  for (int q = lane; q < 2 * W * 32; q += 32) p.cnt[q] = 0;
  const int parity = (int)(e & 1);
  const uint32_t c3 = kTagExch | ((uint32_t)(e >> 32) << 8);
  for (int k = parity + 2 * lane; k + 1 < R; k += 64) {
    const int a = __ldcg(p.slot_of_temp + k), b = __ldcg(p.slot_of_temp + k + 1);
    const int64_t n = __ldcg(p.E_slot + a) - __ldcg(p.E_slot + b);
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
  __syncwarp();
  constexpr uint64_t kTwo32 = 1ull << 32;
  for (int r = lane; r < W * 32; r += 32) {
    const int w = r >> 5, b = r & 31;
    const bool in_use = r < R;
    const int temp = in_use ? __ldcg(p.temp_of_slot + r) : 0;
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

// Runs f(BlockCount<nblk>{}) for nblk in 1..8: one instance of f per block count.
template <class F>
__device__ __forceinline__ void with_block_count(int nblk, const F& f) {
  switch (nblk) {
    case 1: f(BlockCount<1>{}); break;
    case 2: f(BlockCount<2>{}); break;
    case 3: f(BlockCount<3>{}); break;
    case 4: f(BlockCount<4>{}); break;
    case 5: f(BlockCount<5>{}); break;
    case 6: f(BlockCount<6>{}); break;
    case 7: f(BlockCount<7>{}); break;
    default: f(BlockCount<8>{}); break;
  }
}

// ---------------------------------------------------------------------------------------
// One warp tile's half sweep (Eq. 1 on every word of the tile). With `count` (colour 1 of a
// sweep followed by an exchange) the warp also adds, from the words it holds, the
// unsatisfied bonds of its updated sites (all four bonds of a colour-1 site; every bond has
// exactly one colour-1 end) and, in the generic case, the up spins of its sites and of
// their colour-0 neighbours one row up (a one-to-one map between the colours), into the
// problem's counters. thr / gen: this warp's shared-memory threshold slot. Every word of
// another warp that it reads was written before the launch, or before a release that the
// caller has acquired, so plain (L1-cached) loads see it; NB_L2 reads the neighbour words
// through L2 instead.
// ---------------------------------------------------------------------------------------
template <int MODE, bool COUNT, bool NB_L2>
__device__ __forceinline__ void tile_half(const FlatProblem& fp, const Tile& tl, int colour,
                                          int64_t j, bool count, uint4* thr,
                                          PlaneGeneric* gen) {
  const int lane = threadIdx.x & 31;
  const uint64_t t = fp.t0 + (uint64_t)j;
  const DevProblem& p = fp.p;
  const int w = tl.w;
  const int L = p.L, half = L >> 1;
  const int nblk = (min(32, p.R - 32 * w) + 3) >> 2;
  const uint32_t c3 = kTagSpin | ((uint32_t)(t >> 32) << 8);
  RoundKeys rk;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = p.key0 + (uint32_t)r * kPhiloxW0;
    rk.k1[r] = p.key1 + (uint32_t)r * kPhiloxW1;
  }
  BlockTerms bt;
  block_terms((uint32_t)(8 * w), (uint32_t)t, rk, bt);
  const size_t own_base = word_index(L, w, colour, 0, 0);
  uint32_t* own = p.spins + own_base;
  const uint32_t* oth = p.spins + word_index(L, w, colour ^ 1, 0, 0);
  const int nwords = L * half;  // words of one colour of a plane (the debug checks' range)
  (void)nwords;
  const int q_start = tl.q0 + lane;
  int y = q_start / half, i = q_start - y * half;
  const int dy = 32 / half, di = 32 - dy * half;
  // the inputs of one word: the lane's word, its four neighbours (other colour) and site
  struct WordIn {
    uint32_t s, n0, n1, n2, n3, site;
  };
  // the neighbours as offsets from the lane's own word q = yy * half + ii (rows yy - 1 and
  // yy + 1 at the same ii, row yy at ii -+ 1 by the row parity, all mod L): no multiplies
  // (measured: 2% fewer instructions than row * half + column addressing)
  const int wrap = nwords - half;  // (L - 1) * half
  const auto load_word = [&](int q, int yy, int ii) {
    const int par = (yy + colour) & 1;
    const int o0 = (yy == 0) ? wrap : -half;
    const int o1 = (yy == L - 1) ? -wrap : half;
    const int o3 = par ? ((ii + 1 == half) ? -ii : 1) : ((ii == 0) ? half - 1 : -1);
    WordIn a;
    a.s = own[PT_DBG_IDX(p, q, nwords, kDbgSpinLoad)];  // this lane's word
    a.n0 = ld_nb<NB_L2>(oth + PT_DBG_IDX(p, q + o0, nwords, kDbgSpinLoad));
    a.n1 = ld_nb<NB_L2>(oth + PT_DBG_IDX(p, q + o1, nwords, kDbgSpinLoad));
    a.n2 = ld_nb<NB_L2>(oth + PT_DBG_IDX(p, q, nwords, kDbgSpinLoad));
    a.n3 = ld_nb<NB_L2>(oth + PT_DBG_IDX(p, q + o3, nwords, kDbgSpinLoad));
    a.site = (uint32_t)(2 * q + par);  // y L + x with x = 2 ii + par
    return a;
  };
  const auto step = [&]() {
    i += di;
    y += dy;
    if (i >= half) {
      i -= half;
      y += 1;
    }
  };
  if (MODE == kModeFerro) {
    // the tile's thresholds in the warp's shared slot, interleaved for 16-byte broadcast
    // loads (the previous tile's readers are done at the warp barrier)
    const PlaneFerro* pl = reinterpret_cast<const PlaneFerro*>(p.planes) + w;
    __syncwarp();
    if (lane < 16) {
      const int b = 2 * lane;
      thr[lane] = make_uint4(pl->T0[b], pl->T1[b], pl->T0[b + 1], pl->T1[b + 1]);
    }
    __syncwarp();
    const uint32_t alw0 = pl->alw0, alw1 = pl->alw1, used = pl->used;
    BitCounter<13, 8> Uf;
    if (COUNT) Uf.zero();
    // one loop per block count: the word update runs with NB blocks fixed at compile time
    // (measured: 131.5 -> 122.9 us per batched-256 sweep without swaps; with the wide
    // multiplies the counting kernel gains from it too, 135.3 -> 134.0 us per sweep with a
    // swap iteration, where before it cost registers and time)
    const auto finish_word = [&](int q, const WordIn& a, uint32_t ns) {
      if (PT_DBG_STORE(p, q, nwords, own_base, t, colour)) own[q] = ns;
      if (COUNT && count) {
        // with h = 0 the exchange needs only the bonds: U of the new state, all four bonds
        // of this colour-1 site (the colour-0 neighbours are final for this sweep)
        const NbCount k = count4(ns ^ a.n0, ns ^ a.n1, ns ^ a.n2, ns ^ a.n3);
        Uf.add3(k.b0, k.b1, k.b2);
      }
    };
    const auto word_loop = [&](auto nbc) {
      constexpr int NB = decltype(nbc)::value;
      const auto update = [&](const WordIn& a) {
        const SiteTerms st = site_terms(a.site, c3, rk);
        const auto draw = [&](int jb) { return philox_site_block(st, bt, jb, rk); };
        return update_word_ferro_smem<NB>(a.s, a.n0, a.n1, a.n2, a.n3, nblk, thr, alw0, alw1,
                                          used, draw);
      };
      int q = q_start;
      for (; q < tl.q1; q += 32) {
        const WordIn a = load_word(q, y, i);
        finish_word(q, a, update(a));
        step();
      }
    };
    with_block_count(nblk, word_loop);
    if (COUNT && count) {
      const uint32_t u = Uf.warp_total_for_lane();
      if (u) atomicAdd(&p.cnt[PT_DBG_IDX(p, w * 32 + lane, 2 * p.W * 32, kDbgCount)], u);
      if (p.trace_E != nullptr) {
        // a trace row needs M too: the up spins of this lane's colour-1 words and of the
        // colour-0 words one row up, in a second pass
        BitCounter<13, 8> N;
        N.zero();
        int yc = q_start / half, ic = q_start - yc * half;
        for (int q = q_start; q < tl.q1; q += 32) {
          const int ym = (yc == 0) ? L - 1 : yc - 1;
          const uint32_t ns = own[PT_DBG_IDX(p, q, nwords, kDbgSpinLoad)];
          const uint32_t n0 = ld_nb<NB_L2>(oth + PT_DBG_IDX(p, ym * half + ic, nwords, kDbgSpinLoad));
          N.add2(ns ^ n0, ns & n0);
          ic += di;
          yc += dy;
          if (ic >= half) {
            ic -= half;
            yc += 1;
          }
        }
        const uint32_t nn = N.warp_total_for_lane();
        if (nn)
          atomicAdd(&p.cnt[PT_DBG_IDX(p, p.W * 32 + w * 32 + lane, 2 * p.W * 32, kDbgCount)], nn);
      }
    }
  } else {
    // the warp's generic thresholds live in its own shared slot
    {
      __syncwarp();
      const uint32_t* src = reinterpret_cast<const uint32_t*>(
          reinterpret_cast<const PlaneGeneric*>(p.planes) + w);
      uint32_t* dst = reinterpret_cast<uint32_t*>(gen);
      for (int q = lane; q < (int)(sizeof(PlaneGeneric) / 4); q += 32)
        dst[q] = src[q];
      __syncwarp();
    }
    const PlaneGeneric& pl = *gen;
    // few classes with dE > 0 (five for J > 0, 0 < |h| < 2 J): compare with all of them
    const uint32_t cm = (uint32_t)p.cmp_classes;
    // the five-class paths count the bonds and up spins of the words they write in the word
    // loop (158.7 -> 155.5 us per batched-256 sweep at h = 0.1 with a swap iteration every
    // sweep); the lookup path counts them in a second pass
    BitCounter<13, 8> Ug, Ng;
    if (COUNT) {
      Ug.zero();
      Ng.zero();
    }
    const auto gen_loop = [&](auto in_loop, const auto& update) {
      constexpr bool CNT_IN_LOOP = decltype(in_loop)::value;
      for (int q = q_start; q < tl.q1; q += 32) {
        const WordIn a = load_word(q, y, i);
        const SiteTerms st = site_terms(a.site, c3, rk);
        const uint32_t ns = update(a.s, a.n0, a.n1, a.n2, a.n3, [&](int jb) {
          return philox_site_block(st, bt, jb, rk);
        });
        if (PT_DBG_STORE(p, q, nwords, own_base, t, colour)) own[q] = ns;
        if (COUNT && CNT_IN_LOOP && count) {
          const NbCount k = count4(ns ^ a.n0, ns ^ a.n1, ns ^ a.n2, ns ^ a.n3);
          Ug.add3(k.b0, k.b1, k.b2);
          Ng.add2(ns ^ a.n0, ns & a.n0);
        }
        step();
      }
    };
    // J > 0 and 0 < h < 2 J (the served mix's field problems): the classes with dE > 0 are
    // 0..4 (k = 0, 1 with either spin, k = 2 against the field); h < 0 mirrors it (0..3, 5).
    // With the class set known at compile time the threshold rows are read at fixed offsets
    // (181.3 / 160.7 -> 174.3 / 154.5 us per batched-256 sweep at h = 0.1, with / without a
    // swap iteration every sweep), and with the Philox block count fixed too, one loop per
    // count: 158.3 / 138.6 us. The other class sets keep the per-slot lookup and the block
    // count at run time (with the lookup, a fixed count measured 17% slower).
    if (cm == 0x1Fu) {
      constexpr int cls_pos[5] = {0, 1, 2, 3, 4};
      with_block_count(nblk, [&](auto nbc) {
        constexpr int NB = decltype(nbc)::value;
        gen_loop(std::true_type{}, [&](uint32_t s, uint32_t n0, uint32_t n1, uint32_t n2,
                                       uint32_t n3, const auto& draw) {
          return update_word_generic_cmp<5, NB>(s, n0, n1, n2, n3, nblk, pl, cls_pos, draw);
        });
      });
    } else if (cm == 0x2Fu) {
      constexpr int cls_neg[5] = {0, 1, 2, 3, 5};
      with_block_count(nblk, [&](auto nbc) {
        constexpr int NB = decltype(nbc)::value;
        gen_loop(std::true_type{}, [&](uint32_t s, uint32_t n0, uint32_t n1, uint32_t n2,
                                       uint32_t n3, const auto& draw) {
          return update_word_generic_cmp<5, NB>(s, n0, n1, n2, n3, nblk, pl, cls_neg, draw);
        });
      });
    } else if (__popc(cm) == 5) {
      int cls[5];
      uint32_t rest = cm;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        cls[c] = __ffs(rest) - 1;
        rest &= rest - 1;
      }
      gen_loop(std::false_type{}, [&](uint32_t s, uint32_t n0, uint32_t n1, uint32_t n2,
                                      uint32_t n3, const auto& draw) {
        return update_word_generic_cmp<5>(s, n0, n1, n2, n3, nblk, pl, cls, draw);
      });
    } else {
      gen_loop(std::false_type{}, [&](uint32_t s, uint32_t n0, uint32_t n1, uint32_t n2,
                                      uint32_t n3, const auto& draw) {
        return update_word_generic_with(s, n0, n1, n2, n3, nblk, pl, draw);
      });
    }
    if (COUNT && count && (cm == 0x1Fu || cm == 0x2Fu)) {
      const uint32_t u = Ug.warp_total_for_lane();
      const uint32_t nn = Ng.warp_total_for_lane();
      if (u) atomicAdd(&p.cnt[PT_DBG_IDX(p, w * 32 + lane, 2 * p.W * 32, kDbgCount)], u);
      if (nn)
        atomicAdd(&p.cnt[PT_DBG_IDX(p, p.W * 32 + w * 32 + lane, 2 * p.W * 32, kDbgCount)], nn);
    } else if (COUNT && count) {
      // second pass over the words this lane just wrote and their colour-0 neighbours
      BitCounter<13, 8> U, N;
      U.zero();
      N.zero();
      int yc = q_start / half, ic = q_start - yc * half;
      for (int q = q_start; q < tl.q1; q += 32) {
        const int par = (yc + colour) & 1;
        const int ym = (yc == 0) ? L - 1 : yc - 1;
        const int yp = (yc == L - 1) ? 0 : yc + 1;
        const int ih = par ? ((ic + 1 == half) ? 0 : ic + 1) : ((ic == 0) ? half - 1 : ic - 1);
        const uint32_t ns = own[PT_DBG_IDX(p, q, nwords, kDbgSpinLoad)];
        const uint32_t n0 = ld_nb<NB_L2>(oth + PT_DBG_IDX(p, ym * half + ic, nwords, kDbgSpinLoad));
        const NbCount k = count4(
            ns ^ n0, ns ^ ld_nb<NB_L2>(oth + PT_DBG_IDX(p, yp * half + ic, nwords, kDbgSpinLoad)),
            ns ^ ld_nb<NB_L2>(oth + PT_DBG_IDX(p, q, nwords, kDbgSpinLoad)),
            ns ^ ld_nb<NB_L2>(oth + PT_DBG_IDX(p, yc * half + ih, nwords, kDbgSpinLoad)));
        U.add3(k.b0, k.b1, k.b2);
        N.add2(ns ^ n0, ns & n0);
        ic += di;
        yc += dy;
        if (ic >= half) {
          ic -= half;
          yc += 1;
        }
      }
      const uint32_t u = U.warp_total_for_lane();
      const uint32_t nn = N.warp_total_for_lane();
      if (u) atomicAdd(&p.cnt[PT_DBG_IDX(p, w * 32 + lane, 2 * p.W * 32, kDbgCount)], u);
      if (nn)
        atomicAdd(&p.cnt[PT_DBG_IDX(p, p.W * 32 + w * 32 + lane, 2 * p.W * 32, kDbgCount)], nn);
    }
  }
}

// ---------------------------------------------------------------------------------------
// host side (pt_flat.cu)
// ---------------------------------------------------------------------------------------
// Problems with n > 0 and their tiles (split by mode: [0] ferro, [1] generic); returns the
// largest n.
// Tiles hold about tile_words words (a problem's words of one colour and plane in
// max(1, round(words / tile_words)) equal parts, so at most 1.5 tile_words: a lane's counts
// over one tile stay below 2^8); with `refine` (the queued schedule) the tiles of the
// cheapest quarter of the work are then cut in two. Returns the largest n, or -1 when a
// tile would fall outside its plane.
int64_t build_flat_lists(pt_problem* const* ps, int count, const int64_t* n, const int* every,
                         int tile_words, bool refine, std::vector<FlatProblem>* probs,
                         std::vector<Tile> tiles[2]);
// Longest-processing-time-first assignment of tiles to `nwarps` warps: the tiles reordered
// warp by warp and the CSR offsets first[0..nwarps].
void deal_tiles(const std::vector<Tile>& in, const std::vector<FlatProblem>& probs,
                int nwarps, std::vector<Tile>* out, std::vector<int>* first);
int64_t tile_cost(const Tile& t, int R);

}  // namespace ptb
