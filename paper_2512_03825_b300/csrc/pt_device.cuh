// pt_device.cuh -- device building blocks of the parallel-tempering sweep (sm_103a).
//
// Everything here is integer arithmetic on CUDA cores: nothing in the method is a dense
// contraction, so the tensor cores have no role.
#pragma once
#include <stdint.h>

#include "pt_types.h"

namespace ptb {

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32 -> 64-bit
// products whose halves are xored with the other counter words and the round key; the key
// advances by the Weyl constants between rounds.
// ---------------------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

struct Philox4 {
  uint32_t x, y, z, w;
};

// hi:lo = a * b, the full 64-bit product of two 32-bit words, as one wide multiply. Written
// as __umulhi(a, b) and a * b, the two halves were formed by separate multiplies: measured
// on batched-256, 122.2 -> 115.7 us per sweep without swaps with the single wide product,
// L = 1024, R = 64 56.7 -> 55.4 us.
__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
  uint64_t p;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
  lo = (uint32_t)p;
  hi = (uint32_t)(p >> 32);
}

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                  uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mul_wide(kPhiloxM0, c0, hi0, lo0);
    mul_wide(kPhiloxM1, c2, hi1, lo1);
    const uint32_t rk0 = k0 + (uint32_t)r * kPhiloxW0;
    const uint32_t rk1 = k1 + (uint32_t)r * kPhiloxW1;
    c0 = hi1 ^ c1 ^ rk0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ rk1;
    c3 = lo0;
  }
  return Philox4{c0, c1, c2, c3};
}

// The ten round keys (k + r * W, mod 2^32) of one seed, computed on the host. Held in a
// __grid_constant__ kernel parameter and indexed with constants, each key is an operand
// straight from the constant bank: no register and no instruction per round.
struct RoundKeys {
  uint32_t k0[10], k1[10];
};

__device__ __forceinline__ Philox4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2,
                                                     uint32_t c3, const RoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mul_wide(kPhiloxM0, c0, hi0, lo0);
    mul_wide(kPhiloxM1, c2, hi1, lo1);
    c0 = hi1 ^ c1 ^ rk.k0[r];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ rk.k1[r];
    c3 = lo0;
  }
  return Philox4{c0, c1, c2, c3};
}

// One swap attempt of pair k in the statistics: reductions at L2, so the counting thread
// does not wait for the old values (and a later CTA never reads a stale L1 copy).
__device__ __forceinline__ void count_swap(uint64_t* attempted, uint64_t* accepted, int k,
                                           bool accept) {
  atomicAdd(reinterpret_cast<unsigned long long*>(attempted + k), 1ull);
  if (accept) atomicAdd(reinterpret_cast<unsigned long long*>(accepted + k), 1ull);
}

// The exchange threshold of one temperature pair at energy difference n (SwapPair): the
// saturated constants outside the tabulated range, else the table entry; the index stays
// inside the table for every n in [n_lo, n_hi].
__device__ __forceinline__ uint64_t pair_threshold(const SwapPair& sp, const uint32_t* table,
                                                   int shift, int64_t n) {
  if (n < sp.n_lo) return sp.S_below;
  if (n > sp.n_hi) return sp.S_above;
  return table[sp.offset + ((n - sp.n_lo) >> shift)];
}

// The eight blocks j of one site in one sweep have the counters {site, lo32(t), blk0 + j, c3}:
// they differ in counter word 2 only. In round 1 the product of word 0 depends on the site
// alone and that of word 2 on j alone; in round 2 the product of word 0 (which came from
// word 2's product) depends on j and the sweep alone and that of word 2 on the site alone.
// So a site needs two products for rounds 1-2 instead of 4 per block, and the j-dependent
// round-1/2 terms are computed once per sweep and plane (BlockTerms). Same numbers, bit for
// bit: only the order in which the products are formed changes.
struct BlockTerms {
  uint32_t X[8], Y[8], Z[8];  // per block: round-2 output terms that do not depend on the site
};
struct SiteTerms {
  uint32_t H, Hlo, L0;  // round-1/2 products that do not depend on the block
};

__device__ __forceinline__ void block_terms(uint32_t blk0, uint32_t t_lo, const RoundKeys& rk,
                                            BlockTerms& bt) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t c2 = blk0 + (uint32_t)j;
    uint32_t h1, l1, hA, lA;
    mul_wide(kPhiloxM1, c2, h1, l1);             // round 1, word 2
    const uint32_t c0 = h1 ^ t_lo ^ rk.k0[0];    // round-1 output 0
    mul_wide(kPhiloxM0, c0, hA, lA);             // round 2, word 0
    bt.X[j] = l1 ^ rk.k0[1];
    bt.Y[j] = hA ^ rk.k1[1];
    bt.Z[j] = lA;
  }
}

__device__ __forceinline__ SiteTerms site_terms(uint32_t site, uint32_t c3, const RoundKeys& rk) {
  SiteTerms st;
  uint32_t h0;
  mul_wide(kPhiloxM0, site, h0, st.L0);      // round 1, word 0
  const uint32_t c2 = h0 ^ c3 ^ rk.k1[0];    // round-1 output 2
  mul_wide(kPhiloxM1, c2, st.H, st.Hlo);     // round 2, word 2
  return st;
}

// Rounds 3-10 of Philox4x32-10 from the round-2 state (c0, c1, c2, c3).
__device__ __forceinline__ Philox4 philox_rounds_3_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                      uint32_t c3, const RoundKeys& rk) {
#pragma unroll
  for (int r = 2; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mul_wide(kPhiloxM0, c0, hi0, lo0);
    mul_wide(kPhiloxM1, c2, hi1, lo1);
    c0 = hi1 ^ c1 ^ rk.k0[r];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ rk.k1[r];
    c3 = lo0;
  }
  return Philox4{c0, c1, c2, c3};
}

// Philox4x32-10 block j of the site: the round-2 state from the shared terms, then rounds
// 3-10.
__device__ __forceinline__ Philox4 philox_site_block(const SiteTerms& st, const BlockTerms& bt,
                                                     int j, const RoundKeys& rk) {
  return philox_rounds_3_10(st.H ^ bt.X[j], st.Hlo, bt.Y[j] ^ st.L0, bt.Z[j], rk);
}


// Counter words shared by every spin-update draw of one sweep.
struct SweepCtr {
  uint32_t t_lo;  // lo32(t)
  uint32_t c3;    // kTagSpin | hi32(t) << 8
  uint32_t k0, k1;
};

__device__ __forceinline__ SweepCtr make_sweep_ctr(uint64_t t, uint32_t k0, uint32_t k1) {
  return SweepCtr{(uint32_t)t, kTagSpin | ((uint32_t)(t >> 32) << 8), k0, k1};
}

// ---------------------------------------------------------------------------------------
// Anti-aligned neighbour count, bit-sliced over the 32 slots of a word.
// a_j = s ^ n_j marks the slots whose neighbour j points the other way; k = sum_j a_j.
// ---------------------------------------------------------------------------------------
struct NbCount {
  uint32_t b0, b1, b2;  // binary digits of k (0..4)
};

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) {
  return (a & b) | (a & c) | (b & c);
}

__device__ __forceinline__ NbCount count4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3) {
  const uint32_t x01 = a0 ^ a1, c01 = a0 & a1;
  const uint32_t x23 = a2 ^ a3, c23 = a2 & a3;
  const uint32_t c0 = x01 & x23;
  NbCount k;
  k.b0 = x01 ^ x23;
  k.b1 = c01 ^ c23 ^ c0;
  k.b2 = maj3(c01, c23, c0);
  return k;
}

// ---------------------------------------------------------------------------------------
// Metropolis update of one word = 32 slots at one site (Eq. 1 with the Boltzmann target of
// Eq. 2 on the local energy change of Eq. 3). Returns the new word.
//   s        centre word; n0..n3 its four neighbour words (other colour)
//   site     y * L + x;  blk0 = 8 * plane (Philox counter word 2 of the first block)
//   nblk     Philox blocks needed (4 slots each; ceil(used slots / 4))
// ---------------------------------------------------------------------------------------

// acc * 2 + [u >= T]: the carry out of u - T shifted into the low end of acc. Fed from
// bit 31 down to bit 0, a word of 32 such calls is the mask of rejected trials. Two integer
// instructions per trial on the ALU pipe; no predicate or select.
__device__ __forceinline__ uint32_t shift_in_reject(uint32_t acc, uint32_t u, uint32_t T) {
  uint32_t r;
  asm("{\n\t.reg .u32 d;\n\tsub.cc.u32 d, %1, %2;\n\taddc.u32 %0, %3, %3;\n\t}"
      : "=r"(r)
      : "r"(u), "r"(T), "r"(acc));
  return r;
}

// h = 0, J > 0: dE = 4 J (2 - k); classes k = 0 and k = 1 need a random number, k >= 2
// always flips. Each trial is compared with both thresholds: rej0 / rej1 collect u >= T0 and
// u >= T1, and because T0 <= T1 bit by bit, "not rej0, or k == 1 and not rej1" is the exact
// rule for both random classes.
__device__ __forceinline__ uint32_t update_word_ferro(uint32_t s, uint32_t n0, uint32_t n1,
                                                      uint32_t n2, uint32_t n3, uint32_t site,
                                                      uint32_t blk0, int nblk,
                                                      const uint32_t (&T0)[32],
                                                      const uint32_t (&T1)[32], uint32_t alw0,
                                                      uint32_t alw1, uint32_t used,
                                                      const SweepCtr& cx) {
  const uint32_t a0 = s ^ n0, a1 = s ^ n1, a2 = s ^ n2, a3 = s ^ n3;
  const uint32_t x01 = a0 ^ a1, x23 = a2 ^ a3;
  const uint32_t ge2 = (a0 & a1) | (a2 & a3) | (x01 & x23);
  const uint32_t eq1 = (x01 ^ x23) & ~ge2;
  // slots of blocks j >= nblk are unused: their bits start out as "rejected" and no
  // compare is spent on them
  uint32_t rej0 = nblk >= 8 ? 0u : (0xffffffffu >> (4 * nblk));
  uint32_t rej1 = rej0;
#pragma unroll
  for (int j = 7; j >= 0; --j) {
    if (j < nblk) {
      const Philox4 r = philox4x32_10(site, cx.t_lo, blk0 + (uint32_t)j, cx.c3, cx.k0, cx.k1);
      const uint32_t u[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
      for (int q = 3; q >= 0; --q) {
        const int b = 4 * j + q;
        rej0 = shift_in_reject(rej0, u[q], T0[b]);
        rej1 = shift_in_reject(rej1, u[q], T1[b]);
      }
    }
  }
  const uint32_t acc = ~rej0 | (eq1 & ~rej1);
  const uint32_t flip = (ge2 | alw0 | (eq1 & alw1) | acc) & used;
  return s ^ flip;
}

// update_word_ferro with the thresholds in shared memory, interleaved so that one 16-byte
// broadcast load serves two slots: thr[m] = {T0[2m], T1[2m], T0[2m+1], T1[2m+1]}.
// `draw(j)` returns Philox block j of this site (slots 4j .. 4j+3). Same decisions, bit for
// bit. NBC > 0 fixes the block count at compile time (nblk is then ignored).
template <int NBC = 0, class Draw>
__device__ __forceinline__ uint32_t update_word_ferro_smem(uint32_t s, uint32_t n0, uint32_t n1,
                                                           uint32_t n2, uint32_t n3, int nblk_rt,
                                                           const uint4* thr, uint32_t alw0,
                                                           uint32_t alw1, uint32_t used,
                                                           const Draw& draw) {
  const int nblk = NBC > 0 ? NBC : nblk_rt;
  const uint32_t a0 = s ^ n0, a1 = s ^ n1, a2 = s ^ n2, a3 = s ^ n3;
  const uint32_t x01 = a0 ^ a1, x23 = a2 ^ a3;
  const uint32_t ge2 = (a0 & a1) | (a2 & a3) | (x01 & x23);
  const uint32_t eq1 = (x01 ^ x23) & ~ge2;
  uint32_t rej0 = nblk >= 8 ? 0u : (0xffffffffu >> (4 * nblk));
  uint32_t rej1 = rej0;
#pragma unroll
  for (int j = 7; j >= 0; --j) {
    if (j < nblk) {
      const Philox4 r = draw(j);
      const uint4 lo = thr[2 * j], hi = thr[2 * j + 1];  // slots 4j, 4j+1 | 4j+2, 4j+3
      rej0 = shift_in_reject(rej0, r.w, hi.z);
      rej1 = shift_in_reject(rej1, r.w, hi.w);
      rej0 = shift_in_reject(rej0, r.z, hi.x);
      rej1 = shift_in_reject(rej1, r.z, hi.y);
      rej0 = shift_in_reject(rej0, r.y, lo.z);
      rej1 = shift_in_reject(rej1, r.y, lo.w);
      rej0 = shift_in_reject(rej0, r.x, lo.x);
      rej1 = shift_in_reject(rej1, r.x, lo.y);
    }
  }
  const uint32_t acc = ~rej0 | (eq1 & ~rej1);
  const uint32_t flip = (ge2 | alw0 | (eq1 & alw1) | acc) & used;
  return s ^ flip;
}

// The Philox block count of a word as a type: BlockCount<n> fixes it at compile time, so the
// blocks of the word carry no runtime condition and can be interleaved; BlockCount<0> leaves
// it to the nblk argument.
template <int NB>
struct BlockCount {
  static constexpr int value = NB;
};

// Any J, h: class c = 2 k + (sigma == +1) per bit; thresholds from the plane table.
// `draw(j)` returns Philox block j of this site (slots 4j .. 4j+3).
template <class Draw>
__device__ __forceinline__ uint32_t update_word_generic_with(uint32_t s, uint32_t n0,
                                                             uint32_t n1, uint32_t n2,
                                                             uint32_t n3, int nblk,
                                                             const PlaneGeneric& pl,
                                                             const Draw& draw) {
  const NbCount k = count4(s ^ n0, s ^ n1, s ^ n2, s ^ n3);
  const uint32_t z[5] = {~(k.b0 | k.b1 | k.b2), k.b0 & ~k.b1 & ~k.b2, ~k.b0 & k.b1 & ~k.b2,
                         k.b0 & k.b1, k.b2};
  uint32_t always = 0;
#pragma unroll
  for (int kk = 0; kk < 5; ++kk)
    always |= z[kk] & ((s & pl.alw[2 * kk + 1]) | (~s & pl.alw[2 * kk]));
  uint32_t rej = nblk >= 8 ? 0u : (0xffffffffu >> (4 * nblk));
#pragma unroll
  for (int j = 7; j >= 0; --j) {
    if (j < nblk) {
      const Philox4 r = draw(j);
      const uint32_t u[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
      for (int q = 3; q >= 0; --q) {
        const int b = 4 * j + q;
        const uint32_t kb = ((k.b0 >> b) & 1u) | (((k.b1 >> b) & 1u) << 1) |
                            (((k.b2 >> b) & 1u) << 2);
        const uint32_t cls = 2u * kb + ((s >> b) & 1u);
        rej = shift_in_reject(rej, u[q], pl.T[cls][b]);
      }
    }
  }
  const uint32_t flip = (always | ~rej) & pl.used;
  return s ^ flip;
}

// update_word_generic_with for a problem whose classes with dE > 0 are few (NC of them,
// cls[0..NC-1]; every other class has dE <= 0, so its threshold is 2^32 and its slots are in
// the always-masks): each trial is compared with the thresholds of all NC classes (read four
// slots at a time), and bit-sliced class masks pick the result of the slot's own class,
// instead of a class extracted and looked up per slot. Same decisions, bit for bit. NBC > 0
// fixes the block count at compile time (nblk_rt is then ignored).
template <int NC, int NBC = 0, class Draw>
__device__ __forceinline__ uint32_t update_word_generic_cmp(uint32_t s, uint32_t n0, uint32_t n1,
                                                            uint32_t n2, uint32_t n3, int nblk_rt,
                                                            const PlaneGeneric& pl,
                                                            const int (&cls)[NC],
                                                            const Draw& draw) {
  const int nblk = NBC > 0 ? NBC : nblk_rt;
  const NbCount k = count4(s ^ n0, s ^ n1, s ^ n2, s ^ n3);
  const uint32_t z[5] = {~(k.b0 | k.b1 | k.b2), k.b0 & ~k.b1 & ~k.b2, ~k.b0 & k.b1 & ~k.b2,
                         k.b0 & k.b1, k.b2};
  uint32_t always = 0;
#pragma unroll
  for (int kk = 0; kk < 5; ++kk)
    always |= z[kk] & ((s & pl.alw[2 * kk + 1]) | (~s & pl.alw[2 * kk]));
  uint32_t rej[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) rej[c] = nblk >= 8 ? 0u : (0xffffffffu >> (4 * nblk));
#pragma unroll
  for (int j = 7; j >= 0; --j) {
    if (j < nblk) {
      const Philox4 r = draw(j);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const uint4 t = *reinterpret_cast<const uint4*>(&pl.T[cls[c]][4 * j]);
        rej[c] = shift_in_reject(rej[c], r.w, t.w);
        rej[c] = shift_in_reject(rej[c], r.z, t.z);
        rej[c] = shift_in_reject(rej[c], r.y, t.y);
        rej[c] = shift_in_reject(rej[c], r.x, t.x);
      }
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const uint32_t mine = z[cls[c] >> 1] & ((cls[c] & 1) ? s : ~s);
    acc |= mine & ~rej[c];
  }
  const uint32_t flip = (always | acc) & pl.used;
  return s ^ flip;
}

__device__ __forceinline__ uint32_t update_word_generic(uint32_t s, uint32_t n0, uint32_t n1,
                                                        uint32_t n2, uint32_t n3,
                                                        uint32_t site, uint32_t blk0, int nblk,
                                                        const PlaneGeneric& pl,
                                                        const SweepCtr& cx) {
  return update_word_generic_with(s, n0, n1, n2, n3, nblk, pl, [&](int j) {
    return philox4x32_10(site, cx.t_lo, blk0 + (uint32_t)j, cx.c3, cx.k0, cx.k1);
  });
}

// ---------------------------------------------------------------------------------------
// Bit-sliced per-slot counters: level l holds bit l of 32 independent counts. Additions by
// one thread ripple through the low NT levels only (its counts must stay below 2^NT); the
// warp sum uses all NB levels (the warp's counts must stay below 2^NB).
// ---------------------------------------------------------------------------------------
template <int NB, int NT>
struct BitCounter {
  static_assert(NT >= 3 && NT <= NB, "counter depth");
  uint32_t c[NB];

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int l = 0; l < NB; ++l) c[l] = 0;
  }
  // add a per-slot number given by its binary digits d0 (+ 2 d1 + 4 d2)
  __device__ __forceinline__ void add3(uint32_t d0, uint32_t d1, uint32_t d2) {
    uint32_t carry = c[0] & d0;
    c[0] ^= d0;
    uint32_t nc = maj3(c[1], d1, carry);
    c[1] ^= d1 ^ carry;
    carry = nc;
    nc = maj3(c[2], d2, carry);
    c[2] ^= d2 ^ carry;
    carry = nc;
#pragma unroll
    for (int l = 3; l < NT; ++l) {
      nc = c[l] & carry;
      c[l] ^= carry;
      carry = nc;
    }
  }
  __device__ __forceinline__ void add2(uint32_t d0, uint32_t d1) {
    uint32_t carry = c[0] & d0;
    c[0] ^= d0;
    uint32_t nc = maj3(c[1], d1, carry);
    c[1] ^= d1 ^ carry;
    carry = nc;
#pragma unroll
    for (int l = 2; l < NT; ++l) {
      nc = c[l] & carry;
      c[l] ^= carry;
      carry = nc;
    }
  }
  // sum over the warp (every lane ends with the total), then lane b returns the count of
  // slot bit b. Counts must fit NB bits after the sum.
  __device__ __forceinline__ uint32_t warp_total_for_lane() {
    // before round r (r = 0..4) a lane's counts are below 2^(NT + r): levels NT + r and up
    // are zero on both sides, so level NT + r takes the carry and the rest stay zero
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const int off = 16 >> r;
      uint32_t carry = 0;
#pragma unroll
      for (int l = 0; l < NB; ++l) {
        if (l < NT + r) {
          const uint32_t o = __shfl_xor_sync(0xffffffffu, c[l], off);
          const uint32_t sum = c[l] ^ o ^ carry;
          carry = maj3(c[l], o, carry);
          c[l] = sum;
        } else if (l == NT + r) {
          c[l] = carry;
        }
      }
    }
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t v = 0;
#pragma unroll
    for (int l = 0; l < NB; ++l) v |= ((c[l] >> lane) & 1u) << l;
    return v;
  }
};

// ---------------------------------------------------------------------------------------
// Waiting inside persistent kernels: relaxed polls of a counter, release/acquire ordering
// and the global nanosecond timer that bounds every wait.
// ---------------------------------------------------------------------------------------
// Polling a counter with a relaxed load leaves the SM's L1 alone; the one acquire fence
// after the wait is what orders the reads that follow it.
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// Release-ordered add: every write of this thread (and, after a warp or block barrier, of
// the threads it synchronised with) is visible to whoever acquires the new value.
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned atom_release_add_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;"
               : "=r"(old)
               : "l"(p), "r"(v)
               : "memory");
  return old;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------------------
// Word addressing
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ size_t word_index(int L, int w, int c, int y, int i) {
  return (((size_t)w * 2 + c) * L + y) * (size_t)(L >> 1) + i;
}

}  // namespace ptb
