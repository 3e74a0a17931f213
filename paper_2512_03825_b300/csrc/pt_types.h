// pt_types.h -- data layout shared by the host side (pt_host.cpp) and the sm_103a kernels.
//
// Spins: multispin-coded bitplanes. Slot r lives in plane w = r / 32, bit b = r % 32; a set
// bit is sigma = +1. Each plane is a full checkerboard lattice split by colour:
//   word(w, c, y, i) = spins[((w * 2 + c) * L + y) * (L / 2) + i]
// holds site (x, y) with x = 2 i + ((y + c) & 1), colour c = (x + y) & 1. Unused bits of the
// last plane stay 0. The four neighbours of (x, y) are all of the other colour: rows y - 1
// and y + 1 at the same i, and row y at i and at i - 1 (x even) or i + 1 (x odd), mod L / 2.
#pragma once
#include <stdint.h>

namespace ptb {

constexpr uint32_t kTagSpin = 0u;
constexpr uint32_t kTagExch = 1u;
constexpr uint32_t kTagInit = 2u;
constexpr uint32_t kTagFlip = 3u;  // single-spin-flip iterations
constexpr int kClasses = 10;  // class c = 2 k + (sigma == +1), k = anti-aligned neighbours 0..4

enum Mode : int {
  kModeFerro = 0,    // h_int == 0 and J_int > 0: random classes k = 0 (dE = 8J), k = 1 (4J)
  kModeGeneric = 1,  // any other J, h: per-bit threshold chosen from the ten classes
};

// Thresholds of one plane under the current slot -> temperature assignment, ferromagnetic
// zero-field case. T0 <= T1 holds bit by bit (dE(k=0) > dE(k=1) > 0).
struct PlaneFerro {
  uint32_t T0[32];  // min(T(beta, 8 J_int), 2^32 - 1)
  uint32_t T1[32];  // min(T(beta, 4 J_int), 2^32 - 1)
  uint32_t alw0;    // bits whose k = 0 threshold is 2^32 (always accept)
  uint32_t alw1;    // same for k = 1
  uint32_t used;    // bits that hold a slot (< R)
  uint32_t pad;
};

struct PlaneGeneric {
  uint32_t T[kClasses][32];  // min(T(beta, dE_c), 2^32 - 1)
  uint32_t alw[kClasses];    // bits whose class-c threshold is 2^32 (includes dE_c <= 0)
  uint32_t used;
  uint32_t pad;
};
// Kept a multiple of 16 bytes, so that in a 16-byte aligned array every table row T[c]
// starts on a 16-byte boundary (rows are read four slots at a time).
static_assert(sizeof(PlaneGeneric) % 16 == 0, "PlaneGeneric size");

// Exchange threshold of temperature pair (k, k+1) as a function of n = E_int(k) - E_int(k+1):
// table[offset + ((n - n_lo) >> table_shift)] for n_lo <= n <= n_hi, S_below / S_above
// outside. Every n that can occur is a multiple of 2^table_shift (DevProblem), and so are
// n_lo and n_hi: the table holds those n only. Values in [0, 2^32]; table entries are < 2^32.
struct SwapPair {
  int64_t n_lo, n_hi;
  uint64_t S_below, S_above;
  int64_t offset;
};

// The debug build's record of failed checks (PT_DEBUG; see pt_debug.cuh).
struct DebugRecord {
  unsigned long long violations;   // checks that failed
  unsigned long long first_index;  // the index the first failed check was given
  unsigned int first_kind;         // DebugKind of the first failed check (0: none)
  unsigned int pad;
};

// Device-side view of one problem (all pointers are device memory).
struct DevProblem {
  uint32_t* spins;         // [W][2][L][L/2]
  int L, R, W, mode;
  uint32_t key0, key1;     // Philox key = seed
  int32_t table_shift;     // log2 of the exchange tables' stride in n (SwapPair)
  int32_t cmp_classes;     // bit c: class c (= 2 k + (sigma == +1)) has dE > 0 (a random draw decides)
  int64_t J_int, h_int, s;
  const uint64_t* T_temp;  // [R][kClasses] thresholds by temperature index, in [0, 2^32]
  void* planes;            // PlaneFerro[W] or PlaneGeneric[W]
  int32_t* temp_of_slot;   // [R]
  int32_t* slot_of_temp;   // [R]
  uint32_t* cnt;           // [2][W * 32]: unsatisfied bonds, up spins per slot
  int64_t* E_slot;         // [R] E_int per slot (after the last energy pass)
  int64_t* M_slot;         // [R]
  uint64_t* attempted;     // [max(R-1, 1)]
  uint64_t* accepted;      // [max(R-1, 1)]
  const SwapPair* pairs;   // [max(R-1, 1)]
  const uint32_t* swap_table;
  int32_t* status;         // device error word (0 = fine)
  // observable trace (null when off): after sweep t (and its swap iteration), row
  // (t - trace_t0) % trace_cap of trace_E / trace_M [trace_cap][R] holds E_int and M of
  // every temperature index
  int64_t* trace_E;
  int64_t* trace_M;
  int64_t trace_cap;
  uint64_t trace_t0;
  // debug build only (null / 0 otherwise): per spin word, the number of the half sweep that
  // last wrote it (2 t + colour, mod 2^31 - 1, plus 1); the record of failed checks; a test
  // hook that makes the next launch of the plain half-sweep kernel perform one planted
  // mistake that its checks must catch (1: a second store of an unchanged word, 2: a
  // neighbour index one past its colour)
  uint32_t* dbg_tag;
  DebugRecord* dbg;
  int32_t dbg_inject;
  int32_t dbg_pad;
  // the band form of the persistent kernel (null until a band plan allocated it): a second
  // copy of colour 1, [W][L][L/2], so that the sweeps of a launch alternate between the two
  // copies (see k_persist)
  uint32_t* band_c1;
};

}  // namespace ptb
