// pt_debug.cuh -- the checks of the debug build (compiled with PT_DEBUG), which stand in for a
// memory and race checker on small cases:
//   * bounds: every spin-word index a kernel reads or writes is checked against the word
//     range of its plane and colour, every count-buffer and trace index against its buffer,
//     before the access;
//   * write set: every store of a half sweep tags its word with the half sweep's number, so
//     a word stored twice in one half sweep (two threads owning one site: a race) is seen,
//     and after a call the host can check that the last sweep stored every word of each
//     colour exactly in its own half sweep (pt_debug_report).
// A failed check never traps: it records the kind and index in the problem's DebugRecord,
// sets the problem's status word (so the next synchronising call reports PT_EINTERNAL), and
// the access is redirected to index 0 of the same array or skipped. Without PT_DEBUG every
// macro below is the bare index (or `true`), and the release kernels are unchanged.
#pragma once
#include <stdint.h>

#include "pt_types.h"

namespace ptb {

enum DebugKind : unsigned int {
  kDbgNone = 0,
  kDbgSpinLoad = 1,   // a spin-word load outside its plane and colour
  kDbgSpinStore = 2,  // a spin-word store outside its plane and colour
  kDbgTwice = 3,      // a spin word stored twice in one half sweep
  kDbgCount = 4,      // a count-buffer index outside [0, 2 W 32)
  kDbgTrace = 5,      // a trace row outside the ring
  kDbgFlip = 6,       // a single-spin-flip word outside its plane
};

// The status a failed check leaves in the problem's status word (reported as PT_EINTERNAL).
constexpr int32_t kStatusDebug = 3;

// Where a failed check is recorded: the problem's DebugRecord and status word (kernels that
// see only part of a problem carry these two pointers).
struct DbgSink {
  DebugRecord* rec;
  int32_t* status;
};

#ifdef PT_DEBUG
#define PT_DBG_ON 1
#else
#define PT_DBG_ON 0
#endif

#if defined(PT_DEBUG) && defined(__CUDACC__)
__device__ __forceinline__ DbgSink dbg_sink(const DevProblem& p) { return DbgSink{p.dbg, p.status}; }
__device__ __forceinline__ DbgSink dbg_sink(const DbgSink& s) { return s; }

__device__ __noinline__ inline void dbg_fail(DbgSink s, unsigned int kind, long long index) {
  if (s.rec == nullptr) return;
  atomicAdd(&s.rec->violations, 1ull);
  if (atomicCAS(&s.rec->first_kind, 0u, kind) == 0u)
    s.rec->first_index = (unsigned long long)index;
  atomicCAS(reinterpret_cast<int*>(s.status), 0, kStatusDebug);
}

// i when 0 <= i < n; otherwise the failure is recorded and 0 is returned, so the access
// stays inside the array.
template <class P>
__device__ __forceinline__ long long dbg_index(const P& p, long long i, long long n,
                                               unsigned int kind) {
  if (i >= 0 && i < n) return i;
  dbg_fail(dbg_sink(p), kind, i);
  return 0;
}

// May half sweep (t, colour) store word q of the colour's n words, whose first word is word
// `base` of the problem's spins? Checks the range and tags the word; a second store of the
// word in the same half sweep is recorded (the store itself still happens: it is in range).
__device__ __forceinline__ bool dbg_store(const DevProblem& p, long long q, long long n,
                                          long long base, uint64_t t, int colour) {
  if (q < 0 || q >= n) {
    dbg_fail(dbg_sink(p), kDbgSpinStore, q);
    return false;
  }
  if (p.dbg_tag != nullptr) {
    const unsigned int tag = (unsigned int)((2 * t + (uint64_t)colour) % 0x7fffffffull) + 1u;
    const unsigned int old = atomicExch(p.dbg_tag + base + q, tag);
    if (old == tag) dbg_fail(dbg_sink(p), kDbgTwice, base + q);
  }
  return true;
}

#define PT_DBG_IDX(p, i, n, kind) ((int)::ptb::dbg_index((p), (long long)(i), (long long)(n), (kind)))
#define PT_DBG_STORE(p, q, n, base, t, colour) \
  ::ptb::dbg_store((p), (long long)(q), (long long)(n), (long long)(base), (uint64_t)(t), (colour))
#define PT_DBG_CHECK(p, i, n, kind) \
  ((void)::ptb::dbg_index((p), (long long)(i), (long long)(n), (kind)))
#else
#define PT_DBG_IDX(p, i, n, kind) (i)
#define PT_DBG_STORE(p, q, n, base, t, colour) true
#define PT_DBG_CHECK(p, i, n, kind) ((void)0)
#endif

}  // namespace ptb
