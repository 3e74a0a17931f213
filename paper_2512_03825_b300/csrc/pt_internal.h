// pt_internal.h -- the host-side problem object shared by the host translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <vector>

#include "pt.h"
#include "pt_launch.h"
#include "pt_persist.h"

struct pt_problem {
  int L = 0, R = 0, W = 0, mode = 0;
  std::vector<double> betas;
  double J = 0, h = 0;
  int64_t s = 1, J_int = 0, h_int = 0;
  uint64_t seed = 0;
  int swap_rule = PT_SWAP_BARKER;
  uint64_t t = 0, e = 0;  // sweeps and swap iterations enqueued so far
  uint64_t it = 0;        // single-spin-flip iterations enqueued so far
  bool flip_shared = true;  // pt_flip keeps the replicas in shared memory when they fit
  cudaStream_t stream = 0;
  void* dmem = nullptr;   // the problem's single device allocation
  size_t dbytes = 0;
  pt_free_fn allocator_free = nullptr;
  void* allocator_ctx = nullptr;
  ptb::DevProblem dev{};
  ptb::DeviceInfo dev_info{};
  int poisoned = 0;       // sticky PT_E* code once device work failed
  int sweep_strategy = PT_SWEEP_AUTO;
  int words_per_thread = ptb::kPersistDefaultWords;
  bool plan_valid = false;  // plan is computed on first use
  ptb::PersistPlan plan{};
  uint64_t wait_limit_ns = 1000000000ull;
  int stall = 0;            // pt_debug_stall_barrier, one launch
  void* dbg_mem = nullptr;    // debug build: write tags and the check record, own allocation
  pt_free_fn dbg_free = nullptr;
  void* dbg_ctx = nullptr;
  uint64_t dbg_t0 = 0;        // debug build: sweeps done when the tags were last cleared
  void* band_mem = nullptr;   // the band form's second copy of colour 1 (dev.band_c1)
  pt_free_fn band_free = nullptr;
  void* band_ctx = nullptr;
  void* trace_mem = nullptr;  // observable trace ring (dev.trace_E / trace_M), own allocation
  size_t trace_bytes = 0;
  pt_free_fn trace_free = nullptr;
  void* trace_ctx = nullptr;
  // the page-locked creation image the first copy was queued from: kept until destroy, when
  // the stream has been synchronised (null when the image was not page-locked)
  std::shared_ptr<const void> image;
};

namespace ptb {
// Records the message for pt_last_error() and returns code.
int fail(int code, const char* fmt, ...);
int problem_fail(pt_problem* p, int code, const char* what, cudaError_t err);
int problem_check(pt_problem* p);
int problem_device_guard(pt_problem* p);
}  // namespace ptb
