// pt_persist.h -- the persistent single-problem sweep (one cooperative launch per call).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pt_launch.h"

namespace ptb {

constexpr int kPersistThreads = 256;
// Per-thread bit-sliced counts hold 4 x words per thread < 2^10; the warp sum < 2^15.
constexpr int kPersistMaxWordsPerThread = 255;
// Sweeps per launch: keeps the barrier targets of one launch (2 per sweep x CTAs) far
// below 2^31.
constexpr int kPersistChunk = 1 << 16;
constexpr int kPersistDefaultWords = 1;

// The largest grid that runs as one thread-block cluster (non-portable size on B300).
constexpr int kPersistMaxCluster = 16;

// The largest plane (both colours) that a CTA owning a whole plane keeps in shared memory.
constexpr int kPersistMaxLocalBytes = 64 * 1024;

struct PersistPlan {
  int grid;              // CTAs (a multiple of W), 0 when the problem does not fit one wave
  int words_per_thread;  // words of each colour per thread
  bool cluster;          // the grid can run as one cluster (hardware cluster barrier)
  bool local;            // one CTA per plane, its plane in shared memory
};

// The device count buffer holds, in 32-bit words: [2][W * 32] for the per-launch kernels,
// then two [2][W * 32] buffers for the persistent kernel and its barrier counter.
inline size_t count_words(int W) { return (size_t)6 * W * 32 + 16; }
inline size_t persist_clear_bytes(int W) { return ((size_t)4 * W * 32 + 1) * 4; }

size_t persist_smem(int R, int mode);
// Dynamic shared memory of a launch: persist_smem, then (local) the plane's L*L words.
size_t persist_launch_smem(int L, int R, int mode, bool local);
cudaError_t persist_plan(const DevProblem& p, const DeviceInfo& dev, int words_per_thread,
                         PersistPlan* plan);
cudaError_t launch_persist(const DevProblem& p, const PersistPlan& plan, uint64_t t0,
                           uint64_t e0, int n, int m, int stall, uint64_t limit_ns,
                           cudaStream_t st);

}  // namespace ptb
