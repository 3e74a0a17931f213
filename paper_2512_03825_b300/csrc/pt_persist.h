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

// The largest band (both colours' shared copies) that a CTA of the band form keeps in shared
// memory.
constexpr int kPersistMaxBandBytes = 48 * 1024;

// How the persistent kernel lays out a plane's words over its CTAs (a template parameter).
enum PersistForm : int {
  kFormStrided = 0,  // each thread takes every (CTAs x threads)-th word of a colour
  kFormLocal = 1,    // one CTA per plane, the whole plane in shared memory
  kFormBand = 2,     // each CTA owns a band of rows, shared copies, one grid barrier a sweep
};

// Whether a plan may or must use the band form.
enum BandChoice : int { kBandNever = 0, kBandAuto = 1, kBandForce = 2 };
// kBandAuto takes the band form where it measured faster: where the strided form would need
// a cooperative grid (more CTAs than one cluster takes) at one word per thread and the rows
// are at most this many words (L <= 128), so that bands of at least two rows plus their halo
// rows make one pass of a CTA. L = 128, R = 32: 7.23 -> 5.77 us per sweep with a swap
// iteration every sweep, 5.44 -> 4.11 without. The cluster grids of smaller lattices
// (L = 32, 64: 4.95 -> 5.17 and 5.08 -> 5.31 us) and the larger lattices (L = 256: 7.45 ->
// 8.99 us; L = 512 and 1024 lose 17-23%) keep the strided form.
constexpr int kBandAutoMaxHalf = 64;

struct PersistPlan {
  int grid;              // CTAs (a multiple of W), 0 when the problem does not fit one wave
  int words_per_thread;  // words of each colour per thread
  bool cluster;          // the grid can run as one cluster (hardware cluster barrier)
  bool local;            // one CTA per plane, its plane in shared memory
  bool band;             // the band form: a band of rows per CTA (grid / W bands per plane)
};

// The device count buffer holds, in 32-bit words: [2][W * 32] for the per-launch kernels,
// then three [2][W * 32] buffers for the persistent kernel and its barrier counter.
inline size_t count_words(int W) { return (size_t)8 * W * 32 + 16; }
inline size_t persist_clear_bytes(int W) { return ((size_t)6 * W * 32 + 1) * 4; }

size_t persist_smem(int R, int mode);
// Dynamic shared memory of a launch: persist_smem, then (kFormLocal) the plane's L*L words
// or (kFormBand, `bands` bands per plane) the band's shared copies.
size_t persist_launch_smem(int L, int R, int mode, int form, int bands);
// The launch shape for this problem; `band`: whether the band form may (kBandAuto: where it
// is the measured better form) or must be used (kBandForce: plan->grid = 0 if it cannot).
cudaError_t persist_plan(const DevProblem& p, const DeviceInfo& dev, int words_per_thread,
                         int band, PersistPlan* plan);
cudaError_t launch_persist(const DevProblem& p, const PersistPlan& plan, uint64_t t0,
                           uint64_t e0, int n, int m, int stall, uint64_t limit_ns,
                           cudaStream_t st);

}  // namespace ptb
