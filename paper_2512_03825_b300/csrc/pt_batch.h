// pt_batch.h -- the batched path: many problems advanced by one persistent kernel.
#pragma once
#include <stdint.h>

#include <cuda_runtime.h>

#include "pt.h"

namespace ptb {
// Batched path: strategy PT_BATCH_FLAT or PT_BATCH_QUEUE (lock-step tiles, dealt by the
// host or handed out by a device queue, pt_flat.cu), PT_BATCH_FLOW (the same
// tiles in one persistent dataflow launch, pt_flow.cu) or PT_BATCH_CLUSTER (one persistent
// kernel of whole problems, pt_batch.cu). For the last, cluster = CTAs per cluster (1 = no
// clusters); problems with L >= joint_min_L are spread over a whole cluster, smaller ones run
// on one CTA.
// For the tile strategies, tile_words = target words per warp tile (tile_words / 32 words
// of one colour per lane).
struct BatchTuning {
  int strategy = PT_BATCH_FLAT;
  int cluster = 4;
  int joint_min_L = 128;
  int tile_words = 512;
  int streams = 1;  // PT_BATCH_FLAT / PT_BATCH_QUEUE: parts of the batch on their own streams
  int graphs = 0;   // PT_BATCH_FLAT / PT_BATCH_QUEUE: replay repeated batch shapes from graphs
};
extern BatchTuning g_batch_tuning;  // written and read under the library lock only
// A copy of the batch tuning, read under the library lock (the setters take it too).
BatchTuning batch_tuning();

struct DeviceInfo;
// The lock-step path (pt_flat.cu); problems are already checked.
// queued: tiles handed out by the device queue (PT_BATCH_QUEUE) instead of dealt by the host.
// streams: the batch is split into that many parts of about equal work, each advanced on its
// own stream (the first on st, the others on side streams forked from st and joined to it).
int sweep_batch_flat(pt_problem* const* ps, int count, const int64_t* n, const int* every,
                     cudaStream_t st, const DeviceInfo& di, int tile_words, bool queued,
                     int streams = 1, bool graphs = false);

// The dataflow path (pt_flow.cu); problems are already checked.
int sweep_batch_flow(pt_problem* const* ps, int count, const int64_t* n, const int* every,
                     cudaStream_t st, const DeviceInfo& di, int tile_words);

// The allocation-free variant of the lock-step path (pt_flat.cu); problems are checked.
// At most kStaticMaxBatch problems per call.
constexpr int kStaticMaxBatch = 2048;
int sweep_batch_static(pt_problem* const* ps, int count, const int64_t* n, const int* every,
                       cudaStream_t st, const DeviceInfo& di, int tile_words, bool queued);

int sweep_batch(pt_problem* const* problems, int count, const int64_t* n,
                const int* exchange_every);
int sweep_batch_static_entry(pt_problem* const* problems, int count, const int64_t* n,
                             const int* exchange_every);
}  // namespace ptb
