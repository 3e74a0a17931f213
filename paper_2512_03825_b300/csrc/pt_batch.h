// pt_batch.h -- the batched path: many problems advanced by one persistent kernel.
#pragma once
#include <stdint.h>

#include "pt.h"

namespace ptb {
// Launch shape of the batched kernel: cluster = CTAs per cluster (1 = no clusters);
// problems with L >= joint_min_L are spread over a whole cluster, smaller ones run on one CTA.
struct BatchTuning {
  int cluster = 4;
  int joint_min_L = 128;
};
extern BatchTuning g_batch_tuning;

int sweep_batch(pt_problem* const* problems, int count, const int64_t* n,
                const int* exchange_every);
}  // namespace ptb
