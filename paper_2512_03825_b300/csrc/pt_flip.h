// pt_flip.h -- the single-spin-flip variant (one cooperative launch per pt_flip call).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pt_types.h"

namespace ptb {

// n iterations of every replica from iteration it0 and swap index e0, a swap iteration after
// every m-th (0: none). Reads E_slot / M_slot (current) and writes them back.
cudaError_t launch_flip(const DevProblem& p, uint64_t it0, uint64_t e0, int64_t n, int m,
                        int stall, uint64_t limit_ns, cudaStream_t st);

// The shared-memory form: k replicas per 32-thread block (k a power of two, 0 when no k
// fits one resident wave or the shared memory of a CTA) and its dynamic shared memory.
int flip_smem_plan(const DevProblem& p, int sms, size_t smem_optin, int* k, size_t* bytes);
cudaError_t launch_flip_smem(const DevProblem& p, int k, size_t bytes, uint64_t it0,
                             uint64_t e0, int64_t n, int m, int stall, uint64_t limit_ns,
                             cudaStream_t st);

}  // namespace ptb
