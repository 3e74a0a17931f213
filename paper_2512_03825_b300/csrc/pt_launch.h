// pt_launch.h -- host-side entry points of the kernels (implemented in the .cu files).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pt_types.h"

namespace ptb {

struct DeviceInfo {
  int device;
  int sms;
  int cc_major, cc_minor;
  size_t smem_optin;  // max dynamic shared memory per block (opt-in)
};

enum StepFlags : int {
  kStepEnergy = 1,    // turn the accumulated counts into E_slot / M_slot and clear them
  kStepExchange = 2,  // one swap iteration
  kStepRebuild = 4,   // refresh the per-plane thresholds
  kStepTrace = 8,     // append the trace row of sweep t (after the other steps)
};

cudaError_t launch_init(const DevProblem& p, const DeviceInfo& dev, cudaStream_t st);
cudaError_t launch_half_sweep(const DevProblem& p, const DeviceInfo& dev, int colour,
                              uint64_t t, cudaStream_t st);
cudaError_t launch_energy(const DevProblem& p, const DeviceInfo& dev, cudaStream_t st);
cudaError_t launch_exchange(const DevProblem& p, uint64_t e, int flags, cudaStream_t st,
                            uint64_t t = 0);

// One problem's part of a batched read (pt_read_batch): its record of 1 + 3 R + 2 npairs
// 8-byte words starts `out` words into the packed buffer.
// One problem's record for k_gather. The gather first finishes the energy count as the
// energy exchange step does: E_slot / M_slot from the counts in cnt ([2][W * 32]), which
// it then clears.
struct GatherItem {
  int64_t* E_slot;
  int64_t* M_slot;
  const int32_t* slot_of_temp;
  const uint64_t* attempted;
  const uint64_t* accepted;
  const int32_t* status;
  uint32_t* cnt;
  int64_t J_int, h_int;
  int L, W;
  int R, npairs;  // npairs = R - 1 (0 for R = 1)
  int64_t out;
};
cudaError_t launch_gather(const GatherItem* items, int n, uint64_t* out, int sms,
                          cudaStream_t st);

// A run of colour-0 words of one plane of one problem for the batched energy count:
// words [first, first + count) of plane w, at most kEnergyChunkWords.
struct EnergyChunk {
  const uint32_t* spins;
  uint32_t* cnt;
  int L, W, w, first, count;
  DebugRecord* dbg;  // the debug build's record and status word of the problem (else unused)
  int32_t* status;
};
constexpr int kEnergyChunkWords = 2048;
// Counts unsatisfied bonds and up spins of every chunk into its problem's cnt (one block
// per chunk; the counts must start at zero).
cudaError_t launch_energy_batch(const EnergyChunk* chunks, int n, cudaStream_t st);

}  // namespace ptb
