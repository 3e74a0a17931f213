// Test helper: evaluates PyTorch's own header-only Philox4x32-10 engine
// (ATen/core/PhiloxRNGEngine.h) on the CPU, so that the oracle's Philox can be checked
// against an implementation written by someone else. Engine layout: key = {seed lo, seed hi},
// counter = {offset lo, offset hi, subsequence lo, subsequence hi}; the first four calls
// return the four words of the block at that counter.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>

extern "C" void torch_philox_blocks(const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                                    int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t* c = ctr + 4 * i;
        const uint32_t* k = key + 2 * i;
        uint64_t seed = (uint64_t)k[0] | ((uint64_t)k[1] << 32);
        uint64_t subseq = (uint64_t)c[2] | ((uint64_t)c[3] << 32);
        uint64_t offset = (uint64_t)c[0] | ((uint64_t)c[1] << 32);
        at::Philox4_32 eng(seed, subseq, offset);
        for (int j = 0; j < 4; ++j) out[4 * i + j] = eng();
    }
}
