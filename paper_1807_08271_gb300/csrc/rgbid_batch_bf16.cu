// Instantiations of the persistent batched alignment kernel for bfloat16 I /
// binary16 W planes (one translation unit per plane precision so that they
// compile in parallel).
#include "rgbid_batch.cuh"

namespace rgbid {
template cudaError_t batch_dispatch<RGBID_PLANES_BF16_F16>(int, int, const BatchArgs*, int, int*, cudaStream_t);
}  // namespace rgbid

namespace rgbid {
// out-of-plane gathers counted by this translation unit's kernels (bounds-checked builds)
unsigned int oob_count_batch_bf16() { return oob_count_this_unit(); }
}  // namespace rgbid
