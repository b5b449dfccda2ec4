// Instantiations of the persistent batched alignment kernel for FP32 planes
// (one translation unit per plane precision so that they compile in parallel).
#include "rgbid_batch.cuh"

namespace rgbid {
template cudaError_t batch_dispatch<RGBID_PLANES_F32>(int, int, const BatchArgs*, int, int*, cudaStream_t);
}  // namespace rgbid
