// Host interface of the persistent per-level alignment kernel (rgbid_level.cu),
// used by rgbid_align for the levels whose systematic sample is every pixel.
#pragma once

#include <cuda_runtime.h>

#include "rgbid.h"
#include "rgbid_device.cuh"
#include "rgbid_nu.h"

namespace rgbid {

constexpr int kLevelCL = 16;                         // CTAs of the level kernel's cluster
constexpr int kLevelMaxPixels = kLevelCL * 256 * 5;  // pixels one launch holds (5 per thread)

struct LevelArgs {
    LevelDev A, B;
    AlignState* st;
    float2* partials;         // the workspace's block partials: the previous level's pending
                              // ones are read, then [0, kSlots) holds this level's last step
    int iters;                // Gauss-Newton iterations of the level (host count)
    const int* level_iters;   // device iterations per level (NULL: none); the level runs the minimum
    int level;
    int scale_iters, bisect_steps, estimate_nu, min_valid;
    float nu0;
    double nu_lo, nu_hi;
    float nu_g[kNuGTerms];    // Chebyshev series of the nu equation's constant part on [nu_lo, nu_hi]
};

// Whether a w x h level with sample cap `cap` runs in the level kernel on the current
// device (its sample is every pixel, the pixels fit one launch, and the device
// schedules the 16-CTA cluster with the kernel's shared memory).
bool level_kernel_takes(int precision, int w, int h, int cap);

// Enqueue the level kernel on `stream` (programmatic dependent launch).
cudaError_t launch_level(int precision, const LevelArgs& la, cudaStream_t stream);

}  // namespace rgbid
