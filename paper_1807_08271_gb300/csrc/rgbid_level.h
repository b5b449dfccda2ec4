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

// The split level kernel (a level whose sample is a strict subset of its pixels): one
// 16-CTA cluster solves, samples and estimates the robust parameters; helper CTAs of
// the same cooperative launch evaluate every pixel's terms as soon as the pose is
// published and accumulate them once the parameters are.
constexpr int kSplitTileW = 32, kSplitTileH = 8;   // one pixel per thread per tile
constexpr int kSplitTerms = 15;                    // per pixel in shared memory: r_I, r_W, J_I, J_W, lambda_n
constexpr int kSplitMaxTiles = 13;                 // tiles per helper CTA (shared memory)
constexpr int kSplitMaxHelpers = 8 * 16;           // helper CTAs at most (8 clusters)

// One level of a split-kernel launch (consecutive levels run in one launch, coarse to fine).
struct SplitLevel {
    LevelDev A, B;
    int level;                // pyramid level (the index into level_iters)
    int iters;                // Gauss-Newton iterations of the level (host count)
    int s, nsx, nsamp;        // the systematic sample
    int tiles_x, tiles_y;     // kSplitTileW x kSplitTileH tiles of the level
};
constexpr int kSplitMaxLevels = RGBID_MAX_LEVELS;

struct SplitArgs {
    SplitLevel lv[kSplitMaxLevels];
    int n_levels;             // levels of the launch, coarsest first
    AlignState* st;
    float2* partials;         // pending partials of the previous launch, then one per helper CTA
    const int* level_iters;
    int scale_iters, bisect_steps, estimate_nu, min_valid;
    float nu0;
    double nu_lo, nu_hi;
    float nu_g[kNuGTerms];
    int n_helpers;            // helper CTAs (the grid's CTAs after the first cluster)
    int max_tiles;            // tiles per helper CTA (the largest level's)
};

// Helper CTAs the split kernel launches on the current device (0: not available).
int split_kernel_helpers(int precision);
// Whether a w x h level runs in the split kernel (its tiles fit the helpers).
bool split_kernel_takes(int precision, int w, int h);
// Tiles per helper CTA that a w x h level needs with n_helpers helpers.
int split_tiles_per_helper(int w, int h, int n_helpers);
cudaError_t launch_split(int precision, const SplitArgs& sa, cudaStream_t stream);

// Whether a w x h level with sample cap `cap` runs in the level kernel on the current
// device (its sample is every pixel, the pixels fit one launch, and the device
// schedules the 16-CTA cluster with the kernel's shared memory).
bool level_kernel_takes(int precision, int w, int h, int cap);

// Enqueue the level kernel on `stream` (programmatic dependent launch).
cudaError_t launch_level(int precision, const LevelArgs& la, cudaStream_t stream);

}  // namespace rgbid
