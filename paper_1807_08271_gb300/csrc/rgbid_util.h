// Small host-side helpers shared by the rgbid translation units.
#pragma once
#include <cmath>
#include <cstddef>
#include <cstdint>

namespace rgbid {
static inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
// true if p is not a multiple of a (a power of two) bytes
static inline bool misaligned(const void* p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) != 0; }
// pinhole intrinsics usable by every kernel: finite, positive focal lengths
static inline bool intrinsics_ok(double fx, double fy, double cx, double cy) {
    return fx > 0.0 && fy > 0.0 && std::isfinite(fx) && std::isfinite(fy) && std::isfinite(cx) && std::isfinite(cy);
}
}  // namespace rgbid
