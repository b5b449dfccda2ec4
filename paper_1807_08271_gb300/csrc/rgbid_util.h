// Small host-side helpers shared by the rgbid translation units.
#pragma once
#include <cstddef>

namespace rgbid {
static inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
}  // namespace rgbid
