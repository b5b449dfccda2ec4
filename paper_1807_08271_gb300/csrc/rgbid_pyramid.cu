// Pyramid construction ("Dense motion estimation", "Iterative optimisation").
//
// Level l+1 is the 2x2 box mean of level l: I = ((a + b) + (c + d)) / 4 and
// W = mean of the valid (> 0) children, 0 when none; odd sizes drop the last
// row/column; the intrinsics follow f <- f/2, c <- (c + 0.5)/2 - 0.5.
// A level-0 pixel whose I or W is not a finite number carries no measurement:
// it enters as a hole (W = 0), with I = 0 where I itself is not finite.
// Every level is computed in FP32 from the level-0 planes by the same
// quadtree of 2x2 means (so the reduced-precision storage form rounds each
// level once, never a rounded parent), and stored as interleaved (I, W) pairs.
#include <cstdint>
#include <cstring>

#include "rgbid_device.cuh"
#include "rgbid_util.h"

namespace rgbid {

struct PyrSrc {
    const float* I;
    const float* W;
    int pitch, rows;
};

struct IWf {
    float i, w, n;   // n: 1 if w is a valid measurement (used while combining)
};

__device__ __forceinline__ IWf combine4(const IWf& a, const IWf& b, const IWf& c, const IWf& d) {
    IWf o;
    o.i = ((a.i + b.i) + (c.i + d.i)) * 0.25f;
    const float za = a.w > 0.f ? a.w : 0.f, zb = b.w > 0.f ? b.w : 0.f;
    const float zc = c.w > 0.f ? c.w : 0.f, zd = d.w > 0.f ? d.w : 0.f;
    const float cnt = (float)((a.w > 0.f) + (b.w > 0.f) + (c.w > 0.f) + (d.w > 0.f));
    const float s = (za + zb) + (zc + zd);
    o.w = cnt > 0.f ? __fdiv_rn(s, cnt) : 0.f;
    o.n = cnt;
    return o;
}

// Value of level L at (x, y), computed from level 0 through the quadtree.
template <int L>
struct Down {
    static __device__ __forceinline__ IWf at(const PyrSrc& s, int x, int y) {
        const IWf a = Down<L - 1>::at(s, 2 * x, 2 * y);
        const IWf b = Down<L - 1>::at(s, 2 * x + 1, 2 * y);
        const IWf c = Down<L - 1>::at(s, 2 * x, 2 * y + 1);
        const IWf d = Down<L - 1>::at(s, 2 * x + 1, 2 * y + 1);
        return combine4(a, b, c, d);
    }
};

template <>
struct Down<0> {
    static __device__ __forceinline__ IWf at(const PyrSrc& s, int x, int y) {
        const long long o = in_plane((long long)y * s.pitch + x, (long long)s.pitch * s.rows);
        const float i = __ldg(s.I + o), w = __ldg(s.W + o);
        const bool fi = isfinite(i);
        IWf r;
        r.i = fi ? i : 0.f;
        r.w = (fi && isfinite(w)) ? w : 0.f;
        r.n = 1.f;
        return r;
    }
};

template <int PREC>
__device__ __forceinline__ void store_iw(void* base, size_t idx, float i, float w);

template <>
__device__ __forceinline__ void store_iw<RGBID_PLANES_F32>(void* base, size_t idx, float i, float w) {
    reinterpret_cast<float2*>(base)[idx] = make_float2(i, w);
}

template <>
__device__ __forceinline__ void store_iw<RGBID_PLANES_BF16_F16>(void* base, size_t idx, float i, float w) {
    const unsigned short bi = __bfloat16_as_ushort(__float2bfloat16_rn(i));
    const unsigned short hw = __half_as_ushort(__float2half_rn(w));
    reinterpret_cast<unsigned int*>(base)[idx] = (unsigned int)bi | ((unsigned int)hw << 16);
}

// Every level in one launch: block b belongs to the level whose block range holds
// it (the coarsest levels, whose pixels cost the most loads, come first), and
// each thread computes one pixel exactly as the per-level kernel does.
struct PyrLevelOut {
    void* dst;
    int w, h, pitch, bx, first_block;
};
struct PyrAll {
    PyrSrc src;
    int levels;
    PyrLevelOut lv[RGBID_MAX_LEVELS];
};

template <int PREC>
__global__ void __launch_bounds__(256) pyramid_all_kernel(PyrAll a) {
    const int b = blockIdx.x;
    int l = 0, best = -1;      // the level with the largest first block <= b
#pragma unroll
    for (int k = 0; k < RGBID_MAX_LEVELS; ++k)
        if (k < a.levels && a.lv[k].first_block <= b && a.lv[k].first_block > best) {
            best = a.lv[k].first_block;
            l = k;
        }
    void* dst = a.lv[0].dst;
    int w = a.lv[0].w, h = a.lv[0].h, pitch = a.lv[0].pitch, bx = a.lv[0].bx, fb = a.lv[0].first_block;
#pragma unroll
    for (int k = 1; k < RGBID_MAX_LEVELS; ++k)
        if (k == l) {
            dst = a.lv[k].dst;
            w = a.lv[k].w;
            h = a.lv[k].h;
            pitch = a.lv[k].pitch;
            bx = a.lv[k].bx;
            fb = a.lv[k].first_block;
        }
    const int lb = b - fb;
    const int x = (lb % bx) * 32 + (int)(threadIdx.x & 31);
    const int y = (lb / bx) * 8 + (int)(threadIdx.x >> 5);
    if (x >= w || y >= h) return;
    IWf v;
    switch (l) {
        case 0: v = Down<0>::at(a.src, x, y); break;
        case 1: v = Down<1>::at(a.src, x, y); break;
        case 2: v = Down<2>::at(a.src, x, y); break;
        case 3: v = Down<3>::at(a.src, x, y); break;
        case 4: v = Down<4>::at(a.src, x, y); break;
        default: v = Down<5>::at(a.src, x, y); break;
    }
    store_iw<PREC>(dst, (size_t)y * pitch + x, v.i, v.w);
}

static int level_pitch(int w) { return (w + 15) / 16 * 16; }
static size_t bytes_per_px(int prec) { return prec == RGBID_PLANES_F32 ? 8 : 4; }

}  // namespace rgbid

using namespace rgbid;

extern "C" size_t rgbid_pyramid_bytes(int width, int height, int levels, int precision) {
    if (width < 1 || height < 1 || levels < 1 || levels > RGBID_MAX_LEVELS) return 0;
    if (precision != RGBID_PLANES_F32 && precision != RGBID_PLANES_BF16_F16) return 0;
    size_t tot = 0;
    int w = width, h = height;
    for (int l = 0; l < levels; ++l) {
        tot += align_up((size_t)level_pitch(w) * h * bytes_per_px(precision), 256);
        w /= 2;
        h /= 2;
    }
    return tot;
}

extern "C" int rgbid_build_pyramid(const float* I0, const float* W0, int pitch0, int width, int height,
                                   rgbid_intrinsics K0, int levels, int precision, void* storage,
                                   size_t storage_bytes, rgbid_pyramid* out, void* stream_) {
    if (!I0 || !W0 || !out || levels < 1 || levels > RGBID_MAX_LEVELS || pitch0 < width) return RGBID_ERR_INVALID_ARG;
    if (precision != RGBID_PLANES_F32 && precision != RGBID_PLANES_BF16_F16) return RGBID_ERR_UNSUPPORTED;
    if (((uintptr_t)I0 & 3u) || ((uintptr_t)W0 & 3u)) return RGBID_ERR_INVALID_ARG;
    if ((width >> (levels - 1)) < 4 || (height >> (levels - 1)) < 4) return RGBID_ERR_INVALID_ARG;
    if (!intrinsics_ok(K0.fx, K0.fy, K0.cx, K0.cy)) return RGBID_ERR_INVALID_ARG;
    const size_t need = rgbid_pyramid_bytes(width, height, levels, precision);
    if (!storage || ((uintptr_t)storage & 255u) || storage_bytes < need) return RGBID_ERR_WORKSPACE;
    cudaStream_t stream = (cudaStream_t)stream_;
    rgbid_pyramid P;
    memset(&P, 0, sizeof(P));
    P.levels = levels;
    P.precision = precision;
    PyrAll all;
    memset(&all, 0, sizeof(all));
    all.src = PyrSrc{I0, W0, pitch0, height};
    all.levels = levels;
    char* base = (char*)storage;
    int w = width, h = height;
    rgbid_intrinsics K = K0;
    for (int l = 0; l < levels; ++l) {
        rgbid_level& L = P.lv[l];
        L.width = w;
        L.height = h;
        L.pitch = level_pitch(w);
        L.K = K;
        L.IW = base;
        all.lv[l] = PyrLevelOut{base, w, h, L.pitch, (w + 31) / 32, 0};
        base += align_up((size_t)L.pitch * h * bytes_per_px(precision), 256);
        w /= 2;
        h /= 2;
        K.fx *= 0.5;
        K.fy *= 0.5;
        K.cx = (K.cx + 0.5) * 0.5 - 0.5;
        K.cy = (K.cy + 0.5) * 0.5 - 0.5;
    }
    // block ranges, coarsest level first
    int nblocks = 0;
    for (int l = levels - 1; l >= 0; --l) {
        all.lv[l].first_block = nblocks;
        nblocks += all.lv[l].bx * ((all.lv[l].h + 7) / 8);
    }
    if (precision == RGBID_PLANES_F32) pyramid_all_kernel<RGBID_PLANES_F32><<<nblocks, 256, 0, stream>>>(all);
    else pyramid_all_kernel<RGBID_PLANES_BF16_F16><<<nblocks, 256, 0, stream>>>(all);
    if (cudaGetLastError() != cudaSuccess) return RGBID_ERR_CUDA;
    *out = P;
    return RGBID_OK;
}

namespace rgbid {
// out-of-plane gathers counted by this translation unit's kernels (bounds-checked builds)
unsigned int oob_count_pyramid() { return oob_count_this_unit(); }
}  // namespace rgbid
