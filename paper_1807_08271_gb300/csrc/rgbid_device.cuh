// Device-side building blocks shared by the rgbid kernels (sm_103a).
//
// Per-pixel arithmetic is FP32.  The warp is written as an offset from the
// pixel itself: with q = K^-1 p, X_A = q / W_A and T = [R, t],
//   X_B = R^T (X_A - t) = (q + d) / W_A,   d = (R^T - I) q - W_A R^T t,
// so p_B - p = (fx (d_x - a d_z), fy (d_y - b d_z)) / (1 + d_z) with
// q = (a, b, 1).  The flow is small, so it keeps full FP32 relative precision
// where the absolute coordinate u_B (up to ~1300) would lose ~1e-4 px.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

#include "rgbid.h"

namespace rgbid {

constexpr int kSlots = 32;         // reduction slots: H (21) | g (6) | cost | n_I | n_W | 2 spare
constexpr int kSlotG = 21;
constexpr int kSlotCost = 27;
constexpr int kSlotNI = 28;
constexpr int kSlotNW = 29;

// Pose in the form the per-pixel warp consumes.
struct WarpPose {
    float E[9];     // R^T - I, row-major
    float s[3];     // R^T t
    float R2[3];    // third row of R
    float tz;       // t_z
};

static_assert(sizeof(WarpPose) == 16 * sizeof(float), "copied as 16 floats");

// Robust parameters consumed by the weights (per channel: mu, sigma^2 * nu, nu + 1, ok).
struct RobustParams {
    float mu[2];
    float sigma[2];
    float nu[2];
    int ok[2];
};

struct LevelDev {
    const void* IW;
    int w, h, pitch, pad;
    float fx, fy, cx, cy, ifx, ify;
};

// Hand-over between the roles of the split level kernel (the robust-scale cluster
// and the helper CTAs of one launch): flags counting published iterations, the
// helpers' arrivals and exits.  Zero between launches: the last CTA of a launch
// to leave resets it, and the alignment's initialisation clears it.
struct SplitMailbox {
    unsigned int pose_flag;  // iterations whose pose is published
    unsigned int rob_flag;   // iterations whose robust parameters are published
    unsigned int arrived;    // helper partials posted
    unsigned int exited;     // CTAs done with the mailbox
    int error;               // a wait ran out: every role gives up
    int pad[3];
    WarpPose wp;             // the published pose (FP32 warp form)
    RobustParams rob;        // the published robust parameters
};

// Device-resident state of one alignment (lives at the start of the workspace).
struct AlignState {
    double T[16];           // current estimate A_T_B
    WarpPose wp;            // FP32 warp parameters of T
    RobustParams rob;       // robust parameters of the current iteration
    unsigned int pending;   // blocks of the last sweep whose partials await reduction (0: none)
    int status;
    int iters_done;
    int iters_skipped;
    int timeouts;
    int pad[3];
    SplitMailbox mb;
};

// ---------------------------------------------------------------- pixel loads
template <int PREC>
struct Pix;

template <>
struct Pix<RGBID_PLANES_F32> {
    static constexpr int kBytes = 8;
    static __device__ __forceinline__ float2 load(const void* base, int idx) {
        return __ldg(reinterpret_cast<const float2*>(base) + idx);
    }
    // a pixel of a tile staged in shared memory
    static __device__ __forceinline__ float2 shared(const void* base, int idx) {
        return reinterpret_cast<const float2*>(base)[idx];
    }
};

template <>
struct Pix<RGBID_PLANES_BF16_F16> {
    static constexpr int kBytes = 4;
    static __device__ __forceinline__ float2 unpack(uint32_t raw) {
        __nv_bfloat16 i = __ushort_as_bfloat16((unsigned short)(raw & 0xffffu));
        __half w = __ushort_as_half((unsigned short)(raw >> 16));
        return make_float2(__bfloat162float(i), __half2float(w));
    }
    static __device__ __forceinline__ float2 load(const void* base, int idx) {
        return unpack(__ldg(reinterpret_cast<const unsigned int*>(base) + idx));
    }
    static __device__ __forceinline__ float2 shared(const void* base, int idx) {
        return unpack(reinterpret_cast<const unsigned int*>(base)[idx]);
    }
};

// ---------------------------------------------------------------- bounds-checked builds
// Built with -DRGBID_BOUNDS_CHECK (build(checked=True): librgbid_checked.so), every
// index gathered from an image plane is checked against the plane's allocation (rows x
// pitch elements).  An index outside it is counted in this translation unit's counter
// and replaced by element 0, so the kernel goes on without touching memory outside the
// plane; rgbid_debug_bounds_violations adds up the counters.  This stands in for a
// memory checker the GPUs do not offer here.  Without the macro the check compiles away.
#ifdef RGBID_BOUNDS_CHECK
static __device__ unsigned int g_oob_count;
#endif

__device__ __forceinline__ long long in_plane(long long idx, long long n) {
#ifdef RGBID_BOUNDS_CHECK
    if (idx < 0 || idx >= n) {
        atomicAdd(&g_oob_count, 1u);
        return 0;
    }
#endif
    return idx;
}

// pixel idx of a level's interleaved (I, W) plane
template <int PREC>
__device__ __forceinline__ float2 pix(const LevelDev& L, int idx) {
    return Pix<PREC>::load(L.IW, (int)in_plane(idx, (long long)L.pitch * L.h));
}

// This translation unit's count of out-of-plane indices since the library was loaded
// (0 in a build without the check; (unsigned)-1 if it cannot be read).
static inline unsigned int oob_count_this_unit() {
#ifdef RGBID_BOUNDS_CHECK
    unsigned int n = 0;
    if (cudaMemcpyFromSymbol(&n, g_oob_count, sizeof(n)) != cudaSuccess) {
        (void)cudaGetLastError();
        return ~0u;
    }
    return n;
#else
    return 0u;
#endif
}

// ---------------------------------------------------------------- per-pixel terms
struct PixelTerms {
    float rI, rW;        // residuals r(p, 0)
    float JI[6], JW[6];  // Jacobians (translation first)
    float lam;           // normal weight lambda_n
    bool mI, mW;         // masks
};

// Per-pixel evaluation in four stages so that a thread handling several pixels
// can issue all loads of one stage before it needs their values:
//   stage_a   load I_A, W_A at p and its 4-neighbours (central differences)
//   stage_w   warp p into B (eq. 3d_registration, pixel-offset form)
//   stage_b   load the four bilinear taps of B at p_B
//   finish    residuals r(p, 0) (eqs. res_int, res_depth), Jacobians
//             J = g [I | -[X_A]x] (eq. DeltaX) and the normal weight lambda_n.
struct PxA {
    float2 c, nl, nr, nu, nd;
    float a, b;
    bool ok;
};

struct PxW {
    float du, dv, ax, ay;
    int bi;
    bool ok;
};

struct PxB {
    float2 t00, t10, t01, t11;
};

template <int PREC>
__device__ __forceinline__ void stage_a(const LevelDev& A, int u, int v, PxA& s) {
    s.ok = !(u < 1 || v < 1 || u > A.w - 2 || v > A.h - 2);     // no central gradient on the border
    if (!s.ok) return;
    const int idx = v * A.pitch + u;
    s.c = pix<PREC>(A, idx);
    s.nl = pix<PREC>(A, idx - 1);
    s.nr = pix<PREC>(A, idx + 1);
    s.nu = pix<PREC>(A, idx - A.pitch);
    s.nd = pix<PREC>(A, idx + A.pitch);
    s.a = ((float)u - A.cx) * A.ifx;
    s.b = ((float)v - A.cy) * A.ify;
}

// stage_a from a tile of A staged in shared memory: `i` is the pixel's index in the
// tile, `tw` the tile's row length in pixels.
template <int PREC>
__device__ __forceinline__ void stage_a_shared(const LevelDev& A, const void* tile, int tw, int i, int u, int v,
                                               PxA& s) {
    s.ok = !(u < 1 || v < 1 || u > A.w - 2 || v > A.h - 2);
    if (!s.ok) return;
    s.c = Pix<PREC>::shared(tile, i);
    s.nl = Pix<PREC>::shared(tile, i - 1);
    s.nr = Pix<PREC>::shared(tile, i + 1);
    s.nu = Pix<PREC>::shared(tile, i - tw);
    s.nd = Pix<PREC>::shared(tile, i + tw);
    s.a = ((float)u - A.cx) * A.ifx;
    s.b = ((float)v - A.cy) * A.ify;
}

// stage_a with the neighbours (the central differences' taps) read from a float
// (I, W) plane G of A's size and pitch instead of A itself: the covariance
// iteration takes the gradients of the bilateral-filtered reference there, while
// the centre value (the warp, the residuals) stays A's.  G keeps A's holes.
template <int PREC>
__device__ __forceinline__ void stage_a_grad(const LevelDev& A, const float2* G, int u, int v, PxA& s) {
    s.ok = !(u < 1 || v < 1 || u > A.w - 2 || v > A.h - 2);
    if (!s.ok) return;
    const int idx = v * A.pitch + u;
    const long long n = (long long)A.pitch * A.h;
    s.c = pix<PREC>(A, idx);
    s.nl = __ldg(G + in_plane(idx - 1, n));
    s.nr = __ldg(G + in_plane(idx + 1, n));
    s.nu = __ldg(G + in_plane(idx - A.pitch, n));
    s.nd = __ldg(G + in_plane(idx + A.pitch, n));
    s.a = ((float)u - A.cx) * A.ifx;
    s.b = ((float)v - A.cy) * A.ify;
}

__device__ __forceinline__ void stage_w(const LevelDev& A, const LevelDev& B, const WarpPose& wp, int u, int v,
                                        const PxA& s, PxW& w) {
    w.ok = false;
    const float WA = s.c.y;
    if (!s.ok || !(WA > 0.f)) return;
    const float a = s.a, b = s.b;
    // d = (R^T - I) q - W_A R^T t
    const float dx = fmaf(wp.E[0], a, fmaf(wp.E[1], b, wp.E[2])) - WA * wp.s[0];
    const float dy = fmaf(wp.E[3], a, fmaf(wp.E[4], b, wp.E[5])) - WA * wp.s[1];
    const float dz = fmaf(wp.E[6], a, fmaf(wp.E[7], b, wp.E[8])) - WA * wp.s[2];
    const float mz = 1.f + dz;                       // Z_B * W_A
    if (!(mz > 0.f)) return;
    const float imz = 1.f / mz;
    w.du = A.fx * fmaf(-a, dz, dx) * imz;            // u_B - u
    w.dv = A.fy * fmaf(-b, dz, dy) * imz;            // v_B - v
    const float fdu = floorf(w.du), fdv = floorf(w.dv);
    if (!(fabsf(fdu) < 1.0e7f && fabsf(fdv) < 1.0e7f)) return;
    const int x0 = u + (int)fdu, y0 = v + (int)fdv;
    if (x0 < 0 || y0 < 0 || x0 > B.w - 2 || y0 > B.h - 2) return;
    w.ax = w.du - fdu;
    w.ay = w.dv - fdv;
    w.bi = y0 * B.pitch + x0;
    w.ok = true;
}

template <int PREC>
__device__ __forceinline__ void stage_b(const LevelDev& B, const PxW& w, PxB& t) {
    if (!w.ok) return;
    t.t00 = pix<PREC>(B, w.bi);
    t.t10 = pix<PREC>(B, w.bi + 1);
    t.t01 = pix<PREC>(B, w.bi + B.pitch);
    t.t11 = pix<PREC>(B, w.bi + B.pitch + 1);
}

// Jacobians (eq. DeltaX with the gradient terms of eqs. res_int / res_depth) and
// the normal weight lambda_n of a pixel of A whose masks are decided; W_B^gamma
// enters the inverse-depth row.
__device__ __forceinline__ void pixel_jacobians(const LevelDev& A, const PxA& s, bool okW, float WBw, PixelTerms& o) {
    const float WA = s.c.y, a = s.a, b = s.b;
    // g~_I = grad I_A (K - p e_z^T) = (gx fx, gy fy, -(gx fx a + gy fy b))
    const float gIx = 0.5f * (s.nr.x - s.nl.x) * A.fx;
    const float gIy = 0.5f * (s.nd.x - s.nu.x) * A.fy;
    const float gIz = -fmaf(gIx, a, gIy * b);
    // J_I = (W_A g~_I, q x g~_I), q = (a, b, 1)
    o.JI[0] = WA * gIx;
    o.JI[1] = WA * gIy;
    o.JI[2] = WA * gIz;
    o.JI[3] = fmaf(b, gIz, -gIy);
    o.JI[4] = fmaf(-a, gIz, gIx);
    o.JI[5] = fmaf(a, gIy, -b * gIx);
    if (okW) {
        const float gWx = 0.5f * (s.nr.y - s.nl.y) * A.fx;
        const float gWy = 0.5f * (s.nd.y - s.nu.y) * A.fy;
        const float gWz0 = -fmaf(gWx, a, gWy * b);
        const float gWz = gWz0 + WBw;      // + W_B^gamma e_z
        o.JW[0] = WA * gWx;
        o.JW[1] = WA * gWy;
        o.JW[2] = WA * gWz;
        o.JW[3] = fmaf(b, gWz, -gWy);
        o.JW[4] = fmaf(-a, gWz, gWx);
        o.JW[5] = fmaf(a, gWy, -b * gWx);
        // lambda_n = 1 / (|n_u| |q|), n_u = g~_W / W_A + e_z  (n_u . q = 1)
        const float iW = 1.f / WA;
        const float nx = gWx * iW, ny = gWy * iW, nz = fmaf(gWz0, iW, 1.f);
        const float nn = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
        const float qq = fmaf(a, a, fmaf(b, b, 1.f));
        o.lam = rsqrtf(nn * qq);
    } else {
        o.lam = 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) o.JW[k] = 0.f;
    }
}

template <bool WANT_J>
__device__ __forceinline__ void finish(const LevelDev& A, const WarpPose& wp, const PxA& s, const PxW& w,
                                       const PxB& t, PixelTerms& o) {
    o.mI = false;
    o.mW = false;
    o.rI = 0.f;
    o.rW = 0.f;
    if (!w.ok) return;
    const float WA = s.c.y, a = s.a, b = s.b, ax = w.ax, ay = w.ay;
    const float itop = fmaf(ax, t.t10.x - t.t00.x, t.t00.x);
    const float ibot = fmaf(ax, t.t11.x - t.t01.x, t.t01.x);
    const float IBw = fmaf(ay, ibot - itop, itop);
    o.mI = true;
    o.rI = IBw - s.c.x;

    float WBw = 0.f;
    bool okW = (t.t00.y > 0.f) && (t.t10.y > 0.f) && (t.t01.y > 0.f) && (t.t11.y > 0.f) &&
               (s.nl.y > 0.f) && (s.nr.y > 0.f) && (s.nu.y > 0.f) && (s.nd.y > 0.f);
    if (okW) {
        const float wtop = fmaf(ax, t.t10.y - t.t00.y, t.t00.y);
        const float wbot = fmaf(ax, t.t11.y - t.t01.y, t.t01.y);
        const float WBp = fmaf(ay, wbot - wtop, wtop);
        // W_B^gamma = 1 / e_z^T (R K^-1 p_B / W_B(p_B) + t) = W_B(p_B) / (R_2 . q_B + t_z W_B(p_B))
        const float qbx = a + w.du * A.ifx;
        const float qby = b + w.dv * A.ify;
        const float den = fmaf(wp.R2[0], qbx, fmaf(wp.R2[1], qby, wp.R2[2])) + wp.tz * WBp;
        okW = den > 0.f;
        if (okW) {
            WBw = WBp / den;
            o.rW = WBw - WA;
        }
    }
    o.mW = okW;
    if (!WANT_J) return;
    pixel_jacobians(A, s, okW, WBw, o);
}

// The same residuals and Jacobians from B's warped values given directly (the
// warp at full resolution, reading R22): mask_I needs A's measurement, the
// interior and the warped intensity's validity; mask_W adds the warped inverse
// depth's validity and valid neighbours for grad W.
template <bool WANT_J>
__device__ __forceinline__ void finish_given(const LevelDev& A, const PxA& s, float IBw, bool vI, float WBw, bool vW,
                                             PixelTerms& o) {
    o.mI = false;
    o.mW = false;
    o.rI = 0.f;
    o.rW = 0.f;
    const float WA = s.c.y;
    if (!s.ok || !(WA > 0.f) || !vI) return;
    o.mI = true;
    o.rI = IBw - s.c.x;
    const bool okW = vW && (s.nl.y > 0.f) && (s.nr.y > 0.f) && (s.nu.y > 0.f) && (s.nd.y > 0.f);
    if (okW) o.rW = WBw - WA;
    o.mW = okW;
    if (!WANT_J) return;
    pixel_jacobians(A, s, okW, WBw, o);
}

// ---------------------------------------------------------------- warp at full resolution (reading R22)
// B's maps warped towards A at a level-0 pixel p0, or reduced to a coarser level.
struct Warped {
    float I, W;
    bool vI, vW;
};

// One level-0 pixel: I_B(p_B) and the transferred inverse depth W_B^gamma, valid
// when A has a measurement at p0, p_B lies in front of B and is bilinear-valid
// (the intensity), and also has four valid W_B taps and a positive transferred
// depth (the inverse depth).  No interior condition: gradients are not taken here.
template <int PREC>
__device__ __forceinline__ Warped warp_leaf(const LevelDev& A0, const LevelDev& B0, const WarpPose& wp, int u0,
                                            int v0) {
    Warped r{0.f, 0.f, false, false};
    PxA s;
    s.ok = true;
    s.c = pix<PREC>(A0, v0 * A0.pitch + u0);
    s.a = ((float)u0 - A0.cx) * A0.ifx;
    s.b = ((float)v0 - A0.cy) * A0.ify;
    PxW w;
    stage_w(A0, B0, wp, u0, v0, s, w);
    if (!w.ok) return r;
    PxB t;
    stage_b<PREC>(B0, w, t);
    const float itop = fmaf(w.ax, t.t10.x - t.t00.x, t.t00.x);
    const float ibot = fmaf(w.ax, t.t11.x - t.t01.x, t.t01.x);
    r.I = fmaf(w.ay, ibot - itop, itop);
    r.vI = true;
    if ((t.t00.y > 0.f) && (t.t10.y > 0.f) && (t.t01.y > 0.f) && (t.t11.y > 0.f)) {
        const float wtop = fmaf(w.ax, t.t10.y - t.t00.y, t.t00.y);
        const float wbot = fmaf(w.ax, t.t11.y - t.t01.y, t.t01.y);
        const float WBp = fmaf(w.ay, wbot - wtop, wtop);
        const float qbx = s.a + w.du * A0.ifx;
        const float qby = s.b + w.dv * A0.ify;
        const float den = fmaf(wp.R2[0], qbx, fmaf(wp.R2[1], qby, wp.R2[2])) + wp.tz * WBp;
        if (den > 0.f) {
            r.W = WBp / den;
            r.vW = true;
        }
    }
    return r;
}

// Level-L pixel (u, v): the pyramid's rule applied to the warped maps, each with
// its own validity: the mean of the valid children in the order
// ((top-left + top-right) + (bottom-left + bottom-right)), valid when one child
// is.  The children are visited in a loop, so the code grows linearly in L.
template <int PREC, int L>
__device__ __forceinline__ Warped warped_down(const LevelDev& A0, const LevelDev& B0, const WarpPose& wp, int u,
                                              int v) {
    if constexpr (L == 0) {
        return warp_leaf<PREC>(A0, B0, wp, u, v);
    } else {
        float I0 = 0.f, I1 = 0.f, I2 = 0.f, I3 = 0.f, W0 = 0.f, W1 = 0.f, W2 = 0.f, W3 = 0.f;
        unsigned mI = 0u, mW = 0u;
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
            const Warped k = warped_down<PREC, L - 1>(A0, B0, wp, 2 * u + (c & 1), 2 * v + (c >> 1));
            const float ki = k.vI ? k.I : 0.f, kw = k.vW ? k.W : 0.f;
            if (c == 0) { I0 = ki; W0 = kw; }
            else if (c == 1) { I1 = ki; W1 = kw; }
            else if (c == 2) { I2 = ki; W2 = kw; }
            else { I3 = ki; W3 = kw; }
            mI |= (k.vI ? 1u : 0u) << c;
            mW |= (k.vW ? 1u : 0u) << c;
        }
        const int nI = __popc(mI), nW = __popc(mW);
        Warped r;
        r.vI = nI > 0;
        r.vW = nW > 0;
        r.I = nI > 0 ? ((I0 + I1) + (I2 + I3)) / (float)nI : 0.f;
        r.W = nW > 0 ? ((W0 + W1) + (W2 + W3)) / (float)nW : 0.f;
        return r;
    }
}

template <int PREC>
__device__ __forceinline__ Warped warped_at_level(int L, const LevelDev& A0, const LevelDev& B0, const WarpPose& wp,
                                                  int u, int v) {
    switch (L) {
        case 1: return warped_down<PREC, 1>(A0, B0, wp, u, v);
        case 2: return warped_down<PREC, 2>(A0, B0, wp, u, v);
        case 3: return warped_down<PREC, 3>(A0, B0, wp, u, v);
        case 4: return warped_down<PREC, 4>(A0, B0, wp, u, v);
        case 5: return warped_down<PREC, 5>(A0, B0, wp, u, v);
        default: return warped_down<PREC, 0>(A0, B0, wp, u, v);
    }
}

// Student-t weight omega(x, nu) / sigma^2 = (nu + 1) / (nu sigma^2 + (r - mu)^2).
__device__ __forceinline__ float robust_weight(float r, float mu, float sig, float nu) {
    const float d = r - mu;
    return __fdividef(nu + 1.f, fmaf(d, d, nu * sig * sig));
}

// ---------------------------------------------------------------- reductions
// Butterfly reduce-scatter: 32 per-lane values in, lane l returns the warp sum of value l.
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32]) {
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int n = 16; n >= 1; n >>= 1) {
        const bool upper = (lane & (unsigned)n) != 0u;
#pragma unroll
        for (int i = 0; i < n; ++i) {
            const float send = upper ? v[i] : v[i + n];
            const float keep = upper ? v[i + n] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, n);
        }
    }
    return v[0];
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ---------------------------------------------------------------- compensated sums
// Knuth TwoSum accumulation of floats: the pair (hi, lo) carries the rounding error.
struct F2 {
    float hi, lo;
    __device__ __forceinline__ void add(float b) {
        const float s = hi + b;
        const float bp = s - hi;
        const float e = (hi - (s - bp)) + (b - bp);
        hi = s;
        lo += e;
    }
    __device__ __forceinline__ void add(const F2& o) {
        add(o.hi);
        lo += o.lo;
    }
    __device__ __forceinline__ float value() const { return hi + lo; }
};
__device__ __forceinline__ F2 as_f2(float x) { return F2{x, 0.f}; }
__device__ __forceinline__ F2 as_f2(const F2& x) { return x; }

// Solve of the normal equations H xi = -g ("Iterative optimisation") for one
// thread: H is Jacobi-scaled to unit diagonal (D = diag(H)^-1/2, solve
// (D H D) y = -D g, xi = D y) and factorised by Cholesky in FP32 with pivot
// tolerance 1e-7 (the reduced-precision form refines the result to FP64
// accuracy, warp_solve6_refined below); a non-positive pivot reports a
// degenerate step.  H and g are read straight
// from the reduction slots `s` (H's upper triangle row by row in slots 0..20,
// g in kSlotG..kSlotG+5).  All 27 values are loaded into registers before the
// factorisation starts, so no shared-memory latency sits on its dependent
// chains.
template <typename Real>
struct CholTraits;
template <>
struct CholTraits<float> {
    static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float fma3(float a, float b, float c) { return fmaf(a, b, c); }
    static constexpr float kPivotMin = 1e-7f;
};

__host__ __device__ constexpr int upper_slot(int i, int j) { return i * (11 - i) / 2 + j; }   // i <= j

// Every loop below has a constant trip count and tests its bounds inside, so
// full unrolling turns each array index into a constant and the arrays live
// in registers.
template <typename Real>
__device__ __forceinline__ bool cholesky_solve6_slots(const float* s, Real xi[6]) {
    using C = CholTraits<Real>;
    float Hp[21], gp[6];
#pragma unroll
    for (int k = 0; k < 21; ++k) Hp[k] = s[k];
#pragma unroll
    for (int i = 0; i < 6; ++i) gp[i] = s[kSlotG + i];
    Real D[6], L[6][6], iL[6], y[6];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const Real hii = (Real)Hp[upper_slot(i, i)];
        ok = ok && hii > (Real)0;
        D[i] = C::rsq(hii);
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        Real d = (Real)Hp[upper_slot(j, j)] * D[j] * D[j];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < j) d = C::fma3(-L[j][k], L[j][k], d);
        ok = ok && d > C::kPivotMin;
        const Real r = C::rsq(d);
        L[j][j] = d * r;
        iL[j] = r;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            if (i > j) {
                Real t = (Real)Hp[upper_slot(j, i)] * D[i] * D[j];
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    if (k < j) t = C::fma3(-L[i][k], L[j][k], t);
                L[i][j] = t * r;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        Real t = -(Real)gp[i] * D[i];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < i) t = C::fma3(-L[i][k], y[k], t);
        y[i] = t * iL[i];
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        Real t = y[i];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k > i) t = C::fma3(-L[k][i], xi[k], t);
        xi[i] = t * iL[i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) xi[i] *= D[i];
    return ok;
}

// The FP32 factorisation and the substitutions of the same Jacobi-scaled
// Cholesky, kept apart so that one factorisation serves two right-hand sides
// (the refinement below).  D = diag(H)^-1/2; (D H D) = L L^T; iL = 1 / diag(L).
__device__ __forceinline__ bool chol6_factor_f(const float (&Hp)[21], float (&D)[6], float (&L)[6][6],
                                               float (&iL)[6]) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float hii = Hp[upper_slot(i, i)];
        ok = ok && hii > 0.f;
        D[i] = rsqrtf(hii);
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        float d = Hp[upper_slot(j, j)] * D[j] * D[j];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < j) d = fmaf(-L[j][k], L[j][k], d);
        ok = ok && d > CholTraits<float>::kPivotMin;
        const float r = rsqrtf(d);
        L[j][j] = d * r;
        iL[j] = r;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            if (i > j) {
                float t = Hp[upper_slot(j, i)] * D[i] * D[j];
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    if (k < j) t = fmaf(-L[i][k], L[j][k], t);
                L[i][j] = t * r;
            }
        }
    }
    return ok;
}

// x = H^-1 b with the factors of chol6_factor_f.
__device__ __forceinline__ void chol6_subst_f(const float (&D)[6], const float (&L)[6][6], const float (&iL)[6],
                                              const float (&b)[6], float (&x)[6]) {
    float y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        float t = b[i] * D[i];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < i) t = fmaf(-L[i][k], y[k], t);
        y[i] = t * iL[i];
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        float t = y[i];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k > i) t = fmaf(-L[k][i], x[k], t);
        x[i] = t * iL[i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) x[i] *= D[i];
}

// Solve of the reduced-precision form's normal equations H xi = -g, on one warp
// (all 32 lanes call; every lane returns the same verdict).  Lane 0 factorises
// the Jacobi-scaled H by Cholesky in FP32 and solves for x; lanes 0..5 form the
// residual rho = -g - H x in FP64 from the reduction's values; lane 0 solves
// H d = rho with the same factors, and xi = x + d is returned in FP64 (one step
// of mixed-precision iterative refinement, Wilkinson 1963 / Moler 1967).  H and
// g are sums held in FP32, and one refinement step brings x to the accuracy of
// an FP64 factorisation of them at about the cost of the FP32 solve: the FP64
// work is six lanes' six dependent FMAs and one add, where a factorisation in
// FP64 chains some hundred dependent FP64 operations on one lane.
// `x_sh` (float[6]), `d_sh` (float[6]), `rho_sh` and `xi_sh` (double[6]) are
// shared scratch of the calling warp; xi_sh is 0 when the verdict is false.
__device__ __forceinline__ bool warp_solve6_refined(const float* s, bool ok_in, float* x_sh, float* d_sh,
                                                    double* rho_sh, double* xi_sh) {
    const int lane = threadIdx.x & 31;
    float D[6], L[6][6], iL[6];
    int ok = 0;
    if (lane == 0) {
        float Hp[21], b[6], x[6];
#pragma unroll
        for (int k = 0; k < 21; ++k) Hp[k] = s[k];
#pragma unroll
        for (int i = 0; i < 6; ++i) b[i] = -s[kSlotG + i];
        ok = (ok_in && chol6_factor_f(Hp, D, L, iL)) ? 1 : 0;
        chol6_subst_f(D, L, iL, b, x);
#pragma unroll
        for (int i = 0; i < 6; ++i) x_sh[i] = x[i];
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    if (!ok) {
        if (lane < 6) xi_sh[lane] = 0.0;
        __syncwarp();
        return false;
    }
    if (lane < 6) {
        double acc = -(double)s[kSlotG + lane];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const int lo = lane < j ? lane : j, hi = lane < j ? j : lane;
            acc = fma(-(double)s[upper_slot(lo, hi)], (double)x_sh[j], acc);
        }
        rho_sh[lane] = acc;
    }
    __syncwarp();
    if (lane == 0) {
        float r[6], d[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) r[i] = (float)rho_sh[i];
        chol6_subst_f(D, L, iL, r, d);
#pragma unroll
        for (int i = 0; i < 6; ++i) d_sh[i] = d[i];
    }
    __syncwarp();
    if (lane < 6) xi_sh[lane] = (double)x_sh[lane] + (double)d_sh[lane];
    __syncwarp();
    return true;
}

// ---------------------------------------------------------------- warp-parallel pose arithmetic (double)
// FP64 on this part runs at ~1/64 of the FP32 rate with ~64-cycle latency, so
// the 4x4 pose products are spread over the lanes of one warp (one dependent
// chain of <= 4 FP64 operations per lane).

// out = warp pose of T (all 32 lanes call; T and out may be in shared or global memory).
// Every lane < 16 evaluates one field as a0 b0 + a1 b1 + a2 b2 + c with operands
// chosen by its index, so the warp issues the same three FP64 FMAs and one
// conversion whatever the field (divergent branches would each issue their own):
//   E_l (l < 9, i = l/3, j = l%3) = T_ji - delta_ij,   s_i (l = 9 + i) = sum_k T_ki T_k3,
//   R2_k (l = 12 + k) = T_2k,   tz (l = 15) = T_23.
__device__ __forceinline__ void warp_make_pose(const double* T, WarpPose* out) {
    const int lane = threadIdx.x & 31;
    if (lane < 16) {
        const bool e = lane < 9, sl = lane >= 9 && lane < 12;
        const int i = e ? lane / 3 : lane - 9, j = lane % 3;
        const int i0 = e ? j * 4 + i : (sl ? i : (lane < 15 ? 8 + (lane - 12) : 11));
        const double a0 = T[i0], b0 = sl ? T[3] : 1.0;
        const double a1 = sl ? T[4 + i] : 0.0, b1 = sl ? T[7] : 0.0;
        const double a2 = sl ? T[8 + i] : 0.0, b2 = sl ? T[11] : 0.0;
        const double c = (e && i == j) ? -1.0 : 0.0;
        reinterpret_cast<float*>(out)[lane] = (float)fma(a0, b0, fma(a1, b1, fma(a2, b2, c)));
    }
}

// T <- exp(xi)^-1 T with the decoupled exponential exp(xi) = [exp([theta]x), v; 0, 1]
// (Rodrigues with (1 - cos)/theta^2).  Called by all 32 lanes of one warp;
// xi is uniform across the warp; T is read and written in place (12 lanes write).
__device__ __forceinline__ void warp_apply_update(const float xi[6], double* T) {
    const int lane = threadIdx.x & 31;
    const float tx = xi[3], ty = xi[4], tz = xi[5];
    const float t2 = fmaf(tx, tx, fmaf(ty, ty, tz * tz));
    float A, B;
    if (t2 < 0.25f) {
        // sin t / t and (1 - cos t) / t^2 by their Taylor series (|t| < 0.5: the
        // first omitted terms are below 3e-11)
        A = 1.f - t2 * (1.f / 6.f - t2 * (1.f / 120.f - t2 * (1.f / 5040.f - t2 * (1.f / 362880.f))));
        B = 0.5f - t2 * (1.f / 24.f - t2 * (1.f / 720.f - t2 * (1.f / 40320.f - t2 * (1.f / 3628800.f))));
    } else {
        const float t = sqrtf(t2);
        float sn, cs;
        sincosf(t, &sn, &cs);
        A = sn / t;
        // 1 - cos t = 2 sin^2(t/2) avoids cancellation
        const float sh = sinf(0.5f * t);
        B = 2.f * sh * sh / t2;
    }
    // Mi = exp(xi)^-1 = [R^T, -R^T v], R = I + A [th]x + B ([th][th]^T - t2 I), row i of R^T = column i of R.
    // With R^T = I + D the new 3x4 block is T + (D T_{:,j} - [j = 3] (v + D v)): the correction is
    // formed in FP32 (|D| <= |theta|, so its rounding stays near 1e-8 of the pose's scale) and added
    // to the FP64 pose once, one FP64 add per entry instead of a 3x3 FP64 product.
    double Tn = 0.0;
    if (lane < 12) {
        const int i = lane >> 2, j = lane & 3;
        const float thi = i == 0 ? tx : (i == 1 ? ty : tz);
        const float th[3] = {tx, ty, tz};
        float D[3];   // row i of R^T - I: D_ik = R_ki - delta_ki
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float cross = 0.f;    // ([th]x)_ki
            if (k == 0 && i == 1) cross = -tz;
            if (k == 0 && i == 2) cross = ty;
            if (k == 1 && i == 0) cross = tz;
            if (k == 1 && i == 2) cross = -tx;
            if (k == 2 && i == 0) cross = -ty;
            if (k == 2 && i == 1) cross = tx;
            D[k] = fmaf(A, cross, B * fmaf(th[k], thi, k == i ? -t2 : 0.f));
        }
        float c = fmaf(D[0], (float)T[0 * 4 + j], fmaf(D[1], (float)T[1 * 4 + j], D[2] * (float)T[2 * 4 + j]));
        if (j == 3) {
            const float vi = i == 0 ? xi[0] : (i == 1 ? xi[1] : xi[2]);
            c -= vi + fmaf(D[0], xi[0], fmaf(D[1], xi[1], D[2] * xi[2]));
        }
        Tn = T[i * 4 + j] + (double)c;
    }
    __syncwarp();
    if (lane < 12) T[lane] = Tn;
    __syncwarp();
}

// FP64 variant (reduced-precision form): the step and the Rodrigues
// coefficients are double throughout.
__device__ __forceinline__ void warp_apply_update_d(const double xi[6], double* T) {
    const int lane = threadIdx.x & 31;
    const double tx = xi[3], ty = xi[4], tz = xi[5];
    const double t2d = tx * tx + ty * ty + tz * tz;
    double Ad, Bd;
    if (t2d < 1e-4) {
        // the same series to t^8 (|t| < 0.01: the first omitted terms are below 3e-28)
        Ad = 1.0 - t2d * (1.0 / 6.0 - t2d * (1.0 / 120.0 - t2d * (1.0 / 5040.0 - t2d * (1.0 / 362880.0))));
        Bd = 0.5 - t2d * (1.0 / 24.0 - t2d * (1.0 / 720.0 - t2d * (1.0 / 40320.0 - t2d * (1.0 / 3628800.0))));
    } else if (t2d < 0.25) {
        // Taylor series of sin t / t and (1 - cos t) / t^2 to t^16 (|t| < 0.5: error < 1e-19)
        Ad = 1.0 - t2d * (1.0 / 6.0 - t2d * (1.0 / 120.0 - t2d * (1.0 / 5040.0 - t2d * (1.0 / 362880.0 -
             t2d * (1.0 / 39916800.0 - t2d * (1.0 / 6227020800.0 - t2d * (1.0 / 1307674368000.0 -
             t2d * (1.0 / 355687428096000.0))))))));
        Bd = 0.5 - t2d * (1.0 / 24.0 - t2d * (1.0 / 720.0 - t2d * (1.0 / 40320.0 - t2d * (1.0 / 3628800.0 -
             t2d * (1.0 / 479001600.0 - t2d * (1.0 / 87178291200.0 - t2d * (1.0 / 20922789888000.0 -
             t2d * (1.0 / 6402373705728000.0))))))));
    } else {
        const double t = sqrt(t2d);
        double sn, cs;
        sincos(t, &sn, &cs);
        Ad = sn / t;
        const double sh = sin(0.5 * t);
        Bd = 2.0 * sh * sh / t2d;
    }
    double Tn = 0.0;
    if (lane < 12) {
        const int i = lane / 4, j = lane % 4;
        const double th[3] = {tx, ty, tz};
        double Rt[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double cross = 0.0;
            if (k == 0 && i == 1) cross = -th[2];
            if (k == 0 && i == 2) cross = th[1];
            if (k == 1 && i == 0) cross = th[2];
            if (k == 1 && i == 2) cross = -th[0];
            if (k == 2 && i == 0) cross = -th[1];
            if (k == 2 && i == 1) cross = th[0];
            Rt[k] = (k == i ? 1.0 : 0.0) + Ad * cross + Bd * (th[k] * th[i] - (k == i ? t2d : 0.0));
        }
        Tn = Rt[0] * T[0 * 4 + j] + Rt[1] * T[1 * 4 + j] + Rt[2] * T[2 * 4 + j];
        if (j == 3) Tn -= Rt[0] * xi[0] + Rt[1] * xi[1] + Rt[2] * xi[2];
    }
    __syncwarp();
    if (lane < 12) T[lane] = Tn;
    __syncwarp();
}

}  // namespace rgbid
