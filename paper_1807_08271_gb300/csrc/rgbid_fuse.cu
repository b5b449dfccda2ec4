// Keyframe fusion ("Keyframe fusion", section "RGB-ID SLAM system"), keyframe
// initialisation, the dense covisibility ratio ("Dense frame covisibility
// ratio") with the covisibility-driven keyframe decision, and the small pose
// helpers of the tracking front-end.
//
// Fusion warps every keyframe pixel with W_kf > 0 into frame k by the inverse
// geometric warping (eq. 3d_registration with the pixel offset form of the
// alignment kernels), applies the visibility test of "Dense frame
// covisibility ratio" (|W_k(p_k) - w_k| < 3 sigma_W with w_k the keyframe
// point's inverse depth in frame k) and updates the weighted means in place:
//   W_kf <- (W_kf C_kf + C_k W_k*) / (C_kf + C_k),  C_kf <- C_kf + C_k,
// with W_k* = W_k(p_k) / (R_2 . K^-1 p_k + t_z W_k(p_k)) the transferred
// inverse depth and C_k = (dW_k*/dW_k)^-2 = (R_2 . K^-1 p_k + t_z W_k)^4 / (R_2 . K^-1 p_k)^2.
//
// Non-finite input carries no measurement: a keyframe pixel takes part only if
// its I_kf and W_kf are finite (and W_kf > 0), a tap of frame k is valid only
// if its I_k and W_k are finite (and W_k > 0), and the keyframe initialisation
// stores a pixel with a non-finite I or W as a hole (W = 0; I = 0 where I is
// not finite), as the pyramid does.
#include <cstdint>
#include <cstring>

#include "rgbid_device.cuh"
#include "rgbid_util.h"

namespace rgbid {

struct FuseArgs {
    float* I_kf;
    float* W_kf;
    float* C_kf;
    const float* I_k;
    const float* W_k;
    int pitch_kf, pitch_k, w, h;
    float fx, fy, cx, cy, ifx, ify;
    const double* T_dev;       // device pose (kf_T_k) or null
    const double* sigma_dev;   // device sigma_W or null
    double T_val[16];
    double sigma_val;
    int fuse_intensity;
    const int* switch_flag;    // device flag or null: when set, re-initialise the keyframe from frame k
};

__device__ __forceinline__ void init_keyframe_pixel(float* I_kf, float* W_kf, float* C_kf, size_t o, const float* I_k,
                                                    const float* W_k, size_t s) {
    const float ik = I_k[s], wk = W_k[s];
    const bool fi = isfinite(ik);
    I_kf[o] = fi ? ik : 0.f;
    W_kf[o] = (fi && isfinite(wk)) ? wk : 0.f;
    C_kf[o] = 1.f;
}

__global__ void __launch_bounds__(256) fuse_kernel(FuseArgs a) {
    __shared__ WarpPose sh_wp;
    __shared__ float sh_gate;
    __shared__ double sh_T[16];
    if (a.switch_flag && __ldcg(a.switch_flag)) {
        // the frame becomes the keyframe (a uniform branch: every thread reads the same flag)
        const int u = blockIdx.x * blockDim.x + threadIdx.x;
        const int v = blockIdx.y * blockDim.y + threadIdx.y;
        if (u < a.w && v < a.h)
            init_keyframe_pixel(a.I_kf, a.W_kf, a.C_kf, (size_t)v * a.pitch_kf + u, a.I_k, a.W_k,
                                (size_t)v * a.pitch_k + u);
        return;
    }
    if (threadIdx.y == 0) {           // warp 0 derives the FP32 warp pose from the FP64 pose
        const double* T = a.T_dev ? a.T_dev : a.T_val;
        if (threadIdx.x < 16) sh_T[threadIdx.x] = T[threadIdx.x];
        __syncwarp();
        warp_make_pose(sh_T, &sh_wp);
        if (threadIdx.x == 0) sh_gate = (float)(3.0 * (a.sigma_dev ? *a.sigma_dev : a.sigma_val));
    }
    __syncthreads();
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    if (u >= a.w || v >= a.h) return;
    const WarpPose& wp = sh_wp;
    const size_t o = (size_t)v * a.pitch_kf + u;
    const float Wkf = a.W_kf[o];
    const float Ikf = a.I_kf[o];
    if (!(Wkf > 0.f && isfinite(Wkf) && isfinite(Ikf))) return;
    const float qa = ((float)u - a.cx) * a.ifx;
    const float qb = ((float)v - a.cy) * a.ify;
    const float dx = fmaf(wp.E[0], qa, fmaf(wp.E[1], qb, wp.E[2])) - Wkf * wp.s[0];
    const float dy = fmaf(wp.E[3], qa, fmaf(wp.E[4], qb, wp.E[5])) - Wkf * wp.s[1];
    const float dz = fmaf(wp.E[6], qa, fmaf(wp.E[7], qb, wp.E[8])) - Wkf * wp.s[2];
    const float mz = 1.f + dz;                      // Z_k W_kf
    if (!(mz > 0.f)) return;
    const float imz = 1.f / mz;
    const float du = a.fx * fmaf(-qa, dz, dx) * imz;
    const float dv = a.fy * fmaf(-qb, dz, dy) * imz;
    const float fdu = floorf(du), fdv = floorf(dv);
    if (!(fabsf(fdu) < 1.0e7f && fabsf(fdv) < 1.0e7f)) return;
    const int x0 = u + (int)fdu, y0 = v + (int)fdv;
    if (x0 < 0 || y0 < 0 || x0 > a.w - 2 || y0 > a.h - 2) return;
    const float ax = du - fdu, ay = dv - fdv;
    const size_t bi = (size_t)y0 * a.pitch_k + x0;
    const long long nk = (long long)a.pitch_k * a.h;
    const long long b00 = in_plane((long long)bi, nk), b10 = in_plane((long long)bi + 1, nk);
    const long long b01 = in_plane((long long)bi + a.pitch_k, nk), b11 = in_plane((long long)bi + a.pitch_k + 1, nk);
    const float w00 = __ldg(a.W_k + b00), w10 = __ldg(a.W_k + b10);
    const float w01 = __ldg(a.W_k + b01), w11 = __ldg(a.W_k + b11);
    if (!(w00 > 0.f && w10 > 0.f && w01 > 0.f && w11 > 0.f)) return;
    const float i00 = __ldg(a.I_k + b00), i10 = __ldg(a.I_k + b10);
    const float i01 = __ldg(a.I_k + b01), i11 = __ldg(a.I_k + b11);
    // a tap is a measurement only if both of its values are finite (w > 0 is checked above)
    if (!(isfinite(w00) && isfinite(w10) && isfinite(w01) && isfinite(w11) && isfinite(i00) && isfinite(i10) &&
          isfinite(i01) && isfinite(i11)))
        return;
    const float wtop = fmaf(ax, w10 - w00, w00), wbot = fmaf(ax, w11 - w01, w01);
    const float Wkp = fmaf(ay, wbot - wtop, wtop);
    const float wB = Wkf * imz;                     // 1 / Z_k of the keyframe point
    if (!(fabsf(Wkp - wB) < sh_gate)) return;
    const float qbx = qa + du * a.ifx, qby = qb + dv * a.ify;
    const float ar = fmaf(wp.R2[0], qbx, fmaf(wp.R2[1], qby, wp.R2[2]));   // e_z^T R K^-1 p_k
    const float den = fmaf(wp.tz, Wkp, ar);
    if (!(den > 0.f)) return;
    const float Wstar = Wkp / den;
    const float den2 = den * den;
    const float Ck = __fdividef(den2 * den2, ar * ar);
    const float C = a.C_kf[o];
    const float inv = 1.f / (C + Ck);
    a.W_kf[o] = (Wkf * C + Ck * Wstar) * inv;
    if (a.fuse_intensity) {
        const float itop = fmaf(ax, i10 - i00, i00), ibot = fmaf(ax, i11 - i01, i01);
        const float Ik = fmaf(ay, ibot - itop, itop);
        a.I_kf[o] = (Ikf * C + Ck * Ik) * inv;
    }
    a.C_kf[o] = C + Ck;
}

__global__ void init_keyframe_kernel(float* I_kf, float* W_kf, float* C_kf, int pitch_kf, const float* I_k,
                                     const float* W_k, int pitch_k, int w, int h) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    if (u >= w || v >= h) return;
    init_keyframe_pixel(I_kf, W_kf, C_kf, (size_t)v * pitch_kf + u, I_k, W_k, (size_t)v * pitch_k + u);
}

// Warp-parallel rigid-transform arithmetic in FP64 (all 32 lanes call; the
// matrices live in shared memory; lanes 0..11 own entry (i, j) of the 3x4 block).
__device__ __forceinline__ void warp_rigid_mul(const double* A, const double* B, double* C) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    if (lane < 12) {
        const int i = lane >> 2, j = lane & 3;
        s = A[i * 4 + 0] * B[0 * 4 + j] + A[i * 4 + 1] * B[1 * 4 + j] + A[i * 4 + 2] * B[2 * 4 + j];
        if (j == 3) s += A[i * 4 + 3];
    }
    __syncwarp();
    if (lane < 12) C[lane] = s;
    else if (lane < 16) C[lane] = (lane == 15) ? 1.0 : 0.0;
    __syncwarp();
}

__device__ __forceinline__ void warp_rigid_inverse(const double* A, double* Ai) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    if (lane < 12) {
        const int i = lane >> 2, j = lane & 3;
        s = (j < 3) ? A[j * 4 + i] : -(A[0 * 4 + i] * A[3] + A[1 * 4 + i] * A[7] + A[2 * 4 + i] * A[11]);
    }
    __syncwarp();
    if (lane < 12) Ai[lane] = s;
    else if (lane < 16) Ai[lane] = (lane == 15) ? 1.0 : 0.0;
    __syncwarp();
}

// Project the rotation block onto SO(3) by Newton-Schulz iterations of the polar
// factor, X <- X (3 I - X^T X) / 2, which converge quadratically to the nearest
// orthonormal matrix.  Products of rotations read back from FP64 drift off SO(3)
// by rounding, and the constant-velocity composition T1 T2^-1 T1 with the
// transpose inverse amplifies that drift ~2.4x per frame unless it is removed.
__device__ __forceinline__ void warp_orthonormalize(double* T, double* M) {
    const int lane = threadIdx.x & 31;
    for (int it = 0; it < 3; ++it) {
        double m = 0.0;
        if (lane < 9) {
            const int i = lane / 3, j = lane % 3;
            m = T[0 * 4 + i] * T[0 * 4 + j] + T[1 * 4 + i] * T[1 * 4 + j] + T[2 * 4 + i] * T[2 * 4 + j];
        }
        __syncwarp();
        if (lane < 9) M[lane] = m;
        __syncwarp();
        double x = 0.0;
        if (lane < 9) {
            const int i = lane / 3, j = lane % 3;
            x = 0.5 * (3.0 * T[i * 4 + j] - (T[i * 4 + 0] * M[0 * 3 + j] + T[i * 4 + 1] * M[1 * 3 + j] +
                                             T[i * 4 + 2] * M[2 * 3 + j]));
        }
        __syncwarp();
        if (lane < 9) T[(lane / 3) * 4 + (lane % 3)] = x;
        __syncwarp();
    }
}

// rf_T_k(0) = rf_T_{k-1} (rf_T_{k-2})^-1 rf_T_{k-1} ("Camera tracking": constant velocity),
// with the rotation projected onto SO(3).
__global__ void predict_pose_kernel(const double* T1, const double* T2, double* out) {
    __shared__ double a[16], b[16], bi[16], m[16], r[16], M[9];
    const int lane = threadIdx.x & 31;
    if (lane < 16) { a[lane] = T1[lane]; b[lane] = T2[lane]; }
    __syncwarp();
    warp_rigid_inverse(b, bi);
    warp_rigid_mul(a, bi, m);
    warp_rigid_mul(m, a, r);
    warp_orthonormalize(r, M);
    if (lane < 16) out[lane] = r[lane];
}

__global__ void compose_pose_kernel(const double* A, int inv, const double* B, double* out) {
    __shared__ double a[16], b[16], ai[16], r[16];
    const int lane = threadIdx.x & 31;
    if (lane < 16) { a[lane] = A[lane]; b[lane] = B[lane]; }
    __syncwarp();
    if (inv) {
        warp_rigid_inverse(a, ai);
        warp_rigid_mul(ai, b, r);
    } else {
        warp_rigid_mul(a, b, r);
    }
    if (lane < 16) out[lane] = r[lane];
}

// ---------------------------------------------------------------- covisibility
// Dense covisibility ratio ("Dense frame covisibility ratio").  blockIdx.z = 0
// transfers the pixels of A into B with T = A_T_B, blockIdx.z = 1 those of B into
// A with T^-1 (eq. 3d_registration in the pixel-offset form of the alignment).
// A source pixel is in S_H when it is a measurement (W > 0, W and I finite); it
// is in S_V when its transfer lies in front of the other camera and the nearest
// pixel there, floor(p + 1/2), is inside the image, is a measurement, and its
// inverse depth is within 3 sigma_W of the transferred point's 1 / Z.  The
// counts are integer atomics: exact and independent of the order.
struct CovisArgs {
    const float* I[2];
    const float* W[2];
    int pitch[2];
    int w, h;
    float fx, fy, cx, cy, ifx, ify;
    const double* T_dev;
    const double* sigma_dev;
    double T_val[16];
    double sigma_val;
    unsigned int* counts;      // [S_V(A->B), S_H(A), S_V(B->A), S_H(B)]
};

__global__ void __launch_bounds__(256) covisibility_kernel(CovisArgs a) {
    __shared__ WarpPose sh_wp;
    __shared__ double sh_T[16], sh_Ti[16];
    __shared__ float sh_gate;
    __shared__ unsigned int sh_cnt[2];
    const int dir = blockIdx.z;
    if (threadIdx.y == 0) {
        const double* T = a.T_dev ? a.T_dev : a.T_val;
        if (threadIdx.x < 16) sh_T[threadIdx.x] = T[threadIdx.x];
        __syncwarp();
        if (dir == 1) {
            warp_rigid_inverse(sh_T, sh_Ti);
            warp_make_pose(sh_Ti, &sh_wp);
        } else {
            warp_make_pose(sh_T, &sh_wp);
        }
        if (threadIdx.x == 0) {
            sh_gate = (float)(3.0 * (a.sigma_dev ? *a.sigma_dev : a.sigma_val));
            sh_cnt[0] = 0u;
            sh_cnt[1] = 0u;
        }
    }
    __syncthreads();
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    const float* Is = a.I[dir];
    const float* Ws = a.W[dir];
    const float* Id = a.I[dir ^ 1];
    const float* Wd = a.W[dir ^ 1];
    const int ps = a.pitch[dir], pd = a.pitch[dir ^ 1];
    bool valid = false, visible = false;
    if (u < a.w && v < a.h) {
        const long long os = in_plane((long long)v * ps + u, (long long)ps * a.h);
        const float Ws_ = __ldg(Ws + os), Is_ = __ldg(Is + os);
        valid = Ws_ > 0.f && isfinite(Ws_) && isfinite(Is_);
        if (valid) {
            const WarpPose& wp = sh_wp;
            const float qa = ((float)u - a.cx) * a.ifx;
            const float qb = ((float)v - a.cy) * a.ify;
            const float dx = fmaf(wp.E[0], qa, fmaf(wp.E[1], qb, wp.E[2])) - Ws_ * wp.s[0];
            const float dy = fmaf(wp.E[3], qa, fmaf(wp.E[4], qb, wp.E[5])) - Ws_ * wp.s[1];
            const float dz = fmaf(wp.E[6], qa, fmaf(wp.E[7], qb, wp.E[8])) - Ws_ * wp.s[2];
            const float mz = 1.f + dz;                       // Z W of the source point
            if (mz > 0.f) {
                const float imz = 1.f / mz;
                const float du = a.fx * fmaf(-qa, dz, dx) * imz;
                const float dv = a.fy * fmaf(-qb, dz, dy) * imz;
                const float ru = floorf(du + 0.5f), rv = floorf(dv + 0.5f);
                if (fabsf(ru) < 1.0e7f && fabsf(rv) < 1.0e7f) {
                    const int xn = u + (int)ru, yn = v + (int)rv;
                    if (xn >= 0 && yn >= 0 && xn < a.w && yn < a.h) {
                        const long long od = in_plane((long long)yn * pd + xn, (long long)pd * a.h);
                        const float Wn = __ldg(Wd + od), In = __ldg(Id + od);
                        visible = Wn > 0.f && isfinite(Wn) && isfinite(In) && fabsf(Wn - Ws_ * imz) < sh_gate;
                    }
                }
            }
        }
    }
    const unsigned nv = __popc(__ballot_sync(0xffffffffu, valid));
    const unsigned ns = __popc(__ballot_sync(0xffffffffu, visible));
    if ((threadIdx.x & 31) == 0) {
        if (ns) atomicAdd(&sh_cnt[0], ns);
        if (nv) atomicAdd(&sh_cnt[1], nv);
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        if (sh_cnt[0]) atomicAdd(&a.counts[2 * dir + 0], sh_cnt[0]);
        if (sh_cnt[1]) atomicAdd(&a.counts[2 * dir + 1], sh_cnt[1]);
    }
}

__device__ __forceinline__ double covis_ratio(const unsigned int* c) {
    const double ab = c[1] ? (double)c[0] / (double)c[1] : 0.0;
    const double ba = c[3] ? (double)c[2] / (double)c[3] : 0.0;
    return ab < ba ? ab : ba;
}

__global__ void covisibility_ratio_kernel(const unsigned int* counts, float* ratio) {
    if (threadIdx.x == 0) *ratio = (float)covis_ratio(counts);
}

// Keyframe decision of the tracking front-end ("Keyframe fusion": a new keyframe
// when the covisibility of the current frame with the keyframe falls below a
// threshold) and the constant-velocity model's bookkeeping, on one warp:
//   switch:  T2 <- T_k^-1 T1 (frame k-1 in the new keyframe), T1 <- I;
//   else:    T2 <- T1, T1 <- T_k.
__global__ void keyframe_decide_kernel(const unsigned int* counts, double threshold, const double* Tk, double* T1,
                                       double* T2, int* flag, float* ratio) {
    __shared__ double k[16], ki[16], t1[16], r[16];
    const int lane = threadIdx.x & 31;
    const double vr = covis_ratio(counts);
    const bool sw = vr < threshold;
    if (lane < 16) {
        k[lane] = Tk[lane];
        t1[lane] = T1[lane];
    }
    __syncwarp();
    if (sw) {
        warp_rigid_inverse(k, ki);
        warp_rigid_mul(ki, t1, r);
        if (lane < 16) {
            T2[lane] = r[lane];
            T1[lane] = (lane % 5 == 0) ? 1.0 : 0.0;
        }
    } else if (lane < 16) {
        T2[lane] = t1[lane];
        T1[lane] = k[lane];
    }
    if (lane == 0) {
        *flag = sw ? 1 : 0;
        if (ratio) *ratio = (float)vr;
    }
}

}  // namespace rgbid

using namespace rgbid;

static int fuse_impl(float* I_kf, float* W_kf, float* C_kf, int pitch_kf, const float* I_k, const float* W_k,
                     int pitch_k, int width, int height, rgbid_intrinsics K, const double* T_kf_k,
                     const double* sigma_W, int params_on_device, int fuse_intensity, const int* switch_flag,
                     void* stream_) {
    if (!I_kf || !W_kf || !C_kf || !I_k || !W_k || !T_kf_k || !sigma_W) return RGBID_ERR_INVALID_ARG;
    if (misaligned(I_kf, 4) || misaligned(W_kf, 4) || misaligned(C_kf, 4) || misaligned(I_k, 4) || misaligned(W_k, 4))
        return RGBID_ERR_INVALID_ARG;
    if (params_on_device && (misaligned(T_kf_k, 8) || misaligned(sigma_W, 8))) return RGBID_ERR_INVALID_ARG;
    if (width < 2 || height < 2 || pitch_kf < width || pitch_k < width) return RGBID_ERR_INVALID_ARG;
    if (!intrinsics_ok(K.fx, K.fy, K.cx, K.cy)) return RGBID_ERR_INVALID_ARG;
    FuseArgs a;
    memset(&a, 0, sizeof(a));
    a.I_kf = I_kf; a.W_kf = W_kf; a.C_kf = C_kf; a.I_k = I_k; a.W_k = W_k;
    a.pitch_kf = pitch_kf; a.pitch_k = pitch_k; a.w = width; a.h = height;
    a.fx = (float)K.fx; a.fy = (float)K.fy; a.cx = (float)K.cx; a.cy = (float)K.cy;
    a.ifx = (float)(1.0 / K.fx); a.ify = (float)(1.0 / K.fy);
    if (params_on_device) {
        a.T_dev = T_kf_k;
        a.sigma_dev = sigma_W;
    } else {
        for (int i = 0; i < 16; ++i) a.T_val[i] = T_kf_k[i];
        a.sigma_val = *sigma_W;
    }
    a.fuse_intensity = fuse_intensity;
    a.switch_flag = switch_flag;
    dim3 blk(32, 8);
    dim3 grd((width + 31) / 32, (height + 7) / 8);
    fuse_kernel<<<grd, blk, 0, (cudaStream_t)stream_>>>(a);
    return cudaGetLastError() == cudaSuccess ? RGBID_OK : RGBID_ERR_CUDA;
}

extern "C" int rgbid_fuse_keyframe(float* I_kf, float* W_kf, float* C_kf, int pitch_kf, const float* I_k,
                                   const float* W_k, int pitch_k, int width, int height, rgbid_intrinsics K,
                                   const double* T_kf_k, const double* sigma_W, int params_on_device,
                                   int fuse_intensity, void* stream_) {
    return fuse_impl(I_kf, W_kf, C_kf, pitch_kf, I_k, W_k, pitch_k, width, height, K, T_kf_k, sigma_W,
                     params_on_device, fuse_intensity, nullptr, stream_);
}

extern "C" int rgbid_fuse_or_switch_keyframe(float* I_kf, float* W_kf, float* C_kf, int pitch_kf, const float* I_k,
                                             const float* W_k, int pitch_k, int width, int height,
                                             rgbid_intrinsics K, const double* T_kf_k, const double* sigma_W,
                                             int fuse_intensity, const int* d_switch, void* stream_) {
    if (!d_switch || misaligned(d_switch, 4)) return RGBID_ERR_INVALID_ARG;
    return fuse_impl(I_kf, W_kf, C_kf, pitch_kf, I_k, W_k, pitch_k, width, height, K, T_kf_k, sigma_W, 1,
                     fuse_intensity, d_switch, stream_);
}

extern "C" int rgbid_covisibility(const float* I_A, const float* W_A, int pitch_A, const float* I_B, const float* W_B,
                                  int pitch_B, int width, int height, rgbid_intrinsics K, const double* T_AB,
                                  const double* sigma_W, int params_on_device, unsigned int* d_counts,
                                  float* d_ratio, void* stream_) {
    if (!I_A || !W_A || !I_B || !W_B || !T_AB || !sigma_W || !d_counts) return RGBID_ERR_INVALID_ARG;
    if (misaligned(I_A, 4) || misaligned(W_A, 4) || misaligned(I_B, 4) || misaligned(W_B, 4) ||
        misaligned(d_counts, 4) || misaligned(d_ratio, 4))
        return RGBID_ERR_INVALID_ARG;
    if (params_on_device && (misaligned(T_AB, 8) || misaligned(sigma_W, 8))) return RGBID_ERR_INVALID_ARG;
    if (width < 1 || height < 1 || pitch_A < width || pitch_B < width) return RGBID_ERR_INVALID_ARG;
    if (!intrinsics_ok(K.fx, K.fy, K.cx, K.cy)) return RGBID_ERR_INVALID_ARG;
    CovisArgs a;
    memset(&a, 0, sizeof(a));
    a.I[0] = I_A; a.W[0] = W_A; a.pitch[0] = pitch_A;
    a.I[1] = I_B; a.W[1] = W_B; a.pitch[1] = pitch_B;
    a.w = width; a.h = height;
    a.fx = (float)K.fx; a.fy = (float)K.fy; a.cx = (float)K.cx; a.cy = (float)K.cy;
    a.ifx = (float)(1.0 / K.fx); a.ify = (float)(1.0 / K.fy);
    if (params_on_device) {
        a.T_dev = T_AB;
        a.sigma_dev = sigma_W;
    } else {
        for (int i = 0; i < 16; ++i) a.T_val[i] = T_AB[i];
        a.sigma_val = *sigma_W;
    }
    a.counts = d_counts;
    cudaStream_t stream = (cudaStream_t)stream_;
    if (cudaMemsetAsync(d_counts, 0, 4 * sizeof(unsigned int), stream) != cudaSuccess) return RGBID_ERR_CUDA;
    dim3 blk(32, 8);
    dim3 grd((width + 31) / 32, (height + 7) / 8, 2);
    covisibility_kernel<<<grd, blk, 0, stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return RGBID_ERR_CUDA;
    if (d_ratio) {
        covisibility_ratio_kernel<<<1, 32, 0, stream>>>(d_counts, d_ratio);
        if (cudaGetLastError() != cudaSuccess) return RGBID_ERR_CUDA;
    }
    return RGBID_OK;
}

extern "C" int rgbid_keyframe_decide(const unsigned int* d_counts, double threshold, const double* T_k, double* T1,
                                     double* T2, int* d_switch, float* d_ratio, void* stream_) {
    if (!d_counts || !T_k || !T1 || !T2 || !d_switch) return RGBID_ERR_INVALID_ARG;
    if (misaligned(d_counts, 4) || misaligned(T_k, 8) || misaligned(T1, 8) || misaligned(T2, 8) ||
        misaligned(d_switch, 4) || misaligned(d_ratio, 4))
        return RGBID_ERR_INVALID_ARG;
    if (!(threshold >= 0.0 && threshold <= 1.0)) return RGBID_ERR_INVALID_ARG;
    if (T1 == T2 || T_k == T1 || T_k == T2) return RGBID_ERR_INVALID_ARG;
    keyframe_decide_kernel<<<1, 32, 0, (cudaStream_t)stream_>>>(d_counts, threshold, T_k, T1, T2, d_switch, d_ratio);
    return cudaGetLastError() == cudaSuccess ? RGBID_OK : RGBID_ERR_CUDA;
}

extern "C" int rgbid_init_keyframe(float* I_kf, float* W_kf, float* C_kf, int pitch_kf, const float* I_k,
                                   const float* W_k, int pitch_k, int width, int height, void* stream_) {
    if (!I_kf || !W_kf || !C_kf || !I_k || !W_k || width < 1 || height < 1 || pitch_kf < width || pitch_k < width)
        return RGBID_ERR_INVALID_ARG;
    if (misaligned(I_kf, 4) || misaligned(W_kf, 4) || misaligned(C_kf, 4) || misaligned(I_k, 4) || misaligned(W_k, 4))
        return RGBID_ERR_INVALID_ARG;
    dim3 blk(32, 8);
    dim3 grd((width + 31) / 32, (height + 7) / 8);
    init_keyframe_kernel<<<grd, blk, 0, (cudaStream_t)stream_>>>(I_kf, W_kf, C_kf, pitch_kf, I_k, W_k, pitch_k, width,
                                                                height);
    return cudaGetLastError() == cudaSuccess ? RGBID_OK : RGBID_ERR_CUDA;
}

extern "C" int rgbid_predict_pose(const double* T_km1, const double* T_km2, double* T_out, void* stream_) {
    if (!T_km1 || !T_km2 || !T_out) return RGBID_ERR_INVALID_ARG;
    if (misaligned(T_km1, 8) || misaligned(T_km2, 8) || misaligned(T_out, 8)) return RGBID_ERR_INVALID_ARG;
    predict_pose_kernel<<<1, 32, 0, (cudaStream_t)stream_>>>(T_km1, T_km2, T_out);
    return cudaGetLastError() == cudaSuccess ? RGBID_OK : RGBID_ERR_CUDA;
}

extern "C" int rgbid_compose_pose(const double* A, int invert_A, const double* B, double* T_out, void* stream_) {
    if (!A || !B || !T_out || A == T_out) return RGBID_ERR_INVALID_ARG;
    if (misaligned(A, 8) || misaligned(B, 8) || misaligned(T_out, 8)) return RGBID_ERR_INVALID_ARG;
    compose_pose_kernel<<<1, 32, 0, (cudaStream_t)stream_>>>(A, invert_A, B, T_out);
    return cudaGetLastError() == cudaSuccess ? RGBID_OK : RGBID_ERR_CUDA;
}

extern "C" const char* rgbid_status_string(int status) {
    switch (status) {
        case RGBID_OK: return "RGBID_OK";
        case RGBID_ERR_INVALID_ARG: return "RGBID_ERR_INVALID_ARG";
        case RGBID_ERR_CUDA: return "RGBID_ERR_CUDA";
        case RGBID_ERR_WORKSPACE: return "RGBID_ERR_WORKSPACE";
        case RGBID_ERR_DEGENERATE: return "RGBID_ERR_DEGENERATE";
        case RGBID_ERR_TIMEOUT: return "RGBID_ERR_TIMEOUT";
        case RGBID_ERR_UNSUPPORTED: return "RGBID_ERR_UNSUPPORTED";
        default: return "RGBID_UNKNOWN_STATUS";
    }
}

extern "C" void rgbid_default_params(rgbid_align_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->levels = 3;
    p->iters[0] = 5;
    p->iters[1] = 5;
    p->iters[2] = 10;
    p->scale_iters = 10;
    p->bisect_steps = 20;
    p->sample_cap = RGBID_MAX_SAMPLES;
    p->estimate_nu = 1;
    p->min_valid = 60;
    p->nu0 = 5.0;
    p->nu_lo = 2.0;
    p->nu_hi = 10.0;
}

namespace rgbid {
// out-of-plane gathers counted by this translation unit's kernels (bounds-checked builds)
unsigned int oob_count_fuse() { return oob_count_this_unit(); }
}  // namespace rgbid
