// Covariance of a motion estimate ("Dense motion estimation", the paragraph
// after the update rule): one more iteration at the final pose, which does not
// update it, with the reference {I_A, W_A} bilateral-filtered before their
// gradients are taken; the covariance is the inverse of that iteration's
// normal matrix, Sigma = H_filt^-1.
//
//   bilateral_kernel   filters level 0 of the reference into a float (I, W)
//                      plane: each output pixel is the mean of its
//                      (2r+1)^2 window inside the image, weighted by
//                      exp(-d^2 / 2 sigma_s^2) exp(-(f(p) - f(q))^2 / 2 sigma_r^2);
//                      inverse depth only over valid neighbours, and a hole
//                      stays a hole.  The window, with its halo, is staged in
//                      shared memory once per block.
//   (the step)         initialisation, robust scale on the systematic sample
//                      at the given pose, one sweep whose central differences
//                      read the filtered plane, and the closing reduction into
//                      the result record (the alignment's kernels).
//   cov_inverse_kernel H_filt^-1 by an FP64 Cholesky factorisation on one
//                      lane and the six unit right-hand sides on six lanes.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "rgbid_device.cuh"
#include "rgbid_util.h"

namespace rgbid {

int enqueue_eval_step(const rgbid_pyramid* ref, const rgbid_pyramid* cur, int level, const double* T, int T_on_device,
                      const double* robust, const rgbid_align_params& p, void* workspace, float* r_I, float* r_W,
                      uint8_t* mask_I, uint8_t* mask_W, const float2* G, rgbid_align_result* d_result,
                      cudaStream_t stream);
size_t align_workspace_bytes(const rgbid_pyramid& ref);
int check_align_inputs(const rgbid_pyramid* ref, const rgbid_pyramid* cur, const rgbid_align_params* p);

constexpr int kBilTW = 32, kBilTH = 8, kBilMaxR = RGBID_BILATERAL_MAX_RADIUS;

struct BilateralArgs {
    const void* IW;            // level 0 of the reference, interleaved (I, W)
    int w, h, pitch, R;
    float inv2s, inv2rI, inv2rW;   // 1 / (2 sigma^2) of the spatial and the two range kernels
    float2* G;                 // output plane, same pitch
};

template <int PREC>
__global__ void __launch_bounds__(kBilTW * kBilTH) bilateral_kernel(BilateralArgs a) {
    constexpr int TW = kBilTW + 2 * kBilMaxR, TH = kBilTH + 2 * kBilMaxR;
    __shared__ float2 tile[TH][TW];
    __shared__ float gs[2 * kBilMaxR + 1][2 * kBilMaxR + 1];
    const int R = a.R;
    const int u0 = blockIdx.x * kBilTW - R, v0 = blockIdx.y * kBilTH - R;
    const int tw = kBilTW + 2 * R, th = kBilTH + 2 * R;
    const int t = threadIdx.y * kBilTW + threadIdx.x;
    for (int i = t; i < tw * th; i += kBilTW * kBilTH) {
        const int ty = i / tw, tx = i - ty * tw;
        const int u = u0 + tx, v = v0 + ty;
        float2 q = make_float2(0.f, 0.f);
        if (u >= 0 && v >= 0 && u < a.w && v < a.h)
            q = Pix<PREC>::load(a.IW, (int)in_plane(v * a.pitch + u, (long long)a.pitch * a.h));
        tile[ty][tx] = q;
    }
    for (int i = t; i < (2 * R + 1) * (2 * R + 1); i += kBilTW * kBilTH) {
        const int dy = i / (2 * R + 1) - R, dx = i % (2 * R + 1) - R;
        gs[dy + R][dx + R] = expf(-(float)(dx * dx + dy * dy) * a.inv2s);
    }
    __syncthreads();
    const int u = blockIdx.x * kBilTW + threadIdx.x, v = blockIdx.y * kBilTH + threadIdx.y;
    if (u >= a.w || v >= a.h) return;
    const float2 c = tile[threadIdx.y + R][threadIdx.x + R];
    float nI = 0.f, dI = 0.f, nW = 0.f, dW = 0.f;
    for (int dy = -R; dy <= R; ++dy) {
        if (v + dy < 0 || v + dy >= a.h) continue;
        for (int dx = -R; dx <= R; ++dx) {
            if (u + dx < 0 || u + dx >= a.w) continue;
            const float2 q = tile[threadIdx.y + R + dy][threadIdx.x + R + dx];
            const float g = gs[dy + R][dx + R];
            const float eI = q.x - c.x;
            const float kI = g * expf(-eI * eI * a.inv2rI);
            nI = fmaf(kI, q.x, nI);
            dI += kI;
            if (q.y > 0.f) {
                const float eW = q.y - c.y;
                const float kW = g * expf(-eW * eW * a.inv2rW);
                nW = fmaf(kW, q.y, nW);
                dW += kW;
            }
        }
    }
    a.G[(size_t)v * a.pitch + u] = make_float2(nI / dI, c.y > 0.f ? nW / dW : 0.f);
}

// Sigma = H^-1 of the result record's H (FP64).  Lane 0 factorises H = L L^T;
// lanes 0..5 each solve L L^T x = e_j for one column.  A matrix that is not
// positive definite, or fewer than `min_valid` residuals, gives Sigma = 0 and
// status DEGENERATE.
__global__ void cov_inverse_kernel(rgbid_align_result* res, double* Sigma, int min_valid) {
    __shared__ double L[6][6];
    __shared__ int ok_sh;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        bool ok = res->status == RGBID_OK && res->n_valid[0] + res->n_valid[1] >= min_valid;
        for (int j = 0; j < 6 && ok; ++j) {
            double d = res->H[j * 6 + j];
            for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
            if (!(d > 0.0)) {
                ok = false;
                break;
            }
            L[j][j] = sqrt(d);
            for (int i = j + 1; i < 6; ++i) {
                double x = res->H[i * 6 + j];
                for (int k = 0; k < j; ++k) x -= L[i][k] * L[j][k];
                L[i][j] = x / L[j][j];
            }
        }
        ok_sh = ok ? 1 : 0;
        if (!ok) res->status = RGBID_ERR_DEGENERATE;
    }
    __syncwarp();
    if (lane >= 6) return;
    const int j = lane;
    double y[6], x[6];
    if (!ok_sh) {
        for (int i = 0; i < 6; ++i) Sigma[i * 6 + j] = 0.0;
        return;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double t = (i == j) ? 1.0 : 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < i) t -= L[i][k] * y[k];
        y[i] = t / L[i][i];
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        double t = y[i];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k > i) t -= L[k][i] * x[k];
        x[i] = t / L[i][i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) Sigma[i * 6 + j] = x[i];
}

static size_t filtered_plane_bytes(const rgbid_pyramid& ref) {
    return align_up((size_t)ref.lv[0].pitch * ref.lv[0].height * sizeof(float2), 256);
}

}  // namespace rgbid

using namespace rgbid;

extern "C" void rgbid_default_bilateral(rgbid_bilateral* f) {
    if (!f) return;
    memset(f, 0, sizeof(*f));
    f->radius = 2;
    f->sigma_s = 1.5;
    f->sigma_r_I = 0.1;
    f->sigma_r_W = 0.01;
}

extern "C" size_t rgbid_covariance_workspace_bytes(const rgbid_pyramid* ref) {
    if (!ref || ref->levels < 1 || ref->levels > RGBID_MAX_LEVELS) return 0;
    return align_workspace_bytes(*ref) + filtered_plane_bytes(*ref);
}

extern "C" int rgbid_covariance(const rgbid_pyramid* ref, const rgbid_pyramid* cur, const double* T,
                                int T_on_device, const rgbid_align_params* params, const rgbid_bilateral* filter,
                                void* workspace, size_t workspace_bytes, rgbid_align_result* d_result,
                                double* d_sigma, void* stream_) {
    if (!params || !filter || !T || !d_result || !d_sigma) return RGBID_ERR_INVALID_ARG;
    rgbid_align_params p = *params;
    if (p.levels < 1) p.levels = 1;
    int chk = check_align_inputs(ref, cur, &p);
    if (chk != RGBID_OK) return chk;
    if (misaligned(d_result, 8) || misaligned(d_sigma, 8) || (T_on_device && misaligned(T, 8)))
        return RGBID_ERR_INVALID_ARG;
    if (filter->radius < 0 || filter->radius > kBilMaxR) return RGBID_ERR_INVALID_ARG;
    if (!(filter->sigma_s > 0.0) || !(filter->sigma_r_I > 0.0) || !(filter->sigma_r_W > 0.0) ||
        !std::isfinite(filter->sigma_s) || !std::isfinite(filter->sigma_r_I) || !std::isfinite(filter->sigma_r_W))
        return RGBID_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 255u) || workspace_bytes < rgbid_covariance_workspace_bytes(ref))
        return RGBID_ERR_WORKSPACE;
    cudaStream_t stream = (cudaStream_t)stream_;
    const size_t ab = align_workspace_bytes(*ref);
    float2* G = reinterpret_cast<float2*>((char*)workspace + ab);
    const rgbid_level& L0 = ref->lv[0];
    BilateralArgs ba;
    ba.IW = L0.IW;
    ba.w = L0.width;
    ba.h = L0.height;
    ba.pitch = L0.pitch;
    ba.R = filter->radius;
    ba.inv2s = (float)(1.0 / (2.0 * filter->sigma_s * filter->sigma_s));
    ba.inv2rI = (float)(1.0 / (2.0 * filter->sigma_r_I * filter->sigma_r_I));
    ba.inv2rW = (float)(1.0 / (2.0 * filter->sigma_r_W * filter->sigma_r_W));
    ba.G = G;
    dim3 blk(kBilTW, kBilTH);
    dim3 grd((L0.width + kBilTW - 1) / kBilTW, (L0.height + kBilTH - 1) / kBilTH);
    if (ref->precision == RGBID_PLANES_F32) bilateral_kernel<RGBID_PLANES_F32><<<grd, blk, 0, stream>>>(ba);
    else bilateral_kernel<RGBID_PLANES_BF16_F16><<<grd, blk, 0, stream>>>(ba);
    if (cudaGetLastError() != cudaSuccess) return RGBID_ERR_CUDA;
    int e = enqueue_eval_step(ref, cur, 0, T, T_on_device, nullptr, p, workspace, nullptr, nullptr, nullptr, nullptr,
                              G, d_result, stream);
    if (e != RGBID_OK) return e;
    cov_inverse_kernel<<<1, 32, 0, stream>>>(d_result, d_sigma, p.min_valid);
    return cudaGetLastError() == cudaSuccess ? RGBID_OK : RGBID_ERR_CUDA;
}

namespace rgbid {
// out-of-plane gathers counted by this translation unit's kernels (bounds-checked builds)
unsigned int oob_count_covariance() { return oob_count_this_unit(); }
}  // namespace rgbid
