// Seeded synthetic RGB-D renderer on the GPU: the ray caster of textured boxes
// of raycast.c, in single precision, one thread per pixel and many images per
// launch.  It produces INPUT DATA only (camera depth and intensity per pixel)
// for large training sets; it holds none of the alignment arithmetic.
//
// Per image i: T_wc[i] (camera -> world, 4x4 row-major) and the boxes of scene
// scene_of[i] (BOX_STRIDE floats each: center[3], R_world_box[9] row-major,
// half[3], inside, texture id, texel size (m), texture offset u, v; a box with
// half[0] == 0 is absent).  Rays use the unnormalised direction K^-1 (u, v, 1),
// so the ray parameter at a hit is the camera-frame depth.
#include <cuda_runtime.h>

namespace {

constexpr int kBoxStride = 20;

__device__ float tex_lookup(const float* tex, int ts, float s, float t) {
    // periodic bilinear lookup in a ts x ts tile (ts a power of two)
    const float fs0 = floorf(s), ft0 = floorf(t);
    const float fs = s - fs0, ft = t - ft0;
    const long long is = (long long)fs0, it = (long long)ft0;
    const int m = ts - 1;
    const int x0 = (int)(is & m), x1 = (int)((is + 1) & m);
    const int y0 = (int)(it & m), y1 = (int)((it + 1) & m);
    const float a = tex[(size_t)y0 * ts + x0], b = tex[(size_t)y0 * ts + x1];
    const float c = tex[(size_t)y1 * ts + x0], d = tex[(size_t)y1 * ts + x1];
    const float top = a + (b - a) * fs, bot = c + (d - c) * fs;
    return top + (bot - top) * ft;
}

__global__ void render_kernel(int width, int height, float fx, float fy, float cx, float cy, const float* T_wc,
                              const int* scene_of, const float* boxes, int nbox, const float* textures,
                              int tex_size, float lx, float ly, float lz, float* depth_out, float* inten_out) {
    const int img = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= width * height) return;
    const int v = p / width, u = p - v * width;
    const float* T = T_wc + (size_t)img * 16;
    const float* S = boxes + (size_t)scene_of[img] * nbox * kBoxStride;
    const float dcx = ((float)u - cx) / fx, dcy = ((float)v - cy) / fy;
    const float dx = T[0] * dcx + T[1] * dcy + T[2];
    const float dy = T[4] * dcx + T[5] * dcy + T[6];
    const float dz = T[8] * dcx + T[9] * dcy + T[10];
    const float ox = T[3], oy = T[7], oz = T[11];
    float best_t = 3.0e38f;
    int best_box = -1, best_axis = 0;
    for (int b = 0; b < nbox; ++b) {
        const float* B = S + (size_t)b * kBoxStride;
        if (B[12] == 0.f) continue;
        const float* R = B + 3;
        const float px = ox - B[0], py = oy - B[1], pz = oz - B[2];
        const float lo[3] = {R[0] * px + R[3] * py + R[6] * pz, R[1] * px + R[4] * py + R[7] * pz,
                             R[2] * px + R[5] * py + R[8] * pz};
        const float ld[3] = {R[0] * dx + R[3] * dy + R[6] * dz, R[1] * dx + R[4] * dy + R[7] * dz,
                             R[2] * dx + R[5] * dy + R[8] * dz};
        float tmin = -3.0e38f, tmax = 3.0e38f;
        int amin = 0, amax = 0;
        bool miss = false;
        for (int k = 0; k < 3; ++k) {
            const float h = B[12 + k];
            if (ld[k] == 0.f) {
                if (lo[k] < -h || lo[k] > h) { miss = true; break; }
                continue;
            }
            const float t1 = (-h - lo[k]) / ld[k], t2 = (h - lo[k]) / ld[k];
            const float tn = fminf(t1, t2), tf = fmaxf(t1, t2);
            if (tn > tmin) { tmin = tn; amin = k; }
            if (tf < tmax) { tmax = tf; amax = k; }
        }
        if (miss || tmin > tmax) continue;
        const bool inside = B[15] != 0.f;
        const float t = inside ? tmax : tmin;
        const int axis = inside ? amax : amin;
        if (t <= 1e-6f || t >= best_t) continue;
        best_t = t;
        best_box = b;
        best_axis = axis;
    }
    const size_t idx = (size_t)img * width * height + p;
    if (best_box < 0) {
        depth_out[idx] = 0.f;
        inten_out[idx] = 0.f;
        return;
    }
    const float* B = S + (size_t)best_box * kBoxStride;
    const float* R = B + 3;
    const float hx = ox + best_t * dx - B[0], hy = oy + best_t * dy - B[1], hz = oz + best_t * dz - B[2];
    const float hl[3] = {R[0] * hx + R[3] * hy + R[6] * hz, R[1] * hx + R[4] * hy + R[7] * hz,
                         R[2] * hx + R[5] * hy + R[8] * hz};
    const int ia = (best_axis + 1) % 3, ib = (best_axis + 2) % 3;
    const float texel = B[17];
    const float face_off = 97.f * (float)best_axis + (hl[best_axis] > 0.f ? 41.f : 0.f);
    const float s = hl[ia] / texel + B[18] + face_off;
    const float tt = hl[ib] / texel + B[19] + face_off;
    const float* tex = textures + (size_t)((int)B[16]) * tex_size * tex_size;
    const float albedo = tex_lookup(tex, tex_size, s, tt);
    // Lambertian shade from a fixed directional light (face normal only)
    const float ndl = fabsf(R[best_axis] * lx + R[3 + best_axis] * ly + R[6 + best_axis] * lz);
    depth_out[idx] = best_t;
    inten_out[idx] = albedo * (0.55f + 0.45f * ndl);
}

}  // namespace

extern "C" int synth_render_gpu(int n_images, int width, int height, const float* K, const float* T_wc,
                                const int* scene_of, const float* boxes, int nbox, const float* textures,
                                int tex_size, const float* light, float* depth_out, float* inten_out, void* stream) {
    if (n_images <= 0 || width <= 0 || height <= 0 || nbox <= 0 || (tex_size & (tex_size - 1)) != 0) return 1;
    dim3 grid((unsigned)((width * height + 255) / 256), (unsigned)n_images);
    render_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(width, height, K[0], K[1], K[2], K[3], T_wc, scene_of, boxes,
                                                          nbox, textures, tex_size, light[0], light[1], light[2],
                                                          depth_out, inten_out);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
