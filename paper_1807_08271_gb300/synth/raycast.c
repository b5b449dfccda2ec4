/*
 * Seeded synthetic RGB-D renderer: a CPU ray caster of textured boxes.
 *
 * This file produces INPUT DATA only (intensity and camera depth per pixel).
 * It holds none of the alignment or fusion arithmetic. Scenes are built from
 * oriented boxes; a thin box stands in for a plane and a box whose `inside`
 * flag is set is seen from within (the walls of a room).
 *
 * Rays use the unnormalised direction K^-1 (u, v, 1) in the camera frame, so
 * the ray parameter at a hit equals the camera-frame depth z.
 *
 * Built with -ffp-contract=off and only IEEE +,-,*,/ so that x86-64 and
 * aarch64 hosts render bit-identical images.
 */
#include <stddef.h>

#define BOX_STRIDE 20

/* per box (doubles): center[3], R_world_box[9] row-major, half[3], inside,
 * texture id, texel size (m), texture offset u, texture offset v */

static double tex_lookup(const float* tex, int ts, double s, double t)
{
    /* periodic bilinear lookup in a ts x ts tile (ts a power of two) */
    double fs = s - (double)(long long)s;
    double ft = t - (double)(long long)t;
    long long is = (long long)s, it = (long long)t;
    if (fs < 0) { fs += 1.0; is -= 1; }
    if (ft < 0) { ft += 1.0; it -= 1; }
    int m = ts - 1;
    int x0 = (int)(is & m), x1 = (int)((is + 1) & m);
    int y0 = (int)(it & m), y1 = (int)((it + 1) & m);
    double a = tex[(size_t)y0 * ts + x0], b = tex[(size_t)y0 * ts + x1];
    double c = tex[(size_t)y1 * ts + x0], d = tex[(size_t)y1 * ts + x1];
    double top = a + (b - a) * fs;
    double bot = c + (d - c) * fs;
    return top + (bot - top) * ft;
}

void rgbid_synth_raycast(int width, int height, const double* K /* fx fy cx cy */,
                         const double* T_wc /* 4x4 row-major, camera -> world */,
                         int nbox, const double* boxes, int tex_size,
                         const float* textures, const double* light /* unit 3-vector */,
                         double* depth_out, double* inten_out)
{
    const double fx = K[0], fy = K[1], cx = K[2], cy = K[3];
    const double ox = T_wc[3], oy = T_wc[7], oz = T_wc[11];
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int v = 0; v < height; ++v) {
        for (int u = 0; u < width; ++u) {
            double dcx = ((double)u - cx) / fx, dcy = ((double)v - cy) / fy, dcz = 1.0;
            double dx = T_wc[0] * dcx + T_wc[1] * dcy + T_wc[2] * dcz;
            double dy = T_wc[4] * dcx + T_wc[5] * dcy + T_wc[6] * dcz;
            double dz = T_wc[8] * dcx + T_wc[9] * dcy + T_wc[10] * dcz;
            double best_t = 1e300;
            int best_box = -1, best_axis = 0;
            for (int b = 0; b < nbox; ++b) {
                const double* B = boxes + (size_t)b * BOX_STRIDE;
                const double* R = B + 3;
                double px = ox - B[0], py = oy - B[1], pz = oz - B[2];
                /* box-local origin and direction: R^T (.) */
                double lo[3] = { R[0] * px + R[3] * py + R[6] * pz,
                                 R[1] * px + R[4] * py + R[7] * pz,
                                 R[2] * px + R[5] * py + R[8] * pz };
                double ld[3] = { R[0] * dx + R[3] * dy + R[6] * dz,
                                 R[1] * dx + R[4] * dy + R[7] * dz,
                                 R[2] * dx + R[5] * dy + R[8] * dz };
                double tmin = -1e300, tmax = 1e300;
                int amin = 0, amax = 0, miss = 0;
                for (int k = 0; k < 3; ++k) {
                    double h = B[12 + k];
                    if (ld[k] == 0.0) {
                        if (lo[k] < -h || lo[k] > h) { miss = 1; break; }
                        continue;
                    }
                    double t1 = (-h - lo[k]) / ld[k], t2 = (h - lo[k]) / ld[k];
                    double tn = t1 < t2 ? t1 : t2, tf = t1 < t2 ? t2 : t1;
                    if (tn > tmin) { tmin = tn; amin = k; }
                    if (tf < tmax) { tmax = tf; amax = k; }
                }
                if (miss || tmin > tmax) continue;
                double t; int axis;
                if (B[15] != 0.0) { t = tmax; axis = amax; }      /* seen from inside */
                else { t = tmin; axis = amin; }
                if (t <= 1e-6 || t >= best_t) continue;
                best_t = t; best_box = b; best_axis = axis;
            }
            size_t idx = (size_t)v * width + u;
            if (best_box < 0) { depth_out[idx] = 0.0; inten_out[idx] = 0.0; continue; }
            const double* B = boxes + (size_t)best_box * BOX_STRIDE;
            const double* R = B + 3;
            double hx = ox + best_t * dx - B[0], hy = oy + best_t * dy - B[1], hz = oz + best_t * dz - B[2];
            double hl[3] = { R[0] * hx + R[3] * hy + R[6] * hz,
                             R[1] * hx + R[4] * hy + R[7] * hz,
                             R[2] * hx + R[5] * hy + R[8] * hz };
            int ia = (best_axis + 1) % 3, ib = (best_axis + 2) % 3;
            double texel = B[17];
            double face_off = 97.0 * (double)best_axis + (hl[best_axis] > 0 ? 41.0 : 0.0);
            double s = (hl[ia] / texel) + B[18] + face_off;
            double tt = (hl[ib] / texel) + B[19] + face_off;
            const float* tex = textures + (size_t)((int)B[16]) * tex_size * tex_size;
            double albedo = tex_lookup(tex, tex_size, s, tt);
            /* Lambertian shade of the face from a fixed directional light:
             * depends on the face normal only, not on the viewpoint */
            double nx = R[0 + best_axis], ny = R[3 + best_axis], nz = R[6 + best_axis];
            double ndl = nx * light[0] + ny * light[1] + nz * light[2];
            if (ndl < 0) ndl = -ndl;
            double shade = 0.55 + 0.45 * ndl;
            depth_out[idx] = best_t;
            inten_out[idx] = albedo * shade;
        }
    }
}
