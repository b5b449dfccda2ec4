// Host entry points of the batched alignment: argument checks, the per-device
// set-up of the persistent kernel, the launch, and the project's autotuner
// for the kernel's launch shape (cluster size, tile height, clusters launched).
#include <algorithm>
#include <cstring>
#include <vector>

#include "rgbid_batch.cuh"
#include "rgbid_util.h"

namespace rgbid {

// The kernels are instantiated in one translation unit per plane precision.
extern template cudaError_t batch_dispatch<RGBID_PLANES_F32>(int, int, const BatchArgs*, int, int*, cudaStream_t);
extern template cudaError_t batch_dispatch<RGBID_PLANES_BF16_F16>(int, int, const BatchArgs*, int, int*,
                                                                   cudaStream_t);

namespace {

constexpr int kMaxDev = 64;
constexpr int kClusterSizes[3] = {4, 8, 16};
constexpr int kRowOptions[3] = {1, 2, 4};
constexpr int kDefaultCluster = 8;
constexpr int kDefaultRows = 2;

// Resident clusters per device, precision and shape, plus one (0 = not queried
// yet).  A fixed property of the device and the compiled kernel.
int g_resident[kMaxDev][2][3][3];

int index_of(int v, const int (&tbl)[3]) {
    for (int i = 0; i < 3; ++i)
        if (tbl[i] == v) return i;
    return -1;
}

cudaError_t dispatch(int prec, int cl, int rows, const BatchArgs* a, int n_clusters, int* max_clusters,
                     cudaStream_t s) {
    return prec == RGBID_PLANES_F32
               ? batch_dispatch<RGBID_PLANES_F32>(cl, rows, a, n_clusters, max_clusters, s)
               : batch_dispatch<RGBID_PLANES_BF16_F16>(cl, rows, a, n_clusters, max_clusters, s);
}

int resident(int prec, int cl, int rows, int* out) {
    const int ci = index_of(cl, kClusterSizes), ri = index_of(rows, kRowOptions);
    if (ci < 0 || ri < 0) return RGBID_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return RGBID_ERR_CUDA;
    int& slot = g_resident[dev][prec][ci][ri];
    if (slot == 0) {
        int n = 0;
        if (dispatch(prec, cl, rows, nullptr, 0, &n, nullptr) != cudaSuccess) {
            (void)cudaGetLastError();
            return RGBID_ERR_CUDA;
        }
        slot = n + 1;
    }
    *out = slot - 1;
    return RGBID_OK;
}

int resolve_shape(const rgbid_batch_config* cfg, int* cl, int* rows, int* n_clusters) {
    *cl = kDefaultCluster;
    *rows = kDefaultRows;
    *n_clusters = 0;
    if (!cfg) return RGBID_OK;
    if (cfg->cluster) *cl = cfg->cluster;
    if (cfg->rows_per_warp) *rows = cfg->rows_per_warp;
    *n_clusters = cfg->n_clusters;
    if (index_of(*cl, kClusterSizes) < 0 || index_of(*rows, kRowOptions) < 0 || *n_clusters < 0)
        return RGBID_ERR_INVALID_ARG;
    return RGBID_OK;
}

int check_params(const rgbid_align_params* p) {
    if (!p) return RGBID_ERR_INVALID_ARG;
    if (p->sample_cap < 1 || p->sample_cap > RGBID_MAX_SAMPLES) return RGBID_ERR_INVALID_ARG;
    if (p->scale_iters < 0 || p->scale_iters > 1000 || p->bisect_steps < 0 || p->bisect_steps > 60)
        return RGBID_ERR_INVALID_ARG;
    if (!(p->nu_lo > 0.0) || !(p->nu_hi > p->nu_lo) || !(p->nu0 > 0.0) || !(p->nu_hi < 1e6)) return RGBID_ERR_INVALID_ARG;
    // the Chebyshev form of the robustness equation needs (lo + hi)/(hi - lo) >= 1.4
    if (p->nu_lo + p->nu_hi < 1.4 * (p->nu_hi - p->nu_lo)) return RGBID_ERR_UNSUPPORTED;
    // the batched kernel warps B at each level only
    if (p->warp_mode == RGBID_WARP_FULL_RESOLUTION) return RGBID_ERR_UNSUPPORTED;
    if (p->warp_mode != RGBID_WARP_PER_LEVEL) return RGBID_ERR_INVALID_ARG;
    return RGBID_OK;
}

}  // namespace
}  // namespace rgbid

using namespace rgbid;

extern "C" size_t rgbid_align_batched_workspace_bytes(void) { return sizeof(BatchWorkspace); }

extern "C" int rgbid_batch_check_item(const rgbid_batch_item* item, int precision) {
    if (!item) return RGBID_ERR_INVALID_ARG;
    if (precision != RGBID_PLANES_F32 && precision != RGBID_PLANES_BF16_F16) return RGBID_ERR_UNSUPPORTED;
    if (!item->result || ((uintptr_t)item->result & 7u)) return RGBID_ERR_INVALID_ARG;
    return batch_item_ok(*item, precision) ? RGBID_OK : RGBID_ERR_INVALID_ARG;
}

extern "C" int rgbid_batch_resident_clusters(int precision, const rgbid_batch_config* cfg, int* n_resident) {
    if (!n_resident) return RGBID_ERR_INVALID_ARG;
    if (precision != RGBID_PLANES_F32 && precision != RGBID_PLANES_BF16_F16) return RGBID_ERR_UNSUPPORTED;
    int cl, rows, ncl;
    const int rc = resolve_shape(cfg, &cl, &rows, &ncl);
    if (rc != RGBID_OK) return rc;
    return resident(precision, cl, rows, n_resident);
}

extern "C" int rgbid_align_batched(const rgbid_batch_item* d_items, int n_items, int precision,
                                   const rgbid_align_params* params, const rgbid_batch_config* cfg, void* workspace,
                                   size_t workspace_bytes, void* stream_) {
    if (precision != RGBID_PLANES_F32 && precision != RGBID_PLANES_BF16_F16) return RGBID_ERR_UNSUPPORTED;
    int rc = check_params(params);
    if (rc != RGBID_OK) return rc;
    int cl, rows, ncl_req;
    rc = resolve_shape(cfg, &cl, &rows, &ncl_req);
    if (rc != RGBID_OK) return rc;
    if (n_items < 0 || (n_items > 0 && !d_items) || misaligned(d_items, 8)) return RGBID_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 255u) || workspace_bytes < sizeof(BatchWorkspace))
        return RGBID_ERR_WORKSPACE;
    if (n_items == 0) return RGBID_OK;
    int maxc = 0;
    rc = resident(precision, cl, rows, &maxc);
    if (rc != RGBID_OK) return rc;
    if (maxc < 1) return RGBID_ERR_UNSUPPORTED;
    int ncl = ncl_req > 0 ? std::min(ncl_req, maxc) : maxc;
    ncl = std::min(ncl, n_items);

    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.items = d_items;
    a.ws = (BatchWorkspace*)workspace;
    a.n_items = n_items;
    a.precision = precision;
    a.scale_iters = params->scale_iters;
    a.bisect_steps = params->bisect_steps;
    a.sample_cap = params->sample_cap;
    a.estimate_nu = params->estimate_nu;
    a.min_valid = params->min_valid;
    a.nu0 = (float)params->nu0;
    a.nu_lo = (float)params->nu_lo;
    a.nu_hi = (float)params->nu_hi;
    nu_device_series(params->nu_lo, params->nu_hi, a.nu_g);

    cudaStream_t stream = (cudaStream_t)stream_;
    rgbid_timing* tm = params->timing;
    const bool tr = tm && tm->kernel == RGBID_KERNEL_BATCH && tm->count < tm->capacity;
    if (tr && cudaEventRecord((cudaEvent_t)tm->ev_start[tm->count], stream) != cudaSuccess) return RGBID_ERR_CUDA;
    if (dispatch(precision, cl, rows, &a, ncl, nullptr, stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return RGBID_ERR_CUDA;
    }
    if (tr) {
        if (cudaEventRecord((cudaEvent_t)tm->ev_end[tm->count], stream) != cudaSuccess) return RGBID_ERR_CUDA;
        tm->count += 1;
    }
    return RGBID_OK;
}

extern "C" int rgbid_batch_autotune(const rgbid_batch_item* d_items, int n_items, int precision,
                                    const rgbid_align_params* params, void* workspace, size_t workspace_bytes,
                                    int reps, rgbid_batch_config* best, float* best_ms, void* stream_) {
    if (!best || !best_ms || reps < 1 || reps > 100 || n_items < 1) return RGBID_ERR_INVALID_ARG;
    int rc = check_params(params);
    if (rc != RGBID_OK) return rc;
    rgbid_align_params p = *params;
    p.timing = nullptr;
    cudaStream_t stream = (cudaStream_t)stream_;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return RGBID_ERR_CUDA;
    }
    float best_t = -1.f;
    rgbid_batch_config best_c = {0, 0, 0, 0};
    rc = RGBID_OK;
    std::vector<float> times;
    for (int cl : kClusterSizes) {
        for (int rows : kRowOptions) {
            int maxc = 0;
            if (resident(precision, cl, rows, &maxc) != RGBID_OK || maxc < 1) continue;
            const int all = std::min(maxc, n_items);
            const int half = std::max(1, std::min(maxc / 2, n_items));
            for (int variant = 0; variant < 2; ++variant) {
                const int ncl = variant == 0 ? all : half;
                if (variant == 1 && half == all) continue;
                rgbid_batch_config c = {cl, rows, ncl, 0};
                rc = rgbid_align_batched(d_items, n_items, precision, &p, &c, workspace, workspace_bytes, stream_);
                if (rc != RGBID_OK) goto done;
                times.clear();
                for (int r = 0; r < reps; ++r) {
                    float ms = 0.f;
                    if (cudaEventRecord(e0, stream) != cudaSuccess) { rc = RGBID_ERR_CUDA; goto done; }
                    rc = rgbid_align_batched(d_items, n_items, precision, &p, &c, workspace, workspace_bytes, stream_);
                    if (rc != RGBID_OK) goto done;
                    if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        rc = RGBID_ERR_CUDA;
                        goto done;
                    }
                    times.push_back(ms);
                }
                std::sort(times.begin(), times.end());
                const float med = times[times.size() / 2];
                if (best_t < 0.f || med < best_t) {
                    best_t = med;
                    best_c = c;
                }
            }
        }
    }
    if (best_t < 0.f) rc = RGBID_ERR_UNSUPPORTED;
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == RGBID_OK) {
        *best = best_c;
        *best_ms = best_t;
    }
    return rc;
}
