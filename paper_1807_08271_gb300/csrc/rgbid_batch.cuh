// Persistent batched alignment kernel (sm_103a).
//
// One thread-block cluster per alignment, many alignments per launch.  Each
// cluster pops a pair from a device queue and runs its whole coarse-to-fine
// IRLS Gauss-Newton alignment ("Dense motion estimation", "Iterative
// optimisation") without leaving the cluster:
//   sample    the <= 19200 systematic-sample residuals r(p, 0) are computed
//             by all CTAs and kept in each CTA's shared memory;
//   robust    Student-t (mu, sigma) at nu0 by the lagged-weight fixed point and
//             nu by bisection on the robustness equation ("Error distribution
//             and robust optimisation"), each sum exchanged between the CTAs
//             through distributed shared memory; the bisection runs in every
//             CTA on identical sums, so every CTA holds the same parameters;
//   sweep     the CTAs stride over 32 x (8 R) pixel tiles of the level: warp,
//             residuals, Jacobians, weights, and the 27 normal-equation terms
//             (plus cost and counts) accumulated per tile in FP32 and across
//             tiles in compensated FP32 pairs; one exchange sums the CTAs;
//   update    every CTA solves H xi = -g (Jacobi-scaled Cholesky; FP64 for the
//             reduced-precision planes) and applies T <- exp(xi)^-1 T to its
//             copy of the FP64 pose; the copies stay bit-identical.
// All cluster sums use one fixed combine order, so every CTA takes the same
// branches.  The only global synchronisation is the queue's atomic counter.
#pragma once

#include <cooperative_groups.h>

#include "rgbid_cluster.cuh"
#include "rgbid_device.cuh"

namespace rgbid {

constexpr int kBatchNT = 256;                  // threads per CTA (two 128-thread groups bisect nu)
constexpr int kBatchMaxNV = 2 * kChebVals;     // widest exchange: the Chebyshev sums of both channels
constexpr int kBatchMaxIters = 10000;
constexpr int kBatchMaxDim = 16384;
constexpr int kSlotTimeout = 30;               // spare reduction slot: expired waits of the cluster

// Queue state in the caller's workspace (zero between batches).
struct BatchWorkspace {
    unsigned int head;       // next queue position
    unsigned int exited;     // clusters that found the queue empty
    int pad[62];
};
static_assert(sizeof(BatchWorkspace) == 256, "one 256-byte block");

struct BatchArgs {
    const rgbid_batch_item* items;
    BatchWorkspace* ws;
    int n_items;
    int precision;
    int scale_iters, bisect_steps, sample_cap, estimate_nu, min_valid;
    float nu0, nu_lo, nu_hi;
    float nu_g[kNuGTerms];    // Chebyshev series of the nu equation's constant part on [nu_lo, nu_hi]
};

// Per-alignment descriptors held in each CTA's shared memory.
struct BatchJob {
    LevelDev A[RGBID_MAX_LEVELS];
    LevelDev B[RGBID_MAX_LEVELS];
    int iters[RGBID_MAX_LEVELS];
    int lvbad[RGBID_MAX_LEVELS];
    int levels;
    int bad;
    rgbid_align_result* res;
};

__host__ __device__ inline int batch_sample_stride(int w, int h, int cap) {
    int s = 1;
    while ((long long)((w + s - 1) / s) * ((h + s - 1) / s) > cap) ++s;
    return s;
}

// The argument rules of rgbid_align for one level pair (and the kernel's index range).
__host__ __device__ inline bool batch_level_ok(const rgbid_level& a, const rgbid_level& b, int precision) {
    const uintptr_t align = precision == RGBID_PLANES_F32 ? 8u : 4u;
    if (!a.IW || !b.IW) return false;
    if (((uintptr_t)a.IW & (align - 1)) || ((uintptr_t)b.IW & (align - 1))) return false;
    if (a.width != b.width || a.height != b.height) return false;
    if (a.width < 4 || a.height < 4 || a.width > kBatchMaxDim || a.height > kBatchMaxDim) return false;
    if (a.pitch < a.width || b.pitch < b.width || a.pitch > 4 * kBatchMaxDim || b.pitch > 4 * kBatchMaxDim)
        return false;
    if (a.K.fx != b.K.fx || a.K.fy != b.K.fy || a.K.cx != b.K.cx || a.K.cy != b.K.cy) return false;
    if (!(a.K.fx > 0.0) || !(a.K.fy > 0.0) || !(a.K.fx < 1e30) || !(a.K.fy < 1e30)) return false;
    if (!(a.K.cx == a.K.cx) || !(a.K.cy == a.K.cy)) return false;
    return true;
}

__host__ __device__ inline bool batch_item_ok(const rgbid_batch_item& it, int precision) {
    if (it.levels < 1 || it.levels > RGBID_MAX_LEVELS) return false;
    if (it.ref.levels < it.levels || it.ref.levels > RGBID_MAX_LEVELS) return false;
    if (it.cur.levels < it.levels || it.cur.levels > RGBID_MAX_LEVELS) return false;
    if (it.ref.precision != precision || it.cur.precision != precision) return false;
    for (int l = 0; l < it.levels; ++l) {
        if (it.iters[l] < 0 || it.iters[l] > kBatchMaxIters) return false;
        if (!batch_level_ok(it.ref.lv[l], it.cur.lv[l], precision)) return false;
    }
    return true;
}

__device__ __forceinline__ LevelDev batch_level_dev(const rgbid_level& L) {
    LevelDev d;
    d.IW = L.IW;
    d.w = L.width;
    d.h = L.height;
    d.pitch = L.pitch;
    d.pad = 0;
    d.fx = (float)L.K.fx;
    d.fy = (float)L.K.fy;
    d.cx = (float)L.K.cx;
    d.cy = (float)L.K.cy;
    d.ifx = (float)(1.0 / L.K.fx);
    d.ify = (float)(1.0 / L.K.fy);
    return d;
}

// Push exchange of compensated partials between the CTAs of a cluster (the
// protocol of the per-iteration robust kernel: st.async into every CTA's
// receive buffer, completion counted on the receiver's mbarrier, two buffers
// alternating by round parity).  A wait that runs out of budget marks the CTA
// as failed; later waits of a failed CTA give up at once.
template <int CL>
struct BatchXchg {
    float2 (*recv)[CL][kBatchMaxNV];
    unsigned long long* mbar;
    volatile int* failed;
    uint32_t rank;
    int round;

    // A round in three parts, as in the per-iteration kernel: thread 0 arms this
    // CTA's barrier for CL x NV values; send(t, r, s) pushes this CTA's partial of
    // value t into CTA r; threads t < NV receive the total of value t, summed in
    // rank order by the same pairwise tree in every CTA.  The caller ends the round
    // with __syncthreads and next().
    template <int NV>
    __device__ __forceinline__ void arm() {
        if (threadIdx.x == 0) mbar_arrive_expect_tx(&mbar[round & 1], (uint32_t)(CL * NV * sizeof(float2)));
    }
    __device__ __forceinline__ void send(int t, int r, F2 s) {
        const int par = round & 1;
        st_async_f2(map_to_rank(smem_addr(&recv[par][rank][t]), (uint32_t)r), s.hi, s.lo,
                    map_to_rank(smem_addr(&mbar[par]), (uint32_t)r));
    }
    // One thread per value t < NV sends it to every CTA itself and receives.
    template <int NV>
    __device__ __forceinline__ F2 exchange(int t, F2 s) {
        if (t == 0) mbar_arrive_expect_tx(&mbar[round & 1], (uint32_t)(CL * NV * sizeof(float2)));
#pragma unroll
        for (int r = 0; r < CL; ++r) send(t, r, s);
        return receive<NV>(t);
    }
    template <int NV>
    __device__ __forceinline__ F2 receive(int t) {
        const int par = round & 1;
        const uint32_t phase = (uint32_t)(round >> 1) & 1u;
        const long long budget = *failed ? 0 : kWaitBudgetCycles;
        const long long t0 = clock64();
        while (!mbar_try_wait(&mbar[par], phase)) {
            if (clock64() - t0 > budget) {
                *failed = 1;
                break;
            }
        }
        F2 acc[CL];
#pragma unroll
        for (int r = 0; r < CL; ++r) {
            const float2 p = recv[par][r][t];
            acc[r] = F2{p.x, p.y};
        }
#pragma unroll
        for (int step = 1; step < CL; step <<= 1)
#pragma unroll
            for (int r = 0; r < CL; ++r)      // constant trip count: acc stays in registers
                if (r % (2 * step) == 0 && r + step < CL) acc[r].add(acc[r + step]);
        return acc[0];
    }
    __device__ __forceinline__ void next() { ++round; }
};

// A round of NV <= 8 cluster sums of per-thread values (warp sums, then a
// compensated pairwise tree over the warps, then the exchange with its CL x NV
// stores spread over the threads); totals land in tot[0, NV).
template <int CL, int NV>
__device__ __forceinline__ void batch_round_small(BatchXchg<CL>& X, float (&v)[NV], float (*red_w)[64], float* tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const float x = warp_sum(v[j]);
        if (lane == 0) red_w[warp][j] = x;
    }
    __syncthreads();
    X.template arm<NV>();
    for (int p = (int)threadIdx.x; p < NV * CL; p += kBatchNT) {
        const int t = p / CL, r = p - t * CL;
        X.send(t, r, warp_tree<kBatchNT / 32>(red_w, t));
    }
    if ((int)threadIdx.x < NV) tot[threadIdx.x] = X.template receive<NV>((int)threadIdx.x).value();
    __syncthreads();
    X.next();
}

// Uniform parameters (level, pose, robust constants) are re-read from shared
// memory at each stage with broadcast vector loads instead of being held in
// registers across the tile loop; the volatile loads cannot be hoisted.
__device__ __forceinline__ float4 lds_f4(const void* p) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(smem_addr(p)));
    return v;
}

__device__ __forceinline__ LevelDev lds_level(const LevelDev* p) {
    static_assert(sizeof(LevelDev) == 48, "three 16-byte loads");
    const float4 q0 = lds_f4(p), q1 = lds_f4(reinterpret_cast<const char*>(p) + 16),
                 q2 = lds_f4(reinterpret_cast<const char*>(p) + 32);
    LevelDev d;
    const unsigned long long lo = __float_as_uint(q0.x), hi = __float_as_uint(q0.y);
    d.IW = reinterpret_cast<const void*>(lo | (hi << 32));
    d.w = __float_as_int(q0.z);
    d.h = __float_as_int(q0.w);
    d.pitch = __float_as_int(q1.x);
    d.pad = 0;
    d.fx = q1.z;
    d.fy = q1.w;
    d.cx = q2.x;
    d.cy = q2.y;
    d.ifx = q2.z;
    d.ify = q2.w;
    return d;
}

__device__ __forceinline__ WarpPose lds_pose(const WarpPose* p) {
    WarpPose w;
    float* o = reinterpret_cast<float*>(&w);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 q = lds_f4(reinterpret_cast<const float*>(p) + 4 * i);
        o[4 * i] = q.x;
        o[4 * i + 1] = q.y;
        o[4 * i + 2] = q.z;
        o[4 * i + 3] = q.w;
    }
    return w;
}

__device__ __forceinline__ RobustParams lds_rob(const RobustParams* p) {
    static_assert(sizeof(RobustParams) == 32, "two 16-byte loads");
    const float4 q0 = lds_f4(p), q1 = lds_f4(reinterpret_cast<const char*>(p) + 16);
    RobustParams r;
    r.mu[0] = q0.x;
    r.mu[1] = q0.y;
    r.sigma[0] = q0.z;
    r.sigma[1] = q0.w;
    r.nu[0] = q1.x;
    r.nu[1] = q1.y;
    r.ok[0] = __float_as_int(q1.z);
    r.ok[1] = __float_as_int(q1.w);
    return r;
}

template <int PREC, int CL, int R>
__global__ void __launch_bounds__(kBatchNT, 2) batch_align_kernel(BatchArgs a) {
    constexpr int NT = kBatchNT;
    constexpr int NW = NT / 32;
    constexpr int MAXS = (RGBID_MAX_SAMPLES + CL * NT - 1) / (CL * NT);   // samples per thread
    constexpr int TH = NW * R;                                            // tile height
    constexpr int kFlush = R >= 8 ? 1 : 8 / R;                            // tiles per accumulator flush
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t rank = cl.block_rank();
    const int tid = (int)threadIdx.x, lane = tid & 31, warp = tid >> 5;

    extern __shared__ __align__(16) float rs_dyn[];          // [2][MAXS * NT]: r_I, r_W of the samples (NaN = masked)
    float* const rsI = rs_dyn;
    float* const rsW = rs_dyn + MAXS * NT;
    __shared__ __align__(16) float2 recv[2][CL][kBatchMaxNV];
    __shared__ float red_w[NW][64];
    __shared__ F2 red2[NW][kSlots];
    __shared__ float tot[kBatchMaxNV];
    __shared__ double totd[kSlots];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ __align__(16) BatchJob job;
    __shared__ double T_sh[16];
    __shared__ __align__(16) WarpPose wp_sh;
    __shared__ __align__(16) RobustParams rob_sh;
    __shared__ float nuF[2][kNuSeries];
    __shared__ float sh_g[kNuGTerms];
    __shared__ float nu_out[2];
    __shared__ float xi_f[6], d_f[6];
    __shared__ double xi_d[6], rho_d[6];
    __shared__ int ok_flag, n_done, n_skipped, j_status;
    __shared__ int failed;
    __shared__ unsigned int job_idx[2];

    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
#pragma unroll
        for (int k = 0; k < kNuGTerms; ++k) sh_g[k] = a.nu_g[k];
    }
    cl.sync();   // every barrier of the cluster is initialised before any remote store

    BatchXchg<CL> X{recv, mbar, &failed, rank, 0};

    for (int n = 0;; ++n) {
        // ---- take the next pair; rank 0's index is read by the whole cluster
        if (rank == 0 && tid == 0) job_idx[n & 1] = atomicAdd(&a.ws->head, 1u);
        cl.sync();
        const unsigned int jb = *cl.map_shared_rank(&job_idx[n & 1], 0);
        if (jb >= (unsigned int)a.n_items) break;

        const rgbid_batch_item* it = a.items + jb;
        if (tid < RGBID_MAX_LEVELS) {
            const rgbid_level LA = it->ref.lv[tid];
            const rgbid_level LB = it->cur.lv[tid];
            job.A[tid] = batch_level_dev(LA);
            job.B[tid] = batch_level_dev(LB);
            job.lvbad[tid] = batch_level_ok(LA, LB, a.precision) ? 0 : 1;
            job.iters[tid] = it->iters[tid];
        } else if (tid >= 32 && tid < 48) {
            T_sh[tid - 32] = it->T_init[tid - 32];
        } else if (tid == 64) {
            const int L = it->levels;
            job.levels = L;
            rgbid_align_result* const rp = it->result;
            job.res = ((uintptr_t)rp & 7u) ? nullptr : rp;     // a misaligned record is skipped like NULL
            job.bad = (L < 1 || L > RGBID_MAX_LEVELS || it->ref.levels < L || it->ref.levels > RGBID_MAX_LEVELS ||
                       it->cur.levels < L || it->cur.levels > RGBID_MAX_LEVELS || it->ref.precision != a.precision ||
                       it->cur.precision != a.precision) ? 1 : 0;
        }
        __syncthreads();
        if (tid == 0 && !job.bad) {
            for (int l = 0; l < job.levels; ++l)
                if (job.lvbad[l] || job.iters[l] < 0 || job.iters[l] > kBatchMaxIters) job.bad = 1;
        }
        __syncthreads();
        if (!job.res) continue;
        if (job.bad) {
            if (rank == 0 && tid == 0) {
                rgbid_align_result* r = job.res;
                r->status = RGBID_ERR_INVALID_ARG;
                r->iters_done = 0;
                r->iters_skipped = 0;
            }
            continue;
        }
        if (warp == 0) warp_make_pose(T_sh, &wp_sh);
        if (tid < kSlots) {
            totd[tid] = 0.0;
            tot[tid] = 0.f;
        }
        if (tid == 0) {
            n_done = 0;
            n_skipped = 0;
            j_status = RGBID_OK;
            rob_sh = RobustParams{{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0, 0}};
        }
        __syncthreads();

        for (int l = job.levels - 1; l >= 0; --l) {
            const LevelDev* const Ap = &job.A[l];
            const LevelDev* const Bp = &job.B[l];
            const int s = batch_sample_stride(Ap->w, Ap->h, a.sample_cap);
            const int nsx = (Ap->w + s - 1) / s;
            const int nsamp = nsx * ((Ap->h + s - 1) / s);
            const int niters = job.iters[l];
            for (int itn = 0; itn < niters; ++itn) {
                // ======== systematic sample residuals r(p, 0) at the current pose
                {
                    constexpr int G = 2;
                    const int gt = (int)rank * NT + tid;
#pragma unroll 1
                    for (int k0 = 0; k0 < MAXS; k0 += G) {
                        PxA sa[G];
                        PxW sw[G];
                        PxB sb[G];
                        int su[G], sv[G];
                        {
                            const LevelDev A = lds_level(Ap);
#pragma unroll
                            for (int g = 0; g < G; ++g) {
                                const int i = gt + (k0 + g) * (CL * NT);
                                sa[g].ok = false;
                                su[g] = 0;
                                sv[g] = 0;
                                if (k0 + g < MAXS && i < nsamp) {
                                    const int sy = i / nsx, sx = i - sy * nsx;
                                    su[g] = sx * s;
                                    sv[g] = sy * s;
                                    stage_a<PREC>(A, su[g], sv[g], sa[g]);
                                }
                            }
                        }
                        {
                            const LevelDev A = lds_level(Ap), B = lds_level(Bp);
                            const WarpPose wp = lds_pose(&wp_sh);
#pragma unroll
                            for (int g = 0; g < G; ++g) stage_w(A, B, wp, su[g], sv[g], sa[g], sw[g]);
                        }
                        {
                            const LevelDev B = lds_level(Bp);
#pragma unroll
                            for (int g = 0; g < G; ++g) stage_b<PREC>(B, sw[g], sb[g]);
                        }
                        const LevelDev A = lds_level(Ap);
                        const WarpPose wp = lds_pose(&wp_sh);
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            if (k0 + g < MAXS) {
                                PixelTerms o;
                                finish<false>(A, wp, sa[g], sw[g], sb[g], o);
                                rsI[(k0 + g) * NT + tid] = o.mI ? o.rI : __int_as_float(0x7fc00000);
                                rsW[(k0 + g) * NT + tid] = o.mW ? o.rW : __int_as_float(0x7fc00000);
                            }
                        }
                    }
                }

                // ======== counts and mean square -> sigma0 (mu0 = 0)
                float nres[2], mu[2] = {0.f, 0.f}, sig[2];
                bool live[2], ok[2];
                {
                    float v4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
                    for (int k = 0; k < MAXS; ++k) {
                        // masked samples (NaN) add exact zeros: selects, not branches
                        const float r0 = rsI[k * NT + tid], r1 = rsW[k * NT + tid];
                        const bool u0 = r0 == r0, u1 = r1 == r1;
                        const float a0 = u0 ? r0 : 0.f, a1 = u1 ? r1 : 0.f;
                        v4[0] += u0 ? 1.f : 0.f;
                        v4[1] = fmaf(a0, a0, v4[1]);
                        v4[2] += u1 ? 1.f : 0.f;
                        v4[3] = fmaf(a1, a1, v4[3]);
                    }
                    batch_round_small<CL, 4>(X, v4, red_w, tot);
                }
                nres[0] = tot[0];
                nres[1] = tot[2];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float ms = nres[c] > 0.f ? __fdividef(tot[2 * c + 1], nres[c]) : 0.f;
                    sig[c] = ms > 0.f ? ms * rsqrtf(ms) : 0.f;
                    live[c] = nres[c] > 0.f && sig[c] >= 1e-12f;
                }

                // ======== (mu, sigma) fixed point at nu0 with lagged weights
                for (int si = 0; si < a.scale_iters; ++si) {
                    if (!live[0] && !live[1]) break;
                    float v6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const float m = mu[c];
                        const float s2 = sig[c] * sig[c];
                        const float s2nu = s2 * a.nu0;
                        const float num = (a.nu0 + 1.f) * s2;
                        const float* rc = c ? rsW : rsI;
#pragma unroll 2
                        for (int k = 0; k < MAXS; ++k) {
                            const float r = rc[k * NT + tid];
                            const bool use = r == r;
                            const float dr = r - m;
                            const float wr = __fdividef(num, fmaf(dr, dr, s2nu));
                            const float w = use ? wr : 0.f, d = use ? dr : 0.f;
                            v6[3 * c] += w;
                            v6[3 * c + 1] = fmaf(w, d, v6[3 * c + 1]);
                            v6[3 * c + 2] = fmaf(w * d, d, v6[3 * c + 2]);
                        }
                    }
                    batch_round_small<CL, 6>(X, v6, red_w, tot);
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        if (!live[c]) continue;
                        const float S0 = tot[3 * c], S1 = tot[3 * c + 1], S2 = tot[3 * c + 2];
                        const float delta = __fdividef(S1, S0);
                        mu[c] += delta;
                        const float var = __fdividef(fmaf(-S1, delta, S2), nres[c]);
                        sig[c] = var > 0.f ? var * rsqrtf(var) : 0.f;
                        if (!(sig[c] >= 1e-12f)) live[c] = false;
                    }
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) ok[c] = nres[c] > 0.f && sig[c] >= 1e-12f;

                // ======== nu: Chebyshev sums (even warps channel I, odd warps channel W,
                //          each over the samples of its warp pair), then bisection
                float nu[2] = {a.nu0, a.nu0};
                const bool do_nu = a.estimate_nu && (ok[0] || ok[1]);
                if (do_nu) {
                    const int c = warp & 1;
                    const bool okc = c ? ok[1] : ok[0];
                    float v[kChebVals];
#pragma unroll
                    for (int i = 0; i < kChebVals; ++i) v[i] = 0.f;
                    if (okc) {
                        const float is = __fdividef(1.f, c ? sig[1] : sig[0]);
                        const float muc = c ? mu[1] : mu[0];
                        const float* rc = (c ? rsW : rsI) + (warp & ~1) * 32 + lane;
#pragma unroll 1
                        for (int k = 0; k < MAXS; ++k) {
#pragma unroll
                            for (int hh = 0; hh < 2; ++hh) {
                                const float x = (rc[k * NT + hh * 32] - muc) * is;
                                if (x == x) {
                                    const float al = __fdividef(fmaf(x, x, 0.5f * (a.nu_lo + a.nu_hi)), 0.5f * (a.nu_hi - a.nu_lo));
                                    const float s2 = fmaf(al, al, -1.f);
                                    const float gam = rsqrtf(s2);
                                    const float be = fmaf(s2, gam, al);
                                    const float q = __fdividef(1.f, be);
                                    v[0] += __logf(0.5f * be);
                                    v[1 + kChebK] += gam;
                                    float qk = q;
#pragma unroll
                                    for (int kk = 1; kk <= kChebK; ++kk) {
                                        v[kk] += qk;
                                        v[1 + kChebK + kk] = fmaf(gam, qk, v[1 + kChebK + kk]);
                                        qk *= q;
                                    }
                                }
                            }
                        }
                    }
                    {
                        float ch[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) ch[i] = v[i];
                        red_w[warp][lane] = warp_reduce_scatter32(ch);
#pragma unroll
                        for (int i = 0; i < 32; ++i) ch[i] = (32 + i < kChebVals) ? v[32 + i] : 0.f;
                        red_w[warp][32 + lane] = warp_reduce_scatter32(ch);
                    }
                    __syncthreads();
                    if (tid < kBatchMaxNV) {
                        const int cc = tid >= kChebVals ? 1 : 0, j = tid - cc * kChebVals;
                        F2 sacc{0.f, 0.f};
#pragma unroll
                        for (int w = cc; w < NW; w += 2) sacc.add(red_w[w][j]);
                        tot[tid] = X.template exchange<kBatchMaxNV>(tid, sacc).value();
                    }
                    __syncthreads();
                    X.next();
                    // every CTA bisects on the same totals: warp c takes channel c
                    if (tid < 64) {
                        const int cb = tid >> 5;
                        float nuc = a.nu0;
                        if (cb ? ok[1] : ok[0])
                            nuc = bisect_nu_warp(tot + cb * kChebVals, cb ? nres[1] : nres[0], sh_g, a.nu_lo, a.nu_hi,
                                                 a.bisect_steps, nuF[cb]);
                        if ((tid & 31) == 0) nu_out[cb] = nuc;
                    }
                    __syncthreads();
                    nu[0] = nu_out[0];
                    nu[1] = nu_out[1];
                    if (ok[0] && ok[1]) nu[0] = fmaxf(nu[0], nu[1]);
                }
                if (tid == 0) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        rob_sh.mu[c] = mu[c];
                        rob_sh.sigma[c] = sig[c];
                        rob_sh.nu[c] = nu[c];
                        rob_sh.ok[c] = ok[c] ? 1 : 0;
                    }
                }
                __syncthreads();

                // ======== sweep: every pixel of the level, tiles strided over the cluster
                {
                    float acc[kSlots];
#pragma unroll
                    for (int i = 0; i < kSlots; ++i) acc[i] = 0.f;
                    F2 part{0.f, 0.f};
                    // tiles rank, rank + CL, ... in row-major order, stepped without division
                    const int tw = (Ap->w + 31) >> 5;
                    const int th = (Ap->h + TH - 1) / TH;
                    int ty = (int)rank / tw, tx = (int)rank - ((int)rank / tw) * tw;
                    int pending = 0;          // tiles accumulated in acc since the last flush
#pragma unroll 1
                    for (; ty < th; ) {
                        const int u = tx * 32 + lane;
                        const int v0 = ty * TH + warp * R;
                        PxA sa[R];
                        PxW sw[R];
                        PxB sb[R];
                        {
                            const LevelDev A = lds_level(Ap);
#pragma unroll
                            for (int r = 0; r < R; ++r) {
                                sa[r].ok = false;
                                if (u < A.w && v0 + r < A.h) stage_a<PREC>(A, u, v0 + r, sa[r]);
                            }
                        }
                        {
                            const LevelDev A = lds_level(Ap), B = lds_level(Bp);
                            const WarpPose wp = lds_pose(&wp_sh);
#pragma unroll
                            for (int r = 0; r < R; ++r) stage_w(A, B, wp, u, v0 + r, sa[r], sw[r]);
                        }
                        {
                            const LevelDev B = lds_level(Bp);
#pragma unroll
                            for (int r = 0; r < R; ++r) stage_b<PREC>(B, sw[r], sb[r]);
                        }
                        const LevelDev A = lds_level(Ap);
                        const WarpPose wp = lds_pose(&wp_sh);
                        const RobustParams rob = lds_rob(&rob_sh);
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            PixelTerms o;
                            finish<true>(A, wp, sa[r], sw[r], sb[r], o);
                            if (o.mI) {
                                acc[kSlotNI] += 1.f;
                                if (rob.ok[0]) accumulate(acc, o.JI, robust_weight(o.rI, rob.mu[0], rob.sigma[0], rob.nu[0]), o.rI);
                            }
                            if (o.mW) {
                                acc[kSlotNW] += 1.f;
                                if (rob.ok[1])
                                    accumulate(acc, o.JW, o.lam * robust_weight(o.rW, rob.mu[1], rob.sigma[1], rob.nu[1]),
                                               o.rW);
                            }
                        }
                        // every kFlush tiles (about 8 pixels per thread) the warp sums enter the
                        // compensated per-lane partial of slot `lane`
                        if (++pending == kFlush) {
                            pending = 0;
                            part.add(warp_reduce_scatter32(acc));
#pragma unroll
                            for (int i = 0; i < kSlots; ++i) acc[i] = 0.f;
                        }
                        tx += CL;
                        while (tx >= tw) {
                            tx -= tw;
                            ++ty;
                        }
                    }
                    if (pending) part.add(warp_reduce_scatter32(acc));   // warp-uniform: every warp saw the same tiles
                    red2[warp][lane] = part;
                    __syncthreads();
                    if (tid < kSlots) {
                        F2 sacc{0.f, 0.f};
#pragma unroll
                        for (int w = 0; w < NW; ++w) sacc.add(red2[w][tid]);
                        if (tid == kSlotTimeout && failed) sacc.add(1.f);
                        const F2 T2 = X.template exchange<kSlots>(tid, sacc);
                        tot[tid] = T2.value();
                        totd[tid] = (double)T2.hi + (double)T2.lo;
                    }
                    __syncthreads();
                    X.next();
                }

                // ======== solve and update (warp 0 of every CTA, identical inputs)
                if (warp == 0) {
                    const bool ok_in = ((int)tot[kSlotNI] + (int)tot[kSlotNW]) >= a.min_valid;
                    bool okr = false;
                    if constexpr (PREC == RGBID_PLANES_BF16_F16)
                        okr = warp_solve6_refined(tot, ok_in, xi_f, d_f, rho_d, xi_d);
                    if (lane == 0) {
                        bool okl = okr;
                        if constexpr (PREC != RGBID_PLANES_BF16_F16) {
                            float xi[6];
                            okl = ok_in && cholesky_solve6_slots(tot, xi);
#pragma unroll
                            for (int i = 0; i < 6; ++i) xi_f[i] = okl ? xi[i] : 0.f;
                        }
                        ok_flag = okl ? 1 : 0;
                        n_done += 1;
                        if (!okl) {
                            n_skipped += 1;
                            j_status = RGBID_ERR_DEGENERATE;
                        }
                    }
                    __syncwarp();
                    if (ok_flag) {
                        if constexpr (PREC == RGBID_PLANES_BF16_F16) {
                            double xi[6];
#pragma unroll
                            for (int i = 0; i < 6; ++i) xi[i] = xi_d[i];
                            warp_apply_update_d(xi, T_sh);
                        } else {
                            float xi[6];
#pragma unroll
                            for (int i = 0; i < 6; ++i) xi[i] = xi_f[i];
                            warp_apply_update(xi, T_sh);
                        }
                        warp_make_pose(T_sh, &wp_sh);
                    }
                }
                __syncthreads();
            }
        }

        // ---- result of the pair (rank 0)
        if (rank == 0) {
            rgbid_align_result* r = job.res;
            if (tid < 16) {
                r->T[tid] = T_sh[tid];
            } else if (tid >= 32 && tid < 32 + kSlots) {
                const int q = tid - 32;
                const double td = totd[q];
                if (q < 21) {
                    int i = 0, rem = q;
                    while (rem >= 6 - i) { rem -= 6 - i; ++i; }
                    const int j = i + rem;
                    r->H[i * 6 + j] = td;
                    r->H[j * 6 + i] = td;
                } else if (q < 27) {
                    r->g[q - kSlotG] = td;
                } else if (q == kSlotCost) {
                    r->cost = td;
                } else if (q == kSlotNI) {
                    r->n_valid[0] = (int)tot[kSlotNI];
                } else if (q == kSlotNW) {
                    r->n_valid[1] = (int)tot[kSlotNW];
                }
            } else if (tid == 64) {
                for (int c = 0; c < 2; ++c) {
                    r->mu[c] = rob_sh.mu[c];
                    r->sigma[c] = rob_sh.sigma[c];
                    r->nu[c] = rob_sh.nu[c];
                }
                r->iters_done = n_done;
                r->iters_skipped = n_skipped;
                r->status = (failed || tot[kSlotTimeout] > 0.f) ? RGBID_ERR_TIMEOUT : j_status;
            }
        }
    }

    cl.sync();   // no CTA leaves while another may still address its shared memory
    if (rank == 0 && tid == 0) {
        // the last cluster to find the queue empty resets it for the next batch
        const unsigned int left = atomicAdd(&a.ws->exited, 1u);
        if (left == gridDim.x / CL - 1) {
            a.ws->head = 0u;
            a.ws->exited = 0u;
        }
    }
}

// ---------------------------------------------------------------- host-side launch helpers
template <int CL>
constexpr size_t batch_dyn_smem() {
    return 2u * (size_t)((RGBID_MAX_SAMPLES + CL * kBatchNT - 1) / (CL * kBatchNT)) * kBatchNT * sizeof(float);
}

template <int PREC, int CL, int R>
cudaError_t batch_setup_one(int* max_clusters) {
    auto k = batch_align_kernel<PREC, CL, R>;
    cudaError_t e;
    if (CL > 8) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_dyn_smem<CL>());
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(kBatchNT, 1, 1);
    cfg.dynamicSmemBytes = batch_dyn_smem<CL>();
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
    if (e != cudaSuccess) return e;
    *max_clusters = n;
    return cudaSuccess;
}

template <int PREC, int CL, int R>
cudaError_t batch_launch_one(const BatchArgs& a, int n_clusters, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_clusters * CL), 1, 1);
    cfg.blockDim = dim3(kBatchNT, 1, 1);
    cfg.dynamicSmemBytes = batch_dyn_smem<CL>();
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_align_kernel<PREC, CL, R>, a);
}

// a == nullptr: set the kernel attributes and report the resident clusters;
// otherwise launch n_clusters clusters.
template <int PREC>
cudaError_t batch_dispatch(int cl, int rows, const BatchArgs* a, int n_clusters, int* max_clusters,
                           cudaStream_t stream) {
#define RGBID_BATCH_CASE(C, RR)                                                                   \
    if (cl == C && rows == RR)                                                                    \
        return a ? batch_launch_one<PREC, C, RR>(*a, n_clusters, stream)                          \
                 : batch_setup_one<PREC, C, RR>(max_clusters);
    RGBID_BATCH_CASE(4, 1)
    RGBID_BATCH_CASE(4, 2)
    RGBID_BATCH_CASE(4, 4)
    RGBID_BATCH_CASE(8, 1)
    RGBID_BATCH_CASE(8, 2)
    RGBID_BATCH_CASE(8, 4)
    RGBID_BATCH_CASE(16, 1)
    RGBID_BATCH_CASE(16, 2)
    RGBID_BATCH_CASE(16, 4)
#undef RGBID_BATCH_CASE
    return cudaErrorInvalidValue;
}

}  // namespace rgbid
