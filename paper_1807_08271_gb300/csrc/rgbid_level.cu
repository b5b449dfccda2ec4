// Persistent per-level alignment kernel (sm_103a).
//
// On a level whose systematic sample is every pixel (sample stride 1, "Error
// distribution and robust optimisation"), the sample residuals of an iteration
// are the residuals the level's sweep evaluates at the same pose.  One 16-CTA
// cluster then runs all of the level's Gauss-Newton iterations ("Iterative
// optimisation") in one launch, and each pixel is warped once per iteration:
//   terms    every thread warps its <= MAXP pixels with the current pose; it keeps
//            r_I and r_W (NaN where masked out) in registers and the Jacobians
//            and lambda_n in shared memory;
//   robust   Student-t (mu, sigma) at nu0 by the lagged-weight fixed point, then
//            nu by bisection on the robustness equation, from those residuals;
//            every sum goes through the cluster's distributed shared memory, and
//            every CTA bisects the same totals, so all hold the same parameters;
//   normal   the weighted 27 normal-equation terms, cost and counts of the CTA's
//            pixels; one exchange gives every CTA the cluster totals;
//   update   every CTA solves H xi = -g and applies T <- exp(xi)^-1 T to its copy
//            of the FP64 pose; the copies stay bit-identical.
// The level's last step is not solved here.  Its totals stay in the workspace as
// one pending block partial, next to the robust parameters that weighted them,
// exactly as a sweep leaves its partials; the next level's robust-scale kernel,
// or the alignment's closing launch, solves from them and updates the pose.
#include <cooperative_groups.h>
#include <algorithm>
#include <atomic>

#include "rgbid_cluster.cuh"
#include "rgbid_device.cuh"
#include "rgbid_level.h"

// Phase stamps of the split kernel (a diagnostic build, -DRGBID_PHASE_STAMPS): thread 0
// of cluster 0's CTA 0 and of the first helper CTA record %globaltimer (ns) at the
// phases of each iteration, per pyramid level; rgbid_debug_phase_stamps copies them
// out.  Without the macro the stamps compile away.
#ifdef RGBID_PHASE_STAMPS
__device__ long long g_phase[RGBID_MAX_LEVELS][16][16];
__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
#define RGBID_STAMP(role_ok, k)                                                                \
    do {                                                                                       \
        if ((role_ok) && threadIdx.x == 0 && it < 16) g_phase[L.level % RGBID_MAX_LEVELS][it][k] = global_ns(); \
    } while (0)
#else
#define RGBID_STAMP(role_ok, k) \
    do {                        \
    } while (0)
#endif
#define STAMP_C(k) RGBID_STAMP(blockIdx.x == 0, k)
#define STAMP_H(k) RGBID_STAMP((int)blockIdx.x == kLevelCL, k)

namespace cg = cooperative_groups;

namespace rgbid {

constexpr int kJTerms = 13;     // per pixel in shared memory: J_I (6), J_W (6), lambda_n

template <int MAXP>
constexpr size_t level_dyn_smem() {
    return (size_t)MAXP * kJTerms * kRobustNT * sizeof(float);
}

// H xi = -g from the cluster totals (warp 0 of every CTA, identical inputs); a
// solved step updates the CTA's FP64 pose and its FP32 warp form.  cnt holds
// the alignment's iterations done and skipped and its status.
template <int PREC>
__device__ __forceinline__ void level_solve_update(const float* tot, int min_valid, double* T_sh, WarpPose* wp_sh,
                                                   float* xi_f, float* d_f, double* rho_d, double* xi_d,
                                                   int* ok_flag, int* cnt) {
    const int lane = threadIdx.x & 31;
    const bool ok_in = ((int)tot[kSlotNI] + (int)tot[kSlotNW]) >= min_valid;
    if constexpr (PREC == RGBID_PLANES_BF16_F16) {
        // reduced-precision planes: FP32 factorisation refined to an FP64 solution
        const bool okl = warp_solve6_refined(tot, ok_in, xi_f, d_f, rho_d, xi_d);
        if (lane == 0) *ok_flag = okl ? 1 : 0;
    } else if (lane == 0) {
        float xi[6];
        const bool okl = ok_in && cholesky_solve6_slots(tot, xi);
#pragma unroll
        for (int i = 0; i < 6; ++i) xi_f[i] = okl ? xi[i] : 0.f;
        *ok_flag = okl ? 1 : 0;
    }
    __syncwarp();
    const bool ok = *ok_flag != 0;
    if (ok) {
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
        warp_make_pose(T_sh, wp_sh);
    }   // else the pose is kept (a degenerate step)
    if (lane == 0) {
        cnt[0] += 1;
        if (!ok) {
            cnt[1] += 1;
            cnt[2] = RGBID_ERR_DEGENERATE;
        }
    }
    __syncwarp();
}

template <int PREC, int MAXP>
__global__ void __launch_bounds__(kRobustNT, 1) level_kernel(LevelArgs a) {
    constexpr int CL = kLevelCL, NT = kRobustNT, NW = NT / 32;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = (int)threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ __align__(16) float Jsm[];     // [MAXP][kJTerms][NT]
    __shared__ float red_w[NW][kRobustMaxNV];
    __shared__ float2 recv[2][CL][kRobustMaxNV];
    __shared__ float tot[kRobustMaxNV];
    __shared__ float2 tot2[kSlots];                 // the last step's totals as compensated pairs
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ WarpPose sh_wp;
    __shared__ double T_sh[16];
    __shared__ float nu_out[2];
    __shared__ float nuF[2][kNuSeries];
    __shared__ float sh_g[kNuGTerms];
    __shared__ F2 fin2[NW][kSlots];
    __shared__ float xi_f[6], d_f[6];
    __shared__ double xi_d[6], rho_d[6];
    __shared__ int ok_flag;
    __shared__ int sh_cnt[3];                       // iterations done, skipped, status

    // the device count of the level, written before the alignment's first kernel
    const int n_it = a.level_iters ? min(a.iters, __ldg(a.level_iters + a.level)) : a.iters;
    if (n_it <= 0) {
        pdl_wait();   // keeps the chain of dependent launches ordered; never triggers
        return;
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
        for (int k = 0; k < kNuGTerms; ++k) sh_g[k] = a.nu_g[k];
    }
    // no CTA stores into another before every barrier of the cluster is initialised
    cluster_arrive();
    pdl_wait();   // the state and any pending partials of the preceding launches are visible
    if (tid < 16) {
        T_sh[tid] = __ldcg(a.st->T + tid);
    } else if (tid < 32) {
        reinterpret_cast<float*>(&sh_wp)[tid - 16] =
            __ldcg(reinterpret_cast<const float*>(&a.st->wp) + (tid - 16));
    } else if (tid == 32) {
        sh_cnt[0] = __ldcg(&a.st->iters_done);
    } else if (tid == 33) {
        sh_cnt[1] = __ldcg(&a.st->iters_skipped);
    } else if (tid == 34) {
        sh_cnt[2] = __ldcg(&a.st->status);
    }
    const unsigned int nb = __ldcg(&a.st->pending);   // the same value in every CTA
    cluster_wait();
    ClusterSum<CL> R{red_w, recv, tot, mbar, &a.st->timeouts, (uint32_t)rank, 0};

    // ---- a pending step of the previous level: the CTAs sum disjoint subsets of its
    //      block partials, one exchange gives every CTA the totals, and every CTA
    //      solves and updates its copy of the pose
    if (nb) {
        F2 acc{0.f, 0.f};
        constexpr unsigned kStride = (unsigned)CL * NW;
        for (unsigned int b0 = (unsigned)rank + (unsigned)CL * (unsigned)warp; b0 < nb; b0 += 4u * kStride) {
            float2 v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned int b = b0 + (unsigned)q * kStride;
                v[q] = b < nb ? __ldcg(a.partials + (size_t)b * kSlots + lane) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) acc.add(F2{v[q].x, v[q].y});
        }
        fin2[warp][lane] = acc;
        __syncthreads();
        if (tid < kSlots) tot[tid] = R.template exchange<kSlots>(tid, warp_tree<NW>(fin2, tid)).value();
        __syncthreads();
        R.next();
        if (warp == 0) level_solve_update<PREC>(tot, a.min_valid, T_sh, &sh_wp, xi_f, d_f, rho_d, xi_d, &ok_flag, sh_cnt);
    }
    __syncthreads();

    const int w = a.A.w, npix = a.A.w * a.A.h;
    const int gt = rank * NT + tid;
    const float nu0 = a.nu0;
    const float lo0 = (float)a.nu_lo, hi0 = (float)a.nu_hi;
    const float m = 0.5f * (lo0 + hi0), h = 0.5f * (hi0 - lo0);
    float* const Jt = Jsm + tid;                     // this thread's column of the Jacobian store
    for (int it = 0; it < n_it; ++it) {
        const bool last = it + 1 == n_it;
        const WarpPose wp = sh_wp;
        // the next launch may be scheduled while the last step runs; it reads the
        // state only after this grid has completed
        if (last) pdl_trigger();

        // ---- per-pixel terms at the current pose; the pixels of a thread go through
        //      each stage together so their loads overlap
        float rs[2][MAXP];
        {
            PxA sa[MAXP];
            PxW sw[MAXP];
            PxB sb[MAXP];
            int pu[MAXP], pv[MAXP];
#pragma unroll
            for (int k = 0; k < MAXP; ++k) {
                const int i = gt + k * (CL * NT);
                sa[k].ok = false;
                pu[k] = 0;
                pv[k] = 0;
                if (i < npix) {
                    pv[k] = i / w;
                    pu[k] = i - pv[k] * w;
                    stage_a<PREC>(a.A, pu[k], pv[k], sa[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < MAXP; ++k) stage_w(a.A, a.B, wp, pu[k], pv[k], sa[k], sw[k]);
#pragma unroll
            for (int k = 0; k < MAXP; ++k) stage_b<PREC>(a.B, sw[k], sb[k]);
#pragma unroll
            for (int k = 0; k < MAXP; ++k) {
                PixelTerms o;
                finish<true>(a.A, wp, sa[k], sw[k], sb[k], o);
                rs[0][k] = o.mI ? o.rI : __int_as_float(0x7fc00000);
                rs[1][k] = o.mW ? o.rW : __int_as_float(0x7fc00000);
                float* const J = Jt + k * (kJTerms * NT);
                if (o.mI) {
#pragma unroll
                    for (int j = 0; j < 6; ++j) J[j * NT] = o.JI[j];
                }
                if (o.mW) {
#pragma unroll
                    for (int j = 0; j < 6; ++j) J[(6 + j) * NT] = o.JW[j];
                    J[12 * NT] = o.lam;
                }
            }
        }

        // ---- counts and mean square -> sigma0 (mu0 = 0)
        {
            float v4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < MAXP; ++k) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    // masked pixels (NaN) add exact zeros: selects, not branches
                    const float r = rs[c][k];
                    const bool use = r == r;
                    const float rv = use ? r : 0.f;
                    v4[2 * c] += use ? 1.f : 0.f;
                    v4[2 * c + 1] = fmaf(rv, rv, v4[2 * c + 1]);
                }
            }
            R.run(v4);
        }
        const float n[2] = {tot[0], tot[2]};
        float mu[2] = {0.f, 0.f};
        float sig[2];
        bool live[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float ms = n[c] > 0.f ? __fdividef(tot[2 * c + 1], n[c]) : 0.f;
            sig[c] = ms > 0.f ? ms * rsqrtf(ms) : 0.f;
            live[c] = n[c] > 0.f && sig[c] >= 1e-12f;
        }

        // ---- (mu, sigma) fixed point at nu0 with lagged weights:
        //      mu <- sum w r / sum w ; sigma^2 <- sum w (r - mu_new)^2 / n, with d = r - mu_old
        //      sum w (r - mu_new)^2 = S2 - S1^2 / S0.
        for (int si = 0; si < a.scale_iters; ++si) {
            if (!live[0] && !live[1]) break;
            float v6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float mc = mu[c];
                const float s2 = sig[c] * sig[c];
                const float s2nu = s2 * nu0;
                const float num = (nu0 + 1.f) * s2;
#pragma unroll
                for (int k = 0; k < MAXP; ++k) {
                    const float r = rs[c][k];
                    const bool use = r == r;
                    const float dr = r - mc;
                    const float wr = __fdividef(num, fmaf(dr, dr, s2nu));   // omega((r - mu)/sigma, nu0)
                    const float wv = use ? wr : 0.f, d = use ? dr : 0.f;
                    v6[3 * c] += wv;
                    v6[3 * c + 1] = fmaf(wv, d, v6[3 * c + 1]);
                    v6[3 * c + 2] = fmaf(wv * d, d, v6[3 * c + 2]);
                }
            }
            R.run(v6);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (!live[c]) continue;
                const float S0 = tot[3 * c], S1 = tot[3 * c + 1], S2 = tot[3 * c + 2];
                const float delta = __fdividef(S1, S0);
                mu[c] += delta;
                const float var = __fdividef(fmaf(-S1, delta, S2), n[c]);
                sig[c] = var > 0.f ? var * rsqrtf(var) : 0.f;
                if (!(sig[c] >= 1e-12f)) live[c] = false;
            }
        }
        bool ok[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) ok[c] = n[c] > 0.f && sig[c] >= 1e-12f;

        // ---- nu by bisection on eq. robustnessValue: the Chebyshev power sums of both
        //      channels in packed pairs (low half I, high half W), exchanged to every CTA
        float nu[2] = {nu0, nu0};
        const bool do_nu = a.estimate_nu && (ok[0] || ok[1]);
        if (do_nu) {
            unsigned long long V[kChebVals];
#pragma unroll
            for (int i = 0; i < kChebVals; ++i) V[i] = 0ull;
            const float is0 = ok[0] ? __fdividef(1.f, sig[0]) : 0.f;
            const float is1 = ok[1] ? __fdividef(1.f, sig[1]) : 0.f;
#pragma unroll 1
            for (int k = 0; k < MAXP; ++k) {
                float r0 = rs[0][0], r1 = rs[1][0];
#pragma unroll
                for (int q = 1; q < MAXP; ++q)
                    if (k == q) {
                        r0 = rs[0][q];
                        r1 = rs[1][q];
                    }
                float q2[2], g2[2], l2[2];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float x = ((c ? r1 : r0) - mu[c]) * (c ? is1 : is0);
                    const bool use = ok[c] && x == x;
                    const float al = __fdividef(fmaf(x, x, m), h);
                    const float s2 = fmaf(al, al, -1.f);
                    const float gam = rsqrtf(s2);
                    const float be = fmaf(s2, gam, al);
                    q2[c] = use ? __fdividef(1.f, be) : 0.f;
                    g2[c] = use ? gam : 0.f;
                    l2[c] = use ? __logf(0.5f * be) : 0.f;
                }
                const unsigned long long Q = f2_pack(q2[0], q2[1]), G = f2_pack(g2[0], g2[1]);
                V[0] = f2_add(V[0], f2_pack(l2[0], l2[1]));
                V[1 + kChebK] = f2_add(V[1 + kChebK], G);          // G_0
                unsigned long long qk = Q;
#pragma unroll
                for (int kk = 1; kk <= kChebK; ++kk) {
                    V[kk] = f2_add(V[kk], qk);                       // P_k
                    V[1 + kChebK + kk] = f2_fma(G, qk, V[1 + kChebK + kk]);   // G_k
                    qk = f2_mul(qk, Q);
                }
            }
            float v[96];
#pragma unroll
            for (int i = 0; i < kChebVals; ++i) {
                v[i] = f2_lo(V[i]);
                v[kChebVals + i] = f2_hi(V[i]);
            }
#pragma unroll
            for (int i = 2 * kChebVals; i < 96; ++i) v[i] = 0.f;
            R.template run_by_loads<96, 2 * kChebVals, false>(v);
            if (tid < 64) {
                // warp c solves channel c, in every CTA on the same totals
                const int c = tid >> 5;
                float nuc = nu0;
                if (ok[c]) nuc = bisect_nu_warp(tot + c * kChebVals, n[c], sh_g, lo0, hi0, a.bisect_steps, nuF[c]);
                if (lane == 0) nu_out[c] = nuc;
            }
            __syncthreads();
            nu[0] = nu_out[0];
            nu[1] = nu_out[1];
            if (ok[0] && ok[1]) nu[0] = fmaxf(nu[0], nu[1]);
        }

        // ---- normal equations of the CTA's pixels with these weights
        {
            float acc[kSlots];
#pragma unroll
            for (int i = 0; i < kSlots; ++i) acc[i] = 0.f;
#pragma unroll
            for (int k = 0; k < MAXP; ++k) {
                const float* const J = Jt + k * (kJTerms * NT);
                const float rI = rs[0][k], rW = rs[1][k];
                if (rI == rI) {
                    acc[kSlotNI] += 1.f;
                    if (ok[0]) {
                        float Jl[6];
#pragma unroll
                        for (int j = 0; j < 6; ++j) Jl[j] = J[j * NT];
                        accumulate(acc, Jl, robust_weight(rI, mu[0], sig[0], nu[0]), rI);
                    }
                }
                if (rW == rW) {
                    acc[kSlotNW] += 1.f;
                    if (ok[1]) {
                        float Jl[6];
#pragma unroll
                        for (int j = 0; j < 6; ++j) Jl[j] = J[(6 + j) * NT];
                        accumulate(acc, Jl, J[12 * NT] * robust_weight(rW, mu[1], sig[1], nu[1]), rW);
                    }
                }
            }
            red_w[warp][lane] = warp_reduce_scatter32(acc);
            __syncthreads();
            if (tid < kSlots) {
                const F2 T2 = R.template exchange<kSlots>(tid, warp_tree<NW>(red_w, tid));
                tot[tid] = T2.value();
                tot2[tid] = make_float2(T2.hi, T2.lo);
            }
            __syncthreads();
            R.next();
        }

        if (!last) {
            if (warp == 0)
                level_solve_update<PREC>(tot, a.min_valid, T_sh, &sh_wp, xi_f, d_f, rho_d, xi_d, &ok_flag, sh_cnt);
            __syncthreads();
        } else if (rank == 0) {
            // the level's last step is left pending, as a sweep leaves its partials
            AlignState* const st = a.st;
            if (tid < kSlots) {
                a.partials[tid] = tot2[tid];
            } else if (tid < kSlots + 16) {
                const int q = tid - kSlots;
                st->T[q] = T_sh[q];
                reinterpret_cast<float*>(&st->wp)[q] = reinterpret_cast<const float*>(&sh_wp)[q];
            } else if (tid == kSlots + 16) {
                RobustParams& rp = st->rob;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    rp.mu[c] = mu[c];
                    rp.sigma[c] = sig[c];
                    rp.nu[c] = nu[c];
                    rp.ok[c] = ok[c] ? 1 : 0;
                }
            } else if (tid == kSlots + 17) {
                st->iters_done = sh_cnt[0];
                st->iters_skipped = sh_cnt[1];
                st->status = sh_cnt[2];
                st->pending = 1u;
            }
        }
    }
    // no CTA leaves before every CTA is past its last exchange
    cluster_arrive();
    cluster_wait();
}

// ---------------------------------------------------------------- split level kernel
// Levels with more than two pixels per thread of the cluster (160x120, 320x240 and
// 640x480 of the sequence; the sample is every pixel at 160x120, a strict subset
// above).  One launch runs consecutive such levels in turn, coarse to fine, each for
// all of its iterations (a level's last step is taken at the next level's first
// iteration, like any other step):
//   cluster 0 (16 CTAs)  reduces the previous step's partials, solves and updates the
//                        pose in every CTA, publishes the pose, evaluates the sample
//                        residuals at it, estimates (mu, sigma, nu) as the robust-scale
//                        kernel does, and publishes the parameters (CTA 0);
//   helper CTAs          evaluate every pixel's residuals, Jacobians and lambda_n as soon
//                        as the pose is published, keep them in shared memory, weight
//                        and accumulate them once the parameters are published, and post
//                        one compensated partial each.
// The pixel work of an iteration thus overlaps the robust-scale chain instead of
// following it.  The roles hand over through the workspace's mailbox: a release store
// of a counter after the data, an acquire load before reading it, every wait bounded.
// The launch is cooperative, so every CTA is resident while others wait on it.  The
// last level's last step stays pending (one partial per helper), as a sweep leaves it.

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 waits until *word >= target; every thread of the CTA gets the verdict
// through its own shared slot.  A wait that runs out counts a timeout and raises the
// mailbox's error flag; a raised flag makes every later wait give up at once.
__device__ __forceinline__ bool cta_wait(AlignState* st, const unsigned int* word, unsigned int target, int* slot,
                                         long long budget = kWaitBudgetCycles) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const long long t0 = clock64();
        while (ld_acquire_u32(word) < target) {
            if (ld_relaxed_s32(&st->mb.error)) {
                ok = 0;
                break;
            }
            if (clock64() - t0 > budget) {
                atomicAdd(&st->timeouts, 1);
                atomicExch(&st->mb.error, 1);
                ok = 0;
                break;
            }
        }
        *slot = ok;
    }
    __syncthreads();
    return *slot != 0;
}

static_assert((offsetof(AlignState, mb) + offsetof(SplitMailbox, wp)) % 16 == 0, "the pose is published as float4");

constexpr int kSampleTerms = 13;   // a sample's cached keyframe-side stage: 5 taps (10), a, b, interior

template <int PREC>
__global__ void __launch_bounds__(kRobustNT, 1) split_kernel(SplitArgs a) {
    constexpr int CL = kLevelCL, NT = kRobustNT, NW = NT / 32;
    constexpr int MAXS = (RGBID_MAX_SAMPLES + CL * NT - 1) / (CL * NT);
    constexpr int G = 4;                             // a helper's tiles in flight
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = (int)threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ __align__(16) float dyn[];     // cluster 0: cached samples; helpers: pixel terms
    __shared__ float red_w[NW][kRobustMaxNV];
    __shared__ float2 recv[2][CL][kRobustMaxNV];
    __shared__ float tot[kRobustMaxNV];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ __align__(16) WarpPose sh_wp;
    __shared__ RobustParams sh_rob;
    __shared__ double T_sh[16];
    __shared__ float nu_out[2];
    __shared__ float nuF[2][kNuSeries];
    __shared__ float sh_g[kNuGTerms];
    __shared__ F2 fin2[NW][kSlots];
    __shared__ float xi_f[6], d_f[6];
    __shared__ double xi_d[6], rho_d[6];
    __shared__ int ok_flag;
    __shared__ int sh_cnt[3];                        // iterations done, skipped, status
    __shared__ int go[3];                            // verdicts of the CTA's mailbox waits, one per site

    // the launch runs its levels coarse to fine, each for its iteration count; `git`
    // below counts the launch's iterations over all levels (the mailbox's flags)
    auto level_its = [&](int l) {
        return a.level_iters ? min(a.lv[l].iters, __ldg(a.level_iters + a.lv[l].level)) : a.lv[l].iters;
    };
    int n_total = 0;
    for (int l = 0; l < a.n_levels; ++l) n_total += max(level_its(l), 0);
    if (n_total <= 0) {
        pdl_wait();   // keeps the chain of dependent launches ordered; never triggers
        return;
    }
    AlignState* const st = a.st;
    SplitMailbox* const mb = &st->mb;

    if (blockIdx.x < CL) {
        // ================================================================ cluster 0
        if (tid == 0) {
            mbar_init(&mbar[0], 1);
            mbar_init(&mbar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
            for (int k = 0; k < kNuGTerms; ++k) sh_g[k] = a.nu_g[k];
        }
        cluster_arrive();
        // the keyframe-side stage of this thread's samples of a level, kept for all of the
        // level's iterations (A's planes do not change during an alignment); each thread
        // writes only its own slots
        float* const Sa = dyn + tid;                 // [MAXS][kSampleTerms][NT]
        const int gt = rank * NT + tid;
        auto stage_samples = [&](const SplitLevel& L) {
#pragma unroll
            for (int k = 0; k < MAXS; ++k) {
                const int i = gt + k * (CL * NT);
                PxA p;
                p.ok = false;
                if (i < L.nsamp) {
                    const int sy = i / L.nsx, sx = i - sy * L.nsx;
                    stage_a<PREC>(L.A, sx * L.s, sy * L.s, p);
                }
                float* const q = Sa + k * (kSampleTerms * NT);
                q[0] = p.c.x; q[NT] = p.c.y; q[2 * NT] = p.nl.x; q[3 * NT] = p.nl.y; q[4 * NT] = p.nr.x;
                q[5 * NT] = p.nr.y; q[6 * NT] = p.nu.x; q[7 * NT] = p.nu.y; q[8 * NT] = p.nd.x; q[9 * NT] = p.nd.y;
                q[10 * NT] = p.a; q[11 * NT] = p.b; q[12 * NT] = p.ok ? 1.f : 0.f;
            }
        };
        int first = 0;                               // the first level that runs iterations
        while (level_its(first) <= 0) ++first;
        stage_samples(a.lv[first]);                  // A is complete before this launch
        pdl_wait();   // the state and the pending partials of the preceding launches are visible
        if (tid < 16) {
            T_sh[tid] = __ldcg(st->T + tid);
        } else if (tid < 32) {
            reinterpret_cast<float*>(&sh_wp)[tid - 16] = __ldcg(reinterpret_cast<const float*>(&st->wp) + (tid - 16));
        } else if (tid == 32) {
            sh_cnt[0] = __ldcg(&st->iters_done);
        } else if (tid == 33) {
            sh_cnt[1] = __ldcg(&st->iters_skipped);
        } else if (tid == 34) {
            sh_cnt[2] = __ldcg(&st->status);
        } else if (tid >= 64 && tid < 64 + (int)(sizeof(RobustParams) / 4)) {
            reinterpret_cast<int*>(&sh_rob)[tid - 64] = __ldcg(reinterpret_cast<const int*>(&st->rob) + (tid - 64));
        }
        const unsigned int nb0 = __ldcg(&st->pending);
        cluster_wait();
        // the cluster barrier's arrive came before these loads: only a CTA barrier
        // makes warp 0's copies of the state visible to the other warps
        __syncthreads();
        ClusterSum<CL> R{red_w, recv, tot, mbar, &st->timeouts, (uint32_t)rank, 0};
        const float nu0 = a.nu0;
        const float lo0 = (float)a.nu_lo, hi0 = (float)a.nu_hi;
        const float m = 0.5f * (lo0 + hi0), h = 0.5f * (hi0 - lo0);

        int git = 0;
        bool broken = false;
        for (int l = first; l < a.n_levels && !broken; ++l) {
          const int n_it = level_its(l);
          if (n_it <= 0) continue;
          const SplitLevel& L = a.lv[l];
          if (l != first) stage_samples(L);
          for (int it = 0; it < n_it; ++it, ++git) {
            // the next launch may be scheduled while the last iteration runs (on the SMs this
            // launch leaves free); it reads the state only after this grid has completed
            if (git == n_total - 1) pdl_trigger();
            // ---- the previous step: the pending partials of the preceding launch, or the
            //      helpers' partials of the previous iteration (of this level or the last)
            STAMP_C(0);
            if (git > 0 && !cta_wait(st, &mb->arrived, (unsigned)a.n_helpers * (unsigned)git, &go[0])) {
                broken = true;
                break;
            }
            STAMP_C(1);
            const unsigned int nb = git == 0 ? nb0 : (unsigned)a.n_helpers;
            if (nb) {
                // every CTA of the cluster sums all nb partials itself in one fixed order
                // (warp w takes partials w, w + 8, ...; then the warps' sums in a fixed
                // tree), so every CTA holds bit-identical totals without an exchange round
                F2 acc{0.f, 0.f};
                constexpr int Q = 12;                // loads in flight per lane (96 helpers: one batch)
                for (unsigned int b0 = (unsigned)warp; b0 < nb; b0 += (unsigned)(Q * NW)) {
                    float2 v[Q];
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        const unsigned int b = b0 + (unsigned)(q * NW);
                        v[q] = b < nb ? __ldcg(a.partials + (size_t)b * kSlots + lane) : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int q = 0; q < Q; ++q) acc.add(F2{v[q].x, v[q].y});
                }
                fin2[warp][lane] = acc;
                __syncthreads();
                if (tid < kSlots) tot[tid] = warp_tree<NW>(fin2, tid).value();
                __syncthreads();
                if (warp == 0)
                    level_solve_update<PREC>(tot, a.min_valid, T_sh, &sh_wp, xi_f, d_f, rho_d, xi_d, &ok_flag, sh_cnt);
                __syncthreads();
            }
            STAMP_C(2);
            // ---- publish this iteration's pose to the helpers: one thread stores the pose
            //      and then releases the flag, so the release orders the pose before it
            if (rank == 0 && tid == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    __stcg(reinterpret_cast<float4*>(&mb->wp) + q, reinterpret_cast<const float4*>(&sh_wp)[q]);
                st_release_u32(&mb->pose_flag, (unsigned)git + 1u);
            }
            const WarpPose wp = sh_wp;
            STAMP_C(3);

            // ---- systematic sample residuals at this pose (NaN = masked out)
            float rs[2][MAXS];
            {
                PxA sa[MAXS];
                PxW sw[MAXS];
                PxB sb[MAXS];
                int su[MAXS], sv[MAXS];
#pragma unroll
                for (int k = 0; k < MAXS; ++k) {
                    const int i = gt + k * (CL * NT);
                    const float* const q = Sa + k * (kSampleTerms * NT);
                    sa[k].c = make_float2(q[0], q[NT]);
                    sa[k].nl = make_float2(q[2 * NT], q[3 * NT]);
                    sa[k].nr = make_float2(q[4 * NT], q[5 * NT]);
                    sa[k].nu = make_float2(q[6 * NT], q[7 * NT]);
                    sa[k].nd = make_float2(q[8 * NT], q[9 * NT]);
                    sa[k].a = q[10 * NT];
                    sa[k].b = q[11 * NT];
                    sa[k].ok = q[12 * NT] != 0.f;
                    const int sy = i < L.nsamp ? i / L.nsx : 0, sx = i < L.nsamp ? i - sy * L.nsx : 0;
                    su[k] = sx * L.s;
                    sv[k] = sy * L.s;
                }
#pragma unroll
                for (int k = 0; k < MAXS; ++k) stage_w(L.A, L.B, wp, su[k], sv[k], sa[k], sw[k]);
#pragma unroll
                for (int k = 0; k < MAXS; ++k) stage_b<PREC>(L.B, sw[k], sb[k]);
#pragma unroll
                for (int k = 0; k < MAXS; ++k) {
                    PixelTerms o;
                    finish<false>(L.A, wp, sa[k], sw[k], sb[k], o);
                    rs[0][k] = o.mI ? o.rI : __int_as_float(0x7fc00000);
                    rs[1][k] = o.mW ? o.rW : __int_as_float(0x7fc00000);
                }
            }

            STAMP_C(4);
            // ---- counts and mean square -> sigma0 (mu0 = 0)
            {
                float v4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int k = 0; k < MAXS; ++k) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const float r = rs[c][k];
                        const bool use = r == r;
                        const float rv = use ? r : 0.f;
                        v4[2 * c] += use ? 1.f : 0.f;
                        v4[2 * c + 1] = fmaf(rv, rv, v4[2 * c + 1]);
                    }
                }
                R.run(v4);
            }
            const float n[2] = {tot[0], tot[2]};
            float mu[2] = {0.f, 0.f};
            float sig[2];
            bool live[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float ms = n[c] > 0.f ? __fdividef(tot[2 * c + 1], n[c]) : 0.f;
                sig[c] = ms > 0.f ? ms * rsqrtf(ms) : 0.f;
                live[c] = n[c] > 0.f && sig[c] >= 1e-12f;
            }
            STAMP_C(5);
            // ---- (mu, sigma) fixed point at nu0 with lagged weights
            for (int si = 0; si < a.scale_iters; ++si) {
                if (!live[0] && !live[1]) break;
                float v6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float mc = mu[c];
                    const float s2 = sig[c] * sig[c];
                    const float s2nu = s2 * nu0;
                    const float num = (nu0 + 1.f) * s2;
#pragma unroll
                    for (int k = 0; k < MAXS; ++k) {
                        const float r = rs[c][k];
                        const bool use = r == r;
                        const float dr = r - mc;
                        const float wr = __fdividef(num, fmaf(dr, dr, s2nu));
                        const float wv = use ? wr : 0.f, d = use ? dr : 0.f;
                        v6[3 * c] += wv;
                        v6[3 * c + 1] = fmaf(wv, d, v6[3 * c + 1]);
                        v6[3 * c + 2] = fmaf(wv * d, d, v6[3 * c + 2]);
                    }
                }
                R.run(v6);
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (!live[c]) continue;
                    const float S0 = tot[3 * c], S1 = tot[3 * c + 1], S2 = tot[3 * c + 2];
                    const float delta = __fdividef(S1, S0);
                    mu[c] += delta;
                    const float var = __fdividef(fmaf(-S1, delta, S2), n[c]);
                    sig[c] = var > 0.f ? var * rsqrtf(var) : 0.f;
                    if (!(sig[c] >= 1e-12f)) live[c] = false;
                }
            }
            bool ok[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) ok[c] = n[c] > 0.f && sig[c] >= 1e-12f;

            STAMP_C(6);
            // ---- nu: the Chebyshev power sums gathered to CTA 0, which bisects
            float nu[2] = {nu0, nu0};
            const bool do_nu = a.estimate_nu && (ok[0] || ok[1]);
            if (do_nu) {
                unsigned long long V[kChebVals];
#pragma unroll
                for (int i = 0; i < kChebVals; ++i) V[i] = 0ull;
                const float is0 = ok[0] ? __fdividef(1.f, sig[0]) : 0.f;
                const float is1 = ok[1] ? __fdividef(1.f, sig[1]) : 0.f;
#pragma unroll 1
                for (int k = 0; k < MAXS; ++k) {
                    float r0 = rs[0][0], r1 = rs[1][0];
#pragma unroll
                    for (int q = 1; q < MAXS; ++q)
                        if (k == q) {
                            r0 = rs[0][q];
                            r1 = rs[1][q];
                        }
                    float q2[2], g2[2], l2[2];
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const float x = ((c ? r1 : r0) - mu[c]) * (c ? is1 : is0);
                        const bool use = ok[c] && x == x;
                        const float al = __fdividef(fmaf(x, x, m), h);
                        const float s2 = fmaf(al, al, -1.f);
                        const float gam = rsqrtf(s2);
                        const float be = fmaf(s2, gam, al);
                        q2[c] = use ? __fdividef(1.f, be) : 0.f;
                        g2[c] = use ? gam : 0.f;
                        l2[c] = use ? __logf(0.5f * be) : 0.f;
                    }
                    const unsigned long long Q = f2_pack(q2[0], q2[1]), Gp = f2_pack(g2[0], g2[1]);
                    V[0] = f2_add(V[0], f2_pack(l2[0], l2[1]));
                    V[1 + kChebK] = f2_add(V[1 + kChebK], Gp);
                    unsigned long long qk = Q;
#pragma unroll
                    for (int kk = 1; kk <= kChebK; ++kk) {
                        V[kk] = f2_add(V[kk], qk);
                        V[1 + kChebK + kk] = f2_fma(Gp, qk, V[1 + kChebK + kk]);
                        qk = f2_mul(qk, Q);
                    }
                }
                float v[96];
#pragma unroll
                for (int i = 0; i < kChebVals; ++i) {
                    v[i] = f2_lo(V[i]);
                    v[kChebVals + i] = f2_hi(V[i]);
                }
#pragma unroll
                for (int i = 2 * kChebVals; i < 96; ++i) v[i] = 0.f;
                R.template run<96, 2 * kChebVals, true>(v);   // only CTA 0 bisects
            }
            STAMP_C(7);
            if (rank == 0) {
                if (do_nu && tid < 64) {
                    const int c = tid >> 5;
                    float nuc = nu0;
                    if (ok[c]) nuc = bisect_nu_warp(tot + c * kChebVals, n[c], sh_g, lo0, hi0, a.bisect_steps, nuF[c]);
                    if (lane == 0) nu_out[c] = nuc;
                }
                __syncthreads();
                if (do_nu) {
                    nu[0] = nu_out[0];
                    nu[1] = nu_out[1];
                    if (ok[0] && ok[1]) nu[0] = fmaxf(nu[0], nu[1]);
                }
                if (tid == 0) {
                    RobustParams rp;
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        rp.mu[c] = mu[c];
                        rp.sigma[c] = sig[c];
                        rp.nu[c] = nu[c];
                        rp.ok[c] = ok[c] ? 1 : 0;
                    }
                    sh_rob = rp;
                    // ---- publish the parameters to the helpers
                    const int* const src = reinterpret_cast<const int*>(&rp);
#pragma unroll
                    for (int q = 0; q < (int)(sizeof(RobustParams) / 4); ++q)
                        __stcg(reinterpret_cast<int*>(&mb->rob) + q, src[q]);
                    // the same thread releases the flag: the release orders the stores above
                    st_release_u32(&mb->rob_flag, (unsigned)git + 1u);
                    STAMP_C(8);
                }
            }
        }
        }
        // ---- the last step stays pending: the helpers' partials, weighted with the
        //      parameters published last, at the pose published last
        __syncthreads();
        if (rank == 0) {
            if (tid < 16) {
                st->T[tid] = T_sh[tid];
                reinterpret_cast<float*>(&st->wp)[tid] = reinterpret_cast<const float*>(&sh_wp)[tid];
            } else if (tid == 16) {
                st->rob = sh_rob;
            } else if (tid == 17) {
                st->iters_done = sh_cnt[0];
                st->iters_skipped = sh_cnt[1];
                st->status = sh_cnt[2];
                st->pending = (unsigned)a.n_helpers;
            }
        }
        // no CTA leaves before every CTA is past its last exchange
        cluster_arrive();
        cluster_wait();
    } else {
        // ================================================================ helper CTAs
        const int hc = (int)blockIdx.x - CL;
        float* const Tm = dyn + tid;                 // [max_tiles][kSplitTerms][NT]
        pdl_wait();
        int git = 0;
        bool broken = false;
        for (int l = 0; l < a.n_levels && !broken; ++l) {
          const int n_it = level_its(l);
          if (n_it <= 0) continue;
          const SplitLevel& L = a.lv[l];
          const int ntiles = L.tiles_x * L.tiles_y;
          const int mt = min(a.max_tiles, (ntiles + a.n_helpers - 1) / a.n_helpers);   // this level's tiles per CTA
          for (int it = 0; it < n_it; ++it, ++git) {
            if (git == n_total - 1) pdl_trigger();
            if (!cta_wait(st, &mb->pose_flag, (unsigned)git + 1u, &go[1])) {
                broken = true;
                break;
            }
            STAMP_H(9);
            if (tid < 16) reinterpret_cast<float*>(&sh_wp)[tid] = __ldcg(reinterpret_cast<const float*>(&mb->wp) + tid);
            __syncthreads();
            const WarpPose wp = sh_wp;
            // ---- the terms of every pixel of this CTA's tiles at the published pose
#pragma unroll 1
            for (int j0 = 0; j0 < mt; j0 += G) {
                PxA sa[G];
                PxW sw[G];
                PxB sb[G];
                int pu[G], pv[G];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    sa[g].ok = false;
                    pu[g] = 0;
                    pv[g] = 0;
                    const int t = hc + (j0 + g) * a.n_helpers;
                    if (j0 + g < mt && t < ntiles) {
                        const int ty = t / L.tiles_x, tx = t - ty * L.tiles_x;
                        const int u = tx * kSplitTileW + lane, v = ty * kSplitTileH + warp;
                        if (u < L.A.w && v < L.A.h) {
                            pu[g] = u;
                            pv[g] = v;
                            stage_a<PREC>(L.A, u, v, sa[g]);
                        }
                    }
                }
#pragma unroll
                for (int g = 0; g < G; ++g) stage_w(L.A, L.B, wp, pu[g], pv[g], sa[g], sw[g]);
#pragma unroll
                for (int g = 0; g < G; ++g) stage_b<PREC>(L.B, sw[g], sb[g]);
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    if (j0 + g >= mt) continue;
                    PixelTerms o;
                    finish<true>(L.A, wp, sa[g], sw[g], sb[g], o);
                    float* const T = Tm + (j0 + g) * (kSplitTerms * NT);
                    T[0] = o.mI ? o.rI : __int_as_float(0x7fc00000);
                    T[NT] = o.mW ? o.rW : __int_as_float(0x7fc00000);
                    if (o.mI) {
#pragma unroll
                        for (int q = 0; q < 6; ++q) T[(2 + q) * NT] = o.JI[q];
                    }
                    if (o.mW) {
#pragma unroll
                        for (int q = 0; q < 6; ++q) T[(8 + q) * NT] = o.JW[q];
                        T[14 * NT] = o.lam;
                    }
                }
            }
            STAMP_H(10);
            // ---- weighted normal equations once the parameters are published
            if (!cta_wait(st, &mb->rob_flag, (unsigned)git + 1u, &go[2])) {
                broken = true;
                break;
            }
            STAMP_H(11);
            if (tid < (int)(sizeof(RobustParams) / 4))
                reinterpret_cast<int*>(&sh_rob)[tid] = __ldcg(reinterpret_cast<const int*>(&mb->rob) + tid);
            __syncthreads();
            const RobustParams rob = sh_rob;
            float acc[kSlots];
#pragma unroll
            for (int i = 0; i < kSlots; ++i) acc[i] = 0.f;
#pragma unroll 1
            for (int j = 0; j < mt; ++j) {
                const float* const T = Tm + j * (kSplitTerms * NT);
                const float rI = T[0], rW = T[NT];
                if (rI == rI) {
                    acc[kSlotNI] += 1.f;
                    if (rob.ok[0]) {
                        float Jl[6];
#pragma unroll
                        for (int q = 0; q < 6; ++q) Jl[q] = T[(2 + q) * NT];
                        accumulate(acc, Jl, robust_weight(rI, rob.mu[0], rob.sigma[0], rob.nu[0]), rI);
                    }
                }
                if (rW == rW) {
                    acc[kSlotNW] += 1.f;
                    if (rob.ok[1]) {
                        float Jl[6];
#pragma unroll
                        for (int q = 0; q < 6; ++q) Jl[q] = T[(8 + q) * NT];
                        accumulate(acc, Jl, T[14 * NT] * robust_weight(rW, rob.mu[1], rob.sigma[1], rob.nu[1]), rW);
                    }
                }
            }
            red_w[warp][lane] = warp_reduce_scatter32(acc);
            __syncthreads();
            if (warp == 0) {
                F2 sum{0.f, 0.f};
#pragma unroll
                for (int w = 0; w < NW; ++w) sum.add(red_w[w][lane]);
                __stcg(a.partials + (size_t)hc * kSlots + lane, make_float2(sum.hi, sum.lo));
                __threadfence();
                __syncwarp();
                if (lane == 0) atomicAdd(&mb->arrived, 1u);
                if (lane == 0) STAMP_H(12);
            }
          }
        }
    }
    // ---- the last CTA to leave resets the mailbox for the next launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned int done = atomicAdd(&mb->exited, 1u) + 1u;
        if (done == gridDim.x) {
            mb->pose_flag = 0u;
            mb->rob_flag = 0u;
            mb->arrived = 0u;
            mb->error = 0;
            __threadfence();
            mb->exited = 0u;
        }
    }
}

// ---------------------------------------------------------------- mailbox wait probe
// The split kernel's mailbox wait on a counter that nothing advances: the first wait
// (budget `budget`) runs out, counts a timeout and raises the error flag; the second
// (the full ~2 s budget) must then give up at once.  out = {timeouts, verdict of the
// first wait, verdict of the second, error flag}.  The mailbox is left clear.
__global__ void mailbox_probe_kernel(AlignState* st, long long budget, int* out) {
    __shared__ int go[2];
    if (threadIdx.x == 0) {
        st->timeouts = 0;
        st->mb.pose_flag = 0u;
        st->mb.error = 0;
        __threadfence();
    }
    __syncthreads();
    const bool first = cta_wait(st, &st->mb.pose_flag, 1u, &go[0], budget);
    const bool second = cta_wait(st, &st->mb.pose_flag, 1u, &go[1]);
    if (threadIdx.x == 0) {
        out[0] = st->timeouts;
        out[1] = first ? 1 : 0;
        out[2] = second ? 1 : 0;
        out[3] = ld_relaxed_s32(&st->mb.error);
        st->mb.error = 0;
        st->timeouts = 0;
    }
}

// ---------------------------------------------------------------- host side
template <int PREC, int MAXP>
static cudaError_t level_attributes() {
    cudaError_t e = cudaFuncSetAttribute(level_kernel<PREC, MAXP>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(level_kernel<PREC, MAXP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)level_dyn_smem<MAXP>());
}

template <int PREC, int MAXP>
static void level_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, cudaStream_t stream) {
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3(kLevelCL, 1, 1);
    cfg.blockDim = dim3(kRobustNT, 1, 1);
    cfg.dynamicSmemBytes = level_dyn_smem<MAXP>();
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kLevelCL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
}

// Whether the device schedules the 16-CTA cluster of both pixel capacities with
// their shared memory; a fixed property of the device, cached per ordinal.
template <int PREC>
static bool level_kernel_schedulable() {
    static std::atomic<int> cached[64];   // 0 unknown, 1 yes, 2 no
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return false;
    }
    int c = cached[dev].load(std::memory_order_relaxed);
    if (c == 0) {
        bool ok = level_attributes<PREC, 2>() == cudaSuccess && level_attributes<PREC, 5>() == cudaSuccess;
        if (ok) {
            cudaLaunchConfig_t cfg;
            cudaLaunchAttribute attr[2];
            level_config<PREC, 5>(cfg, attr, 0);
            cfg.numAttrs = 1;   // the cluster shape alone
            int nclusters = 0;
            ok = cudaOccupancyMaxActiveClusters(&nclusters, level_kernel<PREC, 5>, &cfg) == cudaSuccess &&
                 nclusters > 0;
        }
        (void)cudaGetLastError();
        c = ok ? 1 : 2;
        cached[dev].store(c, std::memory_order_relaxed);
    }
    return c == 1;
}

bool level_kernel_takes(int precision, int w, int h, int cap) {
    const long long n = (long long)w * h;
    if (n > cap || n > kLevelMaxPixels) return false;   // the sample must be every pixel
    return precision == RGBID_PLANES_F32 ? level_kernel_schedulable<RGBID_PLANES_F32>()
                                         : level_kernel_schedulable<RGBID_PLANES_BF16_F16>();
}

template <int PREC>
static cudaError_t launch_level_t(const LevelArgs& la, cudaStream_t stream) {
    const long long n = (long long)la.A.w * la.A.h;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    if (n <= (long long)kLevelCL * kRobustNT * 2) {
        cudaError_t e = level_attributes<PREC, 2>();
        if (e != cudaSuccess) return e;
        level_config<PREC, 2>(cfg, attr, stream);
        return cudaLaunchKernelEx(&cfg, level_kernel<PREC, 2>, la);
    }
    cudaError_t e = level_attributes<PREC, 5>();
    if (e != cudaSuccess) return e;
    level_config<PREC, 5>(cfg, attr, stream);
    return cudaLaunchKernelEx(&cfg, level_kernel<PREC, 5>, la);
}

cudaError_t launch_level(int precision, const LevelArgs& la, cudaStream_t stream) {
    const long long n = (long long)la.A.w * la.A.h;
    if (n < 1 || n > kLevelMaxPixels) return cudaErrorInvalidValue;
    return precision == RGBID_PLANES_F32 ? launch_level_t<RGBID_PLANES_F32>(la, stream)
                                         : launch_level_t<RGBID_PLANES_BF16_F16>(la, stream);
}

// ---- split kernel
constexpr size_t kSplitMaxSmem = (size_t)kSplitMaxTiles * kSplitTerms * kRobustNT * sizeof(float);
constexpr size_t kSplitSampleSmem =
    (size_t)((RGBID_MAX_SAMPLES + kLevelCL * kRobustNT - 1) / (kLevelCL * kRobustNT)) * kSampleTerms * kRobustNT *
    sizeof(float);

static size_t split_smem(int max_tiles) {
    return std::max((size_t)max_tiles * kSplitTerms * kRobustNT * sizeof(float), kSplitSampleSmem);
}

template <int PREC>
static cudaError_t split_attributes() {
    cudaError_t e = cudaFuncSetAttribute(split_kernel<PREC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(split_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSplitMaxSmem);
}

// Helper CTAs: every co-resident 16-CTA cluster after the first (at the largest
// shared memory a launch takes), at most 8 clusters; a fixed property of the
// device, cached per ordinal.
template <int PREC>
static int split_helpers_t() {
    static std::atomic<int> cached[64];   // 0 unknown, -1 none, else helper CTAs
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return 0;
    }
    int c = cached[dev].load(std::memory_order_relaxed);
    if (c == 0) {
        int nclusters = 0;
        if (split_attributes<PREC>() == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(kLevelCL, 1, 1);
            cfg.blockDim = dim3(kRobustNT, 1, 1);
            cfg.dynamicSmemBytes = kSplitMaxSmem;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = kLevelCL;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if (cudaOccupancyMaxActiveClusters(&nclusters, split_kernel<PREC>, &cfg) != cudaSuccess) nclusters = 0;
        }
        (void)cudaGetLastError();
        c = nclusters >= 2 ? std::min(kLevelCL * (nclusters - 1), kSplitMaxHelpers) : -1;
        cached[dev].store(c, std::memory_order_relaxed);
    }
    return c > 0 ? c : 0;
}

int split_kernel_helpers(int precision) {
    return precision == RGBID_PLANES_F32 ? split_helpers_t<RGBID_PLANES_F32>()
                                         : split_helpers_t<RGBID_PLANES_BF16_F16>();
}

int split_tiles_per_helper(int w, int h, int n_helpers) {
    const long long tiles = (long long)((w + kSplitTileW - 1) / kSplitTileW) * ((h + kSplitTileH - 1) / kSplitTileH);
    return n_helpers > 0 ? (int)((tiles + n_helpers - 1) / n_helpers) : 0x7fffffff;
}

bool split_kernel_takes(int precision, int w, int h) {
    const int nh = split_kernel_helpers(precision);
    if (nh <= 0) return false;
    return split_tiles_per_helper(w, h, nh) <= kSplitMaxTiles;
}

template <int PREC>
static cudaError_t launch_split_t(const SplitArgs& sa, cudaStream_t stream) {
    cudaError_t e = split_attributes<PREC>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(kLevelCL + sa.n_helpers), 1, 1);
    cfg.blockDim = dim3(kRobustNT, 1, 1);
    cfg.dynamicSmemBytes = split_smem(sa.max_tiles);
    cfg.stream = stream;
    cudaLaunchAttribute attr[3];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kLevelCL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeCooperative;   // every CTA resident: the roles wait on one another
    attr[1].val.cooperative = 1;
    attr[2].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[2].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 3;
    return cudaLaunchKernelEx(&cfg, split_kernel<PREC>, sa);
}

cudaError_t launch_split(int precision, const SplitArgs& sa, cudaStream_t stream) {
    if (sa.n_helpers <= 0 || sa.n_helpers > kSplitMaxHelpers || sa.n_helpers % kLevelCL ||
        sa.n_helpers != split_kernel_helpers(precision))
        return cudaErrorInvalidValue;
    if (sa.max_tiles < 1 || sa.max_tiles > kSplitMaxTiles) return cudaErrorInvalidValue;
    if (sa.n_levels < 1 || sa.n_levels > kSplitMaxLevels) return cudaErrorInvalidValue;
    for (int l = 0; l < sa.n_levels; ++l) {
        const SplitLevel& L = sa.lv[l];
        if ((long long)sa.max_tiles * sa.n_helpers < (long long)L.tiles_x * L.tiles_y) return cudaErrorInvalidValue;
        if (L.tiles_x * kSplitTileW < L.A.w || L.tiles_y * kSplitTileH < L.A.h) return cudaErrorInvalidValue;
        if (L.nsamp < 1 || L.nsamp > RGBID_MAX_SAMPLES) return cudaErrorInvalidValue;
    }
    return precision == RGBID_PLANES_F32 ? launch_split_t<RGBID_PLANES_F32>(sa, stream)
                                         : launch_split_t<RGBID_PLANES_BF16_F16>(sa, stream);
}

}  // namespace rgbid

extern "C" int rgbid_probe_mailbox_timeout(long long budget_cycles, void* d_scratch, size_t scratch_bytes, int* d_out,
                                           void* stream) {
    static_assert(sizeof(rgbid::AlignState) <= 1024, "probe scratch");
    if (!d_scratch || !d_out || scratch_bytes < 1024 || budget_cycles < 0 || budget_cycles > 20000000000LL)
        return RGBID_ERR_INVALID_ARG;
    if (((uintptr_t)d_scratch & 15u) || ((uintptr_t)d_out & 3u)) return RGBID_ERR_INVALID_ARG;
    rgbid::mailbox_probe_kernel<<<1, 64, 0, (cudaStream_t)stream>>>(reinterpret_cast<rgbid::AlignState*>(d_scratch),
                                                                    budget_cycles, d_out);
    if (cudaGetLastError() != cudaSuccess) return RGBID_ERR_CUDA;
    return RGBID_OK;
}

namespace rgbid {
// out-of-plane gathers counted by this translation unit's kernels (bounds-checked builds)
unsigned int oob_count_level() { return oob_count_this_unit(); }
}  // namespace rgbid

extern "C" int rgbid_debug_phase_stamps(long long* out, int n) {
#ifdef RGBID_PHASE_STAMPS
    constexpr int kN = RGBID_MAX_LEVELS * 16 * 16;
    if (!out || n < kN) return RGBID_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpyFromSymbol(out, g_phase, sizeof(long long) * kN) != cudaSuccess) {
        (void)cudaGetLastError();
        return RGBID_ERR_CUDA;
    }
    return RGBID_OK;
#else
    (void)out;
    (void)n;
    return RGBID_ERR_UNSUPPORTED;
#endif
}
