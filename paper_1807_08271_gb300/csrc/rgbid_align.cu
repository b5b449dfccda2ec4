// Dense IRLS alignment kernels and the rgbid_align / rgbid_eval_step entry points.
//
// Per Gauss-Newton iteration two kernels run on the caller's stream:
//   robust_kernel  one thread-block cluster.  It first finishes the previous
//                  iteration's sweep: the CTAs sum disjoint subsets of its block
//                  partials (compensated FP32), one exchange through distributed
//                  shared memory gives every CTA the totals, and every CTA solves
//                  H xi = -g by a Jacobi-scaled Cholesky and applies
//                  T <- exp(xi)^-1 T to its copy of the FP64 pose ("Iterative
//                  optimisation"); CTA 0 writes the new state and the step's
//                  results.  It then warps the <= 19200 systematic sample pixels
//                  with the new pose and estimates the Student-t (mu, sigma) at
//                  nu0 by the lagged-weight fixed point (every round exchanged
//                  across the cluster), then gathers the sums of the robustness
//                  equation to CTA 0, which finds nu by bisection ("Error
//                  distribution and robust optimisation").
//   sweep_kernel   the whole level: warp, residuals, Jacobians, weights and the
//                  per-block compensated partials of the 27 normal-equation terms
//                  (plus cost and counts).
// A closing robust_kernel launch (finalize_only) finishes the last sweep of an
// alignment.
#include <cooperative_groups.h>
#include <cuda.h>
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>

#include "rgbid_cluster.cuh"
#include "rgbid_device.cuh"
#include "rgbid_level.h"
#include "rgbid_util.h"

namespace cg = cooperative_groups;

namespace rgbid {

constexpr int kSweepNT = 256;       // 8 warps
constexpr int kTileW = 32;
// Rows per thread of the sweep: 4 on a level of at least kSweepWidePixels (its blocks
// still fill the GPU in one wave), else 1, so a coarse level's blocks are four times
// as many and each thread's serial work a quarter as long.
constexpr long long kSweepWidePixels = 250000;

struct InitArgs {
    AlignState* st;
    rgbid_align_result* res;
    const double* T_dev;     // device pose or null
    double T_val[16];        // host pose (used when T_dev is null)
    int use_fixed;
    float fixed[6];          // mu_I, sigma_I, nu_I, mu_W, sigma_W, nu_W
};

struct RobustArgs {
    LevelDev A, B;
    LevelDev A0, B0;          // level 0 (the warp at full resolution)
    int full_level;           // > 0: warp at level 0 and reduce to this level (reading R22); 0: warp here
    AlignState* st;
    int s, nsx, nsamp;
    int scale_iters, bisect_steps, estimate_nu;
    float nu0;
    double nu_lo, nu_hi;
    const int* level_iters;   // device iterations per level (NULL: none skipped)
    int level, iter;
    // reduction of the previous sweep's block partials, solve and update
    const float2* partials;
    rgbid_align_result* res;
    int update;               // 0: results only (one evaluated step), 1: also update the pose
    int min_valid;
    int finalize_only;        // 1: finish the previous sweep and stop (no robust estimation)
    int state_after_wait;     // 1: the preceding launch writes the state (a level kernel): read it after the wait
    float nu_g[kNuGTerms];    // Chebyshev series of the nu equation's constant part on [nu_lo, nu_hi]
};

struct SweepArgs {
    LevelDev A, B;
    LevelDev A0, B0;          // level 0 (the warp at full resolution)
    int full_level;           // > 0: warp at level 0 and reduce to this level (reading R22); 0: warp here
    const float2* G;          // optional plane for the reference's gradients (the covariance iteration)
    AlignState* st;
    float* partials;
    float* r_I;
    float* r_W;
    uint8_t* m_I;
    uint8_t* m_W;
    const int* level_iters;   // device iterations per level (NULL: none skipped)
    int level, iter;
};

// An iteration beyond the device-side count of its level does nothing.  Its
// CTAs still wait for the preceding grid (griddepcontrol.wait) before they
// return, and they never trigger the next launch, so the chain of dependent
// launches stays ordered end to end whichever levels are skipped.  The counts
// are written before the alignment's first kernel runs.
__device__ __forceinline__ bool iteration_skipped(const int* level_iters, int level, int iter) {
    return level_iters && iter >= __ldg(level_iters + level);
}

// ---------------------------------------------------------------- init
__global__ void init_kernel(InitArgs a) {
    AlignState* st = a.st;
    __shared__ double T[16];
    if (threadIdx.x < 16) {
        T[threadIdx.x] = a.T_dev ? a.T_dev[threadIdx.x] : a.T_val[threadIdx.x];
        st->T[threadIdx.x] = T[threadIdx.x];
        a.res->T[threadIdx.x] = T[threadIdx.x];
    }
    __syncwarp();
    warp_make_pose(T, &st->wp);
    if (threadIdx.x != 0) return;
    st->pending = 0u;
    st->status = RGBID_OK;
    st->iters_done = 0;
    st->iters_skipped = 0;
    st->timeouts = 0;
    st->mb.pose_flag = 0u;
    st->mb.rob_flag = 0u;
    st->mb.arrived = 0u;
    st->mb.exited = 0u;
    st->mb.error = 0;
    if (a.use_fixed) {
        for (int c = 0; c < 2; ++c) {
            st->rob.mu[c] = a.fixed[3 * c + 0];
            st->rob.sigma[c] = a.fixed[3 * c + 1];
            st->rob.nu[c] = a.fixed[3 * c + 2];
            st->rob.ok[c] = a.fixed[3 * c + 1] >= 1e-12f;
        }
    }
    rgbid_align_result* r = a.res;
    for (int i = 0; i < 36; ++i) r->H[i] = 0.0;
    for (int i = 0; i < 6; ++i) r->g[i] = 0.0;
    for (int c = 0; c < 2; ++c) { r->mu[c] = 0.0; r->sigma[c] = 0.0; r->nu[c] = 0.0; r->n_valid[c] = 0; }
    r->cost = 0.0;
    r->iters_done = 0;
    r->iters_skipped = 0;
    r->status = RGBID_OK;
}

// ---------------------------------------------------------------- robust scale (cluster)
template <int PREC, int CL, bool FULL>
__global__ void __launch_bounds__(kRobustNT) robust_kernel(RobustArgs a) {
    constexpr int MAXS = (RGBID_MAX_SAMPLES + CL * kRobustNT - 1) / (CL * kRobustNT);
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    __shared__ float red_w[kRobustNT / 32][kRobustMaxNV];
    __shared__ float2 recv[2][CL][kRobustMaxNV];
    __shared__ float tot[kRobustMaxNV];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ WarpPose sh_wp;
    __shared__ float nu_out[2];
    __shared__ float nuF[2][kNuSeries];          // per channel: f(nu) as one Chebyshev series
    __shared__ float sh_g[kNuGTerms];            // the host series of f's constant part
    __shared__ F2 fin2[kRobustNT / 32][kSlots];
    __shared__ double T_sh[16];
    __shared__ double totd[kSlots];
    __shared__ float xi_f[6], d_f[6];
    __shared__ double xi_d[6], rho_d[6];
    __shared__ int ok_flag;
    __shared__ RobustParams sh_rob_prev;         // rank 0: the parameters the previous sweep used
    __shared__ int sh_cnt[3];                    // rank 0: iters_done, iters_skipped, status
    if (!a.finalize_only && iteration_skipped(a.level_iters, a.level, a.iter)) {
        pdl_wait();
        return;
    }
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
        for (int k = 0; k < kNuGTerms; ++k) sh_g[k] = a.nu_g[k];
    }
    // No CTA stores into another before every barrier of the cluster is
    // initialised: arrive now, wait once the dependent-launch wait is over.
    cluster_arrive();
    // What this launch reads before the wait comes from grids that completed before
    // it started (the previous robust launch and the alignment's initialisation,
    // both ahead of the sweep it waits for): the state fields that CTA 0 writes back,
    // the pose and its FP32 warp form, and the keyframe-side loads of the systematic
    // sample (A's planes do not change during an alignment).  Only the sweep's
    // partials and their count need the wait.
    // A level kernel writes the state itself, so after one of them the state is read
    // only once the wait is over.
    const auto load_state = [&]() {
        if (rank == 0) {
            constexpr int kRobWords = (int)(sizeof(RobustParams) / 4);
            if (threadIdx.x < kRobWords)
                reinterpret_cast<int*>(&sh_rob_prev)[threadIdx.x] =
                    __ldcg(reinterpret_cast<const int*>(&a.st->rob) + threadIdx.x);
            else if (threadIdx.x == 32) sh_cnt[0] = __ldcg(&a.st->iters_done);
            else if (threadIdx.x == 33) sh_cnt[1] = __ldcg(&a.st->iters_skipped);
            else if (threadIdx.x == 34) sh_cnt[2] = __ldcg(&a.st->status);
        }
        static_assert(sizeof(WarpPose) == 16 * sizeof(float), "the warp pose is 16 floats");
        if (threadIdx.x >= 64 && threadIdx.x < 80) T_sh[threadIdx.x - 64] = __ldcg(a.st->T + (threadIdx.x - 64));
        else if (threadIdx.x >= 96 && threadIdx.x < 112)
            reinterpret_cast<float*>(&sh_wp)[threadIdx.x - 96] =
                __ldcg(reinterpret_cast<const float*>(&a.st->wp) + (threadIdx.x - 96));
    };
    if (!a.state_after_wait) load_state();
    PxA sa[MAXS];
    int su[MAXS], sv[MAXS];
    {
        const int gt = rank * kRobustNT + (int)threadIdx.x;
#pragma unroll
        for (int k = 0; k < MAXS; ++k) {
            const int i = gt + k * (CL * kRobustNT);
            sa[k].ok = false;
            su[k] = 0;
            sv[k] = 0;
            if (!a.finalize_only && i < a.nsamp) {
                const int sy = i / a.nsx, sx = i - sy * a.nsx;
                su[k] = sx * a.s;
                sv[k] = sy * a.s;
                stage_a<PREC>(a.A, su[k], sv[k], sa[k]);
            }
        }
    }
    pdl_wait();  // the previous sweep's partials (and the state) are complete and visible
    if (a.state_after_wait) load_state();
    cluster_wait();
    pdl_trigger();
    ClusterSum<CL> R{red_w, recv, tot, mbar, &a.st->timeouts, (uint32_t)rank, 0};
    const unsigned int nb = __ldcg(&a.st->pending);   // the same value in every CTA

    // ---- finish the previous sweep: the CTAs sum disjoint subsets of its block
    //      partials (compensated pairs), one exchange gives every CTA the totals,
    //      and every CTA solves H xi = -g and updates its copy of the pose
    if (nb) {
        const int t = (int)threadIdx.x, lane = t & 31, grp = t >> 5;
        F2 acc{0.f, 0.f};
        // four partials of this thread in flight at once, summed in ascending block order
        constexpr unsigned kStride = (unsigned)CL * (kRobustNT / 32);
        for (unsigned int b0 = (unsigned)rank + (unsigned)CL * (unsigned)grp; b0 < nb; b0 += 4u * kStride) {
            float2 v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned int b = b0 + (unsigned)q * kStride;
                v[q] = b < nb ? __ldcg(a.partials + (size_t)b * kSlots + lane) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) acc.add(F2{v[q].x, v[q].y});
        }
        fin2[grp][lane] = acc;
        __syncthreads();
        if (t < kSlots) {
            // one sender per slot: with 32 slots, spreading the sends would cost a block barrier
            const F2 T2 = R.template exchange<kSlots>(t, warp_tree<kRobustNT / 32>(fin2, t));
            tot[t] = T2.value();
            if (a.finalize_only) totd[t] = (double)T2.hi + (double)T2.lo;   // for the result record
        }
        __syncthreads();
        R.next();
        if (a.finalize_only) cluster_arrive();   // the launch's only exchange is over
        if (t < 32) {
            const bool ok_in = a.update && ((int)tot[kSlotNI] + (int)tot[kSlotNW]) >= a.min_valid;
            if constexpr (PREC == RGBID_PLANES_BF16_F16) {
                // reduced-precision planes: FP32 factorisation refined to an FP64 solution
                const bool okl = warp_solve6_refined(tot, ok_in, xi_f, d_f, rho_d, xi_d);
                if (lane == 0) ok_flag = okl ? 1 : 0;
            } else if (lane == 0) {
                float xi[6];
                const bool okl = ok_in && cholesky_solve6_slots(tot, xi);
#pragma unroll
                for (int i = 0; i < 6; ++i) xi_f[i] = okl ? xi[i] : 0.f;
                ok_flag = okl ? 1 : 0;
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
                warp_make_pose(T_sh, &sh_wp);
            }   // else sh_wp keeps the pose loaded at the start
            __syncwarp();
            if (rank == 0) {
                // the new state (written once, by CTA 0), and in the alignment's closing
                // launch the result record (no other launch's record would survive)
                AlignState* st = a.st;
                rgbid_align_result* res = a.res;
                const bool rec = a.finalize_only != 0;
                const double td = rec ? totd[lane] : 0.0;
                const float tf = tot[lane];
                if (rec) {
                    if (lane < 21) {
                        int i = 0, rem = lane;
                        while (rem >= 6 - i) { rem -= 6 - i; ++i; }
                        const int j = i + rem;
                        res->H[i * 6 + j] = td;
                        res->H[j * 6 + i] = td;
                    } else if (lane < 27) {
                        res->g[lane - kSlotG] = td;
                    } else if (lane == kSlotCost) {
                        res->cost = td;
                    } else if (lane == kSlotNI) {
                        res->n_valid[0] = (int)tf;
                    } else if (lane == kSlotNW) {
                        res->n_valid[1] = (int)tf;
                    } else if (lane == 30) {
                        const RobustParams rob = sh_rob_prev;  // the parameters the sweep used
                        res->mu[0] = rob.mu[0]; res->mu[1] = rob.mu[1];
                        res->sigma[0] = rob.sigma[0]; res->sigma[1] = rob.sigma[1];
                        res->nu[0] = rob.nu[0]; res->nu[1] = rob.nu[1];
                    }
                }
                if (a.update) {
                    if (ok_flag && lane < 16) {
                        reinterpret_cast<float*>(&st->wp)[lane] = reinterpret_cast<const float*>(&sh_wp)[lane];
                        st->T[lane] = T_sh[lane];
                    }
                    if (rec && lane < 16) res->T[lane] = T_sh[lane];
                    if (lane == 0) {
                        const int done = sh_cnt[0] + 1;
                        int skipped = sh_cnt[1], status = sh_cnt[2];
                        if (!ok_flag) {
                            skipped += 1;
                            status = RGBID_ERR_DEGENERATE;
                            st->iters_skipped = skipped;
                            st->status = status;
                        }
                        st->iters_done = done;
                        if (rec) {
                            res->iters_done = done;
                            res->iters_skipped = skipped;
                            // expired waits of every launch of the alignment, this one included
                            res->status = __ldcg(&st->timeouts) ? RGBID_ERR_TIMEOUT : status;
                        }
                    }
                }
                if (lane == 0) st->pending = 0u;
            }
        }
        __syncthreads();
    } else {
        __syncthreads();   // sh_wp: the pose loaded at the start
        if (a.finalize_only) cluster_arrive();
    }
    // No CTA leaves before every CTA is past its last exchange (a split barrier:
    // each arrives once its exchanges are over and waits only when it leaves, so
    // CTA 0's solve, bisection and writes overlap the barrier's latency).
    if (a.finalize_only) {
        cluster_wait();
        return;
    }
    const WarpPose wp = sh_wp;

    // ---- systematic sample residuals r(p, 0) (NaN = masked out); the samples of a
    //      thread go through each evaluation stage together so their loads overlap
    float rs[2][MAXS];
    if constexpr (FULL) {
#pragma unroll
        for (int k = 0; k < MAXS; ++k) {
            PixelTerms o;
            o.mI = o.mW = false;
            if (sa[k].ok) {
                const Warped wd = warped_at_level<PREC>(a.full_level, a.A0, a.B0, wp, su[k], sv[k]);
                finish_given<false>(a.A, sa[k], wd.I, wd.vI, wd.W, wd.vW, o);
            }
            rs[0][k] = o.mI ? o.rI : __int_as_float(0x7fc00000);
            rs[1][k] = o.mW ? o.rW : __int_as_float(0x7fc00000);
        }
    } else {
        PxW sw[MAXS];
        PxB sb[MAXS];
#pragma unroll
        for (int k = 0; k < MAXS; ++k) stage_w(a.A, a.B, wp, su[k], sv[k], sa[k], sw[k]);
#pragma unroll
        for (int k = 0; k < MAXS; ++k) stage_b<PREC>(a.B, sw[k], sb[k]);
#pragma unroll
        for (int k = 0; k < MAXS; ++k) {
            PixelTerms o;
            finish<false>(a.A, wp, sa[k], sw[k], sb[k], o);
            rs[0][k] = o.mI ? o.rI : __int_as_float(0x7fc00000);
            rs[1][k] = o.mW ? o.rW : __int_as_float(0x7fc00000);
        }
    }

    // ---- counts and mean square -> sigma0 (mu0 = 0)
    {
        float v4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < MAXS; ++k) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                // masked samples (NaN) add exact zeros: selects, not branches
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
    const float nu0 = a.nu0;
    for (int it = 0; it < a.scale_iters; ++it) {
        if (!live[0] && !live[1]) break;
        float v6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float m = mu[c];
            const float s2 = sig[c] * sig[c];
            const float s2nu = s2 * nu0;
            const float num = (nu0 + 1.f) * s2;
#pragma unroll
            for (int k = 0; k < MAXS; ++k) {
                const float r = rs[c][k];
                const bool use = r == r;                  // masked samples add exact zeros
                const float dr = r - m;
                const float wr = __fdividef(num, fmaf(dr, dr, s2nu));   // omega((r - mu)/sigma, nu0)
                const float w = use ? wr : 0.f, d = use ? dr : 0.f;
                v6[3 * c] += w;
                v6[3 * c + 1] = fmaf(w, d, v6[3 * c + 1]);
                v6[3 * c + 2] = fmaf(w * d, d, v6[3 * c + 2]);
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

    // ---- nu by bisection on eq. robustnessValue, f(nu) = n c(nu) + sum_i (ln w_i - w_i)
    float nu[2] = {nu0, nu0};
    const bool do_nu = a.estimate_nu && (ok[0] || ok[1]);
    const float lo0 = (float)a.nu_lo, hi0 = (float)a.nu_hi;
    const float m = 0.5f * (lo0 + hi0), h = 0.5f * (hi0 - lo0);
    if (do_nu) {
        // Both channels' sums advance together in packed pairs (low half: I, high
        // half: W): this phase is bound by instruction issue on the cluster's 16 SMs,
        // and the pairs halve the instructions of the 20-term power sums.  A masked
        // sample contributes exact zeros (q = gamma = 0, no log term).
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
        R.template run<96, 2 * kChebVals, true>(v);   // only CTA 0 bisects: the sums go to it alone
    }
    cluster_arrive();
    if (rank != 0) {
        cluster_wait();
        return;
    }

    if (do_nu && threadIdx.x < 64) {
        // warp c solves channel c
        const int c = threadIdx.x >> 5;
        float nuc = nu0;
        if (ok[c]) nuc = bisect_nu_warp(tot + c * kChebVals, n[c], sh_g, lo0, hi0, a.bisect_steps, nuF[c]);
        if ((threadIdx.x & 31) == 0) nu_out[c] = nuc;
    }
    __syncthreads();
    if (do_nu) {
        nu[0] = nu_out[0];
        nu[1] = nu_out[1];
        if (ok[0] && ok[1]) nu[0] = fmaxf(nu[0], nu[1]);
    }
    if (threadIdx.x == 0) {
        RobustParams& rp = a.st->rob;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            rp.mu[c] = mu[c];
            rp.sigma[c] = sig[c];
            rp.nu[c] = nu[c];
            rp.ok[c] = ok[c] ? 1 : 0;
        }
    }
    cluster_wait();
}

// ---------------------------------------------------------------- sweep + solve
// MODE: kSweepTma, the block's tile of A with a one-pixel halo staged in shared
// memory by one TMA copy (every level whose size holds the tile box);
// kSweepPlain, A's taps read straight from global memory (smaller levels);
// kSweepFull, B warped at level 0 and reduced to this level (reading R22);
// kSweepGrad, the reference's gradients read from the plane G (the covariance
// iteration).
constexpr int kSweepPlain = 0, kSweepFull = 1, kSweepGrad = 2, kSweepTma = 3;

// The TMA tile of A: starts kTmaXOff pixels left of the block (a 16-byte aligned x)
// and one row above it, kTmaW pixels wide, 8 R + 2 rows high.
template <int PREC>
struct TmaTile {
    static constexpr int kXOff = 16 / Pix<PREC>::kBytes;
    static constexpr int kW = kTileW + 2 * kXOff;
};

template <int PREC, int R, int MODE>
__global__ void __launch_bounds__(kSweepNT, 2) sweep_kernel(SweepArgs a, const __grid_constant__ CUtensorMap tmA) {
    constexpr bool FULL = MODE == kSweepFull;
    constexpr bool TMA = MODE == kSweepTma;
    constexpr int kTileH = 8 * R;
    constexpr int kTW = TmaTile<PREC>::kW, kTH = kTileH + 2;
    constexpr int kTileBytes = TMA ? kTW * kTH * Pix<PREC>::kBytes : 16;
    __shared__ float red[kSweepNT / 32][kSlots];
    __shared__ WarpPose sh_wp;
    __shared__ RobustParams sh_rob;
    __shared__ __align__(128) unsigned char tile[kTileBytes];
    __shared__ __align__(8) unsigned long long tile_bar;
    if (iteration_skipped(a.level_iters, a.level, a.iter)) {
        pdl_wait();
        return;
    }
    // the keyframe-side loads need no wait: A's planes do not change during an alignment
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int u = blockIdx.x * kTileW + lane;
    // the thread's rows go through each stage together, so the loads of a stage
    // for all rows are in flight at once
    const int v0 = blockIdx.y * kTileH + warp * R;
    PxA sa[R];
    if constexpr (TMA) {
        if (threadIdx.x == 0) {
            mbar_init(&tile_bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(&tile_bar, (uint32_t)kTileBytes);
            tma_load_2d(tile, &tmA, (int)blockIdx.x * kTileW - TmaTile<PREC>::kXOff, (int)blockIdx.y * kTileH - 1,
                        &tile_bar);
        }
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = v0 + r;
            sa[r].ok = false;
            if (u < a.A.w && v < a.A.h) {
                if constexpr (MODE == kSweepGrad) stage_a_grad<PREC>(a.A, a.G, u, v, sa[r]);
                else stage_a<PREC>(a.A, u, v, sa[r]);
            }
        }
    }
    pdl_wait();   // the robust parameters (and pose) of this iteration are complete and visible
    if (threadIdx.x < 16) {
        reinterpret_cast<float*>(&sh_wp)[threadIdx.x] = __ldcg(reinterpret_cast<const float*>(&a.st->wp) + threadIdx.x);
    } else if (threadIdx.x < 16 + (int)(sizeof(RobustParams) / 4)) {
        const int q = threadIdx.x - 16;
        reinterpret_cast<int*>(&sh_rob)[q] = __ldcg(reinterpret_cast<const int*>(&a.st->rob) + q);
    }
    __syncthreads();
    const WarpPose wp = sh_wp;
    const RobustParams rob = sh_rob;

    float acc[kSlots];
#pragma unroll
    for (int i = 0; i < kSlots; ++i) acc[i] = 0.f;

    const bool wantI = rob.ok[0] != 0, wantW = rob.ok[1] != 0;
    PxW sw[R];
    PxB sb[R];
    if constexpr (TMA) {
        // the tile landed long ago in practice; the wait is bounded all the same
        const long long t0 = clock64();
        bool landed = true;
        while (!mbar_try_wait(&tile_bar, 0)) {
            if (clock64() - t0 > kWaitBudgetCycles) {
                landed = false;
                break;
            }
        }
        if (!landed) {
            if (threadIdx.x == 0) atomicAdd(&a.st->timeouts, 1);
            // the copy may still be in flight: give it a second bounded wait before the tile is read
            const long long t1 = clock64();
            while (!mbar_try_wait(&tile_bar, 0) && clock64() - t1 < kWaitBudgetCycles) {
            }
        }
        // A's taps come from the tile; only the warp's inputs stay live across the B gathers
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int v = v0 + r;
            sa[r].ok = false;
            if (u < a.A.w && v < a.A.h)
                stage_a_shared<PREC>(a.A, tile, kTW, (warp * R + r + 1) * kTW + lane + TmaTile<PREC>::kXOff, u, v,
                                     sa[r]);
            stage_w(a.A, a.B, wp, u, v, sa[r], sw[r]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) stage_b<PREC>(a.B, sw[r], sb[r]);
    } else if constexpr (!FULL) {
#pragma unroll
        for (int r = 0; r < R; ++r) stage_w(a.A, a.B, wp, u, v0 + r, sa[r], sw[r]);
#pragma unroll
        for (int r = 0; r < R; ++r) stage_b<PREC>(a.B, sw[r], sb[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = v0 + r;
        if (u >= a.A.w || v >= a.A.h) continue;
        PixelTerms o;
        if constexpr (FULL) {
            o.mI = o.mW = false;
            o.rI = o.rW = 0.f;
            if (sa[r].ok) {
                const Warped wd = warped_at_level<PREC>(a.full_level, a.A0, a.B0, wp, u, v);
                finish_given<true>(a.A, sa[r], wd.I, wd.vI, wd.W, wd.vW, o);
            }
        } else if constexpr (TMA) {
            PxA sr;   // re-read from the tile rather than kept in registers across the gathers
            stage_a_shared<PREC>(a.A, tile, kTW, (warp * R + r + 1) * kTW + lane + TmaTile<PREC>::kXOff, u, v, sr);
            finish<true>(a.A, wp, sr, sw[r], sb[r], o);
        } else {
            finish<true>(a.A, wp, sa[r], sw[r], sb[r], o);
        }
        if (a.r_I) {
            const int oi = v * a.A.w + u;
            a.r_I[oi] = o.mI ? o.rI : 0.f;
            a.r_W[oi] = o.mW ? o.rW : 0.f;
            a.m_I[oi] = o.mI ? 1 : 0;
            a.m_W[oi] = o.mW ? 1 : 0;
        }
        if (o.mI) {
            acc[kSlotNI] += 1.f;
            if (wantI) accumulate(acc, o.JI, robust_weight(o.rI, rob.mu[0], rob.sigma[0], rob.nu[0]), o.rI);
        }
        if (o.mW) {
            acc[kSlotNW] += 1.f;
            if (wantW) accumulate(acc, o.JW, o.lam * robust_weight(o.rW, rob.mu[1], rob.sigma[1], rob.nu[1]), o.rW);
        }
    }

    // the next kernel may be scheduled once every block has finished its pixels;
    // it waits for this grid to complete before it reads anything written here
    pdl_trigger();

    // block reduction: warp reduce-scatter, then warp 0 sums the 8 warps into
    // compensated pairs; the next robust-scale kernel reduces the blocks
    const float mine = warp_reduce_scatter32(acc);
    red[warp][lane] = mine;
    __syncthreads();
    if (warp == 0) {
        F2 s{0.f, 0.f};
#pragma unroll
        for (int w = 0; w < kSweepNT / 32; ++w) s.add(red[w][lane]);
        const int bid = blockIdx.y * gridDim.x + blockIdx.x;
        reinterpret_cast<float2*>(a.partials)[(size_t)bid * kSlots + lane] = make_float2(s.hi, s.lo);
        if (bid == 0 && lane == 0) a.st->pending = gridDim.x * gridDim.y;
    }
}

// ---------------------------------------------------------------- wait-timeout probe
// One exchange round of the cluster reduction in which every CTA withholds its
// partials: no CTA's barrier can complete, so every wait runs out of `budget`,
// counts a timeout and returns.  Shows on the device that a wait with nothing to
// wait for ends with a status instead of hanging.  No CTA writes to another's
// shared memory, so none can exit with a store to it still in flight.
template <int CL>
__global__ void __launch_bounds__(32) wait_timeout_probe_kernel(long long budget, int* timeouts) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    __shared__ float red_w[kRobustNT / 32][kRobustMaxNV];
    __shared__ float2 recv[2][CL][kRobustMaxNV];
    __shared__ float tot[kRobustMaxNV];
    __shared__ __align__(8) unsigned long long mbar[2];
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cl.sync();
    ClusterSum<CL> R{red_w, recv, tot, mbar, timeouts, (uint32_t)rank, 0};
    R.budget = budget;
    if (threadIdx.x == 0) tot[0] = R.template exchange<1>(0, F2{1.f, 0.f}, false).value();
    __syncwarp();
    cl.sync();
}

// ---------------------------------------------------------------- host side
static LevelDev level_dev(const rgbid_level& L) {
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

static int sample_stride(int w, int h, int cap) {
    int s = 1;
    while ((long long)((w + s - 1) / s) * ((h + s - 1) / s) > cap) ++s;
    return s;
}

static int sweep_rows(int w, int h) { return (long long)w * h >= kSweepWidePixels ? 4 : 1; }
// Blocks of a sweep over a w x h level; `one_row`: the sweeps of the full-resolution
// warp and of the covariance iteration, which take one row per thread on every level.
static int sweep_blocks(int w, int h, bool one_row) {
    const int th = 8 * (one_row ? 1 : sweep_rows(w, h));
    return ((w + kTileW - 1) / kTileW) * ((h + th - 1) / th);
}

// The block partials of the largest sweep over the levels of `ref`, and at least one
// per helper CTA the split kernel may launch.
static size_t workspace_bytes_for(const rgbid_pyramid& ref, bool one_row) {
    int nb = kSplitMaxHelpers;
    for (int l = 0; l < ref.levels && l < RGBID_MAX_LEVELS; ++l)
        nb = std::max(nb, sweep_blocks(ref.lv[l].width, ref.lv[l].height, one_row));
    return align_up(sizeof(AlignState), 256) + align_up((size_t)nb * kSlots * sizeof(float2), 256);
}

static int check_pyramids(const rgbid_pyramid* ref, const rgbid_pyramid* cur, const rgbid_align_params* p) {
    if (!ref || !cur || !p) return RGBID_ERR_INVALID_ARG;
    if (ref->levels < 1 || ref->levels > RGBID_MAX_LEVELS || cur->levels < ref->levels) return RGBID_ERR_INVALID_ARG;
    if (p->levels < 1 || p->levels > ref->levels) return RGBID_ERR_INVALID_ARG;
    if (ref->precision != cur->precision) return RGBID_ERR_INVALID_ARG;
    if (ref->precision != RGBID_PLANES_F32 && ref->precision != RGBID_PLANES_BF16_F16) return RGBID_ERR_UNSUPPORTED;
    const uintptr_t px_bytes = ref->precision == RGBID_PLANES_F32 ? 8u : 4u;   // one interleaved (I, W) pixel
    if (p->level_iters && misaligned(p->level_iters, 4)) return RGBID_ERR_INVALID_ARG;
    if (p->sample_cap < 1 || p->sample_cap > RGBID_MAX_SAMPLES) return RGBID_ERR_INVALID_ARG;
    if (p->warp_mode != RGBID_WARP_PER_LEVEL && p->warp_mode != RGBID_WARP_FULL_RESOLUTION) return RGBID_ERR_INVALID_ARG;
    if (p->no_level_kernel != 0 && p->no_level_kernel != 1) return RGBID_ERR_INVALID_ARG;
    if (p->scale_iters < 0 || p->bisect_steps < 0 || p->bisect_steps > 60) return RGBID_ERR_INVALID_ARG;
    if (!(p->nu_lo > 0.0) || !(p->nu_hi > p->nu_lo) || !(p->nu0 > 0.0)) return RGBID_ERR_INVALID_ARG;
    // the Chebyshev form of the robustness equation needs alpha_min = (lo + hi)/(hi - lo) >= 1.4
    if (p->nu_lo + p->nu_hi < 1.4 * (p->nu_hi - p->nu_lo)) return RGBID_ERR_UNSUPPORTED;
    for (int l = 0; l < p->levels; ++l) {
        const rgbid_level& a = ref->lv[l];
        const rgbid_level& b = cur->lv[l];
        if (p->iters[l] < 0) return RGBID_ERR_INVALID_ARG;
        if (!a.IW || !b.IW) return RGBID_ERR_INVALID_ARG;
        if (misaligned(a.IW, px_bytes) || misaligned(b.IW, px_bytes)) return RGBID_ERR_INVALID_ARG;
        if (a.width != b.width || a.height != b.height || a.width < 4 || a.height < 4) return RGBID_ERR_INVALID_ARG;
        if (a.pitch < a.width || b.pitch < b.width) return RGBID_ERR_INVALID_ARG;
        if (a.K.fx != b.K.fx || a.K.fy != b.K.fy || a.K.cx != b.K.cx || a.K.cy != b.K.cy) return RGBID_ERR_INVALID_ARG;
        if (!intrinsics_ok(a.K.fx, a.K.fy, a.K.cx, a.K.cy)) return RGBID_ERR_INVALID_ARG;
    }
    return RGBID_OK;
}

template <int PREC, int CL, bool FULL>
static cudaError_t launch_robust_cl(const RobustArgs& ra, cudaStream_t stream) {
    if (CL > 8) {
        cudaError_t e =
            cudaFuncSetAttribute(robust_kernel<PREC, CL, FULL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(kRobustNT, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, robust_kernel<PREC, CL, FULL>, ra);
}

// 16-CTA clusters (non-portable) where the device can schedule them, else 8.
// The answer is a fixed property of the device, cached per device ordinal.
template <int PREC>
static cudaError_t launch_robust(const RobustArgs& ra, cudaStream_t stream) {
    static std::atomic<int> cached[64];   // 0 = unknown, 8 or 16
    int dev = 0;
    cudaGetDevice(&dev);
    int cl = (dev >= 0 && dev < 64) ? cached[dev].load(std::memory_order_relaxed) : 0;
    if (cl == 0) {
        cl = 8;
        if (cudaFuncSetAttribute(robust_kernel<PREC, 16, false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(16, 1, 1);
            cfg.blockDim = dim3(kRobustNT, 1, 1);
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 16;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, robust_kernel<PREC, 16, false>, &cfg) == cudaSuccess &&
                nclusters > 0)
                cl = 16;
        }
        (void)cudaGetLastError();
        if (dev >= 0 && dev < 64) cached[dev].store(cl, std::memory_order_relaxed);
    }
    if (ra.full_level > 0)
        return cl == 16 ? launch_robust_cl<PREC, 16, true>(ra, stream) : launch_robust_cl<PREC, 8, true>(ra, stream);
    return cl == 16 ? launch_robust_cl<PREC, 16, false>(ra, stream) : launch_robust_cl<PREC, 8, false>(ra, stream);
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link to the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled_fn() {
    static std::atomic<EncodeTiledFn> fn{nullptr};
    EncodeTiledFn f = fn.load(std::memory_order_acquire);
    if (!f) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && p) {
            f = reinterpret_cast<EncodeTiledFn>(p);
            fn.store(f, std::memory_order_release);
        } else {
            (void)cudaGetLastError();
        }
    }
    return f;
}

// The tensor map of a level of A for the sweep's tile (rows of pitch * pixel
// bytes, a multiple of 16; the box of TmaTile<PREC> x (8 R + 2)).  Returns false
// when the level is smaller than the box (the sweep then reads A directly).
template <int PREC>
static bool encode_level_map(CUtensorMap* m, const LevelDev& A, int R, bool* failed) {
    *failed = false;
    const uint32_t bw = (uint32_t)TmaTile<PREC>::kW, bh = (uint32_t)(8 * R + 2);
    if ((uint32_t)A.w < bw || (uint32_t)A.h < bh) return false;
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) {
        *failed = true;
        return false;
    }
    const cuuint64_t gdim[2] = {(cuuint64_t)A.w, (cuuint64_t)A.h};
    const cuuint64_t gstride[1] = {(cuuint64_t)A.pitch * Pix<PREC>::kBytes};
    const cuuint32_t box[2] = {bw, bh};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, Pix<PREC>::kBytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32,
                          2, const_cast<void*>(A.IW), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    *failed = r != CUDA_SUCCESS;
    return r == CUDA_SUCCESS;
}

template <int PREC>
static cudaError_t launch_sweep(const SweepArgs& sa, cudaStream_t stream) {
    const int R = (sa.full_level > 0 || sa.G) ? 1 : sweep_rows(sa.A.w, sa.A.h);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((sa.A.w + kTileW - 1) / kTileW, (sa.A.h + 8 * R - 1) / (8 * R), 1);
    cfg.blockDim = dim3(kSweepNT, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CUtensorMap tm;
    memset(&tm, 0, sizeof(tm));
    if (sa.G) return cudaLaunchKernelEx(&cfg, sweep_kernel<PREC, 1, kSweepGrad>, sa, tm);
    if (sa.full_level > 0) return cudaLaunchKernelEx(&cfg, sweep_kernel<PREC, 1, kSweepFull>, sa, tm);
    bool failed = false;
    const bool tma = encode_level_map<PREC>(&tm, sa.A, R, &failed);
    if (failed) return cudaErrorInvalidValue;
    if (tma)
        return R == 4 ? cudaLaunchKernelEx(&cfg, sweep_kernel<PREC, 4, kSweepTma>, sa, tm)
                      : cudaLaunchKernelEx(&cfg, sweep_kernel<PREC, 1, kSweepTma>, sa, tm);
    return R == 4 ? cudaLaunchKernelEx(&cfg, sweep_kernel<PREC, 4, kSweepPlain>, sa, tm)
                  : cudaLaunchKernelEx(&cfg, sweep_kernel<PREC, 1, kSweepPlain>, sa, tm);
}

static cudaError_t launch_robust_any(int prec, const RobustArgs& ra, cudaStream_t s) {
    // every launch may read the pending partials and writes the state (and the record)
    if (!ra.st || !ra.partials || !ra.res) return cudaErrorInvalidValue;
    return prec == RGBID_PLANES_F32 ? launch_robust<RGBID_PLANES_F32>(ra, s) : launch_robust<RGBID_PLANES_BF16_F16>(ra, s);
}
static cudaError_t launch_sweep_any(int prec, const SweepArgs& sa, cudaStream_t s) {
    return prec == RGBID_PLANES_F32 ? launch_sweep<RGBID_PLANES_F32>(sa, s) : launch_sweep<RGBID_PLANES_BF16_F16>(sa, s);
}

static RobustArgs robust_args(const rgbid_pyramid* ref, const rgbid_pyramid* cur, int l, const rgbid_align_params* p,
                              AlignState* st) {
    RobustArgs ra;
    ra.A = level_dev(ref->lv[l]);
    ra.B = level_dev(cur->lv[l]);
    ra.A0 = level_dev(ref->lv[0]);
    ra.B0 = level_dev(cur->lv[0]);
    ra.full_level = p->warp_mode == RGBID_WARP_FULL_RESOLUTION ? l : 0;
    ra.st = st;
    ra.s = sample_stride(ra.A.w, ra.A.h, p->sample_cap);
    ra.nsx = (ra.A.w + ra.s - 1) / ra.s;
    ra.nsamp = ra.nsx * ((ra.A.h + ra.s - 1) / ra.s);
    ra.scale_iters = p->scale_iters;
    ra.bisect_steps = p->bisect_steps;
    ra.estimate_nu = p->estimate_nu;
    ra.nu0 = (float)p->nu0;
    ra.nu_lo = p->nu_lo;
    ra.nu_hi = p->nu_hi;
    nu_device_series(p->nu_lo, p->nu_hi, ra.nu_g);
    ra.level_iters = nullptr;
    ra.level = l;
    ra.iter = 0;
    ra.partials = nullptr;
    ra.res = nullptr;
    ra.update = 1;
    ra.min_valid = p->min_valid;
    ra.finalize_only = 0;
    ra.state_after_wait = 0;
    return ra;
}

// A small level whose systematic sample is every pixel runs in the persistent level
// kernel.  Above two pixels per thread of its cluster (80x60 takes it, 160x120 does
// not) the split kernel is faster: its helpers take the pixel pass with the Jacobians
// off the cluster's chain (measured on the 640x480 sequence: 160x120 at 24.5 us per
// iteration in the split kernel against 28.4 us in the level kernel, 80x60 the other
// way round), so the level kernel keeps such a level only where the split kernel
// cannot take it.
constexpr long long kLevelKernelPreferredPixels = (long long)kLevelCL * kRobustNT * 2;

static bool use_level_kernel(const rgbid_pyramid* ref, const rgbid_align_params* p, int l) {
    if (p->no_level_kernel || p->warp_mode != RGBID_WARP_PER_LEVEL) return false;
    const rgbid_level& L = ref->lv[l];
    if ((long long)L.width * L.height > kLevelKernelPreferredPixels &&
        split_kernel_takes(ref->precision, L.width, L.height))
        return false;
    return level_kernel_takes(ref->precision, L.width, L.height, p->sample_cap);
}

// Any other level runs in the split kernel when its tiles fit the helper CTAs (its
// sample may be every pixel too).
static bool use_split_kernel(const rgbid_pyramid* ref, const rgbid_align_params* p, int l) {
    if (p->no_level_kernel || p->warp_mode != RGBID_WARP_PER_LEVEL) return false;
    const rgbid_level& L = ref->lv[l];
    return split_kernel_takes(ref->precision, L.width, L.height);
}

// The launch-wide arguments of a split-kernel launch; its levels are added by add_split_level.
static SplitArgs split_args(const RobustArgs& ra, const rgbid_align_params* p, float* partials) {
    SplitArgs sp;
    memset(&sp, 0, sizeof(sp));
    sp.st = ra.st;
    sp.partials = reinterpret_cast<float2*>(partials);
    sp.level_iters = p->level_iters;
    sp.scale_iters = p->scale_iters;
    sp.bisect_steps = p->bisect_steps;
    sp.estimate_nu = p->estimate_nu;
    sp.min_valid = p->min_valid;
    sp.nu0 = (float)p->nu0;
    sp.nu_lo = p->nu_lo;
    sp.nu_hi = p->nu_hi;
    memcpy(sp.nu_g, ra.nu_g, sizeof(sp.nu_g));
    sp.n_helpers = 0;         // set by the caller for the device
    sp.n_levels = 0;
    return sp;
}

// One more level of a split-kernel launch (levels are added coarse to fine).
static void add_split_level(SplitArgs& sp, const RobustArgs& ra, const rgbid_align_params* p) {
    SplitLevel& L = sp.lv[sp.n_levels++];
    L.A = ra.A;
    L.B = ra.B;
    L.level = ra.level;
    L.iters = p->iters[ra.level];
    L.s = ra.s;
    L.nsx = ra.nsx;
    L.nsamp = ra.nsamp;
    L.tiles_x = (ra.A.w + kSplitTileW - 1) / kSplitTileW;
    L.tiles_y = (ra.A.h + kSplitTileH - 1) / kSplitTileH;
}

static LevelArgs level_args(const rgbid_pyramid* ref, const rgbid_pyramid* cur, int l, const rgbid_align_params* p,
                            AlignState* st, float* partials) {
    LevelArgs la;
    memset(&la, 0, sizeof(la));
    la.A = level_dev(ref->lv[l]);
    la.B = level_dev(cur->lv[l]);
    la.st = st;
    la.partials = reinterpret_cast<float2*>(partials);
    la.iters = p->iters[l];
    la.level_iters = p->level_iters;
    la.level = l;
    la.scale_iters = p->scale_iters;
    la.bisect_steps = p->bisect_steps;
    la.estimate_nu = p->estimate_nu;
    la.min_valid = p->min_valid;
    la.nu0 = (float)p->nu0;
    la.nu_lo = p->nu_lo;
    la.nu_hi = p->nu_hi;
    nu_device_series(p->nu_lo, p->nu_hi, la.nu_g);
    return la;
}

}  // namespace rgbid

using namespace rgbid;

namespace rgbid {
unsigned int oob_count_level();
unsigned int oob_count_batch_f32();
unsigned int oob_count_batch_bf16();
unsigned int oob_count_covariance();
unsigned int oob_count_fuse();
unsigned int oob_count_pyramid();
}  // namespace rgbid

extern "C" int rgbid_debug_bounds_violations(unsigned long long* count) {
    if (!count) return RGBID_ERR_INVALID_ARG;
#ifdef RGBID_BOUNDS_CHECK
    if (cudaDeviceSynchronize() != cudaSuccess) {
        (void)cudaGetLastError();
        return RGBID_ERR_CUDA;
    }
    const unsigned int c[7] = {oob_count_this_unit(), rgbid::oob_count_level(), rgbid::oob_count_batch_f32(),
                               rgbid::oob_count_batch_bf16(), rgbid::oob_count_covariance(), rgbid::oob_count_fuse(),
                               rgbid::oob_count_pyramid()};
    unsigned long long n = 0;
    for (unsigned int v : c) {
        if (v == ~0u) return RGBID_ERR_CUDA;
        n += v;
    }
    *count = n;
    return RGBID_OK;
#else
    *count = 0;
    return RGBID_ERR_UNSUPPORTED;
#endif
}

extern "C" size_t rgbid_align_workspace_bytes(const rgbid_pyramid* ref, const rgbid_align_params* params) {
    if (!ref || ref->levels < 1 || ref->levels > RGBID_MAX_LEVELS) return 0;
    return workspace_bytes_for(*ref, params && params->warp_mode == RGBID_WARP_FULL_RESOLUTION);
}

extern "C" int rgbid_align_launches(const rgbid_pyramid* ref, const rgbid_align_params* params) {
    if (check_pyramids(ref, ref, params) != RGBID_OK) return -1;
    int n = 2;   // the initialisation and the closing launch
    bool in_split = false;   // consecutive split-kernel levels share one launch
    for (int l = params->levels - 1; l >= 0; --l) {
        if (params->iters[l] <= 0) continue;
        const bool lk = use_level_kernel(ref, params, l);
        const bool sk = !lk && use_split_kernel(ref, params, l);
        if (sk) {
            if (!in_split) ++n;
            in_split = true;
            continue;
        }
        in_split = false;
        n += lk ? 1 : 2 * params->iters[l];
    }
    return n;
}

extern "C" int rgbid_align(const rgbid_pyramid* ref, const rgbid_pyramid* cur, const double* T_init, int T_init_on_device,
                           const rgbid_align_params* params, void* workspace, size_t workspace_bytes,
                           rgbid_align_result* d_result, void* stream_) {
    int st_chk = check_pyramids(ref, cur, params);
    if (st_chk != RGBID_OK) return st_chk;
    if (!d_result || misaligned(d_result, 8)) return RGBID_ERR_INVALID_ARG;
    if (T_init && T_init_on_device && misaligned(T_init, 8)) return RGBID_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 255u) || workspace_bytes < rgbid_align_workspace_bytes(ref, params))
        return RGBID_ERR_WORKSPACE;
    cudaStream_t stream = (cudaStream_t)stream_;
    AlignState* st = (AlignState*)workspace;
    float* partials = (float*)((char*)workspace + align_up(sizeof(AlignState), 256));

    InitArgs ia;
    memset(&ia, 0, sizeof(ia));
    ia.st = st;
    ia.res = d_result;
    ia.T_dev = (T_init && T_init_on_device) ? T_init : nullptr;
    for (int i = 0; i < 16; ++i) ia.T_val[i] = (i % 5 == 0) ? 1.0 : 0.0;
    if (T_init && !T_init_on_device)
        for (int i = 0; i < 16; ++i) ia.T_val[i] = T_init[i];
    init_kernel<<<1, 32, 0, stream>>>(ia);
    if (cudaGetLastError() != cudaSuccess) return RGBID_ERR_CUDA;

    rgbid_timing* tm = params->timing;
    RobustArgs ra{};
    bool after_level_kernel = false;   // the next robust-scale launch follows a level kernel
    // consecutive levels that run in the split kernel go in one launch (coarse to fine)
    SplitArgs group;
    memset(&group, 0, sizeof(group));
    long long group_units = 0;
    auto flush_split = [&]() -> int {
        if (group.n_levels == 0) return RGBID_OK;
        group.n_helpers = split_kernel_helpers(ref->precision);
        group.max_tiles = 1;
        for (int q = 0; q < group.n_levels; ++q)
            group.max_tiles =
                std::max(group.max_tiles, split_tiles_per_helper(group.lv[q].A.w, group.lv[q].A.h, group.n_helpers));
        const bool tl = tm && tm->kernel == RGBID_KERNEL_SPLIT && tm->count < tm->capacity;
        if (tl && cudaEventRecord((cudaEvent_t)tm->ev_start[tm->count], stream) != cudaSuccess) return RGBID_ERR_CUDA;
        if (launch_split(ref->precision, group, stream) != cudaSuccess) return RGBID_ERR_CUDA;
        if (tl) {
            if (cudaEventRecord((cudaEvent_t)tm->ev_end[tm->count], stream) != cudaSuccess) return RGBID_ERR_CUDA;
            tm->count += 1;
            tm->units += group_units;
        }
        group.n_levels = 0;
        group_units = 0;
        after_level_kernel = true;
        return RGBID_OK;
    };
    for (int l = params->levels - 1; l >= 0; --l) {
        ra = robust_args(ref, cur, l, params, st);
        // set before any level kernel: the closing launch takes `ra` of the finest level
        ra.partials = reinterpret_cast<const float2*>(partials);
        ra.res = d_result;
        ra.level_iters = params->level_iters;
        if (params->iters[l] > 0 && use_split_kernel(ref, params, l) && !use_level_kernel(ref, params, l)) {
            if (group.n_levels == 0) group = split_args(ra, params, partials);
            add_split_level(group, ra, params);
            group_units += (long long)ra.A.w * ra.A.h * params->iters[l];
            continue;
        }
        if (params->iters[l] > 0) {
            const int fe = flush_split();
            if (fe != RGBID_OK) return fe;
        }
        if (params->iters[l] > 0 && use_level_kernel(ref, params, l)) {
            const LevelArgs la = level_args(ref, cur, l, params, st, partials);
            const bool tl = tm && tm->kernel == RGBID_KERNEL_LEVEL && tm->count < tm->capacity;
            if (tl && cudaEventRecord((cudaEvent_t)tm->ev_start[tm->count], stream) != cudaSuccess) return RGBID_ERR_CUDA;
            if (launch_level(ref->precision, la, stream) != cudaSuccess) return RGBID_ERR_CUDA;
            if (tl) {
                if (cudaEventRecord((cudaEvent_t)tm->ev_end[tm->count], stream) != cudaSuccess) return RGBID_ERR_CUDA;
                tm->count += 1;
                tm->units += (long long)la.A.w * la.A.h * params->iters[l];
            }
            after_level_kernel = true;
            continue;
        }
        SweepArgs sa;
        memset(&sa, 0, sizeof(sa));
        sa.A = ra.A;
        sa.B = ra.B;
        sa.A0 = ra.A0;
        sa.B0 = ra.B0;
        sa.full_level = ra.full_level;
        sa.st = st;
        sa.partials = partials;
        sa.level_iters = params->level_iters;
        sa.level = l;
        for (int it = 0; it < params->iters[l]; ++it) {
            ra.iter = it;
            sa.iter = it;
            ra.state_after_wait = after_level_kernel ? 1 : 0;
            after_level_kernel = false;
            const bool tr = tm && tm->kernel == RGBID_KERNEL_ROBUST && tm->count < tm->capacity;
            if (tr && cudaEventRecord((cudaEvent_t)tm->ev_start[tm->count], stream) != cudaSuccess) return RGBID_ERR_CUDA;
            if (launch_robust_any(ref->precision, ra, stream) != cudaSuccess) return RGBID_ERR_CUDA;
            if (tr) {
                if (cudaEventRecord((cudaEvent_t)tm->ev_end[tm->count], stream) != cudaSuccess) return RGBID_ERR_CUDA;
                tm->count += 1;
                tm->units += ra.nsamp;
            }
            const bool ts = tm && tm->kernel == RGBID_KERNEL_SWEEP && tm->count < tm->capacity;
            if (ts && cudaEventRecord((cudaEvent_t)tm->ev_start[tm->count], stream) != cudaSuccess) return RGBID_ERR_CUDA;
            if (launch_sweep_any(ref->precision, sa, stream) != cudaSuccess) return RGBID_ERR_CUDA;
            if (ts) {
                if (cudaEventRecord((cudaEvent_t)tm->ev_end[tm->count], stream) != cudaSuccess) return RGBID_ERR_CUDA;
                tm->count += 1;
                tm->units += (long long)sa.A.w * sa.A.h;
            }
        }
    }
    {
        const int fe = flush_split();
        if (fe != RGBID_OK) return fe;
    }
    // the last sweep's (or level kernel's) pending step: reduction, solve and update
    ra.finalize_only = 1;
    ra.state_after_wait = after_level_kernel ? 1 : 0;
    const bool tr = tm && tm->kernel == RGBID_KERNEL_ROBUST && tm->count < tm->capacity;
    if (tr && cudaEventRecord((cudaEvent_t)tm->ev_start[tm->count], stream) != cudaSuccess) return RGBID_ERR_CUDA;
    if (launch_robust_any(ref->precision, ra, stream) != cudaSuccess) return RGBID_ERR_CUDA;
    if (tr) {
        if (cudaEventRecord((cudaEvent_t)tm->ev_end[tm->count], stream) != cudaSuccess) return RGBID_ERR_CUDA;
        tm->count += 1;
    }
    return RGBID_OK;
}

namespace rgbid {
// One step at a fixed pose, no update: initialisation, the robust-scale kernel
// (unless the robust parameters are given), one sweep and the closing reduction
// into the result record.  The pose is host or device memory; `G` (optional,
// level `level` only) supplies the reference's gradients (the covariance
// iteration).  Arguments are checked by the callers.
int enqueue_eval_step(const rgbid_pyramid* ref, const rgbid_pyramid* cur, int level, const double* T, int T_on_device,
                      const double* robust, const rgbid_align_params& p, void* workspace, float* r_I, float* r_W,
                      uint8_t* mask_I, uint8_t* mask_W, const float2* G, rgbid_align_result* d_result,
                      cudaStream_t stream) {
    AlignState* st = (AlignState*)workspace;
    float* partials = (float*)((char*)workspace + align_up(sizeof(AlignState), 256));
    InitArgs ia;
    memset(&ia, 0, sizeof(ia));
    ia.st = st;
    ia.res = d_result;
    if (T_on_device) ia.T_dev = T;
    else
        for (int i = 0; i < 16; ++i) ia.T_val[i] = T[i];
    if (robust) {
        ia.use_fixed = 1;
        for (int i = 0; i < 6; ++i) ia.fixed[i] = (float)robust[i];
    }
    init_kernel<<<1, 32, 0, stream>>>(ia);
    if (cudaGetLastError() != cudaSuccess) return RGBID_ERR_CUDA;
    RobustArgs ra = robust_args(ref, cur, level, &p, st);
    ra.partials = reinterpret_cast<const float2*>(partials);
    ra.res = d_result;
    ra.update = 0;
    if (!robust && launch_robust_any(ref->precision, ra, stream) != cudaSuccess) return RGBID_ERR_CUDA;
    SweepArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.A = ra.A;
    sa.B = ra.B;
    sa.A0 = ra.A0;
    sa.B0 = ra.B0;
    sa.full_level = ra.full_level;
    sa.G = G;
    sa.st = st;
    sa.partials = partials;
    sa.r_I = r_I;
    sa.r_W = r_W;
    sa.m_I = mask_I;
    sa.m_W = mask_W;
    if (launch_sweep_any(ref->precision, sa, stream) != cudaSuccess) return RGBID_ERR_CUDA;
    // the step's normal equations and results (no update)
    ra.finalize_only = 1;
    if (launch_robust_any(ref->precision, ra, stream) != cudaSuccess) return RGBID_ERR_CUDA;
    return RGBID_OK;
}

size_t align_workspace_bytes(const rgbid_pyramid& ref) { return workspace_bytes_for(ref, true); }
int check_align_inputs(const rgbid_pyramid* ref, const rgbid_pyramid* cur, const rgbid_align_params* p) {
    return check_pyramids(ref, cur, p);
}
}  // namespace rgbid

extern "C" int rgbid_eval_step(const rgbid_pyramid* ref, const rgbid_pyramid* cur, int level, const double* T,
                               const double* robust, const rgbid_align_params* params, void* workspace,
                               size_t workspace_bytes, float* r_I, float* r_W, uint8_t* mask_I, uint8_t* mask_W,
                               rgbid_align_result* d_result, void* stream_) {
    if (!params || !T || !d_result) return RGBID_ERR_INVALID_ARG;
    rgbid_align_params p = *params;
    if (level < 0 || level >= RGBID_MAX_LEVELS) return RGBID_ERR_INVALID_ARG;
    if (p.levels < level + 1) p.levels = level + 1;
    int st_chk = check_pyramids(ref, cur, &p);
    if (st_chk != RGBID_OK) return st_chk;
    const bool any_out = r_I || r_W || mask_I || mask_W;
    if (any_out && !(r_I && r_W && mask_I && mask_W)) return RGBID_ERR_INVALID_ARG;
    if (misaligned(d_result, 8) || misaligned(r_I, 4) || misaligned(r_W, 4)) return RGBID_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 255u) || workspace_bytes < rgbid_align_workspace_bytes(ref, &p))
        return RGBID_ERR_WORKSPACE;
    return enqueue_eval_step(ref, cur, level, T, 0, robust, p, workspace, r_I, r_W, mask_I, mask_W, nullptr, d_result,
                             (cudaStream_t)stream_);
}

// ---------------------------------------------------------------- allocation-free alignment
// Scratch of rgbid_align_noalloc: a fixed device array that every GPU loading this
// library holds until the process exits.  Its host-side name is only a stand-in
// for the symbol; the device address is fetched with cudaGetSymbolAddress once
// per device and cached.  The cache is atomic: host threads making their first
// call on one device at the same time each look the address up and store the
// same value.
namespace rgbid {
constexpr size_t kNoallocScratchBytes = 1024u * 1024u;  // RGBID_NOALLOC_SCRATCH_BYTES
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];
static std::atomic<void*> g_noalloc_ptr[64];
}  // namespace rgbid

extern "C" int rgbid_align_noalloc(const rgbid_pyramid* ref, const rgbid_pyramid* cur, const double* T_init,
                                   int T_init_on_device, const rgbid_align_params* params,
                                   rgbid_align_result* d_result, void* stream) {
    if (!ref || !params) return RGBID_ERR_INVALID_ARG;
    const size_t need = rgbid_align_workspace_bytes(ref, params);
    if (need == 0) return RGBID_ERR_INVALID_ARG;
    if (need > kNoallocScratchBytes) return RGBID_ERR_WORKSPACE;     // the largest level sweep does not fit
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RGBID_ERR_CUDA;
    void* scratch = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!scratch) {
        // set-up on the first call on this device (the device is current here)
        if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess || !scratch) return RGBID_ERR_CUDA;
        g_noalloc_ptr[dev].store(scratch, std::memory_order_release);
    }
    // the alignment's init kernel resets every scratch field that must start at zero
    return rgbid_align(ref, cur, T_init, T_init_on_device, params, scratch, kNoallocScratchBytes, d_result, stream);
}

extern "C" int rgbid_probe_wait_timeout(long long budget_cycles, int* d_timeouts, void* stream) {
    if (!d_timeouts || budget_cycles < 0 || budget_cycles > 20000000000LL) return RGBID_ERR_INVALID_ARG;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(4, 1, 1);
    cfg.blockDim = dim3(32, 1, 1);
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 4;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, wait_timeout_probe_kernel<4>, budget_cycles, d_timeouts) != cudaSuccess) {
        (void)cudaGetLastError();
        return RGBID_ERR_CUDA;
    }
    return RGBID_OK;
}

extern "C" int rgbid_nu_constant_series(double nu_lo, double nu_hi, float* out, int n_out) {
    if (!out || n_out < 1 || !(nu_lo > 0.0) || !(nu_hi > nu_lo) || !(nu_hi < 1e6)) return -RGBID_ERR_INVALID_ARG;
    // the intervals the alignment accepts: (lo + hi)/(hi - lo) >= 1.4 keeps nu = 0 far enough
    // from the interval for 22 terms to reach FP32 accuracy
    if (nu_lo + nu_hi < 1.4 * (nu_hi - nu_lo)) return -RGBID_ERR_UNSUPPORTED;
    float g[kNuGTerms];
    nu_g_series(nu_lo, nu_hi, g);
    const int n = n_out < kNuGTerms ? n_out : kNuGTerms;
    for (int k = 0; k < n; ++k) out[k] = g[k];
    return n;
}
