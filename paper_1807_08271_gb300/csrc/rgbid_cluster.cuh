// Cluster-level building blocks shared by the per-iteration alignment kernels
// and the persistent batched alignment kernel (sm_103a): distributed-shared-
// memory stores completed on mbarriers, programmatic dependent launch, the
// Chebyshev form of the robustness equation and the normal-equation
// accumulation of one residual.
#pragma once

#include "rgbid_device.cuh"
#include "rgbid_nu.h"

namespace rgbid {

// ---- distributed-shared-memory exchange (push model)
// Each CTA sends its compensated partials to every CTA of the cluster with
// st.async, which completes transaction bytes on the receiver's mbarrier; a
// receiver waits only on its own barrier, so no cluster-wide barrier is needed
// per round.  Two receive buffers and two barriers alternate between rounds: a
// CTA cannot send round k+2 before it holds round k+1 from every CTA, which
// each CTA sends only after it has consumed round k.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(addr), "r"(rank));
    return out;
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// One 2D tile of a tensor map into this CTA's shared memory (the tensor memory
// accelerator), completing its bytes on `bar`.  x must be a multiple of 16 bytes
// over the element size; the box may reach outside the tensor (zeros there).
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void st_async_f2(uint32_t remote_addr, float a, float b, uint32_t remote_bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(
                     remote_addr),
                 "f"(a), "f"(b), "r"(remote_bar)
                 : "memory");
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while its predecessor is still running; it must wait
// (griddepcontrol.wait) before reading anything the predecessor writes, and it
// lets its own successor start early with griddepcontrol.launch_dependents.
// Split cluster barrier: every thread of every CTA arrives and later waits, so the
// latency between the two is hidden behind other work.  The arrive is relaxed (it
// orders no memory: mbarrier initialisation is published by its own
// fence.mbarrier_init, and the barrier at exit carries no data); the wait acquires.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

constexpr long long kWaitBudgetCycles = 4000000000LL;   // ~2 s: a wait that exceeds it reports a timeout

// Chebyshev form of the sample sums of eq. robustnessValue.  With
// nu = m + h tau (tau in [-1, 1] over [nu_lo, nu_hi]) and alpha_i = (m + x_i^2)/h > 1:
//   ln(nu + x_i^2)  = ln h + ln(beta_i/2) + 2 sum_k (-1)^(k+1) q_i^k / k T_k(tau)
//   1/(nu + x_i^2)  = (gamma_i / h) (1 + 2 sum_k (-1)^k q_i^k T_k(tau))
// with beta = alpha + sqrt(alpha^2 - 1), q = 1/beta, gamma = 1/sqrt(alpha^2 - 1)
// (the classical expansions of ln(alpha + tau) and 1/(alpha + tau)).  One cluster
// reduction of the power sums P_k = sum q^k, G_k = sum gamma q^k and sum ln(beta/2)
// then gives f(nu) at any nu without revisiting the samples; truncating at K
// terms errs by < q_max^(K+1) per sample (q_max = 0.382 for [2, 10], K = 20).
// Packed pairs of FP32 (Blackwell's f32x2 arithmetic): element-wise, round to
// nearest, so each half is exactly the scalar fmaf / + / * of its operands.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float f2_lo(unsigned long long v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float f2_hi(unsigned long long v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

constexpr int kChebK = 20;
constexpr int kChebVals = 2 * kChebK + 2;      // SL, P_1..P_K, G_0..G_K per channel
constexpr int kNuSeries = kChebK + 2;          // terms of f(nu) as one series in tau (degree K + 1)
static_assert(kNuSeries == kNuGTerms, "the constant part's series has as many terms as f's");

// f(nu) = n (g(nu) - ln h) - SL - A(tau) - (nu + 1) B(tau) / h, with
//   g(nu) - ln h = sum_k g_k T_k(tau)   (host series, g = psi((nu+1)/2) - psi(nu/2) + 1 + ln nu),
//   A(tau) = sum_i ln(alpha_i + tau) - SL = sum_{k>=1} a_k T_k,   a_k = 2 (-1)^(k+1) P_k / k,
//   B(tau) = sum_i 1/(alpha_i + tau)      = sum_{k>=0} b_k T_k,   b_0 = G_0, b_k = 2 (-1)^k G_k,
// and (nu + 1) B / h = ((m + 1)/h) B + tau B, tau T_0 = T_1, tau T_k = (T_{k+1} + T_{k-1})/2.
// So f is one Chebyshev series F_0 .. F_{K+1} in tau; coefficient j of tau B is
//   d_j = [j = 1] b_0 + [j >= 2] b_{j-1}/2 + [j + 1 <= K] b_{j+1}/2.
// Called by the threads lt < kNuSeries of a bisection group; T = the channel's sums.
__device__ __forceinline__ float nu_series_coefficient(const float* T, float n, const float* g, float m, float h,
                                                       int j) {
    auto b = [&](int k) -> float {
        if (k == 0) return T[1 + kChebK];
        if (k > kChebK) return 0.f;
        return ((k & 1) ? -2.f : 2.f) * T[1 + kChebK + k];
    };
    const float a = (j >= 1 && j <= kChebK) ? ((j & 1) ? 2.f : -2.f) * __fdividef(T[j], (float)j) : 0.f;
    float d = 0.f;
    if (j == 1) d += b(0);
    if (j >= 2) d += 0.5f * b(j - 1);
    if (j + 1 <= kChebK) d += 0.5f * b(j + 1);
    float F = fmaf(n, g[j], -a) - __fdividef(m + 1.f, h) * b(j) - d;
    if (j == 0) F -= T[0];
    return F;
}

// sum_k F_k T_k(tau) by Clenshaw's recurrence (FP32; F held in registers)
__device__ __forceinline__ float nu_series_eval(const float (&F)[kNuSeries], float tau) {
    const float t2 = 2.f * tau;
    float b1 = 0.f, b2 = 0.f;
#pragma unroll
    for (int k = kNuSeries - 1; k >= 1; --k) {
        const float bn = fmaf(t2, b1, F[k] - b2);
        b2 = b1;
        b1 = bn;
    }
    return fmaf(tau, b1, F[0] - b2);
}

// nu of one channel by bisection on eq. robustnessValue over [lo0, hi0], run by
// one warp (all 32 lanes call; every lane returns the same nu).  T holds the
// channel's cluster sums (SL, P_1..P_K, G_0..G_K), nc its residual count, g the
// host series of the constant part; F (kNuSeries floats of shared memory) is
// the warp's scratch for f's series.  Each round evaluates f at the 31 interior
// dyadic points of the current bracket (5 halvings; the first round also at
// hi and lo) and replays the bisection's decisions on the ballot of their signs,
// so the result is the midpoint of the bracket the plain bisection reaches
// after `steps` halvings at the same points.
__device__ __forceinline__ float bisect_nu_warp(const float* T, float nc, const float* g, float lo0, float hi0,
                                                int steps, float* F) {
    const int lane = threadIdx.x & 31;
    const float m = 0.5f * (lo0 + hi0), h = 0.5f * (hi0 - lo0);
    if (lane < kNuSeries) F[lane] = nu_series_coefficient(T, nc, g, m, h, lane);
    __syncwarp();
    float Fr[kNuSeries];       // every lane's own copy: no shared-memory load on the recurrence
#pragma unroll
    for (int k = 0; k < kNuSeries; ++k) Fr[k] = F[k];
    const float invh = 1.f / h;
    // the ends: f(hi) >= 0 -> hi, f(lo) <= 0 -> lo (as the plain bisection decides first)
    const float fe = nu_series_eval(Fr, ((lane == 0 ? hi0 : lo0) - m) * invh);
    const unsigned ends = __ballot_sync(0xffffffffu, lane == 0 ? fe >= 0.f : (lane == 1 && fe <= 0.f));
    if (ends & 1u) return hi0;
    if (ends & 2u) return lo0;
    float lo = lo0, hi = hi0;
    for (int left = steps; left > 0;) {
        const int st = left < 5 ? left : 5;
        const int np = 1 << st;                              // sub-intervals this round
        const float step = (hi - lo) * __int_as_float((127 - st) << 23);   // exact: times 2^-st
        const int j = lane + 1;                              // interior point j of this lane
        const bool eval = j < np;
        const float f = eval ? nu_series_eval(Fr, (fmaf((float)j, step, lo) - m) * invh) : 0.f;
        const unsigned pos = __ballot_sync(0xffffffffu, eval && f > 0.f);   // bit j-1: f at point j > 0
        int jl = 0, jh = np;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            if (q < st) {
                const int jm = (jl + jh) >> 1;
                if ((pos >> (jm - 1)) & 1u) jl = jm; else jh = jm;
            }
        }
        const float nlo = fmaf((float)jl, step, lo), nhi = fmaf((float)jh, step, lo);
        lo = nlo;
        hi = nhi;
        left -= st;
    }
    return 0.5f * (lo + hi);
}

// Sum of the NW per-warp partials of value t in a fixed pairwise tree (depth
// log2 NW instead of a chain of NW compensated adds); the same order everywhere.
template <int NW, typename Row>
__device__ __forceinline__ F2 warp_tree(const Row* rows, int t) {
    F2 a[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) a[w] = as_f2(rows[w][t]);
#pragma unroll
    for (int step = 1; step < NW; step <<= 1)
#pragma unroll
        for (int w = 0; w < NW; ++w)
            if (w % (2 * step) == 0 && w + step < NW) a[w].add(a[w + step]);
    return a[0];
}

__device__ __forceinline__ void accumulate(float (&acc)[kSlots], const float (&J)[6], float w, float r) {
    float wj[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) wj[i] = w * J[i];
    int s = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = i; j < 6; ++j) { acc[s] = fmaf(wj[i], J[j], acc[s]); ++s; }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[kSlotG + i] = fmaf(wj[i], r, acc[kSlotG + i]);
    acc[kSlotCost] = fmaf(w * r, r, acc[kSlotCost]);
}

// ---- cluster-wide sums of the per-pair alignment kernels
constexpr int kRobustNT = 256;      // threads per CTA of the robust-scale cluster
constexpr int kRobustMaxNV = 96;    // widest cluster reduction (the Chebyshev sums of both channels)

// All cluster-wide sums use the same fixed combine tree (warp butterfly, then
// a shuffle tree over the 8 warps of a CTA, then a shuffle tree over the CTAs
// of the cluster with compensated (TwoSum) pairs), so every thread of every
// CTA sees bit-identical totals and takes identical branches.

template <int CL>
struct ClusterSum {
    float (*red_w)[kRobustMaxNV];             // per-warp partials [8][NV]
    float2 (*recv)[CL][kRobustMaxNV];         // receive buffers [2][CL][NV]
    float* out;                               // [NV] cluster totals
    unsigned long long* mbar;                 // [2]
    int* timeouts;                            // device counter of expired waits
    uint32_t rank;
    int round;
    long long budget = kWaitBudgetCycles;     // clock64 cycles a wait may take before it gives up

    // One all-to-all round in three parts.  arm<NV>(): thread 0 announces the round's
    // bytes (CL sources x NV values) on this CTA's barrier.  send(t, r, s): the calling
    // thread pushes this CTA's compensated partial of value t into CTA r (st.async
    // completes the bytes on r's barrier).  receive<NV>(t): threads t < NV wait for
    // value t from every CTA and return the total, summed over the ranks in the same
    // pairwise tree in every CTA, so every CTA holds bit-identical totals.  Spreading
    // the CL x NV sends over the threads keeps the issue of the round's stores short.
    // The caller separates rounds with __syncthreads and next().
    template <int NV>
    __device__ __forceinline__ void arm() {
        if (threadIdx.x == 0) mbar_arrive_expect_tx(&mbar[round & 1], (uint32_t)(CL * NV * sizeof(float2)));
    }
    __device__ __forceinline__ void send(int t, int r, F2 s) {
        const int par = round & 1;
        st_async_f2(map_to_rank(smem_addr(&recv[par][rank][t]), (uint32_t)r), s.hi, s.lo,
                    map_to_rank(smem_addr(&mbar[par]), (uint32_t)r));
    }
    template <int NV>
    __device__ __forceinline__ F2 receive(int t) {
        const int par = round & 1;
        const uint32_t phase = (uint32_t)(round >> 1) & 1u;
        const long long t0 = clock64();
        while (!mbar_try_wait(&mbar[par], phase)) {
            if (clock64() - t0 > budget) {
                atomicAdd(timeouts, 1);
                budget = 0;       // the cluster's exchanges are broken: later waits give up at once
                break;
            }
        }
        // fixed pairwise tree over the CL source CTAs
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
    // All CL x NV sends of a round, value t's partial given by part(t).
    template <int NV, typename Part>
    __device__ __forceinline__ void send_all(Part part) {
        for (int p = (int)threadIdx.x; p < NV * CL; p += kRobustNT) {
            const int t = p / CL, r = p - t * CL;
            send(t, r, part(t));
        }
    }
    // A round by one thread per value t < NV, which sends to every CTA itself
    // (`do_send` = false withholds this CTA's partials: the wait-timeout probe).
    template <int NV>
    __device__ __forceinline__ F2 exchange(int t, F2 s, bool do_send = true) {
        if (t == 0) mbar_arrive_expect_tx(&mbar[round & 1], (uint32_t)(CL * NV * sizeof(float2)));
        if (do_send) {
#pragma unroll
            for (int r = 0; r < CL; ++r) send(t, r, s);
        }
        return receive<NV>(t);
    }
    __device__ __forceinline__ void next() { ++round; }

    // The same round towards CTA 0 alone: every CTA pushes its partial of value t
    // into CTA 0, which waits and returns the total (the same tree over the ranks);
    // the other CTAs return at once.  For sums only CTA 0 consumes.  The other CTAs
    // still complete their own barrier's phase of the round (an arrival with no
    // bytes), so every CTA's phases keep counting the rounds when more follow.
    template <int NV>
    __device__ __forceinline__ F2 gather(int t, F2 s) {
        if (t == 0) {
            if (rank == 0) mbar_arrive_expect_tx(&mbar[round & 1], (uint32_t)(CL * NV * sizeof(float2)));
            else mbar_arrive(&mbar[round & 1]);
        }
        send(t, 0, s);
        if (rank != 0) return F2{0.f, 0.f};
        return receive<NV>(t);
    }

    // The same round by loads instead of pushes: every CTA leaves its partial of value
    // t < NSEND in its own receive buffer, one hardware cluster barrier (arrive.release /
    // wait.acquire) publishes them, and each reader (every CTA, or CTA 0 alone with ROOT)
    // reads the CL partials of each value with ld.shared::cluster and sums them in the
    // same pairwise tree, so the totals equal the pushed round's bit for bit.  Faster
    // than the push for wide rounds (a 16-CTA probe: 1.32 against 1.83 us for 96 values,
    // slower for 4-6), so only the Chebyshev round uses it.  Every CTA still completes its
    // mbarrier's phase of the round (an arrival with no bytes), so the phases of the
    // pushed rounds keep counting.  A CTA overwrites its own partial of this parity only
    // two rounds later, after every reader has finished this round.
    template <int NV, int NSEND, bool ROOT>
    __device__ __forceinline__ void run_by_loads(float (&v)[NV]) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        static_assert(NV % 32 == 0 && NSEND <= NV && NSEND <= kRobustMaxNV, "chunks of 32");
#pragma unroll
        for (int c = 0; c < NV / 32; ++c) {
            float chunk[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) chunk[i] = v[c * 32 + i];
            red_w[warp][c * 32 + lane] = warp_reduce_scatter32(chunk);
        }
        __syncthreads();
        const int t = threadIdx.x, par = round & 1;
        if (t < NSEND) {
            const F2 p = warp_tree<kRobustNT / 32>(red_w, t);
            recv[par][rank][t] = make_float2(p.hi, p.lo);
        }
        if (t == 0) mbar_arrive(&mbar[par]);
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
        if ((!ROOT || rank == 0) && t < NSEND) {
            const uint32_t a = smem_addr(&recv[par][0][t]);
            F2 acc[CL];
#pragma unroll
            for (int r = 0; r < CL; ++r) {
                float2 q;
                // source r's partial sits at [par][r][t] of CTA r's own buffer
                asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];"
                             : "=f"(q.x), "=f"(q.y)
                             : "r"(map_to_rank(a + (uint32_t)(r * kRobustMaxNV * sizeof(float2)), (uint32_t)r))
                             : "memory");
                acc[r] = F2{q.x, q.y};
            }
#pragma unroll
            for (int step = 1; step < CL; step <<= 1)
#pragma unroll
                for (int r = 0; r < CL; ++r)
                    if (r % (2 * step) == 0 && r + step < CL) acc[r].add(acc[r + step]);
            out[t] = acc[0].value();
        }
        __syncthreads();
        next();
    }

    // Block reduction of per-thread partials v[0..NV) (NV <= 8: one warp sum each;
    // a multiple of 32: reduce-scatter chunks) into per-warp partials, summed over the
    // warps in a fixed pairwise tree; then values t < NSEND go through the cluster: to
    // every CTA (ROOT = false; out[] bit-identical in all CTAs) or to CTA 0 alone
    // (ROOT = true; out[] valid in CTA 0 only).
    template <int NV, int NSEND = NV, bool ROOT = false>
    __device__ __forceinline__ void run(float (&v)[NV]) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if constexpr (NV <= 8) {
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                const float x = warp_sum(v[j]);
                if (lane == 0) red_w[warp][j] = x;
            }
        } else {
            static_assert(NV % 32 == 0, "chunks of 32");
#pragma unroll
            for (int c = 0; c < NV / 32; ++c) {
                float chunk[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) chunk[i] = v[c * 32 + i];
                red_w[warp][c * 32 + lane] = warp_reduce_scatter32(chunk);
            }
        }
        __syncthreads();
        const auto part = [&](int t) { return warp_tree<kRobustNT / 32>(red_w, t); };
        const int t = threadIdx.x;
        if constexpr (ROOT) {
            if (t < NSEND) out[t] = gather<NSEND>(t, part(t)).value();
        } else if constexpr (NSEND <= 8) {
            // a few values: each is sent to every CTA by its own thread (shorter than
            // spreading the sends, which makes every sender rebuild its warp tree)
            if (t < NSEND) out[t] = exchange<NSEND>(t, part(t)).value();
        } else {
            arm<NSEND>();
            send_all<NSEND>(part);
            if (t < NSEND) out[t] = receive<NSEND>(t).value();
        }
        __syncthreads();
        next();
    }
};

}  // namespace rgbid
