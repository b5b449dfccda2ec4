// Cluster-level building blocks shared by the per-iteration alignment kernels
// and the persistent batched alignment kernel (sm_103a): distributed-shared-
// memory stores completed on mbarriers, programmatic dependent launch, the
// Chebyshev form of the robustness equation and the normal-equation
// accumulation of one residual.
#pragma once

#include "rgbid_device.cuh"

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
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

constexpr long long kWaitBudgetCycles = 4000000000LL;   // ~2 s: a wait that exceeds it reports a timeout

// c(nu) = -psi(nu/2) + ln(nu/2) + psi((nu+1)/2) - ln((nu+1)/2) + 1 (eq. robustnessValue),
// written as D(nu) + 1 - ln(1 + 1/nu) with D(nu) = psi(y + 1/2) - psi(y), y = nu/2.
// D uses the recurrence psi(z) = psi(z + 1) - 1/z six times (each difference
// 1/(y+j) - 1/(y+j+1/2) = 0.5/((y+j)(y+j+1/2)) taken in product form) and the
// asymptotic series of psi (Abramowitz & Stegun 6.3.5, 6.3.18) for the
// difference at z = y + 6, so no term cancels in FP32.
__device__ __forceinline__ float nu_const_f(float nu) {
    const float y = 0.5f * nu;
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const float z = y + (float)j;
        acc += __fdividef(0.5f, z * (z + 0.5f));
    }
    const float z = y + 6.f, zh = z + 0.5f;
    const float iz2 = __fdividef(1.f, z * z), ih2 = __fdividef(1.f, zh * zh);
    // psi(zh) - psi(z) = ln(zh/z) - 1/(2 zh) + 1/(2 z) - sum_k B_2k/(2k) (zh^-2k - z^-2k)
    auto tail = [](float i2) {
        return i2 * (1.f / 12.f - i2 * (1.f / 120.f - i2 * (1.f / 252.f - i2 * (1.f / 240.f))));
    };
    const float asym = log1pf(__fdividef(0.5f, z)) + __fdividef(0.25f, z * zh) - (tail(ih2) - tail(iz2));
    return (asym + acc) + 1.f - log1pf(__fdividef(1.f, nu));
}

// Chebyshev form of the sample sums of eq. robustnessValue.  With
// nu = m + h tau (tau in [-1, 1] over [nu_lo, nu_hi]) and alpha_i = (m + x_i^2)/h > 1:
//   ln(nu + x_i^2)  = ln h + ln(beta_i/2) + 2 sum_k (-1)^(k+1) q_i^k / k T_k(tau)
//   1/(nu + x_i^2)  = (gamma_i / h) (1 + 2 sum_k (-1)^k q_i^k T_k(tau))
// with beta = alpha + sqrt(alpha^2 - 1), q = 1/beta, gamma = 1/sqrt(alpha^2 - 1)
// (the classical expansions of ln(alpha + tau) and 1/(alpha + tau)).  One cluster
// reduction of the power sums P_k = sum q^k, G_k = sum gamma q^k and sum ln(beta/2)
// then gives f(nu) at any nu without revisiting the samples; truncating at K
// terms errs by < q_max^(K+1) per sample (q_max = 0.382 for [2, 10], K = 20).
constexpr int kChebK = 20;
constexpr int kChebVals = 2 * kChebK + 2;      // SL, P_1..P_K, G_0..G_K per channel

// f(nu) from the Chebyshev coefficients (FP32 Clenshaw): ca[k] = 2 (-1)^(k+1) P_k / k,
// cb[k] = 2 (-1)^k G_k for k >= 1, so that sum_i ln(alpha_i + tau) = SL + sum_k ca_k T_k(tau)
// and sum_i 1/(alpha_i + tau) = G_0 + sum_k cb_k T_k(tau).
__device__ __forceinline__ float nu_equation_cheb(const float* ca, const float* cb, float G0, float n, float SL,
                                                  float nu, float m, float invh, float lnh) {
    const float tau = (nu - m) * invh;
    const float t2 = 2.f * tau;
    float a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
    for (int k = kChebK; k >= 1; --k) {
        const float an = fmaf(t2, a1, ca[k] - a2);
        const float bn = fmaf(t2, b1, cb[k] - b2);
        a2 = a1; a1 = an;
        b2 = b1; b1 = bn;
    }
    const float A = fmaf(tau, a1, -a2);            // Clenshaw end with c_0 = 0
    const float B = fmaf(tau, b1, G0 - b2);
    // f = n [c(nu) + ln(nu + 1) - ln h] - SL - A - (nu + 1) B / h
    const float base = n * (nu_const_f(nu) + logf(nu + 1.f) - lnh) - SL;
    return base - A - (nu + 1.f) * B * invh;
}

// nu of one channel by bisection on eq. robustnessValue over [lo0, hi0], run by
// a group of 128 threads that synchronise on named barrier `bar_id` (lt = the
// thread's index in the group).  T holds the channel's cluster sums (SL,
// P_1..P_K, G_0..G_K), nc its residual count.  The first section evaluates
// f(hi), f(lo) and 63 interior points (6 halvings), later sections 127 points
// (7 halvings); each replays exactly the bisection's decisions at the same
// dyadic midpoints.  ca, cb (K + 1 floats each), mask (4 words) and ends (2
// ints) are the group's shared-memory scratch.  Every thread of the group
// returns the same nu.
__device__ __forceinline__ float bisect_nu_group(const float* T, float nc, float lo0, float hi0, int steps, int lt,
                                                 int bar_id, float* ca, float* cb, unsigned* mask, int* ends) {
    const int lane = lt & 31, gw = lt >> 5;
    const float m = 0.5f * (lo0 + hi0), h = 0.5f * (hi0 - lo0);
    if (lt >= 1 && lt <= kChebK) {
        const float sgn = (lt & 1) ? 2.f : -2.f;
        ca[lt] = sgn * __fdividef(T[lt], (float)lt);
        cb[lt] = -sgn * T[1 + kChebK + lt];
    }
    asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
    const float G0 = T[1 + kChebK], SL = T[0];
    const float invh = 1.f / h, lnh = logf(h);
    float lo = lo0, hi = hi0, nuc = 0.5f * (lo0 + hi0);
    int left = steps;
    bool first = true, done = false;
    while (!done) {
        const int st = left < (first ? 6 : 7) ? left : (first ? 6 : 7);
        const int np = 1 << st;                  // sub-intervals this round
        const int off = first ? 2 : 0;           // lanes 0, 1 take the endpoints first
        const float step = (hi - lo) / (float)np;
        const int j = lt - off + 1;              // interior point index of this lane
        float x = 0.f;
        bool eval = false;
        if (first && lt == 0) { x = hi; eval = true; }
        else if (first && lt == 1) { x = lo; eval = true; }
        else if (j >= 1 && j < np) { x = fmaf((float)j, step, lo); eval = true; }
        const float f = eval ? nu_equation_cheb(ca, cb, G0, nc, SL, x, m, invh, lnh) : 0.f;
        const unsigned pos = __ballot_sync(0xffffffffu, eval && f > 0.f);
        if (lane == 0) mask[gw] = pos;
        if (first && lt == 0) ends[0] = (f >= 0.f) ? 1 : 0;   // f(hi) >= 0
        if (first && lt == 1) ends[1] = (f <= 0.f) ? 1 : 0;   // f(lo) <= 0
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        if (first && ends[0]) { nuc = hi0; done = true; }
        else if (first && ends[1]) { nuc = lo0; done = true; }
        else {
            int jl = 0, jh = np;
            for (int q = 0; q < st; ++q) {
                const int jm = (jl + jh) >> 1;
                const int L = jm - 1 + off;
                if ((mask[L >> 5] >> (L & 31)) & 1u) jl = jm; else jh = jm;
            }
            const float nlo = fmaf((float)jl, step, lo), nhi = fmaf((float)jh, step, lo);
            lo = nlo;
            hi = nhi;
            left -= st;
            first = false;
            if (left == 0) { nuc = 0.5f * (lo + hi); done = true; }
        }
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");   // masks are reused next round
    }
    return nuc;
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

}  // namespace rgbid
