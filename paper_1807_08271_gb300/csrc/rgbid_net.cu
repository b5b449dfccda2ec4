// Learned initialiser: forward and backward passes of the network on bfloat16
// tensor cores, its loss, Adam, parameter initialisation, input packing from
// pyramid levels, and the plan that turns proposals into batch items.
//
// Every layer pass is one implicit GEMM C[M x N] = A[M x K] B[K x N] computed
// by tcgen05.mma (bf16 operands in shared memory, FP32 accumulator in tensor
// memory) in 128 x 64 tiles with K-slices of 64; a problem type supplies how A and B elements are
// gathered (convolution patches, transposed weights, upstream gradients) and
// what the epilogue does (bias, ReLU, rounding to bf16, the ReLU mask of the
// layer below, or FP32 atomics for split-K weight gradients):
//   forward   conv: M = B Ho Wo pixels, N = c_out, K = 9 c_in   (A = patches, B = W)
//             fc:   M = B,           N = out,   K = in
//   dgrad     conv: M = B H W input pixels, N = c_in, K = 9 c_out
//             (A = upstream gradient at the output pixel each tap reaches)
//             fc:   M = B, N = in, K = out  (B = W transposed)
//   wgrad     conv: M = 9 c_in + 1, N = c_out, K = B Ho Wo  (the extra row of
//             ones gives the bias gradient); fc: M = in + 1, N = out, K = B
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <type_traits>
#include <utility>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "rgbid.h"
#include "rgbid_util.h"

namespace rgbid {
namespace net {

using bf16 = __nv_bfloat16;

enum { kConv = 0, kFc = 1 };

struct LayerDef {
    int kind, cin, cout, hin, win, hout, wout;
};

constexpr LayerDef kLayers[RGBID_NET_LAYERS] = {
    {kConv, 4, 32, 60, 80, 30, 40},
    {kConv, 32, 32, 30, 40, 15, 20},
    {kConv, 32, 64, 15, 20, 8, 10},
    {kConv, 64, 64, 8, 10, 4, 5},
    {kFc, 1280, 256, 1, 1, 1, 1},
    {kFc, 256, RGBID_NET_OUT, 1, 1, 1, 1},
};

constexpr size_t pad64(size_t n) { return (n + 63) / 64 * 64; }
constexpr size_t weight_count(int l) {
    return kLayers[l].kind == kConv ? (size_t)9 * kLayers[l].cin * kLayers[l].cout
                                    : (size_t)kLayers[l].cin * kLayers[l].cout;
}
constexpr size_t w_offset(int l) { return l == 0 ? 0 : pad64(pad64(w_offset(l - 1) + weight_count(l - 1)) + kLayers[l - 1].cout); }
constexpr size_t b_offset(int l) { return pad64(w_offset(l) + weight_count(l)); }
constexpr size_t kParams = pad64(b_offset(RGBID_NET_LAYERS - 1) + RGBID_NET_OUT);
static_assert(kParams == 395712, "parameter layout");

// activation elements per sample of layer l's output (l = 0..4; the last layer's output is y)
constexpr size_t act_per_sample(int l) {
    return kLayers[l].kind == kConv ? (size_t)kLayers[l].hout * kLayers[l].wout * kLayers[l].cout
                                    : (size_t)kLayers[l].cout;
}
constexpr size_t kInPerSample = (size_t)RGBID_NET_IN_H * RGBID_NET_IN_W * RGBID_NET_IN_C;
constexpr size_t kMaxGradPerSample = act_per_sample(0);   // the largest activation gradient (c1's output)

__device__ __forceinline__ bf16 bz() { return __float2bfloat16_rn(0.f); }

// Programmatic dependent launch between the passes' kernels: each kernel lets its
// successor be scheduled at once and waits for its predecessor's completion (and
// memory) before it reads anything, so the launches overlap and the data never does.
__device__ __forceinline__ void pdl_start() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// launch with programmatic stream serialisation (the kernel calls pdl_start first)
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// ---------------------------------------------------------------- GEMM core
// One CTA of 128 threads computes a 128 x TN tile of C (TN = 32 or 64, the
// smallest that covers N) on the fifth-generation tensor cores: the four warps
// gather 64-wide K slices of A (128 rows) and B (TN rows) into shared memory, one
// thread issues tcgen05.mma (M = 128, N = TN, K = 16 per instruction, bf16
// operands, FP32 accumulator in tensor memory) and commits them to an mbarrier.
// Two stages alternate: while the tensor core reads one, each thread's loads of
// the next slice are already in flight in registers and land in the other stage
// once the MMAs that last read it have completed.  The epilogue reads the
// accumulator back with tcgen05.ld (warp w owns rows 32w .. 32w + 31, one row per
// lane) and hands each element to the problem's store.
//
// Shared-memory operand layout (both operands K-major, no swizzle): an 8-row x
// 16-byte core matrix is 128 contiguous bytes; the 8 core matrices along K of one
// 8-row group follow each other (128 B apart, the descriptor's leading-dimension
// offset) and the 8-row groups are 1024 B apart (its stride-dimension offset).
// Element (r, k) of a tile therefore sits at byte
//     (r / 8) * 1024 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// and the 16-byte vector i of a tile (8 consecutive k of one row) at byte 16 i
// when i enumerates rows fastest within a core matrix, then K chunks, then row
// groups.
constexpr int TM = 128, TK = 64, GEMM_NT = 128, kStages = 2;
constexpr int kATile = TM * TK * 2;
constexpr int kVecBNone = 0, kVecBk = 1, kVecBn = 2;   // how B may be loaded 8 elements at a time
constexpr int kVecANone = 0, kVecAk = 1, kVecAm = 2;   // how A may be loaded 8 elements at a time
constexpr int kVecAk4 = 3, kVecAm4 = 4;                 // ... or 4 elements (8 bytes) at a time
constexpr long long kMmaWaitBudget = 4000000000LL;     // clock64 cycles (~2 s) before a wait gives up

template <int TN>
struct TileCfg {
    static constexpr int kBTile = TN * TK * 2;
    static constexpr int kStageBytes = kATile + kBTile;
    static constexpr int kSmem = kStages * kStageBytes + 128;   // + alignment slack
    static constexpr uint32_t kCols = TN;                       // FP32 accumulator columns (a power of 2, >= 32)
    // instruction descriptor of kind::f16: FP32 D (bits 4-5), bf16 A (7-9) and B (10-12),
    // both K-major (bits 15, 16 clear), N >> 3 at bit 17, M >> 4 at bit 24
    static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                                       ((uint32_t)(TM >> 4) << 24);
};

__device__ unsigned int g_mma_timeouts;   // waits on the tensor core that ran out (0 in a healthy run)

__device__ __forceinline__ uint4 ld16(const bf16* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start >> 4 (bits 0-13), leading-dimension offset
// >> 4 (16-29), stride-dimension offset >> 4 (32-45), descriptor version 1 (bit 46),
// base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void mbar_init1(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
}

// waits until the phase of parity `parity` has completed; false if the budget ran out
__device__ __forceinline__ bool mbar_wait_parity(unsigned long long* bar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n"
            " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(su32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kMmaWaitBudget) return false;
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[128 x 16] B[TN x 16]^T
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrives on `bar` once every tcgen05.mma this thread issued so far has completed
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this lane's accumulator row
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    // the registers are defined only once the load has completed
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// byte offset of element (r, k) of an operand tile
__device__ __forceinline__ int tile_off(int r, int k) { return (r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// An operand tile is ROWS rows x TK columns: row r is operand row row0 + r (m of A or
// n of B), column c is k0 + c.  The vector loaders move 16 bytes: 8 consecutive k of
// one row (MODE 1; vector i lands at byte 16 i) or rows row .. row+7 of one k (MODE 2;
// the 8 values go to one core matrix, 16 bytes apart).  fetch() issues a thread's
// loads of one slice into registers, put() stores them into a stage.
template <int ROWS>
struct Vecs {
    static constexpr int n = ROWS * TK / 8 / GEMM_NT;
    uint4 v[n];
};

template <int ROWS, int MODE, class L8>
__device__ __forceinline__ void fetch(Vecs<ROWS>& r, int row0, int nrows, int k0, int k1, int tid, L8 ld8) {
#pragma unroll
    for (int j = 0; j < Vecs<ROWS>::n; ++j) {
        const int i = tid + j * GEMM_NT;
        const int row = MODE == 1 ? row0 + ((i & 7) | ((i >> 6) << 3)) : row0 + (i >> 6) * 8;
        const int k = MODE == 1 ? k0 + ((i >> 3) & 7) * 8 : k0 + (i & (TK - 1));
        r.v[j] = (row < nrows && k < k1) ? ld8(row, k) : make_uint4(0u, 0u, 0u, 0u);
    }
}

template <int ROWS, int MODE>
__device__ __forceinline__ void put(unsigned char* t, const Vecs<ROWS>& r, int tid) {
#pragma unroll
    for (int j = 0; j < Vecs<ROWS>::n; ++j) {
        const int i = tid + j * GEMM_NT;
        if (MODE == 1) {
            *reinterpret_cast<uint4*>(t + 16 * i) = r.v[j];
        } else {
            unsigned char* const base = t + tile_off((i >> 6) * 8, i & (TK - 1));
            const uint32_t w[4] = {r.v[j].x, r.v[j].y, r.v[j].z, r.v[j].w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                *reinterpret_cast<unsigned short*>(base + 32 * q) = (unsigned short)(w[q] & 0xffffu);
                *reinterpret_cast<unsigned short*>(base + 32 * q + 16) = (unsigned short)(w[q] >> 16);
            }
        }
    }
}

// 8-byte variants for operands whose channel count is a multiple of 4 but not of 8:
// 4 consecutive k of one row (MODE 3; vector i lands at byte 8 i when i enumerates
// the two halves of a 16-byte chunk fastest, then the 8 rows of a core matrix, then
// K chunks, then row groups) or rows row .. row+3 of one k (MODE 4).
struct Vecs4 {
    static constexpr int n = TM * TK / 4 / GEMM_NT;
    uint2 v[n];
};

template <int MODE, class L4>
__device__ __forceinline__ void fetch4(Vecs4& r, int row0, int nrows, int k0, int k1, int tid, L4 ld4) {
#pragma unroll
    for (int j = 0; j < Vecs4::n; ++j) {
        const int i = tid + j * GEMM_NT;
        const int row = MODE == 3 ? row0 + (((i >> 1) & 7) | ((i >> 7) << 3)) : row0 + (i >> 6) * 4;
        const int k = MODE == 3 ? k0 + ((i >> 4) & 7) * 8 + (i & 1) * 4 : k0 + (i & (TK - 1));
        r.v[j] = (row < nrows && k < k1) ? ld4(row, k) : make_uint2(0u, 0u);
    }
}

template <int MODE>
__device__ __forceinline__ void put4(unsigned char* t, const Vecs4& r, int tid) {
#pragma unroll
    for (int j = 0; j < Vecs4::n; ++j) {
        const int i = tid + j * GEMM_NT;
        if (MODE == 3) {
            *reinterpret_cast<uint2*>(t + 8 * i) = r.v[j];
        } else {
            unsigned char* const base = t + tile_off((i >> 6) * 4, i & (TK - 1));
            *reinterpret_cast<unsigned short*>(base) = (unsigned short)(r.v[j].x & 0xffffu);
            *reinterpret_cast<unsigned short*>(base + 16) = (unsigned short)(r.v[j].x >> 16);
            *reinterpret_cast<unsigned short*>(base + 32) = (unsigned short)(r.v[j].y & 0xffffu);
            *reinterpret_cast<unsigned short*>(base + 48) = (unsigned short)(r.v[j].y >> 16);
        }
    }
}

// whether a problem type has the 8-byte A loader
template <class P, class = void>
struct HasA4 : std::false_type {};
template <class P>
struct HasA4<P, decltype((void)std::declval<const P&>().loadA4(0, 0))> : std::true_type {};

// element-wise loader (operands whose layout allows no 16-byte vectors)
template <int ROWS, class L1>
__device__ __forceinline__ void load_elements(unsigned char* t, int row0, int nrows, int k0, int k1, int tid, L1 ld1) {
#pragma unroll 4
    for (int i = tid; i < ROWS * TK; i += GEMM_NT) {
        const int c = i & (TK - 1), r = i >> 6;
        const int row = row0 + r, k = k0 + c;
        *reinterpret_cast<bf16*>(t + tile_off(r, c)) = (row < nrows && k < k1) ? ld1(row, k) : bz();
    }
}

// ---------------------------------------------------------------- epilogue helpers
// A lane's 16 accumulator columns c0 .. c0+15 of one row, of which the first nv exist,
// go out as 16-byte vectors where the row segment is whole and aligned.
__device__ __forceinline__ bool al16(const void* p) { return !((uintptr_t)p & 15u); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

__device__ __forceinline__ void put_bf16_row(bf16* dst, const float (&z)[16], int nv) {
    if (nv == 16 && al16(dst)) {
        uint4 a, b;
        a.x = pack_bf16(z[0], z[1]);
        a.y = pack_bf16(z[2], z[3]);
        a.z = pack_bf16(z[4], z[5]);
        a.w = pack_bf16(z[6], z[7]);
        b.x = pack_bf16(z[8], z[9]);
        b.y = pack_bf16(z[10], z[11]);
        b.z = pack_bf16(z[12], z[13]);
        b.w = pack_bf16(z[14], z[15]);
        reinterpret_cast<uint4*>(dst)[0] = a;
        reinterpret_cast<uint4*>(dst)[1] = b;
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < nv) dst[j] = __float2bfloat16_rn(z[j]);
    }
}

__device__ __forceinline__ void put_f32_row(float* dst, const float (&z)[16], int nv) {
    if (nv == 16 && al16(dst)) {
#pragma unroll
        for (int q = 0; q < 4; ++q) reinterpret_cast<float4*>(dst)[q] = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < nv) dst[j] = z[j];
    }
}

// upstream gradient masked by the ReLU of the layer's input (its stored value > 0)
__device__ __forceinline__ void put_masked_row(bf16* gin, const bf16* act, const float (&v)[16], int nv) {
    if (nv == 16 && al16(gin) && al16(act)) {
        const uint4 a0 = __ldg(reinterpret_cast<const uint4*>(act)), a1 = __ldg(reinterpret_cast<const uint4*>(act) + 1);
        const uint32_t w[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float z[16];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float lo = __bfloat162float(__ushort_as_bfloat16((unsigned short)(w[q] & 0xffffu)));
            const float hi = __bfloat162float(__ushort_as_bfloat16((unsigned short)(w[q] >> 16)));
            z[2 * q] = lo > 0.f ? v[2 * q] : 0.f;
            z[2 * q + 1] = hi > 0.f ? v[2 * q + 1] : 0.f;
        }
        put_bf16_row(gin, z, 16);
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < nv) gin[j] = __bfloat162float(act[j]) > 0.f ? __float2bfloat16_rn(v[j]) : bz();
    }
}

__device__ __forceinline__ void add_f32_row(float* dst, const float (&v)[16], int nv) {
    if (nv == 16 && al16(dst)) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            atomicAdd(reinterpret_cast<float4*>(dst) + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < nv) atomicAdd(dst + j, v[j]);
    }
}

// C tile (blockIdx.x, blockIdx.y) over the K range of blockIdx.z
template <class P, int TN>
__global__ void __launch_bounds__(GEMM_NT) gemm_tc(P p, int M, int N, int K, int kchunk, float* scratch) {
    using Cfg = TileCfg<TN>;
    extern __shared__ unsigned char gemm_smem[];
    __shared__ __align__(8) unsigned long long mbar[kStages];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
    const int kb0 = blockIdx.z * kchunk;
    const int kb1 = min(K, kb0 + kchunk);
    const int nk = (kb1 - kb0 + TK - 1) / TK;
    unsigned char* const sm =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(gemm_smem) + 127) & ~(uintptr_t)127);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(Cfg::kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        mbar_init1(&mbar[0]);
        mbar_init1(&mbar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    const int va = p.vecA(), vb = p.vecB();
    auto la1 = [&](int m, int k) { return p.loadA(m, k); };
    auto la8 = [&](int m, int k) { return p.loadA8(m, k); };
    auto lb1 = [&](int n, int k) { return p.loadB(k, n); };
    // B's rows are n: loadB8(k, n) gives k .. k+7 of row n (kVecBk) or rows n .. n+7 of column k (kVecBn)
    auto lb8 = [&](int n, int k) { return p.loadB8(k, n); };
    pdl_start();   // the operands come from the preceding pass
    Vecs<TM> ra;
    Vecs<TN> rb;
    Vecs4 ra4;
    auto fetch_slice = [&](int k0) {
        if (va == kVecAk) fetch<TM, 1>(ra, m0, M, k0, kb1, tid, la8);
        else if (va == kVecAm) fetch<TM, 2>(ra, m0, M, k0, kb1, tid, la8);
        if constexpr (HasA4<P>::value) {
            auto la4 = [&](int m, int k) { return p.loadA4(m, k); };
            if (va == kVecAk4) fetch4<3>(ra4, m0, M, k0, kb1, tid, la4);
            else if (va == kVecAm4) fetch4<4>(ra4, m0, M, k0, kb1, tid, la4);
        }
        if (vb == kVecBk) fetch<TN, 1>(rb, n0, N, k0, kb1, tid, lb8);
        else if (vb == kVecBn) fetch<TN, 2>(rb, n0, N, k0, kb1, tid, lb8);
    };
    fetch_slice(kb0);   // in flight during the set-up barrier

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    bool ok = true;
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt & 1;
        // the stage's previous MMAs (slice kt - 2) have finished reading it
        if (kt >= 2 && !mbar_wait_parity(&mbar[s], (uint32_t)((kt >> 1) - 1) & 1u)) ok = false;
        unsigned char* const As = sm + s * Cfg::kStageBytes;
        unsigned char* const Bs = As + kATile;
        const int k0 = kb0 + kt * TK;
        if (va == kVecAk) put<TM, 1>(As, ra, tid);
        else if (va == kVecAm) put<TM, 2>(As, ra, tid);
        else if (HasA4<P>::value && va == kVecAk4) put4<3>(As, ra4, tid);
        else if (HasA4<P>::value && va == kVecAm4) put4<4>(As, ra4, tid);
        else load_elements<TM>(As, m0, M, k0, kb1, tid, la1);
        if (vb == kVecBk) put<TN, 1>(Bs, rb, tid);
        else if (vb == kVecBn) put<TN, 2>(Bs, rb, tid);
        else load_elements<TN>(Bs, n0, N, k0, kb1, tid, lb1);
        // the next slice's loads stay in flight across the barrier and the MMAs
        if (kt + 1 < nk) fetch_slice(k0 + TK);
        // the generic-proxy stores must be visible to the tensor core's (async-proxy) reads
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = su32(As), b0 = su32(Bs);
#pragma unroll
            for (int ks = 0; ks < TK / 16; ++ks)   // K = 16 is two core matrices along K: 256 bytes
                umma_f16(tmem, umma_desc(a0 + 256u * ks), umma_desc(b0 + 256u * ks), Cfg::kIdesc, (kt | ks) != 0);
            umma_commit(&mbar[s]);
        }
    }
    // the last commit covers every MMA of the tile
    if (!mbar_wait_parity(&mbar[(nk - 1) & 1], (uint32_t)((nk - 1) >> 1) & 1u)) ok = false;
    tc_fence_after();
    if (!ok && lane == 0) atomicAdd(&g_mma_timeouts, 1u);

    const int rr = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < TN; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        const int nv = min(16, N - (n0 + c0));
        if (rr < M && nv > 0) {
            if (scratch) put_f32_row(scratch + ((size_t)blockIdx.z * M + rr) * N + n0 + c0, v, nv);
            else p.store_row(rr, n0 + c0, v, nv);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::kCols) : "memory");
}

// ---------------------------------------------------------------- problem types
// 3x3 stride-2 pad-1 convolution geometry of one layer and batch position decoding.
struct ConvGeo {
    int H, W, C, Ho, Wo, Co;
    // input element feeding output pixel m (b, i, j) through tap/channel k = (kh * 3 + kw) * C + ci
    __device__ __forceinline__ bf16 patch(const bf16* in, int m, int k) const {
        const int hw = Ho * Wo;
        const int b = m / hw, r = m - b * hw;
        const int i = r / Wo, j = r - i * Wo;
        const int tap = k / C, ci = k - tap * C;
        const int kh = tap / 3, kw = tap - kh * 3;
        const int y = 2 * i + kh - 1, x = 2 * j + kw - 1;
        if (y < 0 || y >= H || x < 0 || x >= W) return bz();
        return in[((size_t)(b * H + y) * W + x) * C + ci];
    }
    // patch elements k .. k+3 (C a multiple of 4, k a multiple of 4: one tap)
    __device__ __forceinline__ uint2 patch4(const bf16* in, int m, int k) const {
        const int hw = Ho * Wo;
        const int b = m / hw, r = m - b * hw;
        const int i = r / Wo, j = r - i * Wo;
        const int tap = k / C, ci = k - tap * C;
        const int kh = tap / 3, kw = tap - kh * 3;
        const int y = 2 * i + kh - 1, x = 2 * j + kw - 1;
        if (y < 0 || y >= H || x < 0 || x >= W) return make_uint2(0u, 0u);
        return *reinterpret_cast<const uint2*>(in + ((size_t)(b * H + y) * W + x) * C + ci);
    }
    // patch elements k .. k+7 (C a multiple of 8, k a multiple of 8: one tap)
    __device__ __forceinline__ uint4 patch8(const bf16* in, int m, int k) const {
        const int hw = Ho * Wo;
        const int b = m / hw, r = m - b * hw;
        const int i = r / Wo, j = r - i * Wo;
        const int tap = k / C, ci = k - tap * C;
        const int kh = tap / 3, kw = tap - kh * 3;
        const int y = 2 * i + kh - 1, x = 2 * j + kw - 1;
        if (y < 0 || y >= H || x < 0 || x >= W) return make_uint4(0u, 0u, 0u, 0u);
        return ld16(in + ((size_t)(b * H + y) * W + x) * C + ci);
    }
};

struct ConvFwd {
    ConvGeo geo;
    const bf16* in;
    const bf16* W;
    const float* bias;
    bf16* out;
    __device__ __forceinline__ bf16 loadA(int m, int k) const { return geo.patch(in, m, k); }
    __device__ __forceinline__ bf16 loadB(int k, int n) const { return W[(size_t)k * geo.Co + n]; }
    // (the 8-byte loads need the input 8-byte aligned; the caller's input is checked for 4 only)
    __device__ __forceinline__ int vecA() const {
        return geo.C % 8 == 0 ? kVecAk : (geo.C % 4 == 0 && !((uintptr_t)in & 7u) ? kVecAk4 : kVecANone);
    }
    __device__ __forceinline__ uint4 loadA8(int m, int k) const { return geo.patch8(in, m, k); }
    __device__ __forceinline__ uint2 loadA4(int m, int k) const { return geo.patch4(in, m, k); }
    __device__ __forceinline__ int vecB() const { return geo.Co % 8 == 0 ? kVecBn : kVecBNone; }
    __device__ __forceinline__ uint4 loadB8(int k, int n) const { return ld16(W + (size_t)k * geo.Co + n); }
    __device__ __forceinline__ void store(int m, int n, float v) const {
        out[(size_t)m * geo.Co + n] = __float2bfloat16_rn(fmaxf(v + bias[n], 0.f));
    }
    __device__ __forceinline__ void store_row(int m, int c0, const float (&v)[16], int nv) const {
        float z[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) z[j] = fmaxf(v[j] + (j < nv ? __ldg(bias + c0 + j) : 0.f), 0.f);
        put_bf16_row(out + (size_t)m * geo.Co + c0, z, nv);
    }
};

struct FcFwd {
    const bf16* in;
    const bf16* W;
    const float* bias;
    bf16* out;        // ReLU'd bf16 output, or
    float* outf;      // the float32 network output (no ReLU)
    int Kin, Nout;
    __device__ __forceinline__ bf16 loadA(int m, int k) const { return in[(size_t)m * Kin + k]; }
    __device__ __forceinline__ bf16 loadB(int k, int n) const { return W[(size_t)k * Nout + n]; }
    __device__ __forceinline__ int vecA() const { return Kin % 8 == 0 ? kVecAk : kVecANone; }
    __device__ __forceinline__ uint4 loadA8(int m, int k) const { return ld16(in + (size_t)m * Kin + k); }
    __device__ __forceinline__ int vecB() const { return Nout % 8 == 0 ? kVecBn : kVecBNone; }
    __device__ __forceinline__ uint4 loadB8(int k, int n) const { return ld16(W + (size_t)k * Nout + n); }
    __device__ __forceinline__ void store(int m, int n, float v) const {
        const float z = v + bias[n];
        if (outf) outf[(size_t)m * Nout + n] = z;
        else out[(size_t)m * Nout + n] = __float2bfloat16_rn(fmaxf(z, 0.f));
    }
    __device__ __forceinline__ void store_row(int m, int c0, const float (&v)[16], int nv) const {
        float z[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) z[j] = v[j] + (j < nv ? __ldg(bias + c0 + j) : 0.f);
        if (outf) {
            put_f32_row(outf + (size_t)m * Nout + c0, z, nv);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) z[j] = fmaxf(z[j], 0.f);
            put_bf16_row(out + (size_t)m * Nout + c0, z, nv);
        }
    }
};

// gradient w.r.t. a convolution's input, masked by that input's ReLU (its stored value > 0)
struct ConvDgrad {
    ConvGeo geo;
    const bf16* gout;     // [B, Ho, Wo, Co]
    const bf16* W;
    const bf16* act_in;   // [B, H, W, C]
    bf16* gin;
    __device__ __forceinline__ bf16 loadA(int m, int k) const {
        const int hw = geo.H * geo.W;
        const int b = m / hw, r = m - b * hw;
        const int y = r / geo.W, x = r - y * geo.W;
        const int tap = k / geo.Co, co = k - tap * geo.Co;
        const int kh = tap / 3, kw = tap - kh * 3;
        const int i2 = y + 1 - kh, j2 = x + 1 - kw;          // = 2 i, 2 j of the output pixel the tap reaches
        if (i2 < 0 || j2 < 0 || (i2 & 1) || (j2 & 1)) return bz();
        const int i = i2 >> 1, j = j2 >> 1;
        if (i >= geo.Ho || j >= geo.Wo) return bz();
        return gout[((size_t)(b * geo.Ho + i) * geo.Wo + j) * geo.Co + co];
    }
    __device__ __forceinline__ bf16 loadB(int k, int n) const {
        const int tap = k / geo.Co, co = k - tap * geo.Co;
        return W[((size_t)tap * geo.C + n) * geo.Co + co];
    }
    // the upstream gradient and the weights are contiguous along co for a fixed tap
    __device__ __forceinline__ int vecA() const { return geo.Co % 8 == 0 ? kVecAk : kVecANone; }
    __device__ __forceinline__ uint4 loadA8(int m, int k) const {
        const int hw = geo.H * geo.W;
        const int b = m / hw, r = m - b * hw;
        const int y = r / geo.W, x = r - y * geo.W;
        const int tap = k / geo.Co, co = k - tap * geo.Co;
        const int kh = tap / 3, kw = tap - kh * 3;
        const int i2 = y + 1 - kh, j2 = x + 1 - kw;
        if (i2 < 0 || j2 < 0 || (i2 & 1) || (j2 & 1)) return make_uint4(0u, 0u, 0u, 0u);
        const int i = i2 >> 1, j = j2 >> 1;
        if (i >= geo.Ho || j >= geo.Wo) return make_uint4(0u, 0u, 0u, 0u);
        return ld16(gout + ((size_t)(b * geo.Ho + i) * geo.Wo + j) * geo.Co + co);
    }
    __device__ __forceinline__ int vecB() const { return geo.Co % 8 == 0 ? kVecBk : kVecBNone; }
    __device__ __forceinline__ uint4 loadB8(int k, int n) const {
        const int tap = k / geo.Co, co = k - tap * geo.Co;
        return ld16(W + ((size_t)tap * geo.C + n) * geo.Co + co);
    }
    __device__ __forceinline__ void store(int m, int n, float v) const {
        const size_t o = (size_t)m * geo.C + n;
        gin[o] = __bfloat162float(act_in[o]) > 0.f ? __float2bfloat16_rn(v) : bz();
    }
    __device__ __forceinline__ void store_row(int m, int c0, const float (&v)[16], int nv) const {
        const size_t o = (size_t)m * geo.C + c0;
        put_masked_row(gin + o, act_in + o, v, nv);
    }
};

struct FcDgrad {
    const bf16* gout;     // [B, Nout] bf16, or
    const float* goutf;   // the float32 loss gradient (rounded to bf16 on load)
    const bf16* W;        // [Kin, Nout]
    const bf16* act_in;   // [B, Kin]
    bf16* gin;
    int Kin, Nout;
    __device__ __forceinline__ bf16 loadA(int m, int k) const {
        const size_t o = (size_t)m * Nout + k;
        return goutf ? __float2bfloat16_rn(goutf[o]) : gout[o];
    }
    __device__ __forceinline__ bf16 loadB(int k, int n) const { return W[(size_t)n * Nout + k]; }
    __device__ __forceinline__ int vecA() const { return goutf == nullptr && Nout % 8 == 0 ? kVecAk : kVecANone; }
    __device__ __forceinline__ uint4 loadA8(int m, int k) const { return ld16(gout + (size_t)m * Nout + k); }
    __device__ __forceinline__ int vecB() const { return Nout % 8 == 0 ? kVecBk : kVecBNone; }
    __device__ __forceinline__ uint4 loadB8(int k, int n) const { return ld16(W + (size_t)n * Nout + k); }
    __device__ __forceinline__ void store(int m, int n, float v) const {
        const size_t o = (size_t)m * Kin + n;
        gin[o] = __bfloat162float(act_in[o]) > 0.f ? __float2bfloat16_rn(v) : bz();
    }
    __device__ __forceinline__ void store_row(int m, int c0, const float (&v)[16], int nv) const {
        const size_t o = (size_t)m * Kin + c0;
        put_masked_row(gin + o, act_in + o, v, nv);
    }
};

// weight (rows < 9 C) and bias (row 9 C) gradients of a convolution, split-K over pixels
struct ConvWgrad {
    ConvGeo geo;
    const bf16* in;
    const bf16* gout;
    float* dW;
    float* db;
    __device__ __forceinline__ bf16 loadA(int m, int k) const {
        if (m == 9 * geo.C) return __float2bfloat16_rn(1.f);
        return geo.patch(in, k, m);
    }
    __device__ __forceinline__ bf16 loadB(int k, int n) const { return gout[(size_t)k * geo.Co + n]; }
    // rows m .. m+7 of pixel k: channels of one tap, or the bias row of ones (m = 9 C, the last)
    __device__ __forceinline__ int vecA() const {
        return geo.C % 8 == 0 ? kVecAm : (geo.C % 4 == 0 && !((uintptr_t)in & 7u) ? kVecAm4 : kVecANone);
    }
    __device__ __forceinline__ uint4 loadA8(int m, int k) const {
        if (m == 9 * geo.C) return make_uint4((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(1.f)), 0u, 0u, 0u);
        return geo.patch8(in, k, m);
    }
    // rows m .. m+3 of pixel k (C a multiple of 4)
    __device__ __forceinline__ uint2 loadA4(int m, int k) const {
        if (m == 9 * geo.C) return make_uint2((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(1.f)), 0u);
        return geo.patch4(in, k, m);
    }
    __device__ __forceinline__ int vecB() const { return geo.Co % 8 == 0 ? kVecBn : kVecBNone; }
    __device__ __forceinline__ uint4 loadB8(int k, int n) const { return ld16(gout + (size_t)k * geo.Co + n); }
    __device__ __forceinline__ void store(int m, int n, float v) const {
        if (m == 9 * geo.C) atomicAdd(&db[n], v);
        else atomicAdd(&dW[(size_t)m * geo.Co + n], v);
    }
    __device__ __forceinline__ void store_row(int m, int c0, const float (&v)[16], int nv) const {
        add_f32_row(m == 9 * geo.C ? db + c0 : dW + (size_t)m * geo.Co + c0, v, nv);
    }
};

struct FcWgrad {
    const bf16* in;       // [B, Kin]
    const bf16* gout;
    const float* goutf;
    float* dW;
    float* db;
    int Kin, Nout;
    __device__ __forceinline__ bf16 loadA(int m, int k) const {
        return m == Kin ? __float2bfloat16_rn(1.f) : in[(size_t)k * Kin + m];
    }
    __device__ __forceinline__ bf16 loadB(int k, int n) const {
        const size_t o = (size_t)k * Nout + n;
        return goutf ? __float2bfloat16_rn(goutf[o]) : gout[o];
    }
    __device__ __forceinline__ int vecA() const { return Kin % 8 == 0 ? kVecAm : kVecANone; }
    __device__ __forceinline__ uint4 loadA8(int m, int k) const {
        if (m == Kin) return make_uint4((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(1.f)), 0u, 0u, 0u);
        return ld16(in + (size_t)k * Kin + m);
    }
    __device__ __forceinline__ int vecB() const { return goutf == nullptr && Nout % 8 == 0 ? kVecBn : kVecBNone; }
    __device__ __forceinline__ uint4 loadB8(int k, int n) const { return ld16(gout + (size_t)k * Nout + n); }
    __device__ __forceinline__ void store(int m, int n, float v) const {
        if (m == Kin) atomicAdd(&db[n], v);
        else atomicAdd(&dW[(size_t)m * Nout + n], v);
    }
    __device__ __forceinline__ void store_row(int m, int c0, const float (&v)[16], int nv) const {
        add_f32_row(m == Kin ? db + c0 : dW + (size_t)m * Nout + c0, v, nv);
    }
};

// second stage of a split-K GEMM whose epilogue is not additive: the partial
// tiles are summed in split order (deterministic) and the epilogue applied
template <class P>
__global__ void splitk_reduce(P p, const float* scratch, int M, int N, int splits) {
    pdl_start();
    const size_t MN = (size_t)M * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < MN; i += (size_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int z = 0; z < splits; ++z) acc += scratch[z * MN + i];
        p.store((int)(i / N), (int)(i % N), acc);
    }
}

// scratch of the split-K forward GEMMs: at most kFwdSplitCtas partial tiles of 64 x 64
constexpr int kFwdSplitCtas = 2 * 152;
constexpr size_t kSplitScratchFloats = (size_t)kFwdSplitCtas * 64 * 64;

// The GEMM's shared memory exceeds the default 48 KB, so each problem type's kernel
// needs the attribute once per device.  Set outside any stream capture: the
// workspace-size query does it first, and the passes only read the cached verdict.
template <class P>
static bool gemm_attr() {
    return cudaFuncSetAttribute(gemm_tc<P, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TileCfg<32>::kSmem) ==
               cudaSuccess &&
           cudaFuncSetAttribute(gemm_tc<P, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, TileCfg<64>::kSmem) ==
               cudaSuccess;
}

static bool gemm_prepared() {
    static std::atomic<int> cached[64];   // 0 unknown, 1 set, 2 failed
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return false;
    }
    int c = cached[dev].load(std::memory_order_relaxed);
    if (c == 0) {
        const bool ok = gemm_attr<ConvFwd>() && gemm_attr<FcFwd>() && gemm_attr<ConvDgrad>() && gemm_attr<FcDgrad>() &&
                        gemm_attr<ConvWgrad>() && gemm_attr<FcWgrad>();
        (void)cudaGetLastError();
        c = ok ? 1 : 2;
        cached[dev].store(c, std::memory_order_relaxed);
    }
    return c == 1;
}

static int tile_n(int N) { return N <= 32 ? 32 : 64; }

template <class P>
static cudaError_t gemm(const P& p, int M, int N, int K, int splits, cudaStream_t s, float* scratch = nullptr) {
    if (!gemm_prepared()) return cudaErrorInvalidDeviceFunction;
    if (splits < 1) splits = 1;
    int kchunk = ((K + splits - 1) / splits + TK - 1) / TK * TK;
    if (kchunk < TK) kchunk = TK;
    splits = (K + kchunk - 1) / kchunk;
    const int tn = tile_n(N);
    dim3 grid((unsigned)((M + TM - 1) / TM), (unsigned)((N + tn - 1) / tn), (unsigned)splits);
    float* const sc = splits > 1 ? scratch : nullptr;
    cudaError_t e = tn == 32 ? launch_pdl(gemm_tc<P, 32>, grid, dim3(GEMM_NT), TileCfg<32>::kSmem, s, p, M, N, K, kchunk, sc)
                             : launch_pdl(gemm_tc<P, 64>, grid, dim3(GEMM_NT), TileCfg<64>::kSmem, s, p, M, N, K, kchunk, sc);
    if (e != cudaSuccess) return e;
    if (splits > 1 && scratch) {
        const size_t MN = (size_t)M * N;
        const unsigned nb = (unsigned)((MN + 255) / 256 < 1024 ? (MN + 255) / 256 : 1024);
        e = launch_pdl(splitk_reduce<P>, dim3(nb), dim3(256), 0, s, p, (const float*)scratch, M, N, splits);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// split-K factor of a forward GEMM: enough CTAs to cover the GPU when the output
// tile grid is small, each split at least one 64-wide K-slice, partial tiles
// within the scratch
static int fwd_splits(int M, int N, int K) {
    const long long tiles = (long long)((M + TM - 1) / TM) * ((N + tile_n(N) - 1) / tile_n(N));
    if (tiles >= 152) return 1;
    long long s = (152 + tiles - 1) / tiles;
    const long long ksteps = (K + TK - 1) / TK;
    if (s > ksteps) s = ksteps;
    while (s > 1 && s * M * (long long)N > (long long)kSplitScratchFloats) --s;
    return (int)(s < 1 ? 1 : s);
}

// split-K factor for a weight-gradient GEMM (FP32 atomics sum the slices): about four
// waves of CTAs (four fit an SM), each at least two 64-wide K-slices
static int wgrad_splits(int M, int N, long long K) {
    const long long tiles = (long long)((M + TM - 1) / TM) * ((N + tile_n(N) - 1) / tile_n(N));
    long long s = (4 * 152 + tiles - 1) / tiles;
    const long long most = (K + 2 * TK - 1) / (2 * TK);
    if (s > most) s = most;
    return (int)(s < 1 ? 1 : s);
}

// ---------------------------------------------------------------- elementwise kernels
__global__ void to_bf16_kernel(const float* src, bf16* dst, size_t n) {
    pdl_start();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", 2014)
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct InitSpans {
    unsigned long long w0[RGBID_NET_LAYERS], n[RGBID_NET_LAYERS];
    int fan_in[RGBID_NET_LAYERS];
};

__global__ void init_kernel(float* p, unsigned long long seed, InitSpans sp) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    float v = 0.f;
#pragma unroll
    for (int l = 0; l < RGBID_NET_LAYERS; ++l) {
        if (i >= sp.w0[l] && i < sp.w0[l] + sp.n[l]) {
            const double u = (double)(splitmix64(seed ^ (0xA24BAED4963EE407ull * (i + 1))) >> 11) * (1.0 / 9007199254740992.0);
            v = (float)((2.0 * u - 1.0) * sqrt(6.0 / sp.fan_in[l]));
        }
    }
    p[i] = v;
}

// mean Gaussian NLL over the batch and dL/dy; one block, fixed summation order
__global__ void loss_kernel(const float* y, const float* tgt, int B, float* dy, float* loss) {
    __shared__ double part[256];
    double acc = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float* yb = y + (size_t)b * RGBID_NET_OUT;
        const float s = yb[6];
        const float e = expf(-s);
        float sq = 0.f;
        float d[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            d[i] = yb[i] - tgt[(size_t)b * 6 + i];
            sq = fmaf(d[i], d[i], sq);
        }
        const float invB = 1.f / (float)B;
#pragma unroll
        for (int i = 0; i < 6; ++i) dy[(size_t)b * RGBID_NET_OUT + i] = e * d[i] * invB;
        dy[(size_t)b * RGBID_NET_OUT + 6] = (-0.5f * e * sq + 3.f) * invB;
        acc += 0.5 * (double)e * (double)sq + 3.0 * (double)s;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(part[0] / B);
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// one block per item; x[n][v][u][c] from the 80x60 level of its ref (A) and cur (B) pyramids
__global__ void inputs_kernel(const rgbid_batch_item* items, int precision, bf16* x) {
    pdl_start();
    const rgbid_batch_item* it = items + blockIdx.x;
    __shared__ int lv;
    if (threadIdx.x == 0) {
        int found = -1;
        const int L = it->ref.levels < RGBID_MAX_LEVELS ? it->ref.levels : RGBID_MAX_LEVELS;
        for (int l = 0; l < L && l < it->cur.levels; ++l)
            if (it->ref.lv[l].width == RGBID_NET_IN_W && it->ref.lv[l].height == RGBID_NET_IN_H &&
                it->cur.lv[l].width == RGBID_NET_IN_W && it->cur.lv[l].height == RGBID_NET_IN_H &&
                it->ref.lv[l].IW && it->cur.lv[l].IW &&
                !((uintptr_t)it->ref.lv[l].IW & (precision == RGBID_PLANES_F32 ? 7u : 3u)) &&
                !((uintptr_t)it->cur.lv[l].IW & (precision == RGBID_PLANES_F32 ? 7u : 3u)) &&
                it->ref.lv[l].pitch >= RGBID_NET_IN_W &&
                it->cur.lv[l].pitch >= RGBID_NET_IN_W && it->ref.precision == precision &&
                it->cur.precision == precision)
                found = l;
        lv = found;
    }
    __syncthreads();
    bf16* out = x + (size_t)blockIdx.x * kInPerSample;
    for (int p = threadIdx.x; p < RGBID_NET_IN_H * RGBID_NET_IN_W; p += blockDim.x) {
        const int v = p / RGBID_NET_IN_W, u = p - v * RGBID_NET_IN_W;
        float vals[4] = {0.f, 0.f, 0.f, 0.f};
        if (lv >= 0) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const rgbid_level& L = side ? it->cur.lv[lv] : it->ref.lv[lv];
                const size_t idx = (size_t)v * L.pitch + u;
                float I, W;
                if (precision == RGBID_PLANES_F32) {
                    const float2 q = reinterpret_cast<const float2*>(L.IW)[idx];
                    I = q.x;
                    W = q.y;
                } else {
                    const uint32_t raw = reinterpret_cast<const uint32_t*>(L.IW)[idx];
                    I = __bfloat162float(__ushort_as_bfloat16((unsigned short)(raw & 0xffffu)));
                    W = __half2float(__ushort_as_half((unsigned short)(raw >> 16)));
                }
                vals[2 * side] = I - 0.5f;
                vals[2 * side + 1] = W;
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) out[(size_t)p * 4 + c] = __float2bfloat16_rn(vals[c]);
    }
}

// one warp per item: copy d_in[i] to d_out[i]; in tier k (log-variance below
// thr[k - 1], largest such k) set T_init to the proposed pose and zero the
// iterations of the k coarsest levels
struct Tiers {
    float thr[RGBID_NET_MAX_TIERS];
    int n;
};

__global__ void plan_kernel(const float* y, int n, Tiers tiers, const rgbid_batch_item* d_in, rgbid_batch_item* d_out,
                            int* skipped) {
    pdl_start();
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    static_assert(sizeof(rgbid_batch_item) % 8 == 0, "copied as 8-byte words");
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(d_in + i);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(d_out + i);
    for (int w = lane; w < (int)(sizeof(rgbid_batch_item) / 8); w += 32) dst[w] = src[w];
    __syncwarp();
    if (lane != 0) return;
    const float* yi = y + (size_t)i * RGBID_NET_OUT;
    rgbid_batch_item& o = d_out[i];
    const int L = o.levels < 1 ? 1 : (o.levels > RGBID_MAX_LEVELS ? RGBID_MAX_LEVELS : o.levels);
    int k = 0;
    for (int t = 0; t < tiers.n; ++t)
        if (yi[6] < tiers.thr[t]) k = t + 1;
    if (k > L - 1) k = L - 1;
    if (skipped) skipped[i] = k;
    if (k == 0) return;
    const double sc = RGBID_NET_TWIST_SCALE;
    const double t[3] = {yi[0] * sc, yi[1] * sc, yi[2] * sc};
    const double w[3] = {yi[3] * sc, yi[4] * sc, yi[5] * sc};
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double A, B;
    if (th2 < 1e-12) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
    } else {
        const double th = sqrt(th2);
        A = sin(th) / th;
        const double sh = sin(0.5 * th);
        B = 2.0 * sh * sh / th2;
    }
    // R = I + A [w]x + B ([w]x)^2, ([w]x)^2 = w w^T - th2 I
    const double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c)
            o.T_init[r * 4 + c] = (r == c ? 1.0 : 0.0) + A * K[r * 3 + c] + B * (w[r] * w[c] - (r == c ? th2 : 0.0));
        o.T_init[r * 4 + 3] = t[r];
    }
    o.T_init[12] = 0.0;
    o.T_init[13] = 0.0;
    o.T_init[14] = 0.0;
    o.T_init[15] = 1.0;
    for (int q = 0; q < k; ++q) o.iters[L - 1 - q] = 0;
}

// ---------------------------------------------------------------- workspace
struct Ws {
    bf16* wb;                         // bf16 weights
    bf16* act[RGBID_NET_LAYERS - 1];  // outputs of c1..f1
    bf16* g0;                         // activation-gradient ping-pong buffers
    bf16* g1;
    float* split;                     // partial tiles of split-K forward GEMMs
};

static size_t ws_layout(int batch, char* base, Ws* w) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += align_up(bytes, 256);
        return p;
    };
    bf16* wb = (bf16*)take(kParams * sizeof(bf16));
    bf16* act[RGBID_NET_LAYERS - 1];
    for (int l = 0; l < RGBID_NET_LAYERS - 1; ++l) act[l] = (bf16*)take((size_t)batch * act_per_sample(l) * sizeof(bf16));
    bf16* g0 = (bf16*)take((size_t)batch * kMaxGradPerSample * sizeof(bf16));
    bf16* g1 = (bf16*)take((size_t)batch * kMaxGradPerSample * sizeof(bf16));
    float* split = (float*)take(kSplitScratchFloats * sizeof(float));
    if (w) {
        w->wb = wb;
        for (int l = 0; l < RGBID_NET_LAYERS - 1; ++l) w->act[l] = act[l];
        w->g0 = g0;
        w->g1 = g1;
        w->split = split;
    }
    return off;
}

static ConvGeo geo_of(int l) {
    const LayerDef& d = kLayers[l];
    return ConvGeo{d.hin, d.win, d.cin, d.hout, d.wout, d.cout};
}

static int check_ws(int batch, void* ws, size_t bytes, Ws* w) {
    if (batch < 1 || batch > 65536) return RGBID_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & 255u) || bytes < ws_layout(batch, nullptr, nullptr)) return RGBID_ERR_WORKSPACE;
    ws_layout(batch, (char*)ws, w);
    return RGBID_OK;
}

}  // namespace net
}  // namespace rgbid

using namespace rgbid;
using namespace rgbid::net;

extern "C" size_t rgbid_net_param_count(void) { return kParams; }

extern "C" size_t rgbid_net_param_offset(int layer, int what) {
    if (layer < 0 || layer >= RGBID_NET_LAYERS || (what != 0 && what != 1)) return (size_t)-1;
    static const size_t w[RGBID_NET_LAYERS] = {w_offset(0), w_offset(1), w_offset(2), w_offset(3), w_offset(4), w_offset(5)};
    static const size_t b[RGBID_NET_LAYERS] = {b_offset(0), b_offset(1), b_offset(2), b_offset(3), b_offset(4), b_offset(5)};
    return what == 0 ? w[layer] : b[layer];
}

extern "C" size_t rgbid_net_workspace_bytes(int batch) {
    if (batch < 1 || batch > 65536) return 0;
    (void)gemm_prepared();   // the kernels' attributes, before the passes can be captured
    return ws_layout(batch, nullptr, nullptr);
}

extern "C" unsigned int rgbid_net_wait_timeouts(void) {
    unsigned int n = 0;
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpyFromSymbol(&n, g_mma_timeouts, sizeof(n)) != cudaSuccess) {
        (void)cudaGetLastError();
        return (unsigned int)-1;
    }
    return n;
}

extern "C" int rgbid_net_init(float* params, unsigned long long seed, void* stream) {
    if (!params || misaligned(params, 4)) return RGBID_ERR_INVALID_ARG;
    InitSpans sp;
    for (int l = 0; l < RGBID_NET_LAYERS; ++l) {
        sp.w0[l] = w_offset(l);
        sp.n[l] = weight_count(l);
        sp.fan_in[l] = kLayers[l].kind == kConv ? 9 * kLayers[l].cin : kLayers[l].cin;
    }
    init_kernel<<<(unsigned)((kParams + 255) / 256), 256, 0, (cudaStream_t)stream>>>(params, seed, sp);
    return cudaGetLastError() == cudaSuccess ? RGBID_OK : RGBID_ERR_CUDA;
}

extern "C" int rgbid_net_inputs(const rgbid_batch_item* d_items, int n, int precision, void* x, void* stream) {
    if (n < 0 || (n > 0 && (!d_items || !x))) return RGBID_ERR_INVALID_ARG;
    if (misaligned(d_items, 8) || misaligned(x, 4)) return RGBID_ERR_INVALID_ARG;
    if (precision != RGBID_PLANES_F32 && precision != RGBID_PLANES_BF16_F16) return RGBID_ERR_UNSUPPORTED;
    if (n == 0) return RGBID_OK;
    return launch_pdl(inputs_kernel, dim3((unsigned)n), dim3(256), 0, (cudaStream_t)stream, d_items, precision,
                      (bf16*)x) == cudaSuccess
               ? RGBID_OK
               : RGBID_ERR_CUDA;
}

extern "C" int rgbid_net_forward(const float* params, const void* x, int batch, float* y, void* workspace,
                                 size_t workspace_bytes, void* stream_) {
    if (!params || !x || !y) return RGBID_ERR_INVALID_ARG;
    if (misaligned(params, 4) || misaligned(x, 4) || misaligned(y, 4)) return RGBID_ERR_INVALID_ARG;
    Ws w;
    const int rc = check_ws(batch, workspace, workspace_bytes, &w);
    if (rc != RGBID_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream_;
    if (launch_pdl(to_bf16_kernel, dim3(256), dim3(256), 0, s, params, w.wb, kParams) != cudaSuccess) return RGBID_ERR_CUDA;
    const bf16* in = (const bf16*)x;
    for (int l = 0; l < RGBID_NET_LAYERS; ++l) {
        const LayerDef& d = kLayers[l];
        const bf16* W = w.wb + w_offset(l);
        const float* bias = params + b_offset(l);
        cudaError_t e;
        if (d.kind == kConv) {
            ConvFwd p{geo_of(l), in, W, bias, w.act[l]};
            const int M = batch * d.hout * d.wout;
            e = gemm(p, M, d.cout, 9 * d.cin, fwd_splits(M, d.cout, 9 * d.cin), s, w.split);
        } else {
            const bool last = l == RGBID_NET_LAYERS - 1;
            FcFwd p{in, W, bias, last ? nullptr : w.act[l], last ? y : nullptr, d.cin, d.cout};
            e = gemm(p, batch, d.cout, d.cin, fwd_splits(batch, d.cout, d.cin), s, w.split);
        }
        if (e != cudaSuccess) return RGBID_ERR_CUDA;
        if (l < RGBID_NET_LAYERS - 1) in = w.act[l];
    }
    return RGBID_OK;
}

extern "C" int rgbid_net_backward(const float* params, const void* x, int batch, const float* dy, float* grad,
                                  void* workspace, size_t workspace_bytes, void* stream_) {
    if (!params || !x || !dy || !grad) return RGBID_ERR_INVALID_ARG;
    if (misaligned(params, 4) || misaligned(x, 4) || misaligned(dy, 4) || misaligned(grad, 4)) return RGBID_ERR_INVALID_ARG;
    Ws w;
    const int rc = check_ws(batch, workspace, workspace_bytes, &w);
    if (rc != RGBID_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream_;
    if (cudaMemsetAsync(grad, 0, kParams * sizeof(float), s) != cudaSuccess) return RGBID_ERR_CUDA;
    const bf16* gout = nullptr;    // bf16 gradient w.r.t. layer l's output (nullptr: the float32 dy)
    bf16* bufs[2] = {w.g0, w.g1};
    int next = 0;
    for (int l = RGBID_NET_LAYERS - 1; l >= 0; --l) {
        const LayerDef& d = kLayers[l];
        const bf16* W = w.wb + w_offset(l);
        const bf16* a_in = l == 0 ? (const bf16*)x : w.act[l - 1];
        float* dW = grad + w_offset(l);
        float* db = grad + b_offset(l);
        bf16* gin = bufs[next];
        cudaError_t e;
        if (d.kind == kConv) {
            const ConvGeo geo = geo_of(l);
            const long long K = (long long)batch * d.hout * d.wout;
            ConvWgrad pw{geo, a_in, gout, dW, db};
            e = gemm(pw, 9 * d.cin + 1, d.cout, (int)K, wgrad_splits(9 * d.cin + 1, d.cout, K), s);
            if (e == cudaSuccess && l > 0) {
                ConvDgrad pd{geo, gout, W, a_in, gin};
                e = gemm(pd, batch * d.hin * d.win, d.cin, 9 * d.cout, 1, s);
            }
        } else {
            const float* goutf = gout ? nullptr : dy;
            FcWgrad pw{a_in, gout, goutf, dW, db, d.cin, d.cout};
            e = gemm(pw, d.cin + 1, d.cout, batch, wgrad_splits(d.cin + 1, d.cout, batch), s);
            if (e == cudaSuccess && l > 0) {
                FcDgrad pd{gout, goutf, W, a_in, gin, d.cin, d.cout};
                e = gemm(pd, batch, d.cin, d.cout, 1, s);
            }
        }
        if (e != cudaSuccess) return RGBID_ERR_CUDA;
        gout = gin;
        next ^= 1;
    }
    return RGBID_OK;
}

extern "C" int rgbid_net_loss(const float* y, const float* target, int batch, float* dy, float* loss, void* stream) {
    if (!y || !target || !dy || !loss || batch < 1) return RGBID_ERR_INVALID_ARG;
    if (misaligned(y, 4) || misaligned(target, 4) || misaligned(dy, 4) || misaligned(loss, 4)) return RGBID_ERR_INVALID_ARG;
    loss_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(y, target, batch, dy, loss);
    return cudaGetLastError() == cudaSuccess ? RGBID_OK : RGBID_ERR_CUDA;
}

extern "C" int rgbid_net_adam(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                              float beta2, float eps, void* stream) {
    if (!params || !grad || !m || !v || step < 1) return RGBID_ERR_INVALID_ARG;
    if (misaligned(params, 4) || misaligned(grad, 4) || misaligned(m, 4) || misaligned(v, 4)) return RGBID_ERR_INVALID_ARG;
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f)) return RGBID_ERR_INVALID_ARG;
    const float c1 = (float)(1.0 / (1.0 - pow((double)beta1, step)));
    const float c2 = (float)(1.0 / (1.0 - pow((double)beta2, step)));
    adam_kernel<<<512, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, kParams, lr, beta1, beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? RGBID_OK : RGBID_ERR_CUDA;
}

extern "C" int rgbid_net_plan(const float* y, int n, const float* max_log_var, int n_tiers,
                              const rgbid_batch_item* d_in, rgbid_batch_item* d_out, int* skipped, void* stream) {
    if (n < 0 || (n > 0 && (!y || !d_in || !d_out)) || n_tiers < 0 || n_tiers > RGBID_NET_MAX_TIERS)
        return RGBID_ERR_INVALID_ARG;
    if (n_tiers > 0 && !max_log_var) return RGBID_ERR_INVALID_ARG;
    if (d_in == d_out) return RGBID_ERR_INVALID_ARG;
    if (misaligned(y, 4) || misaligned(d_in, 8) || misaligned(d_out, 8) || misaligned(skipped, 4))
        return RGBID_ERR_INVALID_ARG;
    if (n == 0) return RGBID_OK;
    Tiers tiers;
    tiers.n = n_tiers;
    for (int t = 0; t < RGBID_NET_MAX_TIERS; ++t) tiers.thr[t] = t < n_tiers ? max_log_var[t] : -3.0e38f;
    return launch_pdl(plan_kernel, dim3((unsigned)((n + 7) / 8)), dim3(256), 0, (cudaStream_t)stream, y, n, tiers,
                      d_in, d_out, skipped) == cudaSuccess
               ? RGBID_OK
               : RGBID_ERR_CUDA;
}
