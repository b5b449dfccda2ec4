// Learned initialiser: forward and backward passes of the network on bfloat16
// tensor cores, its loss, Adam, parameter initialisation, input packing from
// pyramid levels, and the plan that turns proposals into batch items.
//
// Every layer pass is one implicit GEMM C[M x N] = A[M x K] B[K x N] computed
// by mma.sync.m16n8k16 (bf16 operands, FP32 accumulation) in 64 x 64 tiles
// with K-steps of 32; a problem type supplies how A and B elements are
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

// ---------------------------------------------------------------- GEMM core
constexpr int BM = 64, BN = 64, BK = 32, LDS = BK + 8, GEMM_NT = 128;
constexpr int kVecBNone = 0, kVecBk = 1, kVecBn = 2;   // how B may be loaded 8 elements at a time
constexpr int kVecANone = 0, kVecAk = 1, kVecAm = 2;   // how A may be loaded 8 elements at a time

__device__ __forceinline__ uint4 ld16(const bf16* p) { return *reinterpret_cast<const uint4*>(p); }

__device__ __forceinline__ uint32_t ld_pair(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C tile (blockIdx.x, blockIdx.y) over the K range of blockIdx.z; 4 warps in a
// 2 x 2 arrangement, each 32 x 32 = 2 (m16) x 4 (n8) mma tiles.
template <class P>
__global__ void __launch_bounds__(GEMM_NT) gemm_bf16(P p, int M, int N, int K, int kchunk, float* scratch) {
    __shared__ __align__(16) bf16 As[BM][LDS];
    __shared__ __align__(16) bf16 Bs[BN][LDS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * kchunk;
    const int kb1 = min(K, kb0 + kchunk);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    // Vector loaders: 8 bf16 (16 bytes) per load where the operand is contiguous along
    // k (A; B with kVecBk) or along n (B with kVecBn); the problem type says when its
    // layout allows it (channel counts that are multiples of 8, so that every vector
    // stays inside one tap and is 16-byte aligned, and K a multiple of 8, so that a
    // vector that starts before the end of the K range ends before it too).
    const bool vecAk = p.vecA() == kVecAk, vecAm = p.vecA() == kVecAm;
    const bool vecBk = p.vecB() == kVecBk, vecBn = p.vecB() == kVecBn;
    for (int k0 = kb0; k0 < kb1; k0 += BK) {
        if (vecAk) {
            for (int i = tid; i < BM * BK / 8; i += GEMM_NT) {
                const int r = i >> 2, c8 = (i & 3) * 8;
                const int m = m0 + r, k = k0 + c8;
                *reinterpret_cast<uint4*>(&As[r][c8]) = (m < M && k < kb1) ? p.loadA8(m, k) : make_uint4(0u, 0u, 0u, 0u);
            }
        } else if (vecAm) {
            // 8 consecutive rows m of one column k (the problem zero-fills rows from M on)
            for (int i = tid; i < BK * BM / 8; i += GEMM_NT) {
                const int c = i >> 3, m8 = (i & 7) * 8;
                const int k = k0 + c, m = m0 + m8;
                const uint4 v = (k < kb1 && m < M) ? p.loadA8(m, k) : make_uint4(0u, 0u, 0u, 0u);
                const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
                for (int j = 0; j < 8; ++j) As[m8 + j][c] = e[j];
            }
        } else {
            for (int i = tid; i < BM * BK; i += GEMM_NT) {
                const int r = i >> 5, c = i & 31;
                const int m = m0 + r, k = k0 + c;
                As[r][c] = (m < M && k < kb1) ? p.loadA(m, k) : bz();
            }
        }
        if (vecBk) {
            for (int i = tid; i < BN * BK / 8; i += GEMM_NT) {
                const int r = i >> 2, c8 = (i & 3) * 8;
                const int n = n0 + r, k = k0 + c8;
                *reinterpret_cast<uint4*>(&Bs[r][c8]) = (n < N && k < kb1) ? p.loadB8(k, n) : make_uint4(0u, 0u, 0u, 0u);
            }
        } else if (vecBn) {
            for (int i = tid; i < BK * BN / 8; i += GEMM_NT) {
                const int c = i >> 3, n8 = (i & 7) * 8;
                const int k = k0 + c, n = n0 + n8;
                const uint4 v = (k < kb1 && n < N) ? p.loadB8(k, n) : make_uint4(0u, 0u, 0u, 0u);
                const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
                for (int j = 0; j < 8; ++j) Bs[n8 + j][c] = e[j];
            }
        } else {
            for (int i = tid; i < BN * BK; i += GEMM_NT) {
                const int r = i >> 5, c = i & 31;
                const int n = n0 + r, k = k0 + c;
                Bs[r][c] = (n < N && k < kb1) ? p.loadB(k, n) : bz();
            }
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int rb = wm * 32 + mi * 16;
                a[mi][0] = ld_pair(&As[rb + g][ks + 2 * t]);
                a[mi][1] = ld_pair(&As[rb + g + 8][ks + 2 * t]);
                a[mi][2] = ld_pair(&As[rb + g][ks + 2 * t + 8]);
                a[mi][3] = ld_pair(&As[rb + g + 8][ks + 2 * t + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int cb = wn * 32 + ni * 8;
                b[ni][0] = ld_pair(&Bs[cb + g][ks + 2 * t]);
                b[ni][1] = ld_pair(&Bs[cb + g][ks + 2 * t + 8]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const int r = m0 + wm * 32 + mi * 16 + g;
            const int c = n0 + wn * 32 + ni * 8 + 2 * t;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int rr = r + (q >> 1) * 8, cc = c + (q & 1);
                if (rr < M && cc < N) {
                    if (scratch) scratch[((size_t)blockIdx.z * M + rr) * N + cc] = acc[mi][ni][q];
                    else p.store(rr, cc, acc[mi][ni][q]);
                }
            }
        }
    }
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
    __device__ __forceinline__ int vecA() const { return geo.C % 8 == 0 ? kVecAk : kVecANone; }
    __device__ __forceinline__ uint4 loadA8(int m, int k) const { return geo.patch8(in, m, k); }
    __device__ __forceinline__ int vecB() const { return geo.Co % 8 == 0 ? kVecBn : kVecBNone; }
    __device__ __forceinline__ uint4 loadB8(int k, int n) const { return ld16(W + (size_t)k * geo.Co + n); }
    __device__ __forceinline__ void store(int m, int n, float v) const {
        out[(size_t)m * geo.Co + n] = __float2bfloat16_rn(fmaxf(v + bias[n], 0.f));
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
    __device__ __forceinline__ int vecA() const { return geo.C % 8 == 0 ? kVecAm : kVecANone; }
    __device__ __forceinline__ uint4 loadA8(int m, int k) const {
        if (m == 9 * geo.C) return make_uint4((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(1.f)), 0u, 0u, 0u);
        return geo.patch8(in, k, m);
    }
    __device__ __forceinline__ int vecB() const { return geo.Co % 8 == 0 ? kVecBn : kVecBNone; }
    __device__ __forceinline__ uint4 loadB8(int k, int n) const { return ld16(gout + (size_t)k * geo.Co + n); }
    __device__ __forceinline__ void store(int m, int n, float v) const {
        if (m == 9 * geo.C) atomicAdd(&db[n], v);
        else atomicAdd(&dW[(size_t)m * geo.Co + n], v);
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
};

// second stage of a split-K GEMM whose epilogue is not additive: the partial
// tiles are summed in split order (deterministic) and the epilogue applied
template <class P>
__global__ void splitk_reduce(P p, const float* scratch, int M, int N, int splits) {
    const size_t MN = (size_t)M * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < MN; i += (size_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int z = 0; z < splits; ++z) acc += scratch[z * MN + i];
        p.store((int)(i / N), (int)(i % N), acc);
    }
}

// scratch of the split-K forward GEMMs: at most kFwdSplitCtas partial tiles of 64 x 64
constexpr int kFwdSplitCtas = 2 * 152;
constexpr size_t kSplitScratchFloats = (size_t)kFwdSplitCtas * BM * BN;

template <class P>
static cudaError_t gemm(const P& p, int M, int N, int K, int splits, cudaStream_t s, float* scratch = nullptr) {
    if (splits < 1) splits = 1;
    int kchunk = ((K + splits - 1) / splits + BK - 1) / BK * BK;
    if (kchunk < BK) kchunk = BK;
    splits = (K + kchunk - 1) / kchunk;
    dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((N + BN - 1) / BN), (unsigned)splits);
    gemm_bf16<P><<<grid, GEMM_NT, 0, s>>>(p, M, N, K, kchunk, splits > 1 ? scratch : nullptr);
    if (splits > 1 && scratch) {
        const size_t MN = (size_t)M * N;
        splitk_reduce<P><<<(unsigned)((MN + 255) / 256 < 1024 ? (MN + 255) / 256 : 1024), 256, 0, s>>>(p, scratch, M, N,
                                                                                                    splits);
    }
    return cudaGetLastError();
}

// split-K factor of a forward GEMM: enough CTAs to cover the GPU when the output
// tile grid is small, each split at least one 32-wide K-step, partial tiles
// within the scratch
static int fwd_splits(int M, int N, int K) {
    const long long tiles = (long long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    if (tiles >= 152) return 1;
    long long s = (152 + tiles - 1) / tiles;
    const long long ksteps = (K + BK - 1) / BK;
    if (s > ksteps) s = ksteps;
    while (s > 1 && s * M * (long long)N > (long long)kSplitScratchFloats) --s;
    return (int)(s < 1 ? 1 : s);
}

// split-K factor for a weight-gradient GEMM: about 1024 reduction elements per CTA, at most 512 slices
static int wgrad_splits(long long K) {
    long long s = (K + 1023) / 1024;
    return (int)(s < 1 ? 1 : (s > 512 ? 512 : s));
}

// ---------------------------------------------------------------- elementwise kernels
__global__ void to_bf16_kernel(const float* src, bf16* dst, size_t n) {
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
    return ws_layout(batch, nullptr, nullptr);
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
    inputs_kernel<<<(unsigned)n, 256, 0, (cudaStream_t)stream>>>(d_items, precision, (bf16*)x);
    return cudaGetLastError() == cudaSuccess ? RGBID_OK : RGBID_ERR_CUDA;
}

extern "C" int rgbid_net_forward(const float* params, const void* x, int batch, float* y, void* workspace,
                                 size_t workspace_bytes, void* stream_) {
    if (!params || !x || !y) return RGBID_ERR_INVALID_ARG;
    if (misaligned(params, 4) || misaligned(x, 4) || misaligned(y, 4)) return RGBID_ERR_INVALID_ARG;
    Ws w;
    const int rc = check_ws(batch, workspace, workspace_bytes, &w);
    if (rc != RGBID_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream_;
    to_bf16_kernel<<<256, 256, 0, s>>>(params, w.wb, kParams);
    if (cudaGetLastError() != cudaSuccess) return RGBID_ERR_CUDA;
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
            e = gemm(pw, 9 * d.cin + 1, d.cout, (int)K, wgrad_splits(K), s);
            if (e == cudaSuccess && l > 0) {
                ConvDgrad pd{geo, gout, W, a_in, gin};
                e = gemm(pd, batch * d.hin * d.win, d.cin, 9 * d.cout, 1, s);
            }
        } else {
            const float* goutf = gout ? nullptr : dy;
            FcWgrad pw{a_in, gout, goutf, dW, db, d.cin, d.cout};
            e = gemm(pw, d.cin + 1, d.cout, batch, wgrad_splits(batch), s);
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
    plan_kernel<<<(unsigned)((n + 7) / 8), 256, 0, (cudaStream_t)stream>>>(y, n, tiers, d_in, d_out, skipped);
    return cudaGetLastError() == cudaSuccess ? RGBID_OK : RGBID_ERR_CUDA;
}
