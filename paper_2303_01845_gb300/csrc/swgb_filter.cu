// swgb_filter.cu -- the learned candidate filter's network on sm_103a: a
// 32 -> 64 -> 128 -> 1 perceptron with ReLU, BF16 weights and activations and
// FP32 accumulation, its forward pass (inference), its gradient of a weighted
// binary cross-entropy, and Adam, with their C-ABI entry points.
//
// The paper keeps a candidate when it shares at least two k-mers (program-
// parameters table) and observes that few candidates end up in the similarity
// graph (Sec. "Blocked 2D Sparse SUMMA"); the network scores candidates from
// their k-mer features so that most of those that would fail the identity and
// coverage filter are never aligned.  Its definition (rounding points
// included) is stated in include/swgb.h.
//
// Layout of the work: a warp owns a tile of 16 samples and runs the whole
// network on it with the bf16 tensor-core instruction mma.m16n8k16 (FP32
// accumulators).  A layer's accumulator fragments (16 x 8 per n-tile, two
// columns per thread) are exactly the A-operand fragments of the next layer's
// k-slices once biased, rectified and rounded to bf16, so activations never
// leave registers.  The backward pass chains the same way (dz2 -> dz1); the
// weight gradients, contractions over the samples, go through shared memory:
// the four warps of a block write their tiles' activations and gradients
// sample-minor, then each warp accumulates one slice of dW2 (and of dW1) in
// registers across every tile the block processes, and adds it to the global
// gradient once at the end.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "swgb_host.cuh"

namespace swgb {
namespace {

constexpr int kIn = 32, kH1 = 64, kH2 = 128;
// packed parameter offsets: W1 [32][64] (row = input), b1, W2 [64][128], b2, w3, b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kIn * kH1;
constexpr int kOffW2 = kOffB1 + kH1;
constexpr int kOffB2 = kOffW2 + kH1 * kH2;
constexpr int kOffW3 = kOffB2 + kH2;
constexpr int kOffB3 = kOffW3 + kH2;
constexpr int kParams = kOffB3 + 1;
static_assert(kParams == SWGB_MLP_PARAMS, "parameter count");

// bf16 weight copies in shared memory, rows padded against bank conflicts
constexpr int kW1tStride = kIn + 8;    // w1t[out][in]
constexpr int kW2tStride = kH1 + 8;    // w2t[out][in]
constexpr int kW2Stride = kH2 + 8;     // w2[in][out]
constexpr int kWarps = 4;
constexpr int kTileRows = 16;
constexpr int kBlockRows = kWarps * kTileRows;   // samples per block step
constexpr int kTStride = kBlockRows + 8;         // sample-minor staging rows

struct MlpArgs {
    const float* params;          // fp32 master, packed
    const __nv_bfloat16* w1t;     // [64][32]
    const __nv_bfloat16* w2t;     // [128][64]
    const __nv_bfloat16* w2;      // [64][128]
    const float* x;               // [*][32]
    const float* y;               // [*] labels 0 / 1 (gradient)
    const int32_t* order;         // sample ids of the batch, or null: first..first+n
    int64_t first, n;
    float pos_weight;
    float* logits;                // [n] (forward)
    float* grad;                  // [kParams] (gradient)
    float* loss;                  // [1] (gradient: sum of weighted losses / n)
    float* part;                  // [blocks][kParams + 1] per-block sums (gradient, loss last)
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }
__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// D = A (16x16, row) * B (16x8, col) + D, bf16 inputs, fp32 accumulators
__device__ __forceinline__ void mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                    uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

// Shared memory of both kernels; the forward kernel uses the part before w2.
struct Smem {
    __nv_bfloat16 w1t[kH1 * kW1tStride];
    __nv_bfloat16 w2t[kH2 * kW2tStride];
    float b1[kH1], b2[kH2], w3[kH2];
    __nv_bfloat16 w2[kH1 * kW2Stride];
    // gradient staging (sample-minor): x^T, a1^T, dz1^T, dz2^T of a block step
    __nv_bfloat16 xt[kIn * kTStride];
    __nv_bfloat16 a1t[kH1 * kTStride];
    __nv_bfloat16 dz1t[kH1 * kTStride];
    __nv_bfloat16 dz2t[kH2 * kTStride];
    // per-warp sums of the bias gradients, w3's gradient and the loss, added
    // in warp order at the end (no atomics: the gradient is reproducible)
    float gb1[kWarps][kH1], gb2[kWarps][kH2], gw3[kWarps][kH2], gb3[kWarps], loss[kWarps];
};

__device__ void load_weights(Smem& s, const MlpArgs& a, bool with_w2) {
    for (int k = threadIdx.x; k < kH1 * kIn; k += blockDim.x)
        s.w1t[(k / kIn) * kW1tStride + k % kIn] = a.w1t[k];
    for (int k = threadIdx.x; k < kH2 * kH1; k += blockDim.x)
        s.w2t[(k / kH1) * kW2tStride + k % kH1] = a.w2t[k];
    if (with_w2)
        for (int k = threadIdx.x; k < kH1 * kH2; k += blockDim.x)
            s.w2[(k / kH2) * kW2Stride + k % kH2] = a.w2[k];
    for (int k = threadIdx.x; k < kH1; k += blockDim.x) s.b1[k] = a.params[kOffB1 + k];
    for (int k = threadIdx.x; k < kH2; k += blockDim.x) {
        s.b2[k] = a.params[kOffB2 + k];
        s.w3[k] = a.params[kOffW3 + k];
    }
}

// Forward pass of one 16-sample tile held by a warp.  Thread (g, q) = (lane /
// 4, lane % 4) holds rows g and g + 8 of every fragment.  Outputs: xa (x as
// A fragments of layer 1), a1f (a1 as A fragments of layer 2), acc2 (z2 =
// a1 W2 + b2, fp32), z3 of rows g and g + 8.
struct Tile {
    uint32_t xa[2][4];
    uint32_t a1f[4][4];
    float acc2[16][4];
    float z3[2];
};

__device__ __forceinline__ void tile_forward(const Smem& s, const MlpArgs& a, int64_t row0, Tile& T,
                                             float b3) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    // x rows (sample ids through the batch order); rows past n are zero
    const float* xr[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t r = row0 + g + 8 * h;
        xr[h] = nullptr;
        if (r < a.n) {
            const int64_t id = a.order ? (int64_t)a.order[a.first + r] : a.first + r;
            xr[h] = a.x + id * kIn;
        }
    }
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int c = ks * 16 + half * 8 + 2 * q;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float2 v = make_float2(0.f, 0.f);
                if (xr[h]) v = *reinterpret_cast<const float2*>(xr[h] + c);
                T.xa[ks][half * 2 + h] = pack_bf16(v.x, v.y);
            }
        }
    }
    // layer 1: [16 x 32] x [32 x 64]
    float acc1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        acc1[nt][0] = acc1[nt][1] = acc1[nt][2] = acc1[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const __nv_bfloat16* w = s.w1t + (nt * 8 + g) * kW1tStride + ks * 16 + 2 * q;
            mma(acc1[nt], T.xa[ks][0], T.xa[ks][1], T.xa[ks][2], T.xa[ks][3], ld32(w), ld32(w + 8));
        }
    }
    // a1 = bf16(relu(z1)) as the A fragments of layer 2 (k-slice kk = n-tiles 2kk, 2kk+1)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int nt = 2 * kk + half;
            const int c = nt * 8 + 2 * q;
            const float bb0 = s.b1[c], bb1 = s.b1[c + 1];
            T.a1f[kk][half * 2 + 0] = pack_bf16(fmaxf(acc1[nt][0] + bb0, 0.f), fmaxf(acc1[nt][1] + bb1, 0.f));
            T.a1f[kk][half * 2 + 1] = pack_bf16(fmaxf(acc1[nt][2] + bb0, 0.f), fmaxf(acc1[nt][3] + bb1, 0.f));
        }
    }
    // layer 2: [16 x 64] x [64 x 128]
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int c = nt * 8 + 2 * q;
        T.acc2[nt][0] = T.acc2[nt][2] = s.b2[c];
        T.acc2[nt][1] = T.acc2[nt][3] = s.b2[c + 1];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const __nv_bfloat16* w = s.w2t + (nt * 8 + g) * kW2tStride + kk * 16 + 2 * q;
            mma(T.acc2[nt], T.a1f[kk][0], T.a1f[kk][1], T.a1f[kk][2], T.a1f[kk][3], ld32(w), ld32(w + 8));
        }
    }
    // layer 3: z3 = bf16(relu(z2)) . w3 + b3, reduced over the 4 threads of a row
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int c = nt * 8 + 2 * q;
        p0 += round_bf16(fmaxf(T.acc2[nt][0], 0.f)) * s.w3[c] + round_bf16(fmaxf(T.acc2[nt][1], 0.f)) * s.w3[c + 1];
        p1 += round_bf16(fmaxf(T.acc2[nt][2], 0.f)) * s.w3[c] + round_bf16(fmaxf(T.acc2[nt][3], 0.f)) * s.w3[c + 1];
    }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        p0 += __shfl_xor_sync(0xffffffffu, p0, o);
        p1 += __shfl_xor_sync(0xffffffffu, p1, o);
    }
    T.z3[0] = p0 + b3;
    T.z3[1] = p1 + b3;
}

__global__ void __launch_bounds__(kWarps * 32) mlp_forward_kernel(MlpArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& s = *reinterpret_cast<Smem*>(smem_raw);
    load_weights(s, a, false);
    __syncthreads();
    const float b3 = a.params[kOffB3];
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int64_t tiles = (a.n + kTileRows - 1) / kTileRows;
    const int64_t wid = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    for (int64_t t = wid; t < tiles; t += (int64_t)gridDim.x * kWarps) {
        Tile T;
        tile_forward(s, a, t * kTileRows, T, b3);
        if (q == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t r = t * kTileRows + g + 8 * h;
                if (r < a.n) a.logits[r] = T.z3[h];
            }
        }
    }
}

// sum over the 8 row groups (lanes with equal lane % 4)
__device__ __forceinline__ float sum_rows(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

__global__ void __launch_bounds__(kWarps * 32) mlp_grad_kernel(MlpArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& s = *reinterpret_cast<Smem*>(smem_raw);
    load_weights(s, a, true);
    for (int k = threadIdx.x; k < kWarps * kH1; k += blockDim.x) s.gb1[k / kH1][k % kH1] = 0.f;
    for (int k = threadIdx.x; k < kWarps * kH2; k += blockDim.x) s.gb2[k / kH2][k % kH2] = s.gw3[k / kH2][k % kH2] = 0.f;
    if (threadIdx.x < kWarps) s.gb3[threadIdx.x] = s.loss[threadIdx.x] = 0.f;
    __syncthreads();
    const float b3 = a.params[kOffB3];
    const float inv_n = 1.0f / (float)a.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    // this warp's slices of the weight gradients, accumulated over all steps:
    // dW2 rows (layer-1 units) 16w .. 16w+15, all 128 columns;
    // dW1 rows (inputs) 16 (w & 1) .., columns 32 (w >> 1) .. + 31
    float gW2[16][4], gW1[4][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) gW2[nt][0] = gW2[nt][1] = gW2[nt][2] = gW2[nt][3] = 0.f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) gW1[nt][0] = gW1[nt][1] = gW1[nt][2] = gW1[nt][3] = 0.f;

    const int64_t steps = (a.n + kBlockRows - 1) / kBlockRows;
    for (int64_t st = blockIdx.x; st < steps; st += gridDim.x) {
        const int64_t row0 = st * kBlockRows + warp * kTileRows;
        Tile T;
        tile_forward(s, a, row0, T, b3);
        // g3 = w (sigmoid(z3) - y) / n of rows g, g + 8 (0 past n)
        float g3[2];
        float lsum = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t r = row0 + g + 8 * h;
            g3[h] = 0.f;
            if (r < a.n) {
                const int64_t id = a.order ? (int64_t)a.order[a.first + r] : a.first + r;
                const float y = a.y[id];
                const float w = y > 0.5f ? a.pos_weight : 1.0f;
                const float z = T.z3[h];
                g3[h] = w * (1.0f / (1.0f + expf(-z)) - y) * inv_n;
                lsum += w * (fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))) - y * z);
            }
        }
        // dw3, db3, loss: rows summed over the warp, one thread per column pair
        if (q == 0) {
            float l = lsum;
            l += __shfl_xor_sync(0x11111111u, l, 4);
            l += __shfl_xor_sync(0x11111111u, l, 8);
            l += __shfl_xor_sync(0x11111111u, l, 16);
            float gb = g3[0] + g3[1];
            gb += __shfl_xor_sync(0x11111111u, gb, 4);
            gb += __shfl_xor_sync(0x11111111u, gb, 8);
            gb += __shfl_xor_sync(0x11111111u, gb, 16);
            if (lane == 0) {
                s.loss[warp] += l * inv_n;
                s.gb3[warp] += gb;
            }
        }
        // dz2 = bf16(g3 w3 [z2 > 0]) in place of acc2; its column sums and a2 . g3
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const int c = nt * 8 + 2 * q;
            const float a00 = round_bf16(fmaxf(T.acc2[nt][0], 0.f)), a01 = round_bf16(fmaxf(T.acc2[nt][1], 0.f));
            const float a10 = round_bf16(fmaxf(T.acc2[nt][2], 0.f)), a11 = round_bf16(fmaxf(T.acc2[nt][3], 0.f));
            float w30 = sum_rows(a00 * g3[0] + a10 * g3[1]);
            float w31 = sum_rows(a01 * g3[0] + a11 * g3[1]);
            const float d00 = T.acc2[nt][0] > 0.f ? round_bf16(g3[0] * s.w3[c]) : 0.f;
            const float d01 = T.acc2[nt][1] > 0.f ? round_bf16(g3[0] * s.w3[c + 1]) : 0.f;
            const float d10 = T.acc2[nt][2] > 0.f ? round_bf16(g3[1] * s.w3[c]) : 0.f;
            const float d11 = T.acc2[nt][3] > 0.f ? round_bf16(g3[1] * s.w3[c + 1]) : 0.f;
            T.acc2[nt][0] = d00;
            T.acc2[nt][1] = d01;
            T.acc2[nt][2] = d10;
            T.acc2[nt][3] = d11;
            const float s0 = sum_rows(d00 + d10), s1 = sum_rows(d01 + d11);
            if (g == 0) {
                s.gw3[warp][c] += w30;
                s.gw3[warp][c + 1] += w31;
                s.gb2[warp][c] += s0;
                s.gb2[warp][c + 1] += s1;
            }
        }
        // da1 = dz2 W2^T: [16 x 128] x [128 x 64], A fragments straight from dz2
        float da1[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            da1[nt][0] = da1[nt][1] = da1[nt][2] = da1[nt][3] = 0.f;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const uint32_t A0 = pack_bf16(T.acc2[2 * kk][0], T.acc2[2 * kk][1]);
                const uint32_t A1 = pack_bf16(T.acc2[2 * kk][2], T.acc2[2 * kk][3]);
                const uint32_t A2 = pack_bf16(T.acc2[2 * kk + 1][0], T.acc2[2 * kk + 1][1]);
                const uint32_t A3 = pack_bf16(T.acc2[2 * kk + 1][2], T.acc2[2 * kk + 1][3]);
                const __nv_bfloat16* w = s.w2 + (nt * 8 + g) * kW2Stride + kk * 16 + 2 * q;
                mma(da1[nt], A0, A1, A2, A3, ld32(w), ld32(w + 8));
            }
        }
        // stage x^T, a1^T, dz2^T and dz1^T = bf16(da1 [z1 > 0])^T sample-minor
        const int sr0 = warp * kTileRows + g, sr1 = sr0 + 8;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int c = ks * 16 + half * 8 + 2 * q;
                const uint32_t v0 = T.xa[ks][half * 2], v1 = T.xa[ks][half * 2 + 1];
                s.xt[c * kTStride + sr0] = __float2bfloat16_rn(bf16_lo(v0));
                s.xt[(c + 1) * kTStride + sr0] = __float2bfloat16_rn(bf16_hi(v0));
                s.xt[c * kTStride + sr1] = __float2bfloat16_rn(bf16_lo(v1));
                s.xt[(c + 1) * kTStride + sr1] = __float2bfloat16_rn(bf16_hi(v1));
            }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int nt = 2 * kk + half, c = nt * 8 + 2 * q;
                const uint32_t v0 = T.a1f[kk][half * 2], v1 = T.a1f[kk][half * 2 + 1];
                const float a00 = bf16_lo(v0), a01 = bf16_hi(v0), a10 = bf16_lo(v1), a11 = bf16_hi(v1);
                s.a1t[c * kTStride + sr0] = __float2bfloat16_rn(a00);
                s.a1t[(c + 1) * kTStride + sr0] = __float2bfloat16_rn(a01);
                s.a1t[c * kTStride + sr1] = __float2bfloat16_rn(a10);
                s.a1t[(c + 1) * kTStride + sr1] = __float2bfloat16_rn(a11);
                const float d00 = a00 > 0.f ? round_bf16(da1[nt][0]) : 0.f;
                const float d01 = a01 > 0.f ? round_bf16(da1[nt][1]) : 0.f;
                const float d10 = a10 > 0.f ? round_bf16(da1[nt][2]) : 0.f;
                const float d11 = a11 > 0.f ? round_bf16(da1[nt][3]) : 0.f;
                s.dz1t[c * kTStride + sr0] = __float2bfloat16_rn(d00);
                s.dz1t[(c + 1) * kTStride + sr0] = __float2bfloat16_rn(d01);
                s.dz1t[c * kTStride + sr1] = __float2bfloat16_rn(d10);
                s.dz1t[(c + 1) * kTStride + sr1] = __float2bfloat16_rn(d11);
                const float s0 = sum_rows(d00 + d10), s1 = sum_rows(d01 + d11);
                if (g == 0) {
                    s.gb1[warp][c] += s0;
                    s.gb1[warp][c + 1] += s1;
                }
            }
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const int c = nt * 8 + 2 * q;
            s.dz2t[c * kTStride + sr0] = __float2bfloat16_rn(T.acc2[nt][0]);
            s.dz2t[(c + 1) * kTStride + sr0] = __float2bfloat16_rn(T.acc2[nt][1]);
            s.dz2t[c * kTStride + sr1] = __float2bfloat16_rn(T.acc2[nt][2]);
            s.dz2t[(c + 1) * kTStride + sr1] = __float2bfloat16_rn(T.acc2[nt][3]);
        }
        __syncthreads();
        // dW2 += a1^T dz2 over the block's 64 samples: rows 16 warp .. of a1^T
#pragma unroll
        for (int ks = 0; ks < kBlockRows / 16; ++ks) {
            const __nv_bfloat16* ar = s.a1t + (warp * 16 + g) * kTStride + ks * 16 + 2 * q;
            const uint32_t A0 = ld32(ar), A1 = ld32(ar + 8 * kTStride), A2 = ld32(ar + 8),
                           A3 = ld32(ar + 8 * kTStride + 8);
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                const __nv_bfloat16* br = s.dz2t + (nt * 8 + g) * kTStride + ks * 16 + 2 * q;
                mma(gW2[nt], A0, A1, A2, A3, ld32(br), ld32(br + 8));
            }
        }
        // dW1 += x^T dz1: rows 16 (warp & 1) .. of x^T, columns 32 (warp >> 1) ..
#pragma unroll
        for (int ks = 0; ks < kBlockRows / 16; ++ks) {
            const __nv_bfloat16* ar = s.xt + ((warp & 1) * 16 + g) * kTStride + ks * 16 + 2 * q;
            const uint32_t A0 = ld32(ar), A1 = ld32(ar + 8 * kTStride), A2 = ld32(ar + 8),
                           A3 = ld32(ar + 8 * kTStride + 8);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const __nv_bfloat16* br = s.dz1t + ((warp >> 1) * 32 + nt * 8 + g) * kTStride + ks * 16 + 2 * q;
                mma(gW1[nt], A0, A1, A2, A3, ld32(br), ld32(br + 8));
            }
        }
        __syncthreads();
    }
    // this block's sums into its own slice of the per-block buffer: every
    // parameter's entry is written once (the warps' dW2 and dW1 slices are
    // disjoint; the bias, w3 and loss sums are added in warp order)
    float* part = a.part + (int64_t)blockIdx.x * (kParams + 1);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int r = warp * 16 + g, c = nt * 8 + 2 * q;
        part[kOffW2 + r * kH2 + c] = gW2[nt][0];
        part[kOffW2 + r * kH2 + c + 1] = gW2[nt][1];
        part[kOffW2 + (r + 8) * kH2 + c] = gW2[nt][2];
        part[kOffW2 + (r + 8) * kH2 + c + 1] = gW2[nt][3];
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int r = (warp & 1) * 16 + g, c = (warp >> 1) * 32 + nt * 8 + 2 * q;
        part[kOffW1 + r * kH1 + c] = gW1[nt][0];
        part[kOffW1 + r * kH1 + c + 1] = gW1[nt][1];
        part[kOffW1 + (r + 8) * kH1 + c] = gW1[nt][2];
        part[kOffW1 + (r + 8) * kH1 + c + 1] = gW1[nt][3];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kH1; k += blockDim.x) {
        float v = 0.f;
        for (int w = 0; w < kWarps; ++w) v += s.gb1[w][k];
        part[kOffB1 + k] = v;
    }
    for (int k = threadIdx.x; k < kH2; k += blockDim.x) {
        float v = 0.f, u = 0.f;
        for (int w = 0; w < kWarps; ++w) {
            v += s.gb2[w][k];
            u += s.gw3[w][k];
        }
        part[kOffB2 + k] = v;
        part[kOffW3 + k] = u;
    }
    if (threadIdx.x == 0) {
        float v = 0.f, u = 0.f;
        for (int w = 0; w < kWarps; ++w) {
            v += s.gb3[w];
            u += s.loss[w];
        }
        part[kOffB3] = v;
        part[kParams] = u;
    }
}

// grad[k] = sum over the blocks of their slices, in block order; the loss likewise.
__global__ void grad_reduce_kernel(const float* __restrict__ part, int blocks, float* grad, float* loss) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= kParams; k += gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int b = 0; b < blocks; ++b) v += part[(int64_t)b * (kParams + 1) + k];
        if (k < kParams) grad[k] = v;
        else *loss = v;
    }
}

// Adam on the fp32 master parameters (bias-corrected with step t), then the
// bf16 copies the products read.
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kParams; k += gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

__global__ void refresh_kernel(const float* p, __nv_bfloat16* w1t, __nv_bfloat16* w2t,
                               __nv_bfloat16* w2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kH1 * kH2; k += gridDim.x * blockDim.x) {
        if (k < kIn * kH1) {
            const int i = k / kH1, o = k % kH1;   // W1[i][o]
            w1t[o * kIn + i] = __float2bfloat16_rn(p[kOffW1 + k]);
        }
        const int i = k / kH2, o = k % kH2;       // W2[i][o]
        const __nv_bfloat16 v = __float2bfloat16_rn(p[kOffW2 + k]);
        w2[k] = v;
        w2t[o * kH1 + i] = v;
    }
}

}  // namespace
}  // namespace swgb

// ===========================================================================
// Host side
// ===========================================================================
struct swgb_mlp {
    swgb_ctx* ctx = nullptr;
    int device = 0;
    float* params = nullptr;      // fp32 master
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    float* loss = nullptr;        // [1]
    float* part = nullptr;        // [part_blocks][kParams + 1] per-block gradient sums
    int part_blocks = 0;
    __nv_bfloat16* w1t = nullptr;
    __nv_bfloat16* w2t = nullptr;
    __nv_bfloat16* w2 = nullptr;
    int64_t step = 0;             // Adam steps taken
};

namespace {

constexpr size_t kSmemBytes = sizeof(Smem);
constexpr size_t kFwdSmemBytes = offsetof(Smem, w2);

MlpArgs base_args(const swgb_mlp* m) {
    MlpArgs a{};
    a.params = m->params;
    a.w1t = m->w1t;
    a.w2t = m->w2t;
    a.w2 = m->w2;
    a.grad = m->grad;
    a.loss = m->loss;
    a.part = m->part;
    return a;
}

int mlp_check(const swgb_mlp* m) { return (m && m->ctx) ? SWGB_OK : SWGB_EINVAL; }

int grad_launch(swgb_mlp* m, const float* x, const float* y, const int32_t* order, int64_t first,
                int64_t n, float pos_weight, cudaStream_t st) {
    swgb_ctx* ctx = m->ctx;
    MlpArgs a = base_args(m);
    a.x = x;
    a.y = y;
    a.order = order;
    a.first = first;
    a.n = n;
    a.pos_weight = pos_weight;
    const int64_t steps = (n + kBlockRows - 1) / kBlockRows;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(steps, (int64_t)m->part_blocks));
    mlp_grad_kernel<<<blocks, kWarps * 32, kSmemBytes, st>>>(a);
    CK(cudaGetLastError(), "mlp_grad kernel");
    grad_reduce_kernel<<<(kParams + 256) / 256, 256, 0, st>>>(m->part, blocks, m->grad, m->loss);
    CK(cudaGetLastError(), "grad_reduce kernel");
    return SWGB_OK;
}

}  // namespace

SWGB_EXPORT int swgb_mlp_create(swgb_ctx* ctx, const float* init, swgb_mlp** out) {
    if (!ctx) return SWGB_EINVAL;
    if (!init || !out) return fail(ctx, SWGB_EINVAL, "mlp: init or out is NULL");
    *out = nullptr;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    swgb_mlp* m = new (std::nothrow) swgb_mlp();
    if (!m) return fail(ctx, SWGB_ENOMEM, "mlp: host allocation");
    m->ctx = ctx;
    m->device = ctx->device;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    };
    alloc(&m->params, sizeof(float) * kParams);
    alloc(&m->m, sizeof(float) * kParams);
    alloc(&m->v, sizeof(float) * kParams);
    alloc(&m->grad, sizeof(float) * kParams);
    alloc(&m->loss, sizeof(float));
    m->part_blocks = std::max(1, ctx->sm_count * 2);
    alloc(&m->part, sizeof(float) * (kParams + 1) * (size_t)m->part_blocks);
    alloc(&m->w1t, sizeof(__nv_bfloat16) * kIn * kH1);
    alloc(&m->w2t, sizeof(__nv_bfloat16) * kH1 * kH2);
    alloc(&m->w2, sizeof(__nv_bfloat16) * kH1 * kH2);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) {
        swgb_mlp_destroy(m);
        return cuda_fail(ctx, e, "mlp: allocation");
    }
    int rc = swgb_mlp_set(m, init);
    if (rc) {
        swgb_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return SWGB_OK;
}

SWGB_EXPORT void swgb_mlp_destroy(swgb_mlp* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    cudaFree(m->params);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->grad);
    cudaFree(m->loss);
    cudaFree(m->part);
    cudaFree(m->w1t);
    cudaFree(m->w2t);
    cudaFree(m->w2);
    delete m;
}

SWGB_EXPORT int swgb_mlp_set(swgb_mlp* m, const float* params) {
    if (mlp_check(m)) return SWGB_EINVAL;
    swgb_ctx* ctx = m->ctx;
    if (!params) return fail(ctx, SWGB_EINVAL, "mlp: params is NULL");
    CK(cudaSetDevice(m->device), "cudaSetDevice");
    CK(cudaMemcpy(m->params, params, sizeof(float) * kParams, cudaMemcpyHostToDevice), "params H2D");
    CK(cudaMemset(m->m, 0, sizeof(float) * kParams), "memset");
    CK(cudaMemset(m->v, 0, sizeof(float) * kParams), "memset");
    refresh_kernel<<<8, 256>>>(m->params, m->w1t, m->w2t, m->w2);
    CK(cudaGetLastError(), "refresh kernel");
    CK(cudaDeviceSynchronize(), "sync");
    m->step = 0;
    return SWGB_OK;
}

SWGB_EXPORT int swgb_mlp_get(swgb_mlp* m, float* params) {
    if (mlp_check(m)) return SWGB_EINVAL;
    swgb_ctx* ctx = m->ctx;
    if (!params) return fail(ctx, SWGB_EINVAL, "mlp: params is NULL");
    CK(cudaSetDevice(m->device), "cudaSetDevice");
    CK(cudaDeviceSynchronize(), "sync");
    CK(cudaMemcpy(params, m->params, sizeof(float) * kParams, cudaMemcpyDeviceToHost), "params D2H");
    return SWGB_OK;
}

SWGB_EXPORT int swgb_mlp_forward(swgb_mlp* m, const float* features, int64_t n, float* logits,
                                 void* stream) {
    if (mlp_check(m)) return SWGB_EINVAL;
    swgb_ctx* ctx = m->ctx;
    if (n < 0 || (n > 0 && (!features || !logits)))
        return fail(ctx, SWGB_EINVAL, "mlp_forward: negative count or NULL buffer");
    if (n == 0) return SWGB_OK;
    CK(cudaSetDevice(m->device), "cudaSetDevice");
    MlpArgs a = base_args(m);
    a.x = features;
    a.n = n;
    a.logits = logits;
    const int64_t tiles = (n + kTileRows - 1) / kTileRows;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + kWarps - 1) / kWarps,
                                                                   (int64_t)ctx->sm_count * 4));
    mlp_forward_kernel<<<blocks, kWarps * 32, kFwdSmemBytes, (cudaStream_t)stream>>>(a);
    CK(cudaGetLastError(), "mlp_forward kernel");
    return SWGB_OK;
}

SWGB_EXPORT int swgb_mlp_grad(swgb_mlp* m, const float* features, const float* labels, int64_t n,
                              float pos_weight, float* grad, float* loss, void* stream) {
    if (mlp_check(m)) return SWGB_EINVAL;
    swgb_ctx* ctx = m->ctx;
    if (n < 1 || !features || !labels || !grad || !loss || !(pos_weight > 0.f))
        return fail(ctx, SWGB_EINVAL, "mlp_grad: bad argument");
    CK(cudaSetDevice(m->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = grad_launch(m, features, labels, nullptr, 0, n, pos_weight, st);
    if (rc) return rc;
    CK(cudaMemcpyAsync(grad, m->grad, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, st), "grad copy");
    CK(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, st), "loss copy");
    return SWGB_OK;
}

SWGB_EXPORT int swgb_mlp_train(swgb_mlp* m, const float* features, const float* labels,
                               const int32_t* order, int64_t n, int64_t batch, float lr,
                               float pos_weight, float* mean_loss, void* stream) {
    if (mlp_check(m)) return SWGB_EINVAL;
    swgb_ctx* ctx = m->ctx;
    if (n < 1 || batch < 1 || !features || !labels || !(lr > 0.f) || !(pos_weight > 0.f))
        return fail(ctx, SWGB_EINVAL, "mlp_train: bad argument");
    CK(cudaSetDevice(m->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double loss_sum = 0.0;
    int64_t batches = 0;
    float* losses = nullptr;
    const int64_t nb = (n + batch - 1) / batch;
    CK(cudaMalloc(&losses, sizeof(float) * nb), "mlp_train scratch");
    int rc = SWGB_OK;
    for (int64_t first = 0; first < n && rc == SWGB_OK; first += batch, ++batches) {
        const int64_t len = std::min(batch, n - first);
        rc = grad_launch(m, features, labels, order, first, len, pos_weight, st);
        if (rc) break;
        m->step += 1;
        const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
        adam_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(m->params, m->grad, m->m, m->v, lr, b1, b2,
                                                          eps, c1, c2);
        refresh_kernel<<<32, 256, 0, st>>>(m->params, m->w1t, m->w2t, m->w2);
        cudaError_t e = cudaMemcpyAsync(losses + batches, m->loss, sizeof(float),
                                        cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "mlp_train kernels");
    }
    if (rc == SWGB_OK) {
        std::vector<float> h((size_t)nb);
        cudaError_t e = cudaMemcpyAsync(h.data(), losses, sizeof(float) * nb, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "mlp_train losses");
        for (float v : h) loss_sum += v;
    }
    cudaFree(losses);
    if (rc == SWGB_OK && mean_loss) *mean_loss = (float)(loss_sum / (double)nb);
    ctx->last_search_launches = (int32_t)(4 * nb);
    return rc;
}

// ---------------------------------------------------------------------------
// Training loop and calibration behind the ABI
// ---------------------------------------------------------------------------
namespace {

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): the state advances by the golden-ratio increment
// and each output is the state passed through the published finalizer.
struct SplitMix64 {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
    // uniform in [0, n) by rejection of the biased tail
    uint64_t below(uint64_t n) {
        const uint64_t lim = UINT64_MAX - UINT64_MAX % n;
        uint64_t x;
        do x = next(); while (x >= lim);
        return x % n;
    }
};

int copy_labels(swgb_ctx* ctx, const float* labels, int64_t n, std::vector<float>& h, cudaStream_t st) {
    h.resize((size_t)n);
    CK(cudaMemcpyAsync(h.data(), labels, sizeof(float) * n, cudaMemcpyDeviceToHost, st), "labels D2H");
    CK(cudaStreamSynchronize(st), "stream sync");
    return SWGB_OK;
}

}  // namespace

SWGB_EXPORT int swgb_mlp_fit(swgb_mlp* m, const float* features, const float* labels, int64_t n, int epochs,
                             int64_t batch, float lr, float pos_weight, uint64_t seed, float* losses,
                             void* stream) {
    if (mlp_check(m)) return SWGB_EINVAL;
    swgb_ctx* ctx = m->ctx;
    if (n < 1 || n > INT32_MAX || epochs < 0 || batch < 1 || !features || !labels || !(lr > 0.f))
        return fail(ctx, SWGB_EINVAL, "mlp_fit: bad argument");
    CK(cudaSetDevice(m->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    if (!(pos_weight > 0.f)) {
        // sqrt(negatives / positives) of the labels, each at least 1
        std::vector<float> h;
        int rc = copy_labels(ctx, labels, n, h, st);
        if (rc) return rc;
        double pos = 0.0;
        for (float v : h) pos += v > 0.5f;
        pos_weight = (float)std::sqrt(std::max(1.0, (double)n - pos) / std::max(1.0, pos));
    }
    std::vector<int32_t> order((size_t)n);
    int32_t* d_order = nullptr;
    CK(cudaMalloc(&d_order, sizeof(int32_t) * (size_t)n), "mlp_fit scratch");
    SplitMix64 rng{seed};
    int rc = SWGB_OK;
    for (int ep = 0; ep < epochs && rc == SWGB_OK; ++ep) {
        // Fisher-Yates from the identity
        for (int64_t k = 0; k < n; ++k) order[(size_t)k] = (int32_t)k;
        for (int64_t k = n - 1; k > 0; --k) std::swap(order[(size_t)k], order[(size_t)rng.below((uint64_t)k + 1)]);
        cudaError_t e = cudaMemcpyAsync(d_order, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // order is reused by the next epoch
        if (e != cudaSuccess) {
            rc = cuda_fail(ctx, e, "mlp_fit order H2D");
            break;
        }
        float mean = 0.f;
        rc = swgb_mlp_train(m, features, labels, d_order, n, batch, lr, pos_weight, &mean, stream);
        if (rc == SWGB_OK && losses) losses[ep] = mean;
    }
    cudaFree(d_order);
    ctx->last_search_launches = (int32_t)(4 * ((n + batch - 1) / batch) * epochs);
    return rc;
}

SWGB_EXPORT int swgb_mlp_calibrate(swgb_mlp* m, const float* features, const float* labels, int64_t n,
                                   float recall, float* threshold, void* stream) {
    if (mlp_check(m)) return SWGB_EINVAL;
    swgb_ctx* ctx = m->ctx;
    if (n < 1 || !features || !labels || !threshold || !(recall >= 0.f && recall <= 1.f))
        return fail(ctx, SWGB_EINVAL, "mlp_calibrate: bad argument");
    CK(cudaSetDevice(m->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    float* d_logits = nullptr;
    CK(cudaMalloc(&d_logits, sizeof(float) * (size_t)n), "mlp_calibrate scratch");
    int rc = swgb_mlp_forward(m, features, n, d_logits, stream);
    std::vector<float> z((size_t)n), y;
    if (rc == SWGB_OK) {
        cudaError_t e = cudaMemcpyAsync(z.data(), d_logits, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "logits D2H");
    }
    if (rc == SWGB_OK) rc = copy_labels(ctx, labels, n, y, st);
    cudaFree(d_logits);
    if (rc) return rc;
    // the largest threshold that keeps at least `recall` of the positives: the
    // k-th smallest positive logit, k = floor((1 - recall) * positives)
    std::vector<float> pos;
    for (int64_t k = 0; k < n; ++k)
        if (y[(size_t)k] > 0.5f) pos.push_back(z[(size_t)k]);
    if (pos.empty()) {
        *threshold = -INFINITY;
        return SWGB_OK;
    }
    size_t k = (size_t)std::floor((1.0 - (double)recall) * (double)pos.size());
    if (k >= pos.size()) k = pos.size() - 1;
    std::nth_element(pos.begin(), pos.begin() + (std::ptrdiff_t)k, pos.end());
    *threshold = pos[k];
    return SWGB_OK;
}
