// swgb_lane.cuh -- device helpers of the DP kernels (swgb_kernels.cu): packed
// 16x2 / 32-bit lane arithmetic, profile word loads, group reductions and the
// transposed score table the profiles are built from.  Not part of the public
// ABI.
#pragma once

#include <climits>
#include <cstdint>

#include "swgb_internal.cuh"

namespace swgb {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void zero_record(swgb_record* r) {
    *r = swgb_record{0, -1, -1, -1, -1};
}

__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
    atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// Lane arithmetic: packed 16x2 (two pairs per register) or 32-bit
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

template <bool P16>
struct Lane;

// Packed path: two pairs per register, every score kept biased by kBias so
// that both 16-bit halves stay in [0, 65535]; unsigned add-max / max then act
// per half, and a 32-bit add of two such words never carries from one half
// into the other (which lets constant shifts run as integer multiply-adds).
constexpr int kBias = 16384;

template <>
struct Lane<true> {
    static constexpr int kPack = 2;
    __device__ __forceinline__ static uint32_t addmax(uint32_t a, uint32_t b, uint32_t c) {
        return __viaddmax_u16x2(a, b, c);
    }
    __device__ __forceinline__ static uint32_t max3(uint32_t a, uint32_t b, uint32_t c) {
        return __vimax3_u16x2(a, b, c);
    }
    __device__ __forceinline__ static uint32_t splat(int v) {
        return ((uint32_t)v & 0xffffu) * 0x10001u;
    }
    __device__ __forceinline__ static int get(uint32_t w, int h) {
        return h ? (int)(w >> 16) : (int)(w & 0xffffu);
    }
    __device__ __forceinline__ static uint32_t min3(uint32_t a, uint32_t b, uint32_t c) {
        return __vimin3_u16x2(a, b, c);
    }
    // score of row b (0..3) of the word pair: low half from a (pair 0),
    // high half from c (pair 1); packed-path profile bytes are 0..127, so
    // extending the sign bit fills zeros
    __device__ __forceinline__ static uint32_t widen(uint32_t a, uint32_t c, int b) {
        const uint32_t sel = (uint32_t)b | ((uint32_t)(b | 8) << 4) | ((uint32_t)(4 + b) << 8) |
                             ((uint32_t)((4 + b) | 8) << 12);
        return prmt(a, c, sel);
    }
};

template <>
struct Lane<false> {
    static constexpr int kPack = 1;
    __device__ __forceinline__ static uint32_t addmax(uint32_t a, uint32_t b, uint32_t c) {
        return (uint32_t)__viaddmax_s32((int)a, (int)b, (int)c);
    }
    __device__ __forceinline__ static uint32_t max3(uint32_t a, uint32_t b, uint32_t c) {
        return (uint32_t)__vimax3_s32((int)a, (int)b, (int)c);
    }
    __device__ __forceinline__ static uint32_t splat(int v) { return (uint32_t)v; }
    __device__ __forceinline__ static int get(uint32_t w, int) { return (int)w; }
    __device__ __forceinline__ static uint32_t min3(uint32_t a, uint32_t b, uint32_t c) {
        return (uint32_t)__vimin3_s32((int)a, (int)b, (int)c);
    }
    __device__ __forceinline__ static uint32_t widen(uint32_t a, uint32_t, int b) {
        const uint32_t s = (uint32_t)(b | 8);
        const uint32_t sel = (uint32_t)b | (s << 4) | (s << 8) | (s << 12);
        return prmt(a, 0u, sel);
    }
};

// Maximum of N values as a tree of 3-input maxima: every level takes the
// values three at a time and carries the one or two left over, so N values cost
// ceil((N - 1) / 2) instructions at depth about log3(N).
template <bool P16, int N>
__device__ __forceinline__ uint32_t max_reduce(const uint32_t (&x)[N]) {
    if constexpr (N == 1) {
        return x[0];
    } else if constexpr (N == 2) {
        return Lane<P16>::max3(x[0], x[1], x[1]);
    } else {
        constexpr int NG = N / 3, NL = N % 3, M = NG + NL;
        uint32_t y[M];
#pragma unroll
        for (int k = 0; k < NG; ++k) y[k] = Lane<P16>::max3(x[3 * k], x[3 * k + 1], x[3 * k + 2]);
#pragma unroll
        for (int k = 0; k < NL; ++k) y[NG + k] = x[3 * NG + k];
        return max_reduce<P16, M>(y);
    }
}

// Maximum of v[0..R) and init.
template <bool P16, int R>
__device__ __forceinline__ uint32_t tree_max(const uint32_t (&v)[R], uint32_t init) {
    uint32_t x[R + 1];
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = v[k];
    x[R] = init;
    return max_reduce<P16, R + 1>(x);
}

// A lane's profile bytes for one query letter: R rows rounded up to whole
// words (LS bytes, 8, 12 or 16), loaded as one 8-byte, three 4-byte or one
// 16-byte access; they start at a multiple of LS.
template <int LS>
struct ProfWords {
    uint32_t w[LS / 4];
};

template <int LS>
__device__ __forceinline__ ProfWords<LS> load_prof(const int8_t* p) {
    ProfWords<LS> out;
    if constexpr (LS == 8) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        out.w[0] = v.x;
        out.w[1] = v.y;
    } else if constexpr (LS == 12) {
        const uint32_t* q = reinterpret_cast<const uint32_t*>(p);
        out.w[0] = q[0];
        out.w[1] = q[1];
        out.w[2] = q[2];
    } else {
        static_assert(LS == 16, "lane stride must be 8, 12 or 16 bytes");
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        out.w[0] = v.x;
        out.w[1] = v.y;
        out.w[2] = v.z;
        out.w[3] = v.w;
    }
    return out;
}

template <int LS>
__device__ __forceinline__ void store_prof(int8_t* p, const uint32_t (&w)[LS / 4]) {
    if constexpr (LS == 8) {
        *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
    } else if constexpr (LS == 12) {
        uint32_t* q = reinterpret_cast<uint32_t*>(p);
        q[0] = w[0];
        q[1] = w[1];
        q[2] = w[2];
    } else {
        *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// (value, i, j) ordering of candidate end cells: larger value first, then the
// row-major-first cell (smaller streamed index i, then smaller held index j).
__device__ __forceinline__ bool better(int v, int i, int j, int bv, int bi, int bj) {
    return v > bv || (v == bv && (i < bi || (i == bi && j < bj)));
}

// The block's copy of the score table, transposed: tabT[y][x] = table(x, y)
// for reference code y (0..24, the pad code last) and profile row x (the pad
// row mapped to the pad code).  Rows are 9 words apart, so lanes reading one
// word of rows of different codes hit different banks.
constexpr int kTabTStride = 36;
constexpr int kTabTBytes = kProfileRows * kTabTStride;   // 900
constexpr int kSmatRegion = 1024;                        // keeps profiles 16-B aligned
static_assert(kTabTBytes <= kSmatRegion, "transposed table exceeds its region");
// Packed per-half maximum over the G lanes of a group.
template <bool P16, int G>
__device__ __forceinline__ uint32_t group_max(uint32_t v) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const uint32_t o = __shfl_xor_sync(kFull, v, off, G);
        v = Lane<P16>::max3(v, o, o);
    }
    return v;
}

template <int G>
__device__ __forceinline__ int group_min(int v) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v = min(v, __shfl_xor_sync(kFull, v, off, G));
    return v;
}

}  // namespace swgb
