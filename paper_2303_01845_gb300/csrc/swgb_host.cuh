// swgb_host.cuh -- host-side objects shared by the C-ABI translation units
// (swgb_api.cu: contexts, sequence sets, alignment; swgb_search.cu: candidate
// discovery and alignment identity).  Not part of the public ABI.
#pragma once

#include <algorithm>
#include <cstring>
#include <string>

#include "swgb_internal.cuh"

using namespace swgb;

#define SWGB_EXPORT extern "C" __attribute__((visibility("default")))

// Device scratch of candidate discovery and alignment identity (swgb_search.cu),
// created on a context's first such call.
struct SearchStore;
void search_store_free(SearchStore* s);

// Growable device workspace of one issuing context: a context owns one for
// swgb_align, every plan owns its own (a captured graph keeps its pointers).
// The status word and counters are the context's and are shared.
struct Store {
    Workspace ws{};
    int64_t bin_capacity = 0;    // ws.bin_of
    int64_t order_capacity = 0;  // ws.order
    int64_t region_off[kClasses][kNumShapes] = {};
    int64_t region_slots[kClasses][kNumShapes] = {};
    int64_t fmax_off_capacity = 0;      // ws.fmax_off
    int64_t band_region_off[kBandShapes] = {};   // chunk-boundary rows of the band kernels
    int64_t band_region_slots[kBandShapes] = {};
};

struct swgb_ctx {
    int device = 0;
    int sm_count = 0;
    std::string err;
    Store store;                     // workspace of swgb_align
    Workspace& ws = store.ws;        // (status and counters live here)
    int32_t* d_pairs = nullptr;      // staging for swgb_align_host
    swgb_record* d_out = nullptr;
    int64_t d_pairs_capacity = 0;
    int64_t d_out_capacity = 0;
    int32_t* d_encode_flag = nullptr;  // [4]: residue check, largest code, offsets check, longest
                                       // sequence of seqset loads
    // resident blocks per SM of each DP kernel, [profile variant][direction]:
    // variant 0 = 21 profile rows (standard letters), 1 = all 25 rows
    int blocks_per_sm[2][2][kClasses][kNumShapes] = {};
    int tile_overhead = kTileOverhead;
    int band_min = kBandMinDefault;  // banded reverse pass from this length (0 = off)
    int band_blocks[2][kBandShapes] = {};   // resident blocks per SM of each band kernel, [variant]
    swgb_tuning tuning{};            // the last swgb_autotune's figures
    cudaEvent_t ev[6] = {};
    // the DP kernels of one direction run on the caller's stream and these
    // side streams (forked and joined with events), so that their tails overlap
    static constexpr int kSide = 3;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kSide] = {};
    // a stream of the greatest priority: the block scheduler places the
    // blocks of its launches before pending blocks of the other streams (the
    // identity's cooperative spans, the critical path of its launches)
    cudaStream_t first = nullptr;
    bool timed = false;
    cudaStream_t last_stream = nullptr;
    int32_t last_launches = 0;
    int32_t last_search_launches = 0;   // of the last swgb_discover / swgb_identity
    int64_t last_pairs = 0;
    unsigned long long* d_probe_cycles = nullptr;
    uint32_t* d_probe_sink = nullptr;
    SearchStore* search = nullptr;
};

struct swgb_seqset {
    swgb_ctx* ctx = nullptr;
    int device = 0;
    uint8_t* d_res = nullptr;
    int64_t* d_off = nullptr;
    int64_t res_capacity = 0;
    int64_t off_capacity = 0;
    int64_t n = 0;
    int64_t total = 0;
    int64_t max_len = 0;
    int32_t max_code = 0;   // largest residue code in the set
};


static inline int fail(swgb_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

static inline int cuda_fail(swgb_ctx* ctx, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(ctx, SWGB_ENOMEM, m);
    return fail(ctx, SWGB_ECUDA, m);
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

template <class T>
static inline cudaError_t grow(T** p, int64_t* cap, int64_t need) {
    if (need <= *cap && *p) return cudaSuccess;
    int64_t n = std::max<int64_t>(need, *cap * 3 / 2);
    if (n < 1) n = 1;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)n);
    if (e == cudaSuccess) *cap = n;
    return e;
}

static inline SeqView view(const swgb_seqset* s) { return SeqView{s->d_res, s->d_off, s->n}; }
