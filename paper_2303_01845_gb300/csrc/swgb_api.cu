// swgb_api.cu -- host side of the C ABI declared in include/swgb.h.
//
// Owns contexts (device workspace, events, the last call's counters) and
// sequence sets (encoded residues + offsets in device memory), validates
// arguments, and enqueues the per-call pipeline on the caller's stream:
//
//   keys (forward)  -> scan -> scatter -> DP forward  x (2 classes x 5 shapes)
//   keys (reverse)  -> scan -> scatter -> DP reverse  x (2 classes x 5 shapes)
//
// Every step runs in the kernels of swgb_kernels.cu; the host never touches
// pair data.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "swgb_internal.cuh"


using namespace swgb;

// The library's BLOSUM62 (Henikoff & Henikoff, PNAS 89:10915, 1992) in the
// NCBI letter order A R N D C Q E G H I L K M F P S T W Y V B Z X *, as text
// rows of the published integer matrix.
static const char* kBlosum62Rows[kAlpha] = {
    " 4 -1 -2 -2  0 -1 -1  0 -2 -1 -1 -1 -1 -2 -1  1  0 -3 -2  0 -2 -1  0 -4",
    "-1  5  0 -2 -3  1  0 -2  0 -3 -2  2 -1 -3 -2 -1 -1 -3 -2 -3 -1  0 -1 -4",
    "-2  0  6  1 -3  0  0  0  1 -3 -3  0 -2 -3 -2  1  0 -4 -2 -3  3  0 -1 -4",
    "-2 -2  1  6 -3  0  2 -1 -1 -3 -4 -1 -3 -3 -1  0 -1 -4 -3 -3  4  1 -1 -4",
    " 0 -3 -3 -3  9 -3 -4 -3 -3 -1 -1 -3 -1 -2 -3 -1 -1 -2 -2 -1 -3 -3 -2 -4",
    "-1  1  0  0 -3  5  2 -2  0 -3 -2  1  0 -3 -1  0 -1 -2 -1 -2  0  3 -1 -4",
    "-1  0  0  2 -4  2  5 -2  0 -3 -3  1 -2 -3 -1  0 -1 -3 -2 -2  1  4 -1 -4",
    " 0 -2  0 -1 -3 -2 -2  6 -2 -4 -4 -2 -3 -3 -2  0 -2 -2 -3 -3 -1 -2 -1 -4",
    "-2  0  1 -1 -3  0  0 -2  8 -3 -3 -1 -2 -1 -2 -1 -2 -2  2 -3  0  0 -1 -4",
    "-1 -3 -3 -3 -1 -3 -3 -4 -3  4  2 -3  1  0 -3 -2 -1 -3 -1  3 -3 -3 -1 -4",
    "-1 -2 -3 -4 -1 -2 -3 -4 -3  2  4 -2  2  0 -3 -2 -1 -2 -1  1 -4 -3 -1 -4",
    "-1  2  0 -1 -3  1  1 -2 -1 -3 -2  5 -1 -3 -1  0 -1 -3 -2 -2  0  1 -1 -4",
    "-1 -1 -2 -3 -1  0 -2 -3 -2  1  2 -1  5  0 -2 -1 -1 -1 -1  1 -3 -1 -1 -4",
    "-2 -3 -3 -3 -2 -3 -3 -3 -1  0  0 -3  0  6 -4 -2 -2  1  3 -1 -3 -3 -1 -4",
    "-1 -2 -2 -1 -3 -1 -1 -2 -2 -3 -3 -1 -2 -4  7 -1 -1 -4 -3 -2 -2 -1 -2 -4",
    " 1 -1  1  0 -1  0  0  0 -1 -2 -2  0 -1 -2 -1  4  1 -3 -2 -2  0  0  0 -4",
    " 0 -1  0 -1 -1 -1 -1 -2 -2 -1 -1 -1 -1 -2 -1  1  5 -2 -2  0 -1 -1  0 -4",
    "-3 -3 -4 -4 -2 -2 -3 -2 -2 -3 -2 -3 -1  1 -4 -3 -2 11  2 -3 -4 -3 -2 -4",
    "-2 -2 -2 -3 -2 -1 -2 -3  2 -1 -1 -2 -1  3 -3 -2 -2  2  7 -1 -3 -2 -1 -4",
    " 0 -3 -3 -3 -1 -2 -2 -3 -3  3  1 -2  1 -1 -2 -2  0 -3 -1  4 -3 -2 -1 -4",
    "-2 -1  3  4 -3  0  1 -1  0 -3 -4  0 -3 -3 -2  0 -1 -4 -3 -3  4  1 -1 -4",
    "-1  0  0  1 -3  3  4 -2  0 -3 -3  1 -1 -3 -1  0 -1 -3 -2 -2  1  4 -1 -4",
    " 0 -1 -1 -1 -2 -1 -1 -1 -1 -1 -1 -1 -1 -1 -2  0  0 -2 -1 -1 -1 -1 -1 -4",
    "-4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4  1",
};

#include "swgb_host.cuh"

namespace {


// Both profile tables of a validated matrix and gap setting (o + e = oe).
void fill_profiles(const int8_t* m, int go, int ge, ScoreArgs* sc) {
    const int oe = go + ge;
    for (int x = 0; x < kProfileRows; ++x)
        for (int y = 0; y < kMatStride; ++y) {
            const bool real = x < kAlpha && y < kAlpha;
            const int s = real ? m[x * kAlpha + y] : 0;
            sc->prof[x][y] = (int8_t)(real ? s + oe : kPadProfile);
            sc->profu[x][y] = (uint8_t)std::min(std::max(real ? s + oe : 0, 0), 127);
        }
    sc->go = go;
    sc->ge = ge;
    sc->one = 1;
    sc->prof_rows = kProfileRows;
}

// Row / column maxima of a validated 24 x 24 matrix for the 16-bit test.  The
// packed path also needs every s + o + e >= 0 (its profile bytes are
// unsigned); other matrices run on the 32-bit path.
ClassArgs make_class_args(const int8_t* m, int oe, int max_score, bool force32) {
    ClassArgs ca{};
    ca.max_score = max_score;
    for (int x = 0; x < kAlpha; ++x) {
        int rmax = 0, cmax = 0;
        for (int y = 0; y < kAlpha; ++y) {
            rmax = std::max<int>(rmax, m[x * kAlpha + y]);
            cmax = std::max<int>(cmax, m[y * kAlpha + x]);
        }
        ca.rowmax[x] = (int8_t)rmax;
        ca.colmax[x] = (int8_t)cmax;
    }
    bool packable = true;
    for (int k = 0; k < kAlpha * kAlpha; ++k)
        packable = packable && m[k] + oe >= 0;
    ca.force32 = (force32 || !packable) ? 1 : 0;
    return ca;
}

}  // namespace

SWGB_EXPORT void swgb_blosum62(int8_t* out) {
    if (!out) return;
    for (int x = 0; x < kAlpha; ++x) {
        const char* p = kBlosum62Rows[x];
        for (int y = 0; y < kAlpha; ++y) {
            char* end = nullptr;
            long v = std::strtol(p, &end, 10);
            out[x * kAlpha + y] = (int8_t)v;
            p = end;
        }
    }
}

SWGB_EXPORT const char* swgb_last_error(const swgb_ctx* ctx) {
    return ctx ? ctx->err.c_str() : "null context";
}

SWGB_EXPORT int swgb_create(int device, swgb_ctx** out) {
    if (!out) return SWGB_EINVAL;
    *out = nullptr;
    swgb_ctx* ctx = new (std::nothrow) swgb_ctx();
    if (!ctx) return SWGB_ENOMEM;
    ctx->device = device;
    auto bail = [&](cudaError_t e, const char* what) {
        int rc = cuda_fail(ctx, e, what);
        fprintf(stderr, "swgb_create: %s\n", ctx->err.c_str());
        swgb_destroy(ctx);
        return rc;
    };
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return bail(e, "cudaSetDevice");
    e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return bail(e, "cudaDeviceGetAttribute");
    Workspace& ws = ctx->ws;
    if ((e = cudaMalloc(&ws.hist, sizeof(uint32_t) * kNumBins)) != cudaSuccess) return bail(e, "alloc");
    if ((e = cudaMalloc(&ws.scan, sizeof(uint32_t) * (kNumBins + 1))) != cudaSuccess) return bail(e, "alloc");
    if ((e = cudaMalloc(&ws.cursor, sizeof(uint32_t) * kNumBins)) != cudaSuccess) return bail(e, "alloc");
    if ((e = cudaMalloc(&ws.task_ctr, sizeof(uint32_t) * kTaskCounters)) != cudaSuccess) return bail(e, "alloc");
    if ((e = cudaMalloc(&ws.status, sizeof(int32_t))) != cudaSuccess) return bail(e, "alloc");
    if ((e = cudaMalloc(&ctx->d_encode_flag, 4 * sizeof(int32_t))) != cudaSuccess) return bail(e, "alloc");
    if ((e = cudaMalloc(&ws.counters, sizeof(unsigned long long) * kNumCounters)) != cudaSuccess) return bail(e, "alloc");
    if ((e = cudaMemset(ws.status, 0, sizeof(int32_t))) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemset(ws.counters, 0, sizeof(unsigned long long) * kNumCounters)) != cudaSuccess) return bail(e, "memset");
    for (int d = 0; d < 2; ++d)
        for (int c = 0; c < kClasses; ++c)
            for (int s = 0; s < kNumShapes; ++s) {
                if ((e = dp_configure(c, s, d == 1)) != cudaSuccess) return bail(e, "cudaFuncSetAttribute");
                for (int v = 0; v < 2; ++v)
                    ctx->blocks_per_sm[v][d][c][s] =
                        std::max(1, dp_blocks_per_sm(c, s, d == 1, v ? kProfileRows : kStdLetters + 1));
            }
    for (int s = kFirstChunkable; s < kBandShapeEnd; ++s)
        for (int v = 0; v < 2; ++v)
            ctx->band_blocks[v][s - kFirstChunkable] =
                std::max(1, dp_blocks_per_sm(0, s, true, v ? kProfileRows : kStdLetters + 1, true));
    for (auto& ev : ctx->ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(e, "cudaEventCreate");
    if ((e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming)) != cudaSuccess)
        return bail(e, "cudaEventCreate");
    for (int k = 0; k < swgb_ctx::kSide; ++k) {
        if ((e = cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking)) != cudaSuccess)
            return bail(e, "cudaStreamCreate");
        if ((e = cudaEventCreateWithFlags(&ctx->join_ev[k], cudaEventDisableTiming)) != cudaSuccess)
            return bail(e, "cudaEventCreate");
    }
    int least_prio = 0, greatest_prio = 0;
    if ((e = cudaDeviceGetStreamPriorityRange(&least_prio, &greatest_prio)) != cudaSuccess)
        return bail(e, "cudaDeviceGetStreamPriorityRange");
    if ((e = cudaStreamCreateWithPriority(&ctx->first, cudaStreamNonBlocking, greatest_prio)) != cudaSuccess)
        return bail(e, "cudaStreamCreate");
    *out = ctx;
    return SWGB_OK;
}

SWGB_EXPORT void swgb_destroy(swgb_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    Workspace& ws = ctx->ws;
    cudaFree(ws.hist);
    cudaFree(ws.scan);
    cudaFree(ws.cursor);
    cudaFree(ws.bin_of);
    cudaFree(ws.order);
    cudaFree(ws.task_ctr);
    cudaFree(ws.status);
    cudaFree(ws.counters);
    cudaFree(ws.boundary);
    cudaFree(ws.fmax);
    cudaFree(ws.fmax_off);
    cudaFree(ctx->d_pairs);
    cudaFree(ctx->d_out);
    cudaFree(ctx->d_encode_flag);
    cudaFree(ctx->d_probe_cycles);
    cudaFree(ctx->d_probe_sink);
    search_store_free(ctx->search);
    for (auto& ev : ctx->ev)
        if (ev) cudaEventDestroy(ev);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    for (int k = 0; k < swgb_ctx::kSide; ++k) {
        if (ctx->side[k]) cudaStreamDestroy(ctx->side[k]);
        if (ctx->join_ev[k]) cudaEventDestroy(ctx->join_ev[k]);
    }
    if (ctx->first) cudaStreamDestroy(ctx->first);
    delete ctx;
}

// ---------------------------------------------------------------------------
// Sequence sets
// ---------------------------------------------------------------------------
// Host residue uploads of at least this many bytes are split over the streams.
constexpr int64_t kSplitCopyBytes = 64ll << 20;

// Device address of a byte of pinned (page-locked, mapped) host memory, or
// null for any other pointer.
static const uint8_t* mapped_byte(const uint8_t* p) {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
        cudaGetLastError();   // a plain host pointer on some drivers: not an error here
        return nullptr;
    }
    if (pa.type != cudaMemoryTypeHost || pa.devicePointer == nullptr) return nullptr;
    return static_cast<const uint8_t*>(pa.devicePointer);
}

// Device address of the host bytes [p, p + n) when all of them are pinned
// host memory (both ends mapped, n - 1 apart), else null.  Kernels may read
// such memory in place over the host link.
static const uint8_t* mapped_host(const uint8_t* p, int64_t n) {
    const uint8_t* first = mapped_byte(p);
    if (!first) return nullptr;
    const uint8_t* last = mapped_byte(p + (n - 1));
    if (!last || last - first != n - 1) return nullptr;
    return first;
}

SWGB_EXPORT int swgb_seqset_load(swgb_seqset* set, const void* residues, const int64_t* offsets,
                                 int64_t n_seqs, uint32_t flags, void* stream) {
    if (!set || !set->ctx) return SWGB_EINVAL;
    swgb_ctx* ctx = set->ctx;
    if (n_seqs < 0 || (flags & ~(SWGB_SEQ_ASCII | SWGB_SEQ_DEVICE | SWGB_SEQ_COPY)))
        return fail(ctx, SWGB_EINVAL, "seqset: negative count or unknown flags");
    if (n_seqs > 0 && !offsets) return fail(ctx, SWGB_EINVAL, "seqset: offsets is NULL");
    if (n_seqs > INT32_MAX) return fail(ctx, SWGB_ERANGE, "seqset: more than 2^31-1 sequences");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    const bool on_dev = flags & SWGB_SEQ_DEVICE;

    // Only the first and last offsets are read on the host (the residue range
    // to copy); the offsets go to the device as given and are checked, measured
    // and rebased there, so a load costs no host pass over the set.
    int64_t ends[2] = {0, 0};
    if (n_seqs > 0) {
        if (on_dev) {
            CK(cudaMemcpyAsync(&ends[0], offsets, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "offsets D2H");
            CK(cudaMemcpyAsync(&ends[1], offsets + n_seqs, sizeof(int64_t), cudaMemcpyDeviceToHost, st),
               "offsets D2H");
            CK(cudaStreamSynchronize(st), "stream sync");
        } else {
            ends[0] = offsets[0];
            ends[1] = offsets[n_seqs];
        }
    }
    const int64_t base = ends[0];
    const int64_t total = ends[1] - ends[0];
    if (total < 0) return fail(ctx, SWGB_ERANGE, "seqset: offsets decrease");
    if (total > 0 && !residues) return fail(ctx, SWGB_EINVAL, "seqset: residues is NULL");

    CK(grow(&set->d_res, &set->res_capacity, std::max<int64_t>(total, 1)), "seqset alloc");
    CK(grow(&set->d_off, &set->off_capacity, n_seqs + 1), "seqset alloc");
    CK(cudaMemsetAsync(ctx->d_encode_flag, 0, 4 * sizeof(int32_t), st), "memset");
    if (n_seqs > 0) {
        CK(cudaMemcpyAsync(set->d_off, offsets, sizeof(int64_t) * (n_seqs + 1),
                           on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st), "offsets copy");
        CK(launch_offsets(set->d_off, n_seqs, base, SWGB_MAX_LENGTH, ctx->d_encode_flag + 2, st),
           "offsets kernel");
    } else {
        CK(cudaMemsetAsync(set->d_off, 0, sizeof(int64_t), st), "memset");
    }
    const uint8_t* src = static_cast<const uint8_t*>(residues);
    if (total > 0) {
        if (on_dev) {
            src += base;
        } else if (const uint8_t* mapped = (flags & SWGB_SEQ_COPY) ? nullptr : mapped_host(src + base, total)) {
            // pinned host memory: the encode pass reads it in place over the
            // host link (no staging copy)
            src = mapped;
        } else {
            // large host sets are copied in parts on the caller's stream and the
            // context's side streams at once, so several copy engines share the
            // upload; the encode waits for all parts
            const int parts = total >= kSplitCopyBytes ? swgb_ctx::kSide + 1 : 1;
            if (parts > 1) {
                CK(cudaEventRecord(ctx->fork_ev, st), "event");
                for (int k = 0; k < swgb_ctx::kSide; ++k)
                    CK(cudaStreamWaitEvent(ctx->side[k], ctx->fork_ev, 0), "stream wait");
            }
            const int64_t part = (total + parts - 1) / parts;
            for (int k = 0; k < parts; ++k) {
                const int64_t b = k * part, e = std::min(total, b + part);
                if (b < e)
                    CK(cudaMemcpyAsync(set->d_res + b, src + base + b, (size_t)(e - b), cudaMemcpyHostToDevice,
                                       k == 0 ? st : ctx->side[k - 1]), "residues H2D");
            }
            if (parts > 1) {
                for (int k = 0; k < swgb_ctx::kSide; ++k) {
                    CK(cudaEventRecord(ctx->join_ev[k], ctx->side[k]), "event");
                    CK(cudaStreamWaitEvent(st, ctx->join_ev[k], 0), "stream wait");
                }
            }
            src = set->d_res;   // encode in place
        }
    }
    CK(launch_encode(src, set->d_res, total, flags & SWGB_SEQ_ASCII, ctx->d_encode_flag, st), "encode kernel");
    int32_t fl[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(fl, ctx->d_encode_flag, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st), "flag D2H");
    CK(cudaStreamSynchronize(st), "stream sync");
    set->n = fl[2] ? 0 : n_seqs;
    set->total = fl[2] ? 0 : total;
    set->max_len = fl[3];
    set->max_code = fl[1];
    if (fl[2] & 1) return fail(ctx, SWGB_ERANGE, "seqset: offsets decrease");
    if (fl[2] & 2) return fail(ctx, SWGB_ERANGE, "seqset: sequence longer than SWGB_MAX_LENGTH");
    if (fl[0]) return fail(ctx, SWGB_EBADRES, "seqset: residue outside the alphabet");
    return SWGB_OK;
}

SWGB_EXPORT int swgb_seqset_create(swgb_ctx* ctx, const void* residues, const int64_t* offsets,
                                   int64_t n_seqs, uint32_t flags, void* stream, swgb_seqset** out) {
    if (!ctx || !out) return SWGB_EINVAL;
    *out = nullptr;
    swgb_seqset* s = new (std::nothrow) swgb_seqset();
    if (!s) return fail(ctx, SWGB_ENOMEM, "seqset: host allocation");
    s->ctx = ctx;
    s->device = ctx->device;
    int rc = swgb_seqset_load(s, residues, offsets, n_seqs, flags, stream);
    if (rc != SWGB_OK) {
        swgb_seqset_destroy(s);
        return rc;
    }
    *out = s;
    return SWGB_OK;
}

SWGB_EXPORT int swgb_seqset_info(const swgb_seqset* set, int64_t* n_seqs, int64_t* max_length) {
    if (!set) return SWGB_EINVAL;
    if (n_seqs) *n_seqs = set->n;
    if (max_length) *max_length = set->max_len;
    return SWGB_OK;
}

SWGB_EXPORT void swgb_seqset_destroy(swgb_seqset* set) {
    if (!set) return;
    cudaSetDevice(set->device);
    cudaFree(set->d_res);
    cudaFree(set->d_off);
    delete set;
}

// ---------------------------------------------------------------------------
// Alignment
// ---------------------------------------------------------------------------
namespace {

int make_score_args(swgb_ctx* ctx, const swgb_params* params, ScoreArgs* sc, int* max_score) {
    if (!params || !params->matrix) return fail(ctx, SWGB_EINVAL, "params or matrix is NULL");
    if (params->gap_open < 0 || params->gap_extend < 1)
        return fail(ctx, SWGB_EINVAL, "gap_open must be >= 0 and gap_extend >= 1");
    if (params->flags & ~(SWGB_FORCE_INT32 | SWGB_TIMING))
        return fail(ctx, SWGB_EINVAL, "unknown params flags");
    const int oe = params->gap_open + params->gap_extend;
    int mx = 0;
    for (int k = 0; k < kAlpha * kAlpha; ++k) mx = std::max<int>(mx, params->matrix[k]);
    if (oe > 127 || mx + oe > 127)
        return fail(ctx, SWGB_EINVAL, "max(matrix) + gap_open + gap_extend must be <= 127");
    fill_profiles(params->matrix, params->gap_open, params->gap_extend, sc);
    *max_score = mx;
    return SWGB_OK;
}

// Pairs handled by one persistent block of a (class, shape) kernel.
int64_t pairs_per_block(int cls, int shape) {
    return (int64_t)(kDPThreads / 32) * (32 / shape_G(shape)) * (cls == 0 ? 2 : 1);
}

// Fixed-size parts of a store (status and counters come from the context).
int alloc_store_fixed(swgb_ctx* ctx, Store& st) {
    Workspace& ws = st.ws;
    CK(cudaMalloc(&ws.hist, sizeof(uint32_t) * kNumBins), "alloc");
    CK(cudaMalloc(&ws.scan, sizeof(uint32_t) * (kNumBins + 1)), "alloc");
    CK(cudaMalloc(&ws.cursor, sizeof(uint32_t) * kNumBins), "alloc");
    CK(cudaMalloc(&ws.task_ctr, sizeof(uint32_t) * kTaskCounters), "alloc");
    return SWGB_OK;
}

void free_store(Store& st, bool with_status) {
    Workspace& ws = st.ws;
    cudaFree(ws.hist);
    cudaFree(ws.scan);
    cudaFree(ws.cursor);
    cudaFree(ws.bin_of);
    cudaFree(ws.order);
    cudaFree(ws.task_ctr);
    cudaFree(ws.boundary);
    cudaFree(ws.fmax);
    cudaFree(ws.fmax_off);
    if (with_status) {
        cudaFree(ws.status);
        cudaFree(ws.counters);
    }
    ws = Workspace{};
}

// Grows a store for n_pairs pairs of the sets q, r (may allocate).
int prepare_store(swgb_ctx* ctx, Store& store, const swgb_seqset* q, const swgb_seqset* r, int64_t n_pairs) {
    Workspace& ws = store.ws;
    if (ctx->band_min > 0) {
        // forward maxima: a slice of 1 + ceil(lr / Rf) entries per recording
        // pair (Rf >= 8), handed out by the keys kernel; pairs past the pool
        // record none and keep the full reverse pass
        const int64_t per_pair = 2 + (std::max<int64_t>(r->max_len, 1) + 7) / 8;
        const int64_t want = std::min<int64_t>(std::max<int64_t>(n_pairs, 1) * per_pair, kFmaxPoolMax);
        if (ws.fmax_capacity < want) {
            cudaFree(ws.fmax);
            ws.fmax = nullptr;
            ws.fmax_capacity = 0;
            CK(cudaMalloc(&ws.fmax, sizeof(int32_t) * (size_t)want), "workspace alloc");
            ws.fmax_capacity = want;
        }
        CK(grow(&ws.fmax_off, &store.fmax_off_capacity, std::max<int64_t>(n_pairs, 1)), "workspace alloc");
        ws.fmax_off_n = store.fmax_off_capacity;
    }
    CK(grow(&ws.bin_of, &store.bin_capacity, std::max<int64_t>(n_pairs, 1)), "workspace alloc");
    CK(grow(&ws.order, &store.order_capacity, std::max<int64_t>(n_pairs, 1)), "workspace alloc");
    // chunk-boundary rows: one row per resident warp of every kernel that can
    // tile long references; kernels run concurrently, so each has its own region
    const int64_t stride = std::max<int64_t>(((q->max_len + 31) / 32) * 32, 32);
    int64_t slots = 0;
    for (int c = 0; c < kClasses; ++c)
        for (int s = kFirstChunkable; s < kNumShapes; ++s) {
            int64_t n = 0;
            for (int d = 0; d < 2; ++d)
                for (int v = 0; v < 2; ++v)
                    n = std::max<int64_t>(n, (int64_t)ctx->sm_count * ctx->blocks_per_sm[v][d][c][s] *
                                                 (kDPThreads / 32));
            store.region_off[c][s] = slots;
            store.region_slots[c][s] = n;
            slots += n;
        }
    // the band kernels run beside the reverse kernels of their shapes
    for (int s = kFirstChunkable; s < kBandShapeEnd; ++s) {
        const int b = s - kFirstChunkable;
        const int64_t n = (int64_t)ctx->sm_count * std::max(ctx->band_blocks[0][b], ctx->band_blocks[1][b]) *
                          (kDPThreads / 32);
        store.band_region_off[b] = slots;
        store.band_region_slots[b] = n;
        slots += n;
    }
    if (stride > ws.boundary_stride || slots > ws.boundary_slots || !ws.boundary) {
        cudaFree(ws.boundary);
        ws.boundary = nullptr;
        ws.boundary_stride = ws.boundary_slots = 0;
        CK(cudaMalloc(&ws.boundary, sizeof(uint2) * (size_t)stride * slots), "boundary alloc");
        ws.boundary_stride = stride;
        ws.boundary_slots = slots;
    }
    return SWGB_OK;
}

// Records a timing event on st.  Under stream capture (swgb_plan_create) the
// event must become an event node of the graph, so that replays record it.
cudaError_t record_timing(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    return cudaEventRecordWithFlags(ev, st, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                                 : cudaEventRecordDefault);
}

// Enqueues the whole pipeline on st (no allocation: the store is prepared).
int enqueue(swgb_ctx* ctx, const Store& store, const swgb_seqset* q, const swgb_seqset* r,
            const int32_t* pairs, int64_t n_pairs, const swgb_params* params, swgb_record* out,
            cudaStream_t st) {
    ScoreArgs sc;
    int max_score = 0;
    int rc = make_score_args(ctx, params, &sc, &max_score);
    if (rc) return rc;
    const Workspace& ws = store.ws;
    const bool force32 = params->flags & SWGB_FORCE_INT32;
    const bool timed = params->flags & SWGB_TIMING;
    ClassArgs ca = make_class_args(params->matrix, params->gap_open + params->gap_extend, max_score,
                                   force32);
    ca.tile_overhead = ctx->tile_overhead;
    // the banded reverse pass needs the packed path and the forward maxima
    // (a store grown for a banded call keeps its maxima arrays when the
    // setting goes back to 0; they are sized for that call's pairs only)
    const bool band = ctx->band_min > 0 && !ca.force32 && ws.fmax && ws.fmax_off && ws.fmax_off_n >= n_pairs;
    ca.band_min = band ? ctx->band_min : 0;
    const int pv = q->max_code < kStdLetters ? 0 : 1;   // profile variant
    sc.prof_rows = pv ? kProfileRows : kStdLetters + 1;

    int launches = 0;
    CK(cudaMemsetAsync(ws.counters, 0, sizeof(unsigned long long) * kNumCounters, st), "memset");
    CK(cudaMemsetAsync(ws.task_ctr, 0, sizeof(uint32_t) * kTaskCounters, st), "memset");
    if (timed) CK(record_timing(ctx->ev[0], st), "event");

    const SeqView qv = view(q), rv = view(r);
    // one round: keys -> scan -> scatter -> the DP kernels of every (class,
    // shape) and, in the reverse round, the band kernels of the chunkable
    // shapes, spread over the caller's stream and the side streams, largest
    // tiles first
    auto round = [&](int mode, int dir) -> int {
        CK(cudaMemsetAsync(ws.hist, 0, sizeof(uint32_t) * kNumBins, st), "memset");
        CK(launch_keys(qv, rv, pairs, n_pairs, out, mode, ca, ws, st), "keys kernel");
        CK(launch_scan(ws, st), "scan kernel");
        CK(launch_scatter(n_pairs, ws, st), "scatter kernel");
        launches += 4;
        // the DP times exclude the bucketing of their first round
        if (timed && mode != kKeysFallback) CK(record_timing(ctx->ev[mode == kKeysForward ? 1 : 3], st), "event");
        CK(cudaEventRecord(ctx->fork_ev, st), "event");
        for (int k = 0; k < swgb_ctx::kSide; ++k)
            CK(cudaStreamWaitEvent(ctx->side[k], ctx->fork_ev, 0), "stream wait");
        int rr = 0;
        auto next_stream = [&]() {
            const int k = rr++ % (swgb_ctx::kSide + 1);
            return k == 0 ? st : ctx->side[k - 1];
        };
        auto dp_args = [&]() {
            DPArgs a;
            a.q = qv;
            a.r = rv;
            a.pairs = pairs;
            a.order = ws.order;
            a.scan = ws.scan;
            a.out = out;
            a.status = ws.status;
            a.boundary_stride = ws.boundary_stride;
            a.fmax = band ? ws.fmax : nullptr;
            a.fmax_off = band ? ws.fmax_off : nullptr;
            a.counters = ws.counters;
            a.sc = sc;
            return a;
        };
        if (mode == kKeysReverse && band) {
            for (int s = kBandShapeEnd - 1; s >= kFirstChunkable; --s) {
                const int b = s - kFirstChunkable;
                DPArgs a = dp_args();
                a.task_ctr = ws.task_ctr + 3 * kNumKernels + b;
                a.boundary = ws.boundary + store.band_region_off[b] * ws.boundary_stride;
                a.boundary_slots = store.band_region_slots[b];
                a.first_bucket = band_first_bucket(s);
                a.end_bucket = band_end_bucket(s);
                int64_t grid = (int64_t)ctx->sm_count * ctx->band_blocks[pv][b];
                const int64_t need = (n_pairs + pairs_per_block(0, s) - 1) / pairs_per_block(0, s);
                grid = std::max<int64_t>(1, std::min(grid, need));
                CK(launch_dp(0, s, true, a, (int)grid, next_stream(), true), "band dp kernel");
                ++launches;
            }
        }
        // band pairs are on the packed path: the fallback round needs no
        // 32-bit launches
        const int classes = mode == kKeysFallback ? 1 : kClasses;
        for (int c = 0; c < classes; ++c) {
            for (int s = kNumShapes - 1; s >= 0; --s) {
                cudaStream_t ks = next_stream();
                DPArgs a = dp_args();
                a.task_ctr = ws.task_ctr + dir * kNumKernels + c * kNumShapes + s;
                const bool chunkable = s >= kFirstChunkable;
                a.boundary = chunkable ? ws.boundary + store.region_off[c][s] * ws.boundary_stride : nullptr;
                a.boundary_slots = chunkable ? store.region_slots[c][s] : 0;
                a.first_bucket = shape_first_bucket(c, s);
                a.end_bucket = shape_end_bucket(c, s);
                // the forward maxima are written by the forward round only
                if (mode != kKeysForward) a.fmax_off = nullptr;
                const int rev = mode != kKeysForward ? 1 : 0;
                int64_t grid = (int64_t)ctx->sm_count * ctx->blocks_per_sm[pv][rev][c][s];
                const int64_t need = (n_pairs + pairs_per_block(c, s) - 1) / pairs_per_block(c, s);
                grid = std::max<int64_t>(1, std::min(grid, need));
                CK(launch_dp(c, s, rev == 1, a, (int)grid, ks), "dp kernel");
                ++launches;
            }
        }
        for (int k = 0; k < swgb_ctx::kSide; ++k) {
            CK(cudaEventRecord(ctx->join_ev[k], ctx->side[k]), "event");
            CK(cudaStreamWaitEvent(st, ctx->join_ev[k], 0), "stream wait");
        }
        return SWGB_OK;
    };

    // forward: score and end cell
    if ((rc = round(kKeysForward, 0))) return rc;
    if (timed) CK(record_timing(ctx->ev[2], st), "event");
    // reverse: start cell (bands where chosen), then the pairs whose band
    // certificate did not hold over the whole rectangle
    if ((rc = round(kKeysReverse, 1))) return rc;
    if (band && (rc = round(kKeysFallback, 2))) return rc;
    if (timed) CK(record_timing(ctx->ev[4], st), "event");
    if (timed) CK(record_timing(ctx->ev[5], st), "event");
    ctx->timed = timed;
    ctx->last_stream = st;
    ctx->last_launches = launches;
    ctx->last_pairs = n_pairs;
    return SWGB_OK;
}

int check_sets(swgb_ctx* ctx, const swgb_seqset* q, const swgb_seqset* r) {
    if (!q || !r) return fail(ctx, SWGB_EINVAL, "sequence set is NULL");
    if (q->device != ctx->device || r->device != ctx->device)
        return fail(ctx, SWGB_EINVAL, "sequence set on another device");
    return SWGB_OK;
}

}  // namespace

SWGB_EXPORT int swgb_align(swgb_ctx* ctx, const swgb_seqset* queries, const swgb_seqset* refs,
                           const int32_t* pairs, int64_t n_pairs, const swgb_params* params,
                           swgb_record* out, void* stream) {
    if (!ctx) return SWGB_EINVAL;
    ctx->err.clear();
    if (n_pairs < 0) return fail(ctx, SWGB_EINVAL, "n_pairs < 0");
    if (n_pairs > INT32_MAX) return fail(ctx, SWGB_EINVAL, "n_pairs > 2^31-1");
    if (n_pairs > 0 && (!pairs || !out)) return fail(ctx, SWGB_EINVAL, "pairs or out is NULL");
    int rc = check_sets(ctx, queries, refs);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (n_pairs == 0) {
        ctx->last_pairs = 0;
        ctx->last_launches = 0;
        ctx->timed = false;
        ctx->last_stream = (cudaStream_t)stream;
        CK(cudaMemsetAsync(ctx->ws.counters, 0, sizeof(unsigned long long) * kNumCounters, (cudaStream_t)stream), "memset");
        return SWGB_OK;
    }
    rc = prepare_store(ctx, ctx->store, queries, refs, n_pairs);
    if (rc) return rc;
    return enqueue(ctx, ctx->store, queries, refs, pairs, n_pairs, params, out, (cudaStream_t)stream);
}

SWGB_EXPORT int swgb_sync(swgb_ctx* ctx, void* stream) {
    if (!ctx) return SWGB_EINVAL;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(st), "stream sync");
    int32_t status = 0;
    CK(cudaMemcpy(&status, ctx->ws.status, sizeof(int32_t), cudaMemcpyDeviceToHost), "status D2H");
    CK(cudaMemset(ctx->ws.status, 0, sizeof(int32_t)), "memset");
    if (status == SWGB_ERANGE) return fail(ctx, SWGB_ERANGE, "a pair index is outside its sequence set");
    if (status != 0) return fail(ctx, status, "device reported an internal inconsistency");
    return SWGB_OK;
}

SWGB_EXPORT int swgb_align_host(swgb_ctx* ctx, const swgb_seqset* queries, const swgb_seqset* refs,
                                const int32_t* pairs_host, int64_t n_pairs, const swgb_params* params,
                                swgb_record* out_host, void* stream) {
    if (!ctx) return SWGB_EINVAL;
    ctx->err.clear();
    if (n_pairs < 0) return fail(ctx, SWGB_EINVAL, "n_pairs < 0");
    if (n_pairs > 0 && (!pairs_host || !out_host)) return fail(ctx, SWGB_EINVAL, "pairs or out is NULL");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    CK(grow(&ctx->d_pairs, &ctx->d_pairs_capacity, std::max<int64_t>(2 * n_pairs, 2)), "staging alloc");
    CK(grow(&ctx->d_out, &ctx->d_out_capacity, std::max<int64_t>(n_pairs, 1)), "staging alloc");
    if (n_pairs > 0)
        CK(cudaMemcpyAsync(ctx->d_pairs, pairs_host, sizeof(int32_t) * 2 * n_pairs,
                           cudaMemcpyHostToDevice, st), "pairs H2D");
    int rc = swgb_align(ctx, queries, refs, ctx->d_pairs, n_pairs, params, ctx->d_out, stream);
    if (rc) return rc;
    if (n_pairs > 0)
        CK(cudaMemcpyAsync(out_host, ctx->d_out, sizeof(swgb_record) * n_pairs,
                           cudaMemcpyDeviceToHost, st), "records D2H");
    return swgb_sync(ctx, stream);
}

SWGB_EXPORT int swgb_last_stats(swgb_ctx* ctx, swgb_stats* out) {
    if (!ctx || !out) return SWGB_EINVAL;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(ctx->last_stream), "stream sync");
    unsigned long long c[kNumCounters];
    CK(cudaMemcpy(c, ctx->ws.counters, sizeof(c), cudaMemcpyDeviceToHost), "counters D2H");
    std::memset(out, 0, sizeof(*out));
    out->n_pairs = ctx->last_pairs;
    out->forward_cells = (int64_t)c[kCtrFwdCells];
    out->reverse_cells = (int64_t)c[kCtrRevCells];
    out->n_int16_pairs = (int64_t)c[kCtrInt16];
    out->n_int32_pairs = (int64_t)c[kCtrInt32];
    out->n_reverse_pairs = (int64_t)c[kCtrRevPairs];
    out->forward_ms = out->reverse_ms = out->total_ms = -1.0f;
    if (ctx->timed) {
        CK(cudaEventElapsedTime(&out->forward_ms, ctx->ev[1], ctx->ev[2]), "event time");
        CK(cudaEventElapsedTime(&out->reverse_ms, ctx->ev[3], ctx->ev[4]), "event time");
        CK(cudaEventElapsedTime(&out->total_ms, ctx->ev[0], ctx->ev[5]), "event time");
    }
    out->kernel_launches = ctx->last_launches;
    out->n_band_pairs = (int64_t)c[kCtrBandPairs];
    out->n_band_certified = (int64_t)c[kCtrBandCertified];
    out->forward_slots = (int64_t)c[kCtrFwdSlots];
    out->reverse_slots = (int64_t)c[kCtrRevSlots];
    return SWGB_OK;
}

SWGB_EXPORT int swgb_probe_addmax_rate(swgb_ctx* ctx, double* ops_per_clk_per_sm, int* sm_count) {
    if (!ctx || !ops_per_clk_per_sm) return SWGB_EINVAL;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int per_sm = 4;   // 4 x 256 threads resident per SM
    const int blocks = ctx->sm_count * per_sm;
    const int iters = 1 << 16;
    if (!ctx->d_probe_cycles) {
        CK(cudaMalloc(&ctx->d_probe_cycles, sizeof(unsigned long long) * blocks), "probe alloc");
        CK(cudaMalloc(&ctx->d_probe_sink, sizeof(uint32_t) * blocks * kProbeThreads), "probe alloc");
    }
    CK(launch_probe_addmax(ctx->d_probe_cycles, ctx->d_probe_sink, blocks, iters / 16, 0), "probe");
    CK(launch_probe_addmax(ctx->d_probe_cycles, ctx->d_probe_sink, blocks, iters, 0), "probe");
    CK(cudaDeviceSynchronize(), "probe sync");
    std::vector<unsigned long long> cyc(blocks);
    CK(cudaMemcpy(cyc.data(), ctx->d_probe_cycles, sizeof(unsigned long long) * blocks,
                  cudaMemcpyDeviceToHost), "probe D2H");
    unsigned long long mx = 1;
    for (auto v : cyc) mx = std::max(mx, v);
    const double ops_per_sm = (double)per_sm * kProbeThreads * kProbeChains * (double)iters;
    *ops_per_clk_per_sm = ops_per_sm / (double)mx;
    if (sm_count) *sm_count = ctx->sm_count;
    return SWGB_OK;
}

// ---------------------------------------------------------------------------
// swgb_align_noalloc: the same pipeline with every piece of device scratch
// taken from one fixed array compiled into the library.
//
// Some callers cannot allocate device memory while they align: code running
// inside a memory pool or arena that owns all of the device's memory, a host
// framework whose allocator must not be bypassed, or a process that has to
// keep its footprint constant after start-up.  This path never calls
// cudaMalloc, cudaFree or any other allocating routine (device or host); the
// caller passes its inputs and outputs as device pointers and the scratch is
// g_noalloc_scratch below.  Every GPU that loads this library holds the
// array (SWGB_NOALLOC_SCRATCH_BYTES) until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoallocBytes = SWGB_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocChunkBlocks = 304;   // grid cap of the kernels that tile long references
constexpr int64_t kNoallocSlots = (int64_t)kNoallocChunkBlocks * (kDPThreads / 32);
constexpr int kNoallocMaxDevices = 64;

constexpr int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

// byte offsets of the pieces inside the array
constexpr int64_t kNaHist = 0;
constexpr int64_t kNaScan = kNaHist + align256(4 * (int64_t)kNumBins);
constexpr int64_t kNaCursor = kNaScan + align256(4 * ((int64_t)kNumBins + 1));
constexpr int64_t kNaTask = kNaCursor + align256(4 * (int64_t)kNumBins);
constexpr int64_t kNaStatus = kNaTask + align256(4 * 2 * (int64_t)kNumKernels);
constexpr int64_t kNaFlags = kNaStatus + 256;
constexpr int64_t kNaCounters = kNaFlags + 256;
constexpr int64_t kNaBinOf = kNaCounters + 256;
static_assert(8 * kNumCounters <= 256, "no-alloc counters exceed their slot");
constexpr int64_t kNaOrder = kNaBinOf + align256(4 * (int64_t)SWGB_NOALLOC_MAX_PAIRS);
constexpr int64_t kNaBoundary = kNaOrder + align256(4 * (int64_t)SWGB_NOALLOC_MAX_PAIRS);
constexpr int64_t kNaEnd = kNaBoundary + 8 * kNoallocSlots * (int64_t)SWGB_NOALLOC_MAX_QUERY_LENGTH;
static_assert(kNaEnd <= kNoallocBytes, "no-alloc scratch layout exceeds the array");

// flag bits written by noalloc_check_kernel
constexpr int32_t kFlagBadCode = 1;
constexpr int32_t kFlagTooLong = 2;
constexpr int32_t kFlagBadOffsets = 4;

struct NoallocDevice {
    bool ready = false;
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch
    int sm_count = 0;
    int blocks_per_sm[2][kClasses][kNumShapes] = {};   // all 25 profile rows
};

NoallocDevice g_noalloc_dev[kNoallocMaxDevices];
std::mutex g_noalloc_mu;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[SWGB_NOALLOC_SCRATCH_BYTES];

// One warp per sequence: offsets non-negative and non-decreasing, codes < 24,
// lengths in [0, max_len].  A sequence with bad offsets reads no residue.
__global__ void noalloc_check_kernel(const uint8_t* __restrict__ res, const int64_t* __restrict__ off,
                                     int64_t n, int64_t max_len, int32_t* flags) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    int32_t f = 0;
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); k < n; k += warps) {
        const int64_t b = off[k], e = off[k + 1];
        if (b < 0 || e < b) {
            f |= kFlagBadOffsets;
            continue;
        }
        if (e - b > max_len) f |= kFlagTooLong;
        for (int64_t i = b + lane; i < e; i += 32)
            if (res[i] >= kAlpha) f |= kFlagBadCode;
    }
    if (f) atomicOr(flags, f);
}

namespace {

// Same acceptance rule as swgb_align, without building any error string.
int noalloc_score_args(const swgb_params* params, ScoreArgs* sc, int* max_score) {
    if (!params || !params->matrix) return SWGB_EINVAL;
    if (params->gap_open < 0 || params->gap_extend < 1) return SWGB_EINVAL;
    if (params->flags & ~(SWGB_FORCE_INT32 | SWGB_TIMING)) return SWGB_EINVAL;
    const int oe = params->gap_open + params->gap_extend;
    int mx = 0;
    for (int k = 0; k < kAlpha * kAlpha; ++k) mx = std::max<int>(mx, params->matrix[k]);
    if (oe > 127 || mx + oe > 127) return SWGB_EINVAL;
    fill_profiles(params->matrix, params->gap_open, params->gap_extend, sc);
    *max_score = mx;
    return SWGB_OK;
}

int noalloc_cuda(cudaError_t e) {
    return e == cudaSuccess ? SWGB_OK : SWGB_ECUDA;
}

#define NA_CK(call)                                     \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return noalloc_cuda(e_); \
    } while (0)

// First call on a device (with that device current): resolve the array's
// device address and configure the kernels.
int noalloc_setup(int dev, NoallocDevice** out) {
    if (dev < 0 || dev >= kNoallocMaxDevices) return SWGB_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDevice& d = g_noalloc_dev[dev];
    if (!d.ready) {
        void* ptr = nullptr;
        NA_CK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        NA_CK(cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev));
        for (int dir = 0; dir < 2; ++dir)
            for (int c = 0; c < kClasses; ++c)
                for (int s = 0; s < kNumShapes; ++s) {
                    NA_CK(dp_configure(c, s, dir == 1));
                    d.blocks_per_sm[dir][c][s] = std::max(1, dp_blocks_per_sm(c, s, dir == 1, kProfileRows));
                }
        d.base = static_cast<unsigned char*>(ptr);
        d.ready = true;
    }
    *out = &d;
    return SWGB_OK;
}

}  // namespace

SWGB_EXPORT int swgb_align_noalloc(const uint8_t* q_codes, const int64_t* q_offsets, int64_t n_q,
                                   const uint8_t* r_codes, const int64_t* r_offsets, int64_t n_r,
                                   const int32_t* pairs, int64_t n_pairs, const swgb_params* params,
                                   swgb_record* out, void* stream) {
    if (n_q < 0 || n_r < 0 || n_pairs < 0) return SWGB_EINVAL;
    if ((n_q > 0 && !q_offsets) || (n_r > 0 && !r_offsets)) return SWGB_EINVAL;
    if (n_pairs > 0 && (!pairs || !out)) return SWGB_EINVAL;
    if (n_q > INT32_MAX || n_r > INT32_MAX) return SWGB_ETOOBIG;
    if (n_pairs > SWGB_NOALLOC_MAX_PAIRS) return SWGB_ETOOBIG;
    ScoreArgs sc;
    int max_score = 0;
    int rc = noalloc_score_args(params, &sc, &max_score);
    if (rc) return rc;
    if (n_pairs == 0) return SWGB_OK;

    int dev = 0;
    NA_CK(cudaGetDevice(&dev));
    NoallocDevice* d = nullptr;
    rc = noalloc_setup(dev, &d);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = d->base;

    Workspace ws{};
    ws.hist = reinterpret_cast<uint32_t*>(base + kNaHist);
    ws.scan = reinterpret_cast<uint32_t*>(base + kNaScan);
    ws.cursor = reinterpret_cast<uint32_t*>(base + kNaCursor);
    ws.task_ctr = reinterpret_cast<uint32_t*>(base + kNaTask);
    ws.status = reinterpret_cast<int32_t*>(base + kNaStatus);
    ws.counters = reinterpret_cast<unsigned long long*>(base + kNaCounters);
    ws.bin_of = reinterpret_cast<int32_t*>(base + kNaBinOf);
    ws.order = reinterpret_cast<int32_t*>(base + kNaOrder);
    ws.boundary = reinterpret_cast<uint2*>(base + kNaBoundary);
    ws.boundary_stride = SWGB_NOALLOC_MAX_QUERY_LENGTH;
    ws.boundary_slots = kNoallocSlots;
    int32_t* flags = reinterpret_cast<int32_t*>(base + kNaFlags);

    // the array keeps the previous call's contents: clear what starts at zero
    NA_CK(cudaMemsetAsync(base + kNaStatus, 0, kNaBinOf - kNaStatus, st));
    NA_CK(cudaMemsetAsync(ws.task_ctr, 0, sizeof(uint32_t) * 2 * kNumKernels, st));

    // sizes and residue codes, checked on the device before any DP launch
    const int64_t check_blocks = std::max<int64_t>(1, std::min<int64_t>(((std::max(n_q, n_r) + 7) / 8),
                                                                       (int64_t)d->sm_count * 8));
    if (n_q > 0)
        noalloc_check_kernel<<<(unsigned)check_blocks, 256, 0, st>>>(q_codes, q_offsets, n_q,
                                                                     SWGB_NOALLOC_MAX_QUERY_LENGTH, flags);
    if (n_r > 0)
        noalloc_check_kernel<<<(unsigned)check_blocks, 256, 0, st>>>(r_codes, r_offsets, n_r,
                                                                     SWGB_MAX_LENGTH, flags);
    NA_CK(cudaGetLastError());
    int32_t host_flags = 0;
    NA_CK(cudaMemcpyAsync(&host_flags, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (host_flags & kFlagBadOffsets) return SWGB_ERANGE;
    if (host_flags & kFlagTooLong) return SWGB_ETOOBIG;
    if (host_flags & kFlagBadCode) return SWGB_EBADRES;

    const SeqView qv{q_codes, q_offsets, n_q}, rv{r_codes, r_offsets, n_r};
    ClassArgs ca = make_class_args(params->matrix, params->gap_open + params->gap_extend, max_score,
                                   params->flags & SWGB_FORCE_INT32);
    ca.tile_overhead = kTileOverhead;
    sc.prof_rows = kProfileRows;
    for (int dir = 0; dir < 2; ++dir) {
        const bool rev = dir == 1;
        NA_CK(cudaMemsetAsync(ws.hist, 0, sizeof(uint32_t) * kNumBins, st));
        NA_CK(launch_keys(qv, rv, pairs, n_pairs, out, rev ? kKeysReverse : kKeysForward, ca, ws, st));
        NA_CK(launch_scan(ws, st));
        NA_CK(launch_scatter(n_pairs, ws, st));
        for (int c = 0; c < kClasses; ++c) {
            for (int s = 0; s < kNumShapes; ++s) {
                DPArgs a;
                a.q = qv;
                a.r = rv;
                a.pairs = pairs;
                a.order = ws.order;
                a.scan = ws.scan;
                a.task_ctr = ws.task_ctr + dir * kNumKernels + c * kNumShapes + s;
                a.out = out;
                a.status = ws.status;
                a.boundary = ws.boundary;
                a.boundary_stride = ws.boundary_stride;
                a.boundary_slots = ws.boundary_slots;
                a.first_bucket = shape_first_bucket(c, s);
                a.end_bucket = shape_end_bucket(c, s);
                a.fmax = nullptr;
                a.fmax_off = nullptr;
                a.counters = ws.counters;
                a.sc = sc;
                int64_t grid = (int64_t)d->sm_count * d->blocks_per_sm[dir][c][s];
                const int64_t per_block = (int64_t)(kDPThreads / 32) * (32 / shape_G(s)) * (c == 0 ? 2 : 1);
                grid = std::min(grid, (n_pairs + per_block - 1) / per_block);
                if (s >= kFirstChunkable) grid = std::min<int64_t>(grid, kNoallocChunkBlocks);
                NA_CK(launch_dp(c, s, rev, a, (int)std::max<int64_t>(grid, 1), st));
            }
        }
    }
    int32_t status = 0;
    NA_CK(cudaMemcpyAsync(&status, ws.status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    return status;
}

// ---------------------------------------------------------------------------
// Plans: the pipeline for fixed buffers captured once into a CUDA graph
// ---------------------------------------------------------------------------
struct swgb_plan {
    swgb_ctx* ctx = nullptr;
    const swgb_seqset* queries = nullptr;
    bool std_profile = false;   // captured with the 21-row profile (codes 0..19 only)
    Store store;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool timed = false;
    int32_t launches = 0;
    int64_t n_pairs = 0;
};

SWGB_EXPORT void swgb_plan_destroy(swgb_plan* plan) {
    if (!plan) return;
    if (plan->ctx) cudaSetDevice(plan->ctx->device);
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    free_store(plan->store, false);
    delete plan;
}

SWGB_EXPORT int swgb_plan_create(swgb_ctx* ctx, const swgb_seqset* queries, const swgb_seqset* refs,
                                 const int32_t* pairs, int64_t n_pairs, const swgb_params* params,
                                 swgb_record* out, swgb_plan** out_plan) {
    if (!ctx || !out_plan) return SWGB_EINVAL;
    *out_plan = nullptr;
    ctx->err.clear();
    if (n_pairs < 1 || n_pairs > INT32_MAX) return fail(ctx, SWGB_EINVAL, "plan: n_pairs must be in [1, 2^31)");
    if (!pairs || !out) return fail(ctx, SWGB_EINVAL, "pairs or out is NULL");
    int rc = check_sets(ctx, queries, refs);
    if (rc) return rc;
    ScoreArgs probe;
    int max_score = 0;
    rc = make_score_args(ctx, params, &probe, &max_score);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    swgb_plan* plan = new (std::nothrow) swgb_plan();
    if (!plan) return fail(ctx, SWGB_ENOMEM, "plan: host allocation");
    plan->ctx = ctx;
    plan->store.ws.status = ctx->ws.status;
    plan->store.ws.counters = ctx->ws.counters;
    rc = alloc_store_fixed(ctx, plan->store);
    if (!rc) rc = prepare_store(ctx, plan->store, queries, refs, n_pairs);
    if (rc) {
        swgb_plan_destroy(plan);
        return rc;
    }
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        if (cs) cudaStreamDestroy(cs);
        swgb_plan_destroy(plan);
        return cuda_fail(ctx, e, "plan: begin capture");
    }
    rc = enqueue(ctx, plan->store, queries, refs, pairs, n_pairs, params, out, cs);
    e = cudaStreamEndCapture(cs, &plan->graph);
    cudaStreamDestroy(cs);
    if (rc == SWGB_OK && e != cudaSuccess) rc = cuda_fail(ctx, e, "plan: end capture");
    if (rc == SWGB_OK) {
        e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "plan: instantiate");
    }
    if (rc) {
        swgb_plan_destroy(plan);
        return rc;
    }
    plan->queries = queries;
    plan->std_profile = queries->max_code < kStdLetters;
    plan->timed = ctx->timed;
    plan->launches = ctx->last_launches;
    plan->n_pairs = n_pairs;
    ctx->last_pairs = 0;
    ctx->last_launches = 0;
    ctx->timed = false;
    *out_plan = plan;
    return SWGB_OK;
}

SWGB_EXPORT int swgb_plan_launch(swgb_plan* plan, void* stream) {
    if (!plan || !plan->ctx || !plan->exec) return SWGB_EINVAL;
    swgb_ctx* ctx = plan->ctx;
    ctx->err.clear();
    // The graph stages one profile row per query letter the set held at
    // capture; a set reloaded since then with codes beyond the 20 standard
    // letters would index rows that were never staged.
    if (plan->std_profile && plan->queries->max_code >= kStdLetters)
        return fail(ctx, SWGB_EINVAL, "plan: the query set now holds codes beyond the 20 standard letters; "
                                      "create a new plan");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaGraphLaunch(plan->exec, (cudaStream_t)stream), "graph launch");
    ctx->timed = plan->timed;
    ctx->last_stream = (cudaStream_t)stream;
    ctx->last_launches = plan->launches;
    ctx->last_pairs = plan->n_pairs;
    return SWGB_OK;
}

// ---------------------------------------------------------------------------
// Tile selection tuning
// ---------------------------------------------------------------------------
SWGB_EXPORT int swgb_set_tile_overhead(swgb_ctx* ctx, int overhead) {
    if (!ctx) return SWGB_EINVAL;
    if (overhead < 0 || overhead > 64) return fail(ctx, SWGB_EINVAL, "tile overhead must be in [0, 64]");
    ctx->tile_overhead = overhead;
    return SWGB_OK;
}

SWGB_EXPORT int swgb_get_tile_overhead(const swgb_ctx* ctx) {
    return ctx ? ctx->tile_overhead : SWGB_EINVAL;
}

SWGB_EXPORT int swgb_set_band_min(swgb_ctx* ctx, int band_min) {
    if (!ctx) return SWGB_EINVAL;
    if (band_min != 0 && (band_min < 32 || band_min > SWGB_MAX_LENGTH))
        return fail(ctx, SWGB_EINVAL, "band_min must be 0 or in [32, SWGB_MAX_LENGTH]");
    ctx->band_min = band_min;
    return SWGB_OK;
}

SWGB_EXPORT int swgb_get_band_min(const swgb_ctx* ctx) {
    return ctx ? ctx->band_min : SWGB_EINVAL;
}

SWGB_EXPORT int swgb_last_tuning(const swgb_ctx* ctx, swgb_tuning* out) {
    if (!ctx || !out) return SWGB_EINVAL;
    *out = ctx->tuning;
    return SWGB_OK;
}

SWGB_EXPORT int swgb_autotune(swgb_ctx* ctx, const swgb_seqset* queries, const swgb_seqset* refs,
                              const int32_t* pairs, int64_t n_pairs, const swgb_params* params,
                              swgb_record* out, void* stream, int* best_overhead, float* best_ms) {
    if (!ctx || !params) return SWGB_EINVAL;
    static const int kOverheads[] = {2, 4, 6, 8, 10, 12, 14, 17, 20, 24, 28, 32, 40};
    static const int kBandMins[] = {0, 256, 320, 384, 512, 768, 1024};
    constexpr int kTimed = 5;
    swgb_params p = *params;
    p.flags |= SWGB_TIMING;
    const int saved_ovh = ctx->tile_overhead, saved_band = ctx->band_min;
    swgb_tuning tu{};
    // whole-call time of one setting: a warm-up call, then the fastest of
    // kTimed (the settings differ by about a percent, as does run-to-run noise)
    auto timed = [&](int ovh, int band_min, float* t) -> int {
        ctx->tile_overhead = ovh;
        ctx->band_min = band_min;
        *t = -1.0f;
        for (int rep = 0; rep <= kTimed; ++rep) {
            int rc = swgb_align(ctx, queries, refs, pairs, n_pairs, &p, out, stream);
            if (!rc) rc = swgb_sync(ctx, stream);
            swgb_stats st;
            if (!rc) rc = swgb_last_stats(ctx, &st);
            if (rc) return rc;
            if (rep > 0 && (*t < 0.0f || st.total_ms < *t)) *t = st.total_ms;
        }
        ++tu.candidates;
        return SWGB_OK;
    };
    auto fail_restore = [&](int rc) {
        ctx->tile_overhead = saved_ovh;
        ctx->band_min = saved_band;
        return rc;
    };
    float t_ovh[sizeof(kOverheads) / sizeof(int)];
    auto sweep_overhead = [&](int band_min, int* best) -> int {
        float bt = -1.0f;
        for (size_t i = 0; i < sizeof(kOverheads) / sizeof(int); ++i) {
            int rc = timed(kOverheads[i], band_min, &t_ovh[i]);
            if (rc) return rc;
            if (bt < 0.0f || t_ovh[i] < bt) {
                bt = t_ovh[i];
                *best = kOverheads[i];
            }
        }
        return SWGB_OK;
    };
    int ovh = saved_ovh, band_min = saved_band, rc;
    if ((rc = sweep_overhead(band_min, &ovh))) return fail_restore(rc);
    float bt = -1.0f;
    for (int bm : kBandMins) {
        float t;
        if ((rc = timed(ovh, bm, &t))) return fail_restore(rc);
        if (bm == 0) tu.band_off_ms = t;
        if (bt < 0.0f || t < bt) {
            bt = t;
            band_min = bm;
        }
    }
    if ((rc = sweep_overhead(band_min, &ovh))) return fail_restore(rc);
    tu.tile_overhead = ovh;
    tu.band_min = band_min;
    tu.best_ms = -1.0f;
    tu.runner_up_ms = -1.0f;
    for (size_t i = 0; i < sizeof(kOverheads) / sizeof(int); ++i) {
        if (kOverheads[i] == ovh) {
            tu.best_ms = t_ovh[i];
        } else if (tu.runner_up_ms < 0.0f || t_ovh[i] < tu.runner_up_ms) {
            tu.runner_up_ms = t_ovh[i];
            tu.runner_up_overhead = kOverheads[i];
        }
    }
    ctx->tile_overhead = ovh;
    ctx->band_min = band_min;
    ctx->tuning = tu;
    if (best_overhead) *best_overhead = ovh;
    if (best_ms) *best_ms = tu.best_ms;
    return SWGB_OK;
}
