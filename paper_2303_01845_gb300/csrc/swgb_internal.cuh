// swgb_internal.cuh -- declarations shared by the host API (swgb_api.cu) and
// the kernels (swgb_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "swgb.h"

namespace swgb {

// ---- alphabet / profile --------------------------------------------------
constexpr int kAlpha = SWGB_ALPHABET_SIZE;  // residue codes 0..23
constexpr int kPadCode = kAlpha;            // code of a padding position
constexpr int kProfileRows = kAlpha + 1;    // one profile row per query code + pad
constexpr int kMatStride = 32;              // padded row of the staged matrix
// Biased profile value of any cell touching padding.  The real value s + o + e
// of a padded cell is <= -1 for every accepted gap setting, so a padded cell
// never scores strictly above the best real cell that feeds it.
constexpr int kPadProfile = -64;

// Scoring parameters as the kernels see them (passed by value).
struct ScoreArgs {
    // prof[x][y] = s(x, y) + o + e for x, y < 24; kPadProfile where x or y is
    // the pad code.  Row = query code, column = reference code.
    int8_t prof[kProfileRows][kMatStride];
    // The packed 16-bit path's table: the same for x, y < 24, and 0 (a score
    // of -(o + e)) at the pad code.  That path takes a matrix only if every
    // s(x, y) + o + e >= 0, so all entries are 0..127.
    uint8_t profu[kProfileRows][kMatStride];
    int32_t go, ge;
    int32_t one;   // always 1; a run-time multiplier the compiler cannot fold
    // rows of the per-pair profile: one per query letter the query set uses
    // plus one for padding.  Sets of the 20 standard letters (codes 0..19)
    // need 21; otherwise all 25.  The pad row is the last.
    int32_t prof_rows;
};
constexpr int kStdLetters = 20;

struct SeqView {
    const uint8_t* res;   // codes
    const int64_t* off;   // n + 1 offsets
    int64_t n;
};

// ---- bucketing -------------------------------------------------------------
// A pair's DP is laid out with the reference along the lanes ("held", rows of
// a tile) and the query streamed through the wavefront.  Tile shapes: G lanes
// per pair group x R rows per lane.
//   shape: 0     1      2     3      4 .. 12               13 .. 20
//   (G,R): (4,8) (4,12) (8,8) (8,12) (16,8) .. (16,16)     (32,9) .. (32,16)
// The 16- and 32-lane tiles step by one row per lane (16 or 32 rows), which
// keeps the rows padded past the end of the reference few; (32,8) would never
// win over (16,16), which has the same rows and half the wavefront fill.  Shapes from kFirstChunkable on (one group per warp) also
// cover references longer than one tile, in chunks of G*R rows.
constexpr int kNumShapes = 21;
constexpr int kFirstChunkable = 13;
__host__ __device__ constexpr int shape_G(int s) { return s < 2 ? 4 : s < 4 ? 8 : s < 13 ? 16 : 32; }
__host__ __device__ constexpr int shape_R(int s) {
    return s < 4 ? ((s & 1) ? 12 : 8) : s < 13 ? 8 + (s - 4) : 9 + (s - 13);
}
// bytes of profile per lane and query letter: R rounded up to whole words
__host__ __device__ constexpr int shape_LS(int s) { return (shape_R(s) + 3) / 4 * 4; }
constexpr int kChunkBuckets = 16;             // chunk-count buckets of a chunkable shape
constexpr int kBucketsPerClass = kFirstChunkable + (kNumShapes - kFirstChunkable) * kChunkBuckets;
constexpr int kClasses = 2;                   // 0 = packed 16x2, 1 = 32-bit
constexpr int kNumBuckets = kClasses * kBucketsPerClass;
constexpr int kQBins = 512;                   // streamed-length bins per bucket
constexpr int kQBinShift = 3;                 // 8 residues per bin
constexpr int kNumKernels = kClasses * kNumShapes;

// ---- banded reverse pass ---------------------------------------------------
// A scored pair on the packed path whose sequences are both at least the
// context's band_min long may run its reverse pass over a staircase band of
// the reversed prefixes (la query x lb reference positions) instead of the
// whole rectangle.  It runs on a 32-lane tile of ROWS = 32 R rows: chunk c
// (reversed reference rows [c ROWS, (c + 1) ROWS)) streams only the window
// [c ROWS - khi, (c + 1) ROWS + W - khi) of query positions, which holds the
// diagonals (khi - W, khi] (row - position) of every row of the chunk.
// band_geometry centres them on the segment from the origin's diagonal 0 to
// the far corner's lb - la, with band_margin(L) diagonals free on each side.
// The DP over the band is anchored (H = 0 only before the origin, kFloorH
// outside the band and as the floor), and its start is kept only under the
// exactness certificate the kernel checks; otherwise the pair is re-run over
// the whole rectangle.
constexpr int kFloorH = -8192;
__host__ __device__ constexpr int64_t band_margin(int64_t L) { return 64 + L / 32; }
__host__ __device__ inline void band_geometry(int64_t la, int64_t lb, int64_t* W, int64_t* khi) {
    const int64_t d = lb - la;
    const int64_t m = band_margin(la > lb ? la : lb);
    *W = (d < 0 ? -d : d) + 2 * m;
    *khi = (d > 0 ? d : 0) + m;
}
// Window [w0, w1) of chunk c (rows per chunk `rows`), clipped to [0, la).
__host__ __device__ inline void band_window(int64_t c, int64_t rows, int64_t W, int64_t khi, int64_t la,
                                            int64_t* w0, int64_t* w1) {
    const int64_t lo = c * rows - khi, hi = (c + 1) * rows + W - khi;
    *w0 = lo < 0 ? 0 : lo;
    *w1 = hi > la ? la : hi;
}
// Per-pair maxima of the forward pass's H over the reference rows of each
// forward lane, the certificate's bound on the part of an alignment beyond a
// band exit.  The keys kernel hands each recording pair a slice of
// 1 + ceil(lr / Rf) entries (fmax_off[p], -1 = none; Rf = its forward tile's
// rows per lane): entry 0 holds Rf, entry 1 + k the largest H of reference
// rows [k Rf, (k + 1) Rf), written once by the forward lane holding them.
// Shortest query and reference (whole sequences) of a pair whose forward pass
// records them; the context's setting, tuned by swgb_autotune (0 = no banded
// reverse pass, the default).
constexpr int kBandMinDefault = 0;
// Entries of a store's forward-maxima pool at most (int32 each, 512 MB).
constexpr int64_t kFmaxPoolMax = int64_t(1) << 27;
// The band tiles are the chunkable shapes with 9 to 13 rows per lane (smaller
// chunks give narrower windows, and these kernels keep all their state in
// registers); their buckets follow the classes' buckets, kChunkBuckets per
// shape (more chunks first).
constexpr int kBandShapeEnd = kFirstChunkable + 5;
constexpr int kBandShapes = kBandShapeEnd - kFirstChunkable;
constexpr int kBandFirstBucket = kNumBuckets;
constexpr int kNumBins = (kNumBuckets + kBandShapes * kChunkBuckets) * kQBins;
__host__ __device__ inline int band_first_bucket(int s) {
    return kBandFirstBucket + (s - kFirstChunkable) * kChunkBuckets;
}
__host__ __device__ inline int band_end_bucket(int s) { return band_first_bucket(s) + kChunkBuckets; }
__host__ __device__ inline int band_bucket_of(int s, int nch) {
    return band_first_bucket(s) + kChunkBuckets - (nch < kChunkBuckets ? nch : kChunkBuckets);
}
// work-queue counters: forward, reverse, reverse fallback (per class and
// shape), then one per band shape
constexpr int kTaskCounters = 3 * kNumKernels + kBandShapes;

// Tile of a pair: the shape (and chunk count) of least modelled cost, where a
// pair costs (streamed steps incl. the G-1 wavefront fill) x chunks x G x
// (R + overhead) -- R cell updates plus the per-step work of a lane counted in
// rows (loop control, letter fetch, max tracking), shared by the 32/G groups
// of a warp.  The overhead is a context setting (default kTileOverhead), tuned
// by swgb_autotune.
constexpr int kTileOverhead = 6;
__host__ __device__ inline void choose_shape(int64_t lq, int64_t lr, int overhead, int* shape, int* nch) {
    int64_t best = -1;
    for (int s = 0; s < kNumShapes; ++s) {
        const int64_t rows = (int64_t)shape_G(s) * shape_R(s);
        int64_t n = 1;
        if (lr > rows) {
            if (s < kFirstChunkable) continue;
            n = (lr + rows - 1) / rows;
        }
        const int64_t cost = (lq + shape_G(s) - 1) * n * shape_G(s) * (shape_R(s) + overhead);
        if (best < 0 || cost < best) {
            best = cost;
            *shape = s;
            *nch = (int)n;
        }
    }
}

__host__ __device__ inline int shape_first_bucket(int cls, int s) {
    return cls * kBucketsPerClass +
           (s < kFirstChunkable ? s : kFirstChunkable + (s - kFirstChunkable) * kChunkBuckets);
}
__host__ __device__ inline int shape_end_bucket(int cls, int s) {
    return shape_first_bucket(cls, s) + (s < kFirstChunkable ? 1 : kChunkBuckets);
}
// more chunks first: the longest pairs start first in the persistent grid
__host__ __device__ inline int bucket_of(int cls, int s, int nch) {
    const int b = shape_first_bucket(cls, s);
    if (s < kFirstChunkable) return b;
    return b + kChunkBuckets - (nch < kChunkBuckets ? nch : kChunkBuckets);
}

// What the keys kernel needs to put a pair on the packed 16-bit path: the
// score can only pass 32767 if max_score * min(lq, lr) does, and never exceeds
// min(sum_i rowmax[q_i], sum_j colmax[r_j]) (every aligned query residue
// contributes at most its best substitution score, likewise every reference
// residue; gaps only subtract).
struct ClassArgs {
    int32_t max_score;            // max(0, largest matrix entry)
    int8_t rowmax[kMatStride];    // max(0, max_y s(x, y)) per query code x
    int8_t colmax[kMatStride];    // max(0, max_x s(x, y)) per reference code y
    int32_t force32;
    int32_t tile_overhead;        // per-step lane work in rows (choose_shape)
    int32_t band_min;             // forward maxima / banded reverse from this length (0 = off)
};

// Tile of a banded reverse pass of query prefix lq, reference prefix lr and
// score S: the band shape of least modelled cost over its chunk windows
// (choose_shape's per-step cost), if that is below the whole rectangle's cost
// by a tenth (the share kept for pairs the certificate sends back); returns
// false otherwise.  The reverse pass stops after the start: an alignment that
// scores S spans about S / 2 streamed positions on these workloads
// (homologous pairs gain 2 to 3 per column), so both models stream at most
// a = min(lq, S / 2 + 1) positions.  The choice changes no result.
// A score large enough that choose_band streams the whole query prefix.
constexpr int64_t kBandAnyScore = int64_t(1) << 40;
__host__ __device__ inline bool choose_band(int64_t lq, int64_t lr, int64_t S, int overhead, int* shape,
                                            int* nch) {
    int64_t a = S / 2 + 1;
    if (a > lq) a = lq;
    int fs = 0, fn = 1;
    choose_shape(a, lr, overhead, &fs, &fn);
    const int64_t full = (a + shape_G(fs) - 1) * fn * shape_G(fs) * (shape_R(fs) + overhead);
    int64_t W = 0, khi = 0;
    band_geometry(lq, lr, &W, &khi);
    int64_t best = -1;
    for (int s = kFirstChunkable; s < kBandShapeEnd; ++s) {
        const int64_t rows = (int64_t)shape_G(s) * shape_R(s);
        const int64_t n = (lr + rows - 1) / rows;
        int64_t steps = 0;
        for (int64_t c = 0; c < n; ++c) {
            int64_t w0 = 0, w1 = 0;
            band_window(c, rows, W, khi, lq, &w0, &w1);
            if (w1 > a) w1 = a;
            if (w1 <= w0) break;
            steps += (w1 - w0 + shape_G(s) + 2) / 4 * 4;
        }
        const int64_t cost = steps * shape_G(s) * (shape_R(s) + overhead);
        if (best < 0 || cost < best) {
            best = cost;
            *shape = s;
            *nch = (int)n;
        }
    }
    return best >= 0 && best * 10 < full * 9;
}

// Per-call device workspace (owned by the context).
struct Workspace {
    uint32_t* hist;        // [kNumBins]
    uint32_t* scan;        // [kNumBins + 1] exclusive scan of hist
    uint32_t* cursor;      // [kNumBins] scatter cursors
    int32_t* bin_of;       // [n_pairs] bin of each pair (-1 = not aligned)
    int32_t* order;        // [n_pairs] pair ids sorted by bin
    uint32_t* task_ctr;    // [kTaskCounters] work-queue counters
    int32_t* status;       // [1] device status word
    unsigned long long* counters;  // [8] cells / class counts
    uint2* boundary;       // chunk-boundary rows, [slots][boundary_stride]
    int64_t boundary_stride;
    int64_t boundary_slots;
    int32_t* fmax;         // forward maxima slices (null: no banded reverse pass)
    int64_t fmax_capacity; // entries of fmax
    int64_t* fmax_off;     // [fmax_off_n] slice of each pair, -1 = none
    int64_t fmax_off_n;    // entries of fmax_off (pairs a call may record)
};

// Arguments of one DP launch.
struct DPArgs {
    SeqView q, r;
    const int32_t* pairs;
    const int32_t* order;
    const uint32_t* scan;       // bin scan: range = [scan[b0*kQBins], scan[b1*kQBins])
    uint32_t* task_ctr;
    swgb_record* out;
    int32_t* status;
    uint2* boundary;
    int64_t boundary_stride;
    int64_t boundary_slots;
    int32_t first_bucket, end_bucket;
    int32_t* fmax;              // forward maxima slices (forward: written; banded reverse: read)
    const int64_t* fmax_off;    // slice of each pair (-1 = none); null: no maxima
    unsigned long long* counters;
    ScoreArgs sc;
};

enum Counter {
    kCtrFwdCells = 0,
    kCtrRevCells = 1,
    kCtrInt16 = 2,
    kCtrInt32 = 3,
    kCtrRevPairs = 4,
    kCtrBandPairs = 5,      // reverse passes run over a band
    kCtrBandCertified = 6,  // of which the certificate held
    kCtrFmaxUsed = 7,       // forward-maxima entries handed out
    kCtrFwdSlots = 8,       // cell updates the forward DP kernels computed (fill, padding included)
    kCtrRevSlots = 9,       // likewise, the reverse pass (all its rounds)
};
constexpr int kNumCounters = 16;

// Marker left in q_start by the banded reverse pass for a pair whose
// certificate did not hold: the fallback keys pass sends it to the full
// reverse pass.
constexpr int32_t kBandFallback = -2;

// ---- launchers (swgb_kernels.cu) -------------------------------------------
// flags[0] |= 1 on a residue outside the alphabet; flags[1] = max(flags[1], code)
cudaError_t launch_encode(const uint8_t* in, uint8_t* out, int64_t n, bool ascii,
                          int32_t* flags, cudaStream_t st);
// Checks the n_seqs + 1 device offsets (flags[0] |= 1 decreasing, 2 longer than
// max_len; flags[1] = longest length) and subtracts base from each.
cudaError_t launch_offsets(int64_t* off, int64_t n_seqs, int64_t base, int64_t max_len, int32_t* flags,
                           cudaStream_t st);
// mode 0: forward keys; 1: reverse keys (band or full rectangle); 2: the
// pairs the banded pass left for the full reverse pass
enum KeysMode { kKeysForward = 0, kKeysReverse = 1, kKeysFallback = 2 };
cudaError_t launch_keys(const SeqView& q, const SeqView& r, const int32_t* pairs, int64_t n_pairs,
                        swgb_record* out, int mode, const ClassArgs& ca,
                        const Workspace& ws, cudaStream_t st);
cudaError_t launch_scan(const Workspace& ws, cudaStream_t st);
cudaError_t launch_scatter(int64_t n_pairs, const Workspace& ws, cudaStream_t st);
// Launches the DP kernel of (class, shape); grid sized from occupancy.  band:
// the banded reverse pass of a chunkable shape on the packed path.
cudaError_t launch_dp(int cls, int shape, bool reverse, const DPArgs& a, int grid_blocks,
                      cudaStream_t st, bool band = false);
// Blocks per SM the DP kernel of (class, shape, direction) can keep resident
// with prof_rows profile rows.
int dp_blocks_per_sm(int cls, int shape, bool reverse, int prof_rows, bool band = false);
// Threads per block of every DP kernel.
constexpr int kDPThreads = 64;
size_t dp_smem_bytes(int cls, int shape, int prof_rows);
cudaError_t dp_configure(int cls, int shape, bool reverse);
cudaError_t launch_probe_addmax(unsigned long long* cycles, uint32_t* sink, int blocks,
                                int iters, cudaStream_t st);
constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

}  // namespace swgb
