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
    int32_t go, ge;
};

struct SeqView {
    const uint8_t* res;   // codes
    const int64_t* off;   // n + 1 offsets
    int64_t n;
};

// ---- bucketing -------------------------------------------------------------
// A pair's DP is laid out with the reference along the lanes ("held", rows of
// a tile) and the query streamed through the wavefront.  Tile shapes (lanes
// per pair group G x rows per lane R):
constexpr int kNumShapes = 5;
constexpr int kShapeG[kNumShapes] = {4, 8, 16, 32, 32};
constexpr int kShapeR[kNumShapes] = {8, 8, 8, 8, 16};
constexpr int kChunkRows = 512;               // rows per chunk of the last shape
constexpr int kChunkBuckets = 16;             // chunk-count buckets of the last shape
constexpr int kBucketsPerClass = (kNumShapes - 1) + kChunkBuckets;
constexpr int kClasses = 2;                   // 0 = packed 16x2, 1 = 32-bit
constexpr int kNumBuckets = kClasses * kBucketsPerClass;
constexpr int kQBins = 1024;                  // streamed-length bins per bucket
constexpr int kQBinShift = 2;                 // 4 residues per bin
constexpr int kNumBins = kNumBuckets * kQBins;
constexpr int kNumKernels = kClasses * kNumShapes;

__host__ __device__ inline int shape_of(int64_t held_len) {
    if (held_len <= 32) return 0;
    if (held_len <= 64) return 1;
    if (held_len <= 128) return 2;
    if (held_len <= 256) return 3;
    return 4;
}

__host__ __device__ inline int bucket_of(int cls, int64_t held_len) {
    int s = shape_of(held_len);
    if (s < kNumShapes - 1) return cls * kBucketsPerClass + s;
    int64_t chunks = (held_len + kChunkRows - 1) / kChunkRows;
    int cb = (int)(chunks < kChunkBuckets ? chunks : kChunkBuckets) - 1;
    return cls * kBucketsPerClass + (kNumShapes - 1) + cb;
}

// first and one-past-last bucket of (class, shape)
__host__ __device__ inline int shape_first_bucket(int cls, int s) {
    return cls * kBucketsPerClass + s;
}
__host__ __device__ inline int shape_end_bucket(int cls, int s) {
    return s < kNumShapes - 1 ? cls * kBucketsPerClass + s + 1 : (cls + 1) * kBucketsPerClass;
}

// Per-call device workspace (owned by the context).
struct Workspace {
    uint32_t* hist;        // [kNumBins]
    uint32_t* scan;        // [kNumBins + 1] exclusive scan of hist
    uint32_t* cursor;      // [kNumBins] scatter cursors
    int32_t* bin_of;       // [n_pairs] bin of each pair (-1 = not aligned)
    int32_t* order;        // [n_pairs] pair ids sorted by bin
    uint32_t* task_ctr;    // [2 * kNumKernels] work-queue counters (fwd, rev)
    int32_t* status;       // [1] device status word
    unsigned long long* counters;  // [8] cells / class counts
    uint2* boundary;       // chunk-boundary rows, [slots][boundary_stride]
    int64_t boundary_stride;
    int64_t boundary_slots;
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
    ScoreArgs sc;
};

enum Counter {
    kCtrFwdCells = 0,
    kCtrRevCells = 1,
    kCtrInt16 = 2,
    kCtrInt32 = 3,
    kCtrRevPairs = 4,
};

// ---- launchers (swgb_kernels.cu) -------------------------------------------
cudaError_t launch_encode(const uint8_t* in, uint8_t* out, int64_t n, bool ascii,
                          int32_t* bad_flag, cudaStream_t st);
cudaError_t launch_keys(const SeqView& q, const SeqView& r, const int32_t* pairs, int64_t n_pairs,
                        swgb_record* out, bool reverse, bool force32, int max_score,
                        const Workspace& ws, cudaStream_t st);
cudaError_t launch_scan(const Workspace& ws, cudaStream_t st);
cudaError_t launch_scatter(int64_t n_pairs, const Workspace& ws, cudaStream_t st);
// Launches the DP kernel of (class, shape); grid sized from occupancy.
cudaError_t launch_dp(int cls, int shape, bool reverse, const DPArgs& a, int grid_blocks,
                      cudaStream_t st);
// Blocks per SM the DP kernel of (class, shape, direction) can keep resident.
int dp_blocks_per_sm(int cls, int shape, bool reverse);
// Threads per block of every DP kernel.
constexpr int kDPThreads = 128;
size_t dp_smem_bytes(int cls, int shape);
cudaError_t dp_configure(int cls, int shape, bool reverse);
cudaError_t launch_probe_addmax(unsigned long long* cycles, uint32_t* sink, int blocks,
                                int iters, cudaStream_t st);
constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

}  // namespace swgb
