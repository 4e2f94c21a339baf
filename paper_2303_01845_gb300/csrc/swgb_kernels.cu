// swgb_kernels.cu -- sm_103a kernels of libswgb.
//
// The hot kernel is dp_kernel: the affine-gap local-alignment recurrence of
// include/swgb.h evaluated over whole score matrices (the paper's alignment
// step; cell updates of the forward pass are its CUPS metric, Sec. "How
// Performance Was Measured").  Layout of one pair group:
//
//   * the reference ("held" sequence) is cut into chunks of G*R rows; lane k
//     of a group of G lanes holds rows [k*R, k*R+R) of the chunk in registers;
//   * the query is streamed: at step t lane k updates query position
//     i = t - k, so the lanes form an anti-diagonal wavefront and each lane
//     receives the values of the row above its first row from lane k-1 by a
//     warp shuffle (the previous step's output of that lane);
//   * on the packed path every register holds two independent pairs (low and
//     high 16 bits, every value biased by kBias so both halves stay unsigned);
//     a cell update is four unsigned dual add-max / max instructions on the
//     integer pipe plus two packed adds issued as multiply-adds on the FMA
//     pipe (a biased 32-bit add never carries between the halves);  pairs
//     whose score could pass 32767 run on 32-bit registers, five add-max
//     instructions per cell;
//   * substitution scores come from a per-pair profile in shared memory,
//     prof[query code][held row] = s + o + e (8-bit), read as R bytes per
//     lane per step and widened by one byte-permute per register.
//
// Work distribution: pairs are bucketed on the device by held length (tile
// shape) and sorted by query length (longest first); one persistent launch per
// (precision class, tile shape) pulls pair groups from an atomic counter.
#include <climits>
#include <cstdint>
#include <type_traits>

#include "swgb_internal.cuh"
#include "swgb_lane.cuh"

namespace swgb {

// SMs of the current device: caps the grids of the grid-stride kernels.
static int64_t sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
        return 1;
    return n;
}

// ---------------------------------------------------------------------------
// Residue encoding (ASCII letters or codes -> codes 0..23)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint8_t ascii_code(int c) {
    if (c >= 'a' && c <= 'z') c -= 'a' - 'A';
    switch (c) {
        case 'A': return 0;  case 'R': return 1;  case 'N': return 2;  case 'D': return 3;
        case 'C': return 4;  case 'Q': return 5;  case 'E': return 6;  case 'G': return 7;
        case 'H': return 8;  case 'I': return 9;  case 'L': return 10; case 'K': return 11;
        case 'M': return 12; case 'F': return 13; case 'P': return 14; case 'S': return 15;
        case 'T': return 16; case 'W': return 17; case 'Y': return 18; case 'V': return 19;
        case 'B': return 20; case 'Z': return 21; case 'X': return 22; case '*': return 23;
        case 'U': case 'O': return 22;
        default: return 255;
    }
}

__global__ void encode_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                              int64_t n, int ascii, int32_t* flags) {
    __shared__ uint8_t tab[256];
    __shared__ int32_t block_max;
    for (int k = threadIdx.x; k < 256; k += blockDim.x)
        tab[k] = ascii ? ascii_code(k) : (k < kAlpha ? (uint8_t)k : (uint8_t)255);
    if (threadIdx.x == 0) block_max = 0;
    __syncthreads();
    int any_bad = 0, mx = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        uint8_t c = tab[in[k]];
        if (c == 255) {
            any_bad = 1;
            c = 0;
        }
        mx = max(mx, (int)c);
        out[k] = c;
    }
    for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&block_max, mx);
    if (__syncthreads_or(any_bad) && threadIdx.x == 0) atomicOr(&flags[0], 1);
    if (threadIdx.x == 0) atomicMax(&flags[1], block_max);
}

// Residues given as codes, 16 per thread: a code of 24 or more becomes 0 and
// sets flags[0]; flags[1] = max(flags[1], largest code).  Per-byte SIMD compare
// and max, so the pass moves at copy speed (also when `in` is pinned host
// memory read over the host link).
__global__ void encode_codes16_kernel(const uint4* __restrict__ in, uint4* __restrict__ out, int64_t n16,
                                      int32_t* flags) {
    __shared__ uint32_t block_max;
    if (threadIdx.x == 0) block_max = 0;
    __syncthreads();
    uint32_t bad = 0, mx = 0;
    const uint32_t lim = 0x18181818u;   // 24 in every byte
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n16; k += stride) {
        uint4 v = in[k];
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t over = __vcmpgeu4(w[j], lim);   // 0xff in bytes >= 24
            bad |= over;
            w[j] &= ~over;
            mx = __vmaxu4(mx, w[j]);
        }
        out[k] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    mx = max(max(mx & 0xffu, (mx >> 8) & 0xffu), max((mx >> 16) & 0xffu, mx >> 24));
    for (int off = 16; off > 0; off >>= 1) {
        mx = max(mx, __shfl_xor_sync(kFull, mx, off));
        bad |= __shfl_xor_sync(kFull, bad, off);
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&block_max, mx);
    if (__syncthreads_or(bad != 0) && threadIdx.x == 0) atomicOr(&flags[0], 1);
    if (threadIdx.x == 0) atomicMax(&flags[1], (int32_t)block_max);
}

cudaError_t launch_encode(const uint8_t* in, uint8_t* out, int64_t n, bool ascii,
                          int32_t* flags, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t head = 0;
    if (!ascii && ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0) {
        const int64_t n16 = n / 16;
        if (n16 > 0) {
            int64_t blocks = (n16 + 255) / 256;
            if (blocks > sm_count() * 8) blocks = sm_count() * 8;
            encode_codes16_kernel<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<const uint4*>(in),
                                                                    reinterpret_cast<uint4*>(out), n16, flags);
        }
        head = n16 * 16;
    }
    if (head < n) {
        int64_t blocks = (n - head + 255) / 256;
        if (blocks > sm_count() * 32) blocks = sm_count() * 32;
        encode_kernel<<<(unsigned)blocks, 256, 0, st>>>(in + head, out + head, n - head, ascii ? 1 : 0, flags);
    }
    return cudaGetLastError();
}

// Sequence offsets of a set being loaded: flags[0] |= 1 where an offset
// decreases, |= 2 where a sequence is longer than max_len; flags[1] = max(
// flags[1], longest length within the limit).  Read only: the lengths are
// differences of neighbours, so the rebase runs as a separate pass.
__global__ void offsets_check_kernel(const int64_t* __restrict__ off, int64_t n, int64_t max_len,
                                     int32_t* flags) {
    int bad = 0, mx = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const int64_t len = off[k + 1] - off[k];
        if (len < 0) bad |= 1;
        else if (len > max_len) bad |= 2;
        else mx = max(mx, (int)len);
    }
    for (int o = 16; o > 0; o >>= 1) {
        bad |= __shfl_xor_sync(kFull, bad, o);
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(&flags[0], bad);
        atomicMax(&flags[1], mx);
    }
}

__global__ void offsets_rebase_kernel(int64_t* off, int64_t n, int64_t base) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) off[k] -= base;
}

cudaError_t launch_offsets(int64_t* off, int64_t n_seqs, int64_t base, int64_t max_len, int32_t* flags,
                           cudaStream_t st) {
    if (n_seqs <= 0) return cudaSuccess;
    int64_t blocks = (n_seqs + 255) / 256;
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    offsets_check_kernel<<<(unsigned)blocks, 256, 0, st>>>(off, n_seqs, max_len, flags);
    if (base != 0) offsets_rebase_kernel<<<(unsigned)blocks, 256, 0, st>>>(off, n_seqs + 1, base);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Bucketing: keys + histogram, scan, scatter
// ---------------------------------------------------------------------------
// Upper bound of the score of a pair from its residues (see ClassArgs).
__device__ int64_t score_bound(const uint8_t* __restrict__ q, int64_t lq, const uint8_t* __restrict__ r,
                               int64_t lr, const ClassArgs& ca) {
    int64_t bq = 0, br = 0;
    for (int64_t i = 0; i < lq; ++i) bq += ca.rowmax[q[i]];
    for (int64_t j = 0; j < lr; ++j) br += ca.colmax[r[j]];
    return bq < br ? bq : br;
}

// Hands each lane of a warp `need` consecutive entries of a shared pool whose
// cursor is *ctr: one atomic per warp.  Every lane of the warp calls it.
__device__ int64_t warp_alloc(unsigned long long* ctr, int64_t need) {
    const int lane = threadIdx.x & 31;
    int64_t incl = need;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t o = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += o;
    }
    const int64_t total = __shfl_sync(kFull, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(ctr, (unsigned long long)total);
    base = __shfl_sync(kFull, base, 31);
    return (int64_t)base + incl - need;
}

__global__ void keys_kernel(SeqView q, SeqView r, const int32_t* __restrict__ pairs,
                            int64_t n_pairs, swgb_record* out, int mode, ClassArgs ca,
                            Workspace ws) {
    unsigned long long cells = 0, n16 = 0, n32 = 0, nband = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // every lane of a warp runs the same iterations (warp_alloc)
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n_pairs; base += stride) {
        const int64_t p = base + threadIdx.x;
        const bool valid = p < n_pairs;
        int bin = -1;
        int64_t lq = 0, lr = 0;
        int cls = 0, band_shape = -1, band_nch = 0;
        int64_t fmax_need = 0, fmax_rows = 0;
        if (valid && mode == kKeysForward) {
            const int32_t qi = pairs[2 * p], ri = pairs[2 * p + 1];
            if (qi < 0 || qi >= q.n || ri < 0 || ri >= r.n) {
                set_status(ws.status, SWGB_ERANGE);
                zero_record(&out[p]);
            } else {
                lq = q.off[qi + 1] - q.off[qi];
                lr = r.off[ri + 1] - r.off[ri];
                if (lq == 0 || lr == 0) {
                    zero_record(&out[p]);
                    lq = lr = 0;
                } else if (ca.force32) {
                    cls = 1;
                } else if ((int64_t)ca.max_score * (lq < lr ? lq : lr) > 32767) {
                    cls = score_bound(q.res + q.off[qi], lq, r.res + r.off[ri], lr, ca) > 32767;
                }
                // a pair long enough for a banded reverse pass, and for which
                // the band would be cheaper if its alignment spanned it,
                // records the maxima of its forward lanes (packed path only)
                int bs = 0, bn = 0;
                if (ws.fmax_off && ca.band_min > 0 && p < ws.fmax_off_n && cls == 0 && lq >= ca.band_min &&
                    lr >= ca.band_min && choose_band(lq, lr, kBandAnyScore, ca.tile_overhead, &bs, &bn)) {
                    int shape = 0, nch = 1;
                    choose_shape(lq, lr, ca.tile_overhead, &shape, &nch);
                    fmax_rows = shape_R(shape);
                    fmax_need = 1 + (lr + fmax_rows - 1) / fmax_rows;
                }
            }
        } else if (valid) {
            const swgb_record rec = out[p];
            const bool take = mode == kKeysReverse ? rec.score > 0 : (rec.score > 0 && rec.q_start == kBandFallback);
            if (take) {
                // The reverse pass reads the prefixes q[0..q_end], r[0..r_end]
                // through the forward record: check that the record lies inside
                // its pair (0 <= q_end < lq, 0 <= r_end < lr) and that its score
                // is attainable there (at most max_score per aligned column),
                // else report EINTERNAL and leave the pair out with a zero record.
                const int32_t qi = pairs[2 * p], ri = pairs[2 * p + 1];
                bool ok = qi >= 0 && qi < q.n && ri >= 0 && ri < r.n;
                int64_t nq = 0, nr = 0;
                if (ok) {
                    nq = q.off[qi + 1] - q.off[qi];
                    nr = r.off[ri + 1] - r.off[ri];
                    ok = rec.q_end >= 0 && rec.q_end < nq && rec.r_end >= 0 && rec.r_end < nr &&
                         (int64_t)rec.score <=
                             (int64_t)ca.max_score * (rec.q_end < rec.r_end ? rec.q_end + 1 : rec.r_end + 1);
                }
                if (ok) {
                    lq = (int64_t)rec.q_end + 1;
                    lr = (int64_t)rec.r_end + 1;
                    // every cell of the reversed prefixes scores at most S
                    cls = (ca.force32 || rec.score > 32767) ? 1 : 0;
                    // a banded pass needs the pair's forward maxima
                    if (mode == kKeysReverse && cls == 0 && ws.fmax_off && ca.band_min > 0 &&
                        p < ws.fmax_off_n && nq >= ca.band_min && nr >= ca.band_min && ws.fmax_off[p] >= 0 &&
                        !choose_band(lq, lr, rec.score, ca.tile_overhead, &band_shape, &band_nch))
                        band_shape = -1;
                } else {
                    set_status(ws.status, SWGB_EINTERNAL);
                    zero_record(&out[p]);
                }
            }
        }
        if (mode == kKeysForward && ws.fmax_off && ca.band_min > 0) {
            // the slice of the forward maxima (all lanes: warp_alloc); only a
            // banded call, whose workspace holds an entry per pair, records
            const int64_t off = warp_alloc(&ws.counters[kCtrFmaxUsed], fmax_need);
            if (valid && p < ws.fmax_off_n) {
                const bool got = fmax_need > 0 && off + fmax_need <= ws.fmax_capacity;
                ws.fmax_off[p] = got ? off : -1;
                if (got) ws.fmax[off] = (int32_t)fmax_rows;
            }
        }
        if (lq > 0) {
            int bucket;
            int64_t qb;
            if (band_shape >= 0) {
                // band pairs sorted by the drift of the end diagonal, so that
                // the two pairs of a warp share most of their windows
                bucket = band_bucket_of(band_shape, band_nch);
                qb = (lr - lq + 4 * (kQBins / 2)) / 4;
                ++nband;
            } else {
                int shape = 0, nch = 1;
                choose_shape(lq, lr, ca.tile_overhead, &shape, &nch);
                bucket = bucket_of(cls, shape, nch);
                qb = lq >> kQBinShift;
            }
            if (qb < 0) qb = 0;
            if (qb > kQBins - 1) qb = kQBins - 1;
            bin = bucket * kQBins + (kQBins - 1 - (int)qb);
            atomicAdd(&ws.hist[bin], 1u);
            if (mode != kKeysFallback) {
                cells += (unsigned long long)(lq * lr);
                if (cls == 0) ++n16; else ++n32;
            }
        }
        if (valid) ws.bin_of[p] = bin;
    }
    // block reduction of the counters
    for (int off = 16; off > 0; off >>= 1) {
        cells += __shfl_xor_sync(kFull, cells, off);
        n16 += __shfl_xor_sync(kFull, n16, off);
        n32 += __shfl_xor_sync(kFull, n32, off);
        nband += __shfl_xor_sync(kFull, nband, off);
    }
    if ((threadIdx.x & 31) == 0 && (cells | n16 | n32 | nband)) {
        if (mode == kKeysForward) {
            atomicAdd(&ws.counters[kCtrFwdCells], cells);
            atomicAdd(&ws.counters[kCtrInt16], n16);
            atomicAdd(&ws.counters[kCtrInt32], n32);
        } else if (mode == kKeysReverse) {
            atomicAdd(&ws.counters[kCtrRevCells], cells);
            atomicAdd(&ws.counters[kCtrRevPairs], n16 + n32);
            atomicAdd(&ws.counters[kCtrBandPairs], nband);
        }
    }
}

cudaError_t launch_keys(const SeqView& q, const SeqView& r, const int32_t* pairs, int64_t n_pairs,
                        swgb_record* out, int mode, const ClassArgs& ca,
                        const Workspace& ws, cudaStream_t st) {
    if (n_pairs <= 0) return cudaSuccess;
    int64_t blocks = (n_pairs + 255) / 256;
    if (blocks > sm_count() * 16) blocks = sm_count() * 16;
    keys_kernel<<<(unsigned)blocks, 256, 0, st>>>(q, r, pairs, n_pairs, out, mode, ca, ws);
    return cudaGetLastError();
}

// Exclusive scan of hist[kNumBins] into scan (and the scatter cursors), in
// two launches over tiles of kScanTile bins, reads and writes coalesced:
// scan_tiles_kernel scans each tile locally and leaves the tile's total in the
// tile's first histogram entry (the histogram is not read again, and only the
// tile's own block reads that entry); scan_offsets_kernel adds to each tile the
// totals of the tiles before it.
constexpr int kScanTile = 1024;
constexpr int kScanTiles = (kNumBins + kScanTile - 1) / kScanTile;

// Block-wide inclusive scan of one value per thread (kScanTile threads).
__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t v, uint32_t* warp_sums) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t o = __shfl_up_sync(kFull, v, off);
        if (lane >= off) v += o;
    }
    if (lane == 31) warp_sums[w] = v;
    __syncthreads();
    if (w == 0) {
        uint32_t x = warp_sums[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(kFull, x, off);
            if (lane >= off) x += o;
        }
        warp_sums[lane] = x;
    }
    __syncthreads();
    return v + (w > 0 ? warp_sums[w - 1] : 0u);
}

__global__ void __launch_bounds__(kScanTile) scan_tiles_kernel(Workspace ws) {
    __shared__ uint32_t warp_sums[32];
    const int b = blockIdx.x * kScanTile + threadIdx.x;
    const uint32_t v = b < kNumBins ? ws.hist[b] : 0u;
    const uint32_t inc = block_inclusive_scan(v, warp_sums);
    if (b < kNumBins) ws.scan[b] = inc - v;
    __syncthreads();   // every thread has read its entry before the total overwrites the first
    if (threadIdx.x == kScanTile - 1) ws.hist[blockIdx.x * kScanTile] = inc;
}

__global__ void __launch_bounds__(kScanTile) scan_offsets_kernel(Workspace ws) {
    __shared__ uint32_t offset;
    if (threadIdx.x < 32) {
        uint32_t sum = 0;
        for (int t = threadIdx.x; t < (int)blockIdx.x; t += 32) sum += ws.hist[t * kScanTile];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(kFull, sum, off);
        if (threadIdx.x == 0) offset = sum;
    }
    __syncthreads();
    const int b = blockIdx.x * kScanTile + threadIdx.x;
    if (b < kNumBins) {
        const uint32_t x = ws.scan[b] + offset;
        ws.scan[b] = x;
        ws.cursor[b] = x;
    }
    if (blockIdx.x == kScanTiles - 1 && threadIdx.x == 0)
        ws.scan[kNumBins] = offset + ws.hist[blockIdx.x * kScanTile];
}

cudaError_t launch_scan(const Workspace& ws, cudaStream_t st) {
    scan_tiles_kernel<<<kScanTiles, kScanTile, 0, st>>>(ws);
    scan_offsets_kernel<<<kScanTiles, kScanTile, 0, st>>>(ws);
    return cudaGetLastError();
}

__global__ void scatter_kernel(int64_t n_pairs, Workspace ws) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs; p += stride) {
        const int bin = ws.bin_of[p];
        if (bin >= 0) {
            const uint32_t pos = atomicAdd(&ws.cursor[bin], 1u);
            ws.order[pos] = (int32_t)p;
        }
    }
}

cudaError_t launch_scatter(int64_t n_pairs, const Workspace& ws, cudaStream_t st) {
    if (n_pairs <= 0) return cudaSuccess;
    int64_t blocks = (n_pairs + 255) / 256;
    if (blocks > sm_count() * 16) blocks = sm_count() * 16;
    scatter_kernel<<<(unsigned)blocks, 256, 0, st>>>(n_pairs, ws);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The DP kernel
// ---------------------------------------------------------------------------
// Steps between refreshes of the group's score bound (forward) and between
// tests for the end of the reverse pass, whose bound is fixed.
__host__ __device__ constexpr int bound_every(bool reverse) { return reverse ? 32 : 16; }

// bytes of profile a warp stages: per group and pair, prof_rows x G x LS
__host__ __device__ constexpr int dp_prof_bytes_per_warp(int G, int R, bool P16, int prof_rows) {
    return (32 / G) * (P16 ? 2 : 1) * prof_rows * G * ((R + 3) / 4 * 4);
}

// REV = false: forward pass over q x r -> score and end cell.
// REV = true : local DP over the reversed prefixes q[q_end..0] x r[r_end..0]
//              of each scored pair -> start cell.  The score S is known, so the
//              pass stops once the wavefront is past the first step holding S.
// FMAX (forward, packed): also records the maxima of each lane's rows for the
//              banded reverse pass, in the tasks holding a pair that records
//              them (the wavefront is compiled with and without the running
//              maximum, chosen per task).
// BAND (reverse, packed, 32-lane tiles): the banded reverse pass.  Chunk c of
//              the reversed reference streams only its window [w0, wend) (the
//              union of the two halves' band windows); lane gl computes the
//              positions [w0 - gl, w0 - gl + steps) of its rows, so the
//              computed region D is a staircase of those ranges.  The DP is
//              anchored: H = 0 only before the origin, the floor kFloorH
//              outside D and below every cell.  Certificate: every cell x of
//              D with a successor y outside D (right, down or diagonal, inside
//              the matrix) is an exit.  An alignment from the origin that
//              leaves D leaves it first through an exit x: its part up to x
//              scores at most H_D(x), and the rest, read in the forward
//              direction, is a local alignment ending at y's cell, which scores
//              at most the forward H there plus o (had it opened with a gap
//              extension) -- at most the forward maximum of y's rows plus o.
//              A cell of value S reached that way lies at a position no
//              earlier than x's, so if every exit at a position <= a* (the
//              first position holding S in D) has H_D(x) + fmax(y's rows) + o
//              < S, the first cell of value S in D is the first in the whole
//              rectangle and the start is exact; otherwise the pair is marked
//              for the full reverse pass.  Exits are tracked per lane with
//              bounds over a few rows (conservative): the last two positions
//              of each lane's range (its right edge) and, for the bottom row
//              of a chunk, the positions the next chunk's first row does not
//              cover.
//
// Position of the maximum.  Every lane keeps lb1 = max(its running maximum,
// T - 1), T a lower bound of the pair's final score (the largest lb1 of the
// group, refreshed every bound_every steps).  When the maximum of a step's R
// rows passes lb1 -- it grew and reached T -- the lane copies its R registers
// (a snapshot per pair half) and the step.  The first row holding the value is
// read from the snapshot once per chunk.  A lane whose maximum never reached T
// holds no cell of the final score, so skipping its positions loses nothing;
// ties with T are recorded.
// Blocks per SM the shared-memory profile of a 21-row, R-row-per-lane launch
// leaves room for (8-, 12- or 16-byte lane strides), given to the compiler as
// the register budget: 65536 / (64 threads x blocks) registers per thread.
__host__ __device__ constexpr int dp_min_blocks(int R) { return R <= 8 ? 8 : R <= 12 ? 6 : 5; }

template <int G, int R, bool P16, bool REV, bool FMAX, bool BAND>
__global__ void __launch_bounds__(kDPThreads, dp_min_blocks(R)) dp_kernel(const DPArgs a) {
    static_assert(!FMAX || (P16 && !REV), "forward maxima are recorded by packed forward kernels");
    static_assert(!BAND || (P16 && REV && G == 32), "the banded reverse pass runs on packed 32-lane tiles");
    using L = Lane<P16>;
    constexpr int PACK = L::kPack;
    constexpr int GROUPS = 32 / G;
    constexpr int ROWS = G * R;                // reference rows per tile
    constexpr int LS = (R + 3) / 4 * 4;        // profile bytes per lane and letter
    constexpr int RS = G * LS;                 // profile bytes per letter
    const int prows = a.sc.prof_rows;          // profile rows, the pad row last
    const int pad_row = prows - 1;
    const int PROF = prows * RS;               // profile bytes per pair
    constexpr int NW = LS / 4;

    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t* tabT = smem;
    for (int k = threadIdx.x; k < kTabTBytes; k += blockDim.x) {
        const int y = k / kTabTStride, x = k % kTabTStride;
        const int xr = x == pad_row ? kPadCode : x;
        tabT[k] = x >= prows ? (uint8_t)0
                             : P16 ? a.sc.profu[xr][y] : (uint8_t)a.sc.prof[xr][y];
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int g = lane / G;    // pair group within the warp
    const int gl = lane % G;   // lane within the group
    int8_t* prof = reinterpret_cast<int8_t*>(smem + kSmatRegion) +
                   (size_t)warp * dp_prof_bytes_per_warp(G, R, P16, prows) + (size_t)g * PACK * PROF;
    const int8_t* plane = prof + gl * LS;   // this lane's rows within a profile row

    const int64_t begin = a.scan[(int64_t)a.first_bucket * kQBins];
    const int64_t end = a.scan[(int64_t)a.end_bucket * kQBins];
    const int64_t slot = (int64_t)blockIdx.x * (kDPThreads / 32) + warp;
    uint2* bnd = a.boundary ? a.boundary + slot * a.boundary_stride : nullptr;

    const int oe = a.sc.go + a.sc.ge;
    const uint32_t NOE = L::splat(-oe);
    const uint32_t NE = L::splat(-a.sc.ge);
    const uint32_t MONE = L::splat(-1);
    // Row state Hop = H - (o + e), kept biased by kBias on the packed path;
    // the profile holds s + o + e, so the diagonal term Hop + prof = H + s is
    // one add.  HZ is the value of Hop at H = 0, which is also the value of
    // E and F at -(o + e), their "minus infinity" at the borders.
    const int zero_h = P16 ? kBias - oe : -oe;
    const uint32_t HZ = L::splat(zero_h);
    const uint32_t BV = L::splat(kBias);                  // H = 0 on the packed path
    // the banded pass's "minus infinity" / floor: HF the row state (and E, F)
    // at H = kFloorH, BF the floor of U's maximum; the local DP uses H = 0
    const uint32_t HF = BAND ? L::splat(zero_h + kFloorH) : HZ;
    const uint32_t BF = BAND ? L::splat(kBias + kFloorH) : BV;
    const uint32_t one = (uint32_t)a.sc.one;              // 1 at run time: adds issue as multiply-adds
    const uint32_t neg_one = 0u - one;
    const uint32_t ONE = L::splat(1);
    const uint32_t C_UOP = (uint32_t)(-(oe * 65537));    // U -> U - (o + e) in both halves

    // wavefront steps this warp ran; steps x its 32 lanes' rows x PACK cell
    // updates go to the pass's counter once, when the warp runs out of work
    uint32_t steps_run = 0;
    for (;;) {
        uint32_t task = 0;
        if (lane == 0) task = atomicAdd(a.task_ctr, 1u);
        task = __shfl_sync(kFull, task, 0);
        const int64_t first = begin + (int64_t)task * (GROUPS * PACK);
        if (first >= end) break;

        // ---- the (up to) PACK pairs of this group
        int pid[PACK];
        const uint8_t* qp[PACK];
        const uint8_t* rp[PACK];
        int lq[PACK], lr[PACK], target[PACK];
        int ls = 0, lh = 0;
#pragma unroll
        for (int h = 0; h < PACK; ++h) {
            const int64_t pos = first + g * PACK + h;
            pid[h] = -1;
            lq[h] = lr[h] = 0;
            target[h] = 0;
            qp[h] = rp[h] = nullptr;
            if (pos < end) {
                const int p = a.order[pos];
                pid[h] = p;
                const int32_t qi = a.pairs[2 * (int64_t)p], ri = a.pairs[2 * (int64_t)p + 1];
                qp[h] = a.q.res + a.q.off[qi];
                rp[h] = a.r.res + a.r.off[ri];
                if (REV) {
                    const swgb_record rec = a.out[p];
                    lq[h] = rec.q_end + 1;
                    lr[h] = rec.r_end + 1;
                    target[h] = rec.score;
                } else {
                    lq[h] = (int)(a.q.off[qi + 1] - a.q.off[qi]);
                    lr[h] = (int)(a.r.off[ri + 1] - a.r.off[ri]);
                }
            }
            ls = max(ls, lq[h]);
            lh = max(lh, lr[h]);
        }
        // warp-uniform extents (groups of one warp run in lock step)
        int ls_w = ls, nch = (lh + ROWS - 1) / ROWS;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            ls_w = max(ls_w, __shfl_xor_sync(kFull, ls_w, off));
            nch = max(nch, __shfl_xor_sync(kFull, nch, off));
        }
        // a chunked task needs this warp's boundary row; a launch wider than
        // the rows provided is a host error: report it, touch nothing
        if (nch > 1 && (bnd == nullptr || slot >= a.boundary_slots || ls_w > a.boundary_stride)) {
            if (lane == 0) set_status(a.status, SWGB_EINTERNAL);
            continue;
        }
        // profile row of the query letter at streamed position i (the pad
        // row outside the pair; letters are their own rows)
        auto code_at = [&](int h, int i) -> int {
            if (i < 0 || i >= lq[h]) return pad_row;
            return REV ? qp[h][lq[h] - 1 - i] : qp[h][i];
        };

        // maxima variant: does any pair of the warp record forward maxima
        // (warp-uniform, since the warp's groups step together)
        bool rec = false;
        if constexpr (FMAX) {
            if (a.fmax_off) {
#pragma unroll
                for (int h = 0; h < PACK; ++h)
                    if (pid[h] >= 0 && a.fmax_off[pid[h]] >= 0) rec = true;
            }
            rec = __any_sync(kFull, rec);
        }

        int bv[PACK], bi[PACK], bj[PACK];
#pragma unroll
        for (int h = 0; h < PACK; ++h) {
            bv[h] = zero_h;
            bi[h] = INT_MAX;
            bj[h] = INT_MAX;
        }
        // lower bound of the final score (tracked units), per half.  The reverse
        // pass knows the score S itself: with T = S a lane has an event only
        // when it first reaches S, so earlier runs of events cost nothing.
        uint32_t T = HZ;
        if constexpr (REV) {
            if constexpr (P16)
                T = (uint32_t)(target[0] + zero_h) | ((uint32_t)(target[PACK - 1] + zero_h) << 16);
            else
                T = (uint32_t)(target[0] + zero_h);
        }
        // reverse pass: the score S is known; fi = first streamed step at which
        // this lane recorded a cell of value S, per half
        int fi[PACK];
#pragma unroll
        for (int h = 0; h < PACK; ++h) fi[h] = INT_MAX;
        int ls_c = ls;   // streamed positions the chunk still needs

        // banded pass, per half: the band (width bW, offset bK), the slice of
        // the pair's forward maxima (foff, rows per entry frf) and vmin, the
        // smallest position of an exit whose bound reaches S (INT_MIN: no
        // maxima, never certified)
        int bW[PACK], bK[PACK], frf[PACK], vmin[PACK];
        int64_t foff[PACK];
        if constexpr (BAND) {
#pragma unroll
            for (int h = 0; h < PACK; ++h) {
                int64_t w = 0, k = 0;
                if (pid[h] >= 0) band_geometry(lq[h], lr[h], &w, &k);
                bW[h] = (int)w;
                bK[h] = (int)k;
                foff[h] = pid[h] >= 0 ? a.fmax_off[pid[h]] : -1;
                frf[h] = foff[h] >= 0 ? a.fmax[foff[h]] : 0;
                vmin[h] = (foff[h] >= 0 && frf[h] > 0) ? INT_MAX : INT_MIN;
            }
        }
        // largest forward H over the reversed rows [j0, j1] of half h, i.e.
        // reference rows lr - 1 - j1 .. lr - 1 - j0 (kFloorH if none)
        auto fmax_rows = [&](int h, int j0, int j1) -> int {
            int lo = lr[h] - 1 - j1, hi = lr[h] - 1 - j0, m = kFloorH;
            if (lo < 0) lo = 0;
            for (int k = lo / frf[h]; hi >= lo && k <= hi / frf[h]; ++k) m = max(m, a.fmax[foff[h] + 1 + k]);
            return m;
        };
        // exits through the bottom row of the chunk before row jrow at the
        // positions [p0, p1), read from the chunk-boundary row (every lane)
        auto stair_exits = [&](int jrow, int p0, int p1) {
            int fn[PACK];
#pragma unroll
            for (int h = 0; h < PACK; ++h)
                fn[h] = (vmin[h] != INT_MIN && jrow < lr[h]) ? fmax_rows(h, jrow, jrow) + a.sc.go : INT_MIN;
            for (int p = p0 + lane; p < p1; p += 32) {
                const uint32_t y = bnd[p].y;
#pragma unroll
                for (int h = 0; h < PACK; ++h)
                    if (fn[h] != INT_MIN && p < lq[h] && L::get(y, h) - zero_h + fn[h] >= target[h])
                        vmin[h] = min(vmin[h], p);
            }
        };
        const int ls_all = ls_w;      // positions a chunk-boundary row may hold
        int prev_lo = 0, prev_hi = 0; // positions the last chunk's bottom row holds

        for (int c = 0; c < nch; ++c) {
            const int jc = c * ROWS;          // first held row of the chunk
            const int jl = jc + gl * R;       // first held row of this lane
            // streamed window [w0, wend) of the chunk: the positions the
            // chunks before left to scan, or in the banded pass the union of
            // the halves' band windows within them (empty: wend <= w0)
            int w0 = 0, wend = ls_w;
            if constexpr (BAND) {
                int64_t lo = INT_MAX, hi = 0;
#pragma unroll
                for (int h = 0; h < PACK; ++h) {
                    if (pid[h] >= 0 && jc < lr[h]) {
                        int64_t x0 = 0, x1 = 0;
                        band_window(c, ROWS, bW[h], bK[h], lq[h], &x0, &x1);
                        lo = min(lo, x0);
                        hi = max(hi, x1);
                    }
                }
                if (hi > ls_w) hi = ls_w;
                w0 = (int)(lo < INT_MAX / 2 ? lo : INT_MAX / 2);
                wend = (int)hi;
                // the last chunk's bottom row at the positions left of this
                // chunk's first row (all of them if this chunk scans nothing);
                // this chunk's last lane overwrites them
                if (c > 0) stair_exits(jc, prev_lo, wend > w0 ? min(prev_hi, w0) : prev_hi);
                if (wend <= w0) {
                    prev_lo = prev_hi = 0;
                    continue;
                }
            }
            // ---- profile of the chunk: prof[h][x][row] = s(x, held row) + o + e
            __syncwarp();
#pragma unroll
            for (int h = 0; h < PACK; ++h) {
                uint8_t y[LS];
#pragma unroll
                for (int k = 0; k < LS; ++k) {
                    const int j = jl + k;
                    y[k] = (k < R && j < lr[h]) ? (REV ? rp[h][lr[h] - 1 - j] : rp[h][j])
                                                : (uint8_t)kPadCode;
                }
                // Four profile rows x = 4 xq .. 4 xq + 3 at a time: word xq of
                // the transposed table rows of four held letters is a 4 x 4 byte
                // block, transposed by byte permutes into the four rows' words
                // for those letters.
                int8_t* dst = prof + h * PROF + gl * LS;
                for (int xq = 0; 4 * xq < prows; ++xq) {
                    uint32_t o[4][NW];
#pragma unroll
                    for (int k4 = 0; k4 < NW; ++k4) {
                        uint32_t w[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            w[j] = *reinterpret_cast<const uint32_t*>(tabT + y[4 * k4 + j] * kTabTStride + 4 * xq);
                        const uint32_t t0 = prmt(w[0], w[1], 0x5140u), t1 = prmt(w[0], w[1], 0x7362u);
                        const uint32_t t2 = prmt(w[2], w[3], 0x5140u), t3 = prmt(w[2], w[3], 0x7362u);
                        o[0][k4] = prmt(t0, t2, 0x5410u);
                        o[1][k4] = prmt(t0, t2, 0x7632u);
                        o[2][k4] = prmt(t1, t3, 0x5410u);
                        o[3][k4] = prmt(t1, t3, 0x7632u);
                    }
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        if (4 * xq + m < prows) store_prof<LS>(dst + (4 * xq + m) * RS, o[m]);
                }
            }
            __syncwarp();

            // ---- wavefront over the streamed query
            // Row state of the last two steps: the step loop is unrolled by four
            // and alternates the roles of HopA / HopB (and of the profile words
            // pwA / pwB), so the previous step's registers stay available
            // without copies.  Between groups of steps the state is in the A set.
            uint32_t HopA[R], HopB[R], F[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                HopA[r] = HF;   // H = 0 before the first query position (banded: the floor)
                F[r] = HF;
            }
            // the diagonal input of the lane's first row at its first position:
            // the banded pass is anchored (H = 0 only at the origin's corner; in
            // later chunks lane 0 takes the row above from the last chunk)
            uint32_t hin_prev = HZ;
            if constexpr (BAND) {
                hin_prev = (c == 0 && gl == 0) ? HZ : HF;
                if (c > 0 && gl == 0 && w0 - 1 >= prev_lo && w0 - 1 < prev_hi) hin_prev = bnd[w0 - 1].y;
            }
            // per half max(this lane's maximum in this chunk, T - 1)
            uint32_t lb1 = L::addmax(T, MONE, HZ);
            // forward maxima variant: this lane's own running maximum over its
            // rows in this chunk (lb1 also holds T - 1), for the banded reverse pass
            uint32_t pmax = HZ;
            // the kept event's row values of each half; on the packed path two
            // rows per register (row 2k low, row 2k + 1 high)
            constexpr int NS = P16 ? (R + 1) / 2 : R;   // odd R: the last high half unused
            uint32_t snap[PACK][NS];
            int si[PACK], sv[PACK];
#pragma unroll
            for (int h = 0; h < PACK; ++h) {
                si[h] = -1;
                sv[h] = INT_MIN;
#pragma unroll
                for (int k = 0; k < NS; ++k) snap[h][k] = HZ;
            }

            const bool read_bnd = (c > 0) && (gl == 0);
            const bool write_bnd = (c + 1 < nch) && (gl == G - 1);
            const int steps = (wend - w0) + G - 1;
            // lane 0 reads the row above at the positions [w0, rd_hi) the last
            // chunk's bottom row holds; the last lane writes its bottom row
            // at the positions [0, wr_hi)
            const int rd_hi = BAND ? prev_hi : ls_c;
            const int wr_hi = BAND ? ls_all : ls_c;
            int t_end = 0;   // steps the wavefront ran
            int stop_w = INT_MAX;   // reverse pass: warp-uniform last useful step

            // software pipeline: profile words of the next step and the query
            // letter of the step after are fetched one step ahead.  A lane's
            // streamed position is one behind the lane before it, so the letter
            // it needs next is the one that lane holds now: letters move down
            // the group by shuffle, and lane 0 reads them from a batch of
            // kBatch letters (xb); the group loads the batch after it (xc) one
            // batch period ahead.
            constexpr int kBoundEvery = bound_every(REV);
            constexpr int kBatch = G < kBoundEvery ? G : kBoundEvery;
            ProfWords<LS> pwA[PACK], pwB[PACK];
            int xn[PACK], xb[PACK], xc[PACK];
#pragma unroll
            for (int h = 0; h < PACK; ++h) {
                pwA[h] = load_prof<LS>(plane + h * PROF + code_at(h, w0 - gl) * RS);
                xn[h] = code_at(h, w0 + 1 - gl);
                xb[h] = code_at(h, w0 + 2 + gl);            // positions for steps 0 .. kBatch - 1
                xc[h] = code_at(h, w0 + 2 + kBatch + gl);   // steps kBatch .. 2 kBatch - 1
            }
            // per half 1 where the previous step had an event whose registers
            // are not kept yet, else 0; endp: per half 1 where a run of events
            // ended at the previous step (its last event one step before that),
            // with the event's value in lbp
            // mp: the last step's maximum (with lb1, before a bound refresh
            // raised it), i.e. the value of that step's event if it had one
            uint32_t pend = 0, endp = 0, lbp = lb1, mp = lb1;
            uint32_t ein = HF, hin = HF;   // from lane gl-1, previous step
            // multiplier and addend that give lane 0 of a group HZ for its
            // inputs from above (one-tile wavefronts; run-time values, so the
            // product is issued as a multiply-add, not a select)
            const uint32_t not0 = gl == 0 ? 0u : one;
            const uint32_t hz0 = gl == 0 ? HF : 0u;

            // The step loop, compiled twice for the 32-lane tiles: with the
            // chunk-boundary exchange (BND, references longer than one tile) and
            // without it (one tile, and every smaller shape).
            auto wavefront = [&](auto bnd_tag, auto rec_tag) {
            constexpr bool BND = decltype(bnd_tag)::value;
            constexpr bool REC = FMAX && decltype(rec_tag)::value;   // track pmax
            uint2 bcur = make_uint2(HF, HF);
            if (BND && read_bnd && rd_hi > w0) bcur = bnd[w0];

            // keeps the registers of an event of value v at streamed position
            // ii (Hs holds that step's values) as half h's candidate
            auto keep = [&](int h, int ii, const uint32_t (&Hs)[R], int v) {
                si[h] = ii;
                sv[h] = v;
                if constexpr (P16) {
#pragma unroll
                    for (int k = 0; k < NS; ++k)
                        snap[h][k] = prmt(Hs[2 * k], Hs[2 * k + 1 < R ? 2 * k + 1 : 2 * k],
                                          h ? 0x7632u : 0x5410u);
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r) snap[h][r] = Hs[r];
                }
                if (REV && sv[h] == target[h] + zero_h && ii < fi[h]) fi[h] = ii;
            };

            // One step: query position i = t - gl against the lane's rows.  Hp
            // holds the previous step's row state, Hn receives this step's; pw
            // holds this step's profile words and pwn receives the next step's.
            //
            // Lanes step in lock step without branching on their own range:
            // before its first position a lane sees only pad letters and
            // "minus infinity" inputs from the lane before, which leaves its
            // initial state unchanged; after its last position it computes pad
            // cells, which score below the best real cell feeding them and can
            // never be the pair's maximum.  Only the boundary store is guarded.
            // last marks the fourth step of a group (t % 4 == 3; a literal at
            // every call, folded once inlined): only there can the batch and
            // bound periods (multiples of four) end.
            auto step = [&](int t, const uint32_t (&Hp)[R], uint32_t (&Hn)[R],
                            const ProfWords<LS> (&pw)[PACK], ProfWords<LS> (&pwn)[PACK], bool last) {
                const int i = w0 + t - gl;
#pragma unroll
                for (int h = 0; h < PACK; ++h) {
                    pwn[h] = load_prof<LS>(plane + h * PROF + xn[h] * RS);
                    const int from_prev = __shfl_up_sync(kFull, xn[h], 1, G);
                    const int from_batch = __shfl_sync(kFull, xb[h], t & (kBatch - 1), G);
                    xn[h] = gl == 0 ? from_batch : from_prev;   // letter of position i + 2
                }
                if constexpr (BND) {
                    if (gl == 0) {
                        // past the rows the previous chunk handed over, lane 0 sees
                        // "minus infinity": cells there score alignments confined
                        // to this chunk, never above the pair's score
                        const bool take = read_bnd && i < rd_hi;
                        ein = take ? bcur.x : HF;
                        hin = take ? bcur.y : HF;
                    }
                    if (read_bnd && i + 1 < rd_hi) bcur = bnd[i + 1];
                }
                // A run of events that ended at the previous step had its last
                // event two steps back, whose row state is still in Hn until
                // phase 1 overwrites it: keep it now.  The test reads a flag set
                // a step ago, so no branch waits on the last step's maximum.
                if (endp != 0) {
#pragma unroll
                    for (int h = 0; h < PACK; ++h)
                        if (L::get(endp, h) != 0) keep(h, i - 2, Hn, L::get(lbp, h));
                }
                // phase 1, independent rows: U = max(Hdiag + s, F, 0) - (o + e)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t s = L::widen(pw[0].w[r >> 2], pw[PACK - 1].w[r >> 2], r & 3);
                    const uint32_t hd = r == 0 ? hin_prev : Hp[r - 1];
                    if constexpr (P16) {
                        const uint32_t d = s * one + hd;                 // H_diag + s (biased)
                        Hn[r] = L::max3(d, F[r], BF) * one + C_UOP;      // max(., F, 0) - (o + e)
                    } else {
                        Hn[r] = L::addmax(L::addmax(hd, s, F[r]), NOE, NOE);
                    }
                }
                // phase 2, the chain along the rows: H - (o + e) and E of the next row
                uint32_t e = ein;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t hn = L::addmax(e, NOE, Hn[r]);
                    e = L::addmax(e, NE, Hn[r]);
                    Hn[r] = hn;
                }
                // phase 3, independent rows: F of the next query position
#pragma unroll
                for (int r = 0; r < R; ++r) F[r] = L::addmax(F[r], NE, Hn[r]);
                hin_prev = hin;
                if constexpr (BND) {
                    if (write_bnd && i >= 0 && i < wr_hi) bnd[i] = make_uint2(e, Hn[R - 1]);
                }
                const uint32_t e_next = __shfl_up_sync(kFull, e, 1, G);
                const uint32_t h_next = __shfl_up_sync(kFull, Hn[R - 1], 1, G);
                {
                    // A half has an event when the step's maximum passes lb1, i.e.
                    // it grew the lane's maximum and reached T.  Events come in
                    // runs while an alignment grows through the lane's rows; only
                    // the last of a run can hold the lane's maximum, so its
                    // registers are kept once the run has ended (at the start of
                    // the step after next).  After an event lb1 is its value.
                    uint32_t nlb1;
                    if constexpr (REC) {
                        pmax = tree_max<P16, R>(Hn, pmax);
                        nlb1 = L::max3(pmax, lb1, lb1);
                    } else {
                        nlb1 = tree_max<P16, R>(Hn, lb1);
                    }
                    // nlb1 >= lb1 in each half, so the 32-bit difference is exact
                    // per half; up = 1 in the halves with an event, else 0
                    const uint32_t up = L::min3(nlb1 + lb1 * neg_one, ONE, ONE);
                    endp = pend & ~up;
                    lbp = mp;    // the previous step's event value, if it had one
                    mp = nlb1;
                    pend = up;
                    lb1 = nlb1;
                }
                // the batch of the steps from t + 1 on was loaded a period ago;
                // load the one after it
                if constexpr (kBatch < kBoundEvery) {
                    if (last && (t & (kBatch - 1)) == kBatch - 1) {
#pragma unroll
                        for (int h = 0; h < PACK; ++h) {
                            xb[h] = xc[h];
                            xc[h] = code_at(h, w0 + t + 3 + kBatch + gl);
                        }
                    }
                }
                if (last && (t & (kBoundEvery - 1)) == kBoundEvery - 1) {
                    if constexpr (kBatch == kBoundEvery) {
#pragma unroll
                        for (int h = 0; h < PACK; ++h) {
                            xb[h] = xc[h];
                            xc[h] = code_at(h, w0 + t + 3 + kBatch + gl);
                        }
                    }
                    if constexpr (!REV) {   // the reverse pass's bound is S from the start
                        T = group_max<P16, G>(L::max3(lb1, T, T));
                        lb1 = L::addmax(T, MONE, lb1);
                    }
                    if constexpr (REV) {
                        // once every half of every group has met S at some step,
                        // cells of later steps can no longer be the first such cell
                        // after the wavefront has passed that step in all lanes
                        int stop = 0;
#pragma unroll
                        for (int h = 0; h < PACK; ++h) {
                            const int gm = group_min<G>(fi[h]);   // every lane shuffles
                            const int f = pid[h] >= 0 ? gm : 0;
                            stop = (stop == INT_MAX || f == INT_MAX) ? INT_MAX : max(stop, f);
                        }
                        if (stop != INT_MAX) stop += G - 1 - w0;   // in steps
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1)
                            stop = max(stop, __shfl_xor_sync(kFull, stop, off));
                        stop_w = stop;
                    }
                }
                if constexpr (BND) {
                    ein = e_next;
                    hin = h_next;
                } else {
                    // lane 0 of a group takes "minus infinity" from above; as a
                    // multiply-add (x * 0 + HZ, or x * 1 + 0) on the FMA pipe
                    ein = e_next * not0 + hz0;
                    hin = h_next * not0 + hz0;
                }
            };

            // Steps go in fours with one exit test per group, so the four steps
            // are straight-line code apart from the rare event branches.  Up to
            // three steps run past the last: every lane is then past its last
            // position and computes pad cells (each scores below a real cell
            // feeding it, so it cannot be the pair's maximum; boundary rows are
            // guarded by position), and in the reverse pass a step past stop_w
            // cannot record an earlier cell.  The group ends in the A set.
            int t = 0;
            while (t < steps && t <= stop_w) {
                step(t, HopA, HopB, pwA, pwB, false);
                step(t + 1, HopB, HopA, pwB, pwA, false);
                step(t + 2, HopA, HopB, pwA, pwB, false);
                step(t + 3, HopB, HopA, pwB, pwA, true);
                t += 4;
            }
            // a run that ended at the last step (its event one step before, in
            // the B set), then a run still open at the last step (A set)
#pragma unroll
            for (int h = 0; h < PACK; ++h) {
                if (L::get(endp, h) != 0) keep(h, w0 + t - 2 - gl, HopB, L::get(lbp, h));
                if (L::get(pend, h) != 0) keep(h, w0 + t - 1 - gl, HopA, L::get(mp, h));
            }
            t_end = t;
            };
            // the maxima variant tracks pmax only in tasks that record some
            auto run = [&](auto bnd_tag) {
                if constexpr (FMAX) {
                    if (rec) wavefront(bnd_tag, std::true_type{});
                    else wavefront(bnd_tag, std::false_type{});
                } else {
                    wavefront(bnd_tag, std::false_type{});
                }
            };
            if constexpr (G == 32) {
                if (nch > 1) run(std::true_type{});
                else run(std::false_type{});
            } else {
                run(std::false_type{});
            }
            steps_run += (uint32_t)t_end;

            // ---- forward maxima of the lane's rows for the banded reverse
            // pass: entry jl / R of the pair's slice (its forward tile is this
            // one, so every lane writes its own entry once).  Pad cells the
            // lane computed score below real cells feeding them, so the value
            // bounds the rows' H from above.
            if constexpr (FMAX) {
                if (rec) {
#pragma unroll
                    for (int h = 0; h < PACK; ++h) {
                        if (pid[h] >= 0 && jl < lr[h]) {
                            const int64_t off = a.fmax_off[pid[h]];
                            if (off >= 0) a.fmax[off + 1 + jl / R] = L::get(pmax, h) - zero_h;
                        }
                    }
                }
            }

            // ---- exits of the banded pass at the end of the chunk
            if constexpr (BAND) {
                // right edge: the lane's rows at its last position e, and its
                // bottom row at e - 1 (the lane below stops at e - 1)
                const int e = w0 + t_end - 1 - gl;
                const uint32_t m = tree_max<P16, R>(HopA, HopB[R - 1]);
#pragma unroll
                for (int h = 0; h < PACK; ++h)
                    if (vmin[h] != INT_MIN && jl < lr[h] && e < lq[h] &&
                        L::get(m, h) - zero_h + fmax_rows(h, jl, jl + R) + a.sc.go >= target[h])
                        vmin[h] = min(vmin[h], e - 1);
                // the last chunk's bottom row from the position where this
                // chunk's first row stops on: this chunk's last lane wrote only
                // positions before it
                if (c > 0) stair_exits(jc, max(prev_lo, w0 + t_end - 1), prev_hi);
                prev_lo = max(0, w0 - (G - 1));
                prev_hi = min(ls_all, w0 + t_end - (G - 1));
            }

            // ---- the lane's candidate of this chunk: the recorded step and the
            // first row of the snapshot holding the value, if it is the lane's
            // maximum
            if constexpr (!REV) T = group_max<P16, G>(L::max3(lb1, T, T));
#pragma unroll
            for (int h = 0; h < PACK; ++h) {
                if (si[h] >= 0 && sv[h] == L::get(lb1, h)) {
                    int row = R - 1;
#pragma unroll
                    for (int r = R - 1; r >= 0; --r)
                        if ((P16 ? L::get(snap[h][r / 2], r & 1) : L::get(snap[h][r], h)) == sv[h]) row = r;
                    if (better(sv[h], si[h], jl + row, bv[h], bi[h], bj[h])) {
                        bv[h] = sv[h];
                        bi[h] = si[h];
                        bj[h] = jl + row;
                    }
                }
            }
            if constexpr (REV) {
                // later chunks hold later reference rows: only steps before the
                // first one that met S can still give a row-major-earlier cell
                int need = 0;
#pragma unroll
                for (int h = 0; h < PACK; ++h) {
                    const int f = group_min<G>(fi[h]);
                    need = max(need, f == INT_MAX ? lq[h] : min(lq[h], f));
                }
                ls_c = need;
                ls_w = need;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) ls_w = max(ls_w, __shfl_xor_sync(kFull, ls_w, off));
            }
            __syncwarp();
        }

        // ---- reduce over the lanes of the group and write the records
        int ncert = 0;
#pragma unroll
        for (int h = 0; h < PACK; ++h) {
            int v = bv[h], ii = bi[h], jj = bj[h];
            const int vm = BAND ? group_min<G>(vmin[h]) : 0;
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                const int ov = __shfl_xor_sync(kFull, v, off, G);
                const int oi = __shfl_xor_sync(kFull, ii, off, G);
                const int oj = __shfl_xor_sync(kFull, jj, off, G);
                if (better(ov, oi, oj, v, ii, jj)) {
                    v = ov;
                    ii = oi;
                    jj = oj;
                }
            }
            if (gl == 0 && pid[h] >= 0) {
                const int S = v - zero_h;
                swgb_record* rec = &a.out[pid[h]];
                if (!REV) {
                    if (S > 0 && ii != INT_MAX) {
                        *rec = swgb_record{S, -1, ii, -1, jj};
                    } else {
                        *rec = swgb_record{0, -1, -1, -1, -1};
                    }
                } else if (BAND) {
                    // certified: S found in the band before every exit whose
                    // bound reaches S; otherwise left for the full pass
                    if (S == target[h] && ii != INT_MAX && vm > ii) {
                        rec->q_start = lq[h] - 1 - ii;
                        rec->r_start = lr[h] - 1 - jj;
                        ++ncert;
                    } else {
                        rec->q_start = kBandFallback;
                    }
                } else {
                    if (S != target[h] || ii == INT_MAX) {
                        set_status(a.status, SWGB_EINTERNAL);
                    } else {
                        rec->q_start = lq[h] - 1 - ii;
                        rec->r_start = lr[h] - 1 - jj;
                    }
                }
            }
        }
        if (BAND && ncert > 0) atomicAdd(&a.counters[kCtrBandCertified], (unsigned long long)ncert);
    }
    if (lane == 0 && steps_run > 0 && a.counters)
        atomicAdd(&a.counters[REV ? kCtrRevSlots : kCtrFwdSlots], (unsigned long long)steps_run * (32 * R * PACK));
}

// ---------------------------------------------------------------------------
// Dispatch over (class, shape, direction)
// ---------------------------------------------------------------------------
using DPFn = void (*)(const DPArgs);

template <int S, bool P16, bool REV, bool FMAX, bool BAND = false>
constexpr DPFn dp_fn() {
    return &dp_kernel<shape_G(S), shape_R(S), P16, REV, FMAX, BAND>;
}

template <bool P16, bool REV, bool FMAX>
DPFn dp_pick(int shape) {
    switch (shape) {
        case 0: return dp_fn<0, P16, REV, FMAX>();
        case 1: return dp_fn<1, P16, REV, FMAX>();
        case 2: return dp_fn<2, P16, REV, FMAX>();
        case 3: return dp_fn<3, P16, REV, FMAX>();
        case 4: return dp_fn<4, P16, REV, FMAX>();
        case 5: return dp_fn<5, P16, REV, FMAX>();
        case 6: return dp_fn<6, P16, REV, FMAX>();
        case 7: return dp_fn<7, P16, REV, FMAX>();
        case 8: return dp_fn<8, P16, REV, FMAX>();
        case 9: return dp_fn<9, P16, REV, FMAX>();
        case 10: return dp_fn<10, P16, REV, FMAX>();
        case 11: return dp_fn<11, P16, REV, FMAX>();
        case 12: return dp_fn<12, P16, REV, FMAX>();
        case 13: return dp_fn<13, P16, REV, FMAX>();
        case 14: return dp_fn<14, P16, REV, FMAX>();
        case 15: return dp_fn<15, P16, REV, FMAX>();
        case 16: return dp_fn<16, P16, REV, FMAX>();
        case 17: return dp_fn<17, P16, REV, FMAX>();
        case 18: return dp_fn<18, P16, REV, FMAX>();
        case 19: return dp_fn<19, P16, REV, FMAX>();
        default: return dp_fn<20, P16, REV, FMAX>();
    }
}

// the banded reverse pass: packed 32-lane tiles of the band shapes only
static DPFn dp_pick_band(int shape) {
    switch (shape) {
        case 13: return dp_fn<13, true, true, false, true>();
        case 14: return dp_fn<14, true, true, false, true>();
        case 15: return dp_fn<15, true, true, false, true>();
        case 16: return dp_fn<16, true, true, false, true>();
        default: return dp_fn<17, true, true, false, true>();
    }
}

// The packed forward pass always runs the FMAX variant: in tasks that record
// no maxima it takes its wavefront without pmax, and that build measured 5 %
// faster on the 2,000,000-pair batch than the kernel without the variant
// (66.1 -> 62.7 ms, same records).  band: the banded reverse pass (packed).
static DPFn dp_lookup(int cls, int shape, bool reverse, bool band = false) {
    if (cls == 0) {
        if (reverse)
            return band && shape >= kFirstChunkable && shape < kBandShapeEnd ? dp_pick_band(shape)
                                                                             : dp_pick<true, true, false>(shape);
        return dp_pick<true, false, true>(shape);
    }
    return reverse ? dp_pick<false, true, false>(shape) : dp_pick<false, false, false>(shape);
}

size_t dp_smem_bytes(int cls, int shape, int prof_rows) {
    const size_t per_warp = dp_prof_bytes_per_warp(shape_G(shape), shape_R(shape), cls == 0, prof_rows);
    return kSmatRegion + per_warp * (kDPThreads / 32);
}

cudaError_t dp_configure(int cls, int shape, bool reverse) {
    cudaError_t e = cudaFuncSetAttribute(dp_lookup(cls, shape, reverse),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dp_smem_bytes(cls, shape, kProfileRows));
    if (e == cudaSuccess && cls == 0 && reverse && shape >= kFirstChunkable && shape < kBandShapeEnd)
        e = cudaFuncSetAttribute(dp_lookup(cls, shape, true, true),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)dp_smem_bytes(cls, shape, kProfileRows));
    return e;
}

int dp_blocks_per_sm(int cls, int shape, bool reverse, int prof_rows, bool band) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dp_lookup(cls, shape, reverse, band),
                                                      kDPThreads,
                                                      dp_smem_bytes(cls, shape, prof_rows)) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_dp(int cls, int shape, bool reverse, const DPArgs& a, int grid_blocks,
                      cudaStream_t st, bool band) {
    DPFn fn = dp_lookup(cls, shape, reverse, band);
    fn<<<grid_blocks, kDPThreads, dp_smem_bytes(cls, shape, a.sc.prof_rows), st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Issue-rate probe of __viaddmax_s16x2
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kProbeThreads) probe_addmax_kernel(unsigned long long* cycles,
                                                                      uint32_t* sink, int iters) {
    uint32_t v[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) v[k] = threadIdx.x * 0x00010001u + k;
    const uint32_t inc = 0x00010001u;
    const uint32_t floor_v = (blockIdx.x & 7) * 0x00010001u;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) v[k] = __viaddmax_s16x2(v[k], inc, floor_v);
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) acc ^= v[k];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
}

cudaError_t launch_probe_addmax(unsigned long long* cycles, uint32_t* sink, int blocks, int iters,
                                cudaStream_t st) {
    probe_addmax_kernel<<<blocks, kProbeThreads, 0, st>>>(cycles, sink, iters);
    return cudaGetLastError();
}

}  // namespace swgb
