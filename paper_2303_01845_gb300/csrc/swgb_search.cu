// swgb_search.cu -- candidate discovery by shared k-mers and the identity of
// alignment records, on sm_103a, with their C-ABI entry points.
//
// Discovery (Sec. "Protein similarity search pipeline": the overlap matrix
// C = A A^T of the sequence-by-k-mer matrix A gives the candidate pairs and
// their common k-mer counts; Sec. "Load balancing techniques": C is symmetric,
// one triangle suffices, and pairs below the common-k-mer threshold are not
// aligned).  The paper forms C with a sparse matrix product on the CPU because
// no GPU semiring product was at hand (Sec. "Implications"); here it is a
// k-mer join on the device:
//
//   1. kmer_sets:  one block per sequence hashes the k-mers of its standard
//      letters into a table (shared memory, or a per-block global region for
//      long sequences) and writes the distinct ones with their first position;
//   2. histogram of the distinct k-mers -> exclusive scan -> scatter: the
//      columns of A as buckets (k-mer -> the sequences holding it), i.e. A^T;
//   3. row_need: per sequence i, the number of (k-mer, j > i) incidences, an
//      upper bound of the distinct partners of row i;
//   4. join (twice: count, then write): one block per row i counts each
//      partner j > i over the buckets of i's k-mers in a hash table, keeps
//      the partners with count >= threshold, sorts them by j and writes them
//      at the row's offset (a scan of the counting pass);
//   so C's upper triangle comes out ordered by (i, j) and deterministic.
//
// Identity (the production filter keeps pairs of identity >= 30 % and
// coverage >= 70 %, program-parameters table; the paper defines neither):
// the identical columns and columns of the alignment that a traceback of the
// record span's global affine DP takes under a fixed preference -- diagonal,
// then a gap in the reference (query residue against a gap), then a gap in
// the query; inside a gap its opening before its extension -- computed by a
// forward wavefront that carries those statistics with the DP (no decision
// matrix, no traceback).  A counting sort lays the pairs out in work lists
// by span class, each longest first; spans of many chunks are shared by the
// warps of a block.
#include <climits>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "swgb_host.cuh"

namespace swgb {
namespace {

constexpr uint32_t kEmpty = 0xffffffffu;
constexpr int kSearchThreads = 256;
// shared-memory hash tables: k-mer sets of sequences with up to
// kSetSmemSlots/2 k-mers, join rows with up to kJoinSmemSlots/2 partners
constexpr int kSetSmemSlots = 4096;
constexpr int kJoinSmemSlots = 4096;
constexpr int kJoinSmemBytes = kJoinSmemSlots * 12;
// rows of at most kWarpJoinNeed partners: one warp each (join_warp_kernel)
constexpr int kWarpJoinSlots = 512;
constexpr int kWarpJoinNeed = kWarpJoinSlots / 2;
constexpr int kWarpJoinWarps = 8;
constexpr int kWarpJoinSmemBytes = kWarpJoinWarps * kWarpJoinSlots * 12;

__host__ __device__ inline uint32_t pow2_at_least(uint64_t v) {
    uint32_t p = 64;
    while (p < v) p <<= 1;
    return p;
}

__device__ __forceinline__ uint32_t slot_of(uint32_t key, uint32_t mask) {
    // multiplicative hashing (Knuth): the high bits of key * 2654435761
    return ((key * 2654435761u) >> 7) & mask;
}

// Block-uniform next task index from a work counter.
__device__ __forceinline__ int64_t next_task(unsigned long long* ctr, int64_t* s_task) {
    __syncthreads();
    if (threadIdx.x == 0) *s_task = (int64_t)atomicAdd(ctr, 1ull);
    __syncthreads();
    return *s_task;
}

// ---------------------------------------------------------------------------
// 1. distinct k-mers of every sequence
// ---------------------------------------------------------------------------
struct SetArgs {
    SeqView s;
    int k;
    uint32_t* ent_kmer;      // [total residues]: sequence i's entries at off[i]
    uint32_t* ent_pos;
    uint32_t* kcount;        // [n]
    uint32_t* gtab;          // per-block global tables (keys then positions)
    uint32_t gslots;         // slots of one global table (power of two)
    unsigned long long* ctr;
    int32_t* status;
};

__global__ void __launch_bounds__(kSearchThreads) kmer_sets_kernel(SetArgs a) {
    __shared__ uint32_t s_keys[kSetSmemSlots];
    __shared__ uint32_t s_pos[kSetSmemSlots];
    __shared__ int64_t s_task;
    __shared__ uint32_t s_cnt;
    const int64_t n = a.s.n;
    for (;;) {
        const int64_t i = next_task(a.ctr, &s_task);
        if (i >= n) break;
        const int64_t o = a.s.off[i];
        const int64_t npos = a.s.off[i + 1] - o - a.k + 1;
        if (npos <= 0) {
            if (threadIdx.x == 0) a.kcount[i] = 0;
            continue;
        }
        const uint32_t cap = pow2_at_least((uint64_t)npos * 2);
        uint32_t* keys;
        uint32_t* pos;
        if (cap <= (uint32_t)kSetSmemSlots) {
            keys = s_keys;
            pos = s_pos;
        } else {
            if (cap > a.gslots) {   // sized by the host from the longest sequence
                if (threadIdx.x == 0) { atomicMax(a.status, 1); a.kcount[i] = 0; }
                continue;
            }
            keys = a.gtab + (size_t)blockIdx.x * 2 * a.gslots;
            pos = keys + a.gslots;
        }
        const uint32_t mask = cap - 1;
        for (uint32_t t = threadIdx.x; t < cap; t += blockDim.x) {
            keys[t] = kEmpty;
            pos[t] = kEmpty;
        }
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        const uint8_t* seq = a.s.res + o;
        for (int64_t p = threadIdx.x; p < npos; p += blockDim.x) {
            uint32_t v = 0;
            bool ok = true;
            for (int t = 0; t < a.k; ++t) {
                const uint32_t c = seq[p + t];
                ok = ok && c < (uint32_t)kStdLetters;
                v = v * kStdLetters + c;
            }
            if (!ok) continue;
            uint32_t h = slot_of(v, mask);
            for (uint32_t probe = 0; probe < cap; ++probe) {
                const uint32_t cur = atomicCAS(&keys[h], kEmpty, v);
                if (cur == kEmpty || cur == v) {
                    atomicMin(&pos[h], (uint32_t)p);
                    break;
                }
                h = (h + 1) & mask;
            }
        }
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < cap; t += blockDim.x) {
            const uint32_t v = keys[t];
            if (v != kEmpty) {
                const uint32_t e = atomicAdd(&s_cnt, 1u);
                a.ent_kmer[o + e] = v;
                a.ent_pos[o + e] = pos[t];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) a.kcount[i] = s_cnt;
    }
}

// ---------------------------------------------------------------------------
// 2. buckets: histogram, scan, scatter
// ---------------------------------------------------------------------------
__global__ void kmer_hist_kernel(SeqView s, const uint32_t* __restrict__ ent_kmer,
                                 const uint32_t* __restrict__ kcount, uint32_t* hist) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < s.n; i += warps) {
        const int64_t o = s.off[i];
        const uint32_t c = kcount[i];
        for (uint32_t e = lane; e < c; e += 32) atomicAdd(&hist[ent_kmer[o + e]], 1u);
    }
}

// Bucket members: each entry takes the next slot of its k-mer's bucket from
// a cursor array (a copy of the bucket starts), four atomics in flight per lane.
__global__ void kmer_scatter_kernel(SeqView s, const uint32_t* __restrict__ ent_kmer,
                                    const uint32_t* __restrict__ kcount,
                                    uint32_t* __restrict__ cursor, int32_t* __restrict__ bseq) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < s.n; i += warps) {
        const int64_t o = s.off[i];
        const uint32_t c = kcount[i];
        for (uint32_t e0 = lane; e0 < c; e0 += 128) {
            uint32_t x[4], slot[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = e0 + 32 * u < c ? ent_kmer[o + e0 + 32 * u] : kEmpty;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (x[u] != kEmpty) slot[u] = atomicAdd(&cursor[x[u]], 1u);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (x[u] != kEmpty) bseq[slot[u]] = (int32_t)i;
        }
    }
}

// Exclusive scan of n counters into out[0..n] (out[n] = total), in three
// launches: block sums, a one-block scan of the sums, block scans.
constexpr int kScanT = 1024;
constexpr int kScanPerThread = 4;
constexpr int kScanTile = kScanT * kScanPerThread;

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* s_warp,
                                                         uint64_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t x = v;
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        uint64_t t = lane < nw ? s_warp[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t += y;
        }
        if (lane < nw) s_warp[lane] = t;
    }
    __syncthreads();
    const uint64_t before = (w ? s_warp[w - 1] : 0) + x - v;
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanT) scan_reduce_kernel(const uint32_t* __restrict__ in,
                                                             int64_t n, uint64_t* part) {
    __shared__ uint64_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPerThread;
    uint64_t v = 0;
    for (int k = 0; k < kScanPerThread; ++k)
        if (base + k < n) v += in[base + k];
    uint64_t total;
    block_exclusive_scan(v, s_warp, &total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanT) scan_part_kernel(uint64_t* part, int64_t nb) {
    __shared__ uint64_t s_warp[32];
    uint64_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanT) {
        const int64_t b = b0 + threadIdx.x;
        const uint64_t v = b < nb ? part[b] : 0;
        uint64_t total;
        const uint64_t ex = block_exclusive_scan(v, s_warp, &total);
        if (b < nb) part[b] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) part[nb] = carry;
}

template <class Out>
__global__ void __launch_bounds__(kScanT) scan_apply_kernel(const uint32_t* __restrict__ in,
                                                            int64_t n, const uint64_t* __restrict__ part,
                                                            int64_t nb, Out* out) {
    __shared__ uint64_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPerThread;
    uint32_t x[kScanPerThread];
    uint64_t v = 0;
    for (int k = 0; k < kScanPerThread; ++k) {
        x[k] = base + k < n ? in[base + k] : 0u;
        v += x[k];
    }
    uint64_t total;
    uint64_t run = part[blockIdx.x] + block_exclusive_scan(v, s_warp, &total);
    for (int k = 0; k < kScanPerThread; ++k)
        if (base + k < n) {
            out[base + k] = (Out)run;
            run += x[k];
        }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (Out)part[nb];
}

// ---------------------------------------------------------------------------
// 3. per-row partner bound and row class
// ---------------------------------------------------------------------------
struct JoinArgs {
    SeqView s;                 // the rows' set (offsets of their k-mer entries)
    const uint32_t* ent_kmer;
    const uint32_t* kcount;
    const uint32_t* start;     // bucket starts [V + 1] of the columns' set
    const int32_t* bseq;
    int64_t n_cols;            // sequences of the columns' set
    int self_pairs;            // rows and columns are one set: only j > i
    uint2* range;              // per row entry: its bucket [begin, end), set by row_need
    uint32_t* need;            // [n] min(partner incidences, possible partners)
    uint32_t* ccount;          // [n] candidates of row i (counting pass)
    const uint64_t* coff;      // [n + 1] scan of ccount (writing pass)
    int32_t* out_pairs;        // caller's [capacity][2]
    int32_t* out_counts;       // caller's [capacity] or null
    int64_t capacity;
    int min_shared;
    uint32_t* gtab;            // per-block global tables of large rows
    uint32_t gslots;
    unsigned long long* ctr;
    unsigned long long* stats; // [0] max need, [1] rows above the shared-memory table
    int32_t* status;
    int32_t* large_rows;       // [n] the rows above the shared-memory table
    int64_t n_tasks;           // LARGE launches: tasks are large_rows[0, n_tasks); else rows
    // counting pass with a stash: each row's sorted list (j << 32 | count) also
    // goes to stash[stash_off[i] ..) (slices handed out by stash_ctr; -1 where
    // the stash is full), so that a copy replaces the writing pass
    uint64_t* stash;           // [stash_cap] or null
    int64_t stash_cap;
    int64_t* stash_off;        // [n]
    unsigned long long* stash_ctr;
};

__global__ void row_need_kernel(JoinArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t n = a.s.n;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int64_t o = a.s.off[i];
        const uint32_t c = a.kcount[i];
        uint64_t inc = 0;
        for (uint32_t e = lane; e < c; e += 32) {
            const uint32_t x = a.ent_kmer[o + e];
            const uint32_t b0 = a.start[x], b1 = a.start[x + 1];
            a.range[o + e] = make_uint2(b0, b1);
            if (a.self_pairs) {
                // a bucket of one holds only row i itself
                if (b1 - b0 > 1)
                    for (uint32_t b = b0; b < b1; ++b) inc += a.bseq[b] > i;
            } else {
                inc += b1 - b0;
            }
        }
        for (int d = 16; d; d >>= 1) inc += __shfl_xor_sync(0xffffffffu, inc, d);
        if (lane == 0) {
            const uint64_t lim = (uint64_t)(a.self_pairs ? a.n_cols - 1 - i : a.n_cols);
            const uint32_t need = (uint32_t)(inc < lim ? inc : lim);
            a.need[i] = inc < (uint64_t)a.min_shared ? 0u : need;
            if (inc >= (uint64_t)a.min_shared) {
                atomicMax(&a.stats[0], (unsigned long long)need);
                if (2ull * need > (unsigned long long)kJoinSmemSlots)
                    a.large_rows[atomicAdd(&a.stats[1], 1ull)] = (int32_t)i;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 4. the join: per row i, partners j > i with at least min_shared common
//    k-mers, sorted by j.  LARGE: rows whose table does not fit in shared
//    memory use a per-block global table.  WRITE: second pass, writes the
//    pairs at coff[i]; otherwise counts them into ccount[i].
// ---------------------------------------------------------------------------
template <bool LARGE, bool WRITE>
__global__ void __launch_bounds__(kSearchThreads) join_kernel(JoinArgs a) {
    // dynamic shared layout (small rows, kJoinSmemBytes): list[kJoinSmemSlots
    // / 2] u64 (j << 32 | count), keys[kJoinSmemSlots] u32, counts[...] u32
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint64_t* s_list = reinterpret_cast<uint64_t*>(s_dyn);
    uint32_t* s_keys = reinterpret_cast<uint32_t*>(s_list + kJoinSmemSlots / 2);
    uint32_t* s_cnts = s_keys + kJoinSmemSlots;
    __shared__ int64_t s_task;
    __shared__ uint32_t s_n;
    __shared__ int64_t s_off;
    const int64_t n = a.s.n;
    for (;;) {
        int64_t i = next_task(a.ctr, &s_task);
        if (i >= (LARGE ? a.n_tasks : n)) break;
        if (LARGE) i = a.large_rows[i];
        const uint32_t need = a.need[i];
        const bool large = 2ull * need > (unsigned long long)kJoinSmemSlots;
        // rows of at most kWarpJoinNeed partners belong to join_warp_kernel
        if (need == 0 || large != LARGE || need <= (uint32_t)kWarpJoinNeed) {
            if (!WRITE && need == 0 && threadIdx.x == 0) a.ccount[i] = 0;
            continue;
        }
        const uint32_t cap = pow2_at_least(2ull * need);
        uint32_t* keys;
        uint32_t* cnts;
        uint64_t* list;
        if (!LARGE) {
            keys = s_keys;
            cnts = s_cnts;
            list = s_list;
        } else {
            if (cap > a.gslots) {
                if (threadIdx.x == 0) atomicMax(a.status, 1);
                continue;
            }
            // one region per block: keys, counts, then the list (u64, 8-aligned)
            keys = a.gtab + (size_t)blockIdx.x * 3 * a.gslots;
            cnts = keys + a.gslots;
            list = reinterpret_cast<uint64_t*>(cnts + a.gslots);
        }
        const uint32_t mask = cap - 1;
        for (uint32_t t = threadIdx.x; t < cap; t += blockDim.x) {
            keys[t] = kEmpty;
            cnts[t] = 0;
        }
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        const int64_t o = a.s.off[i];
        const uint32_t c = a.kcount[i];
        for (uint32_t e = threadIdx.x; e < c; e += blockDim.x) {
            const uint2 rg = a.range[o + e];
            if (a.self_pairs && rg.y - rg.x <= 1) continue;   // only row i itself
            for (uint32_t b = rg.x; b < rg.y; ++b) {
                const int32_t j = a.bseq[b];
                if (a.self_pairs && j <= i) continue;
                uint32_t h = slot_of((uint32_t)j, mask);
                for (uint32_t probe = 0; probe < cap; ++probe) {
                    const uint32_t cur = atomicCAS(&keys[h], kEmpty, (uint32_t)j);
                    if (cur == kEmpty || cur == (uint32_t)j) {
                        atomicAdd(&cnts[h], 1u);
                        break;
                    }
                    h = (h + 1) & mask;
                }
            }
        }
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < cap; t += blockDim.x) {
            const uint32_t j = keys[t];
            if (j != kEmpty && cnts[t] >= (uint32_t)a.min_shared) {
                const uint32_t e = atomicAdd(&s_n, 1u);
                if (WRITE || a.stash) list[e] = ((uint64_t)j << 32) | cnts[t];
            }
        }
        __syncthreads();
        const uint32_t m = s_n;
        if (!WRITE) {
            if (threadIdx.x == 0) a.ccount[i] = m;
            if (!a.stash) continue;
        }
        if (m == 0) continue;
        // bitonic sort of list[0, P) by j (padding sorts last); P <= cap / 2
        const uint32_t P = m <= 1 ? 1 : 1u << (32 - __clz(m - 1));
        for (uint32_t t = m + threadIdx.x; t < P; t += blockDim.x) list[t] = ~0ull;
        __syncthreads();
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
                for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) {
                    const uint32_t u = t ^ jj;
                    if (u > t) {
                        const uint64_t x = list[t], y = list[u];
                        const bool up = (t & k) == 0;
                        if ((x > y) == up) {
                            list[t] = y;
                            list[u] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (!WRITE) {
            // the counting pass stashes the sorted row
            if (threadIdx.x == 0) {
                int64_t off = (int64_t)atomicAdd(a.stash_ctr, (unsigned long long)m);
                if (off + m > a.stash_cap) off = -1;
                a.stash_off[i] = off;
                s_off = off;
            }
            __syncthreads();
            const int64_t off = s_off;
            if (off >= 0)
                for (uint32_t t = threadIdx.x; t < m; t += blockDim.x) a.stash[off + t] = list[t];
            __syncthreads();
            continue;
        }
        const int64_t base = (int64_t)a.coff[i];
        for (uint32_t t = threadIdx.x; t < m; t += blockDim.x) {
            const int64_t d = base + t;
            if (d < a.capacity) {
                const uint64_t v = list[t];
                a.out_pairs[2 * d] = (int32_t)i;
                a.out_pairs[2 * d + 1] = (int32_t)(v >> 32);
                if (a.out_counts) a.out_counts[d] = (int32_t)(v & 0xffffffffu);
            }
        }
    }
}

// Copies every row's stashed list to its place in (i, j) order (one warp per
// row): what the writing pass would write, without its second join.
__global__ void join_copy_kernel(JoinArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < a.s.n; i += warps) {
        const uint32_t m = a.ccount[i];
        if (m == 0) continue;
        const int64_t src = a.stash_off[i], base = (int64_t)a.coff[i];
        for (uint32_t t = lane; t < m; t += 32) {
            const int64_t d = base + t;
            if (d < a.capacity) {
                const uint64_t v = a.stash[src + t];
                a.out_pairs[2 * d] = (int32_t)i;
                a.out_pairs[2 * d + 1] = (int32_t)(v >> 32);
                if (a.out_counts) a.out_counts[d] = (int32_t)(v & 0xffffffffu);
            }
        }
    }
}

// The join of rows with at most kWarpJoinNeed possible partners: one warp
// per row, its hash table and candidate list in the warp's share of shared
// memory, warp-level synchronisation only.  Same results as join_kernel.

template <bool WRITE>
__global__ void __launch_bounds__(kWarpJoinWarps * 32) join_warp_kernel(JoinArgs a) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ uint32_t s_n[kWarpJoinWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* const list = reinterpret_cast<uint64_t*>(s_dyn) + w * (kWarpJoinSlots / 2);
    uint32_t* const keys = reinterpret_cast<uint32_t*>(reinterpret_cast<uint64_t*>(s_dyn) +
                                                       kWarpJoinWarps * (kWarpJoinSlots / 2)) +
                           w * 2 * kWarpJoinSlots;
    uint32_t* const cnts = keys + kWarpJoinSlots;
    const int64_t n = a.s.n;
    for (;;) {
        int64_t i = 0;
        if (lane == 0) i = (int64_t)atomicAdd(a.ctr, 1ull);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= n) break;
        const uint32_t need = a.need[i];
        if (need == 0 || need > (uint32_t)kWarpJoinNeed) {
            if (!WRITE && need == 0 && lane == 0) a.ccount[i] = 0;
            continue;
        }
        const uint32_t cap = pow2_at_least(2ull * need);
        const uint32_t mask = cap - 1;
        for (uint32_t t = lane; t < cap; t += 32) {
            keys[t] = kEmpty;
            cnts[t] = 0;
        }
        if (lane == 0) s_n[w] = 0;
        __syncwarp();
        const int64_t o = a.s.off[i];
        const uint32_t c = a.kcount[i];
        for (uint32_t e = lane; e < c; e += 32) {
            const uint2 rg = a.range[o + e];
            if (a.self_pairs && rg.y - rg.x <= 1) continue;   // only row i itself
            for (uint32_t b = rg.x; b < rg.y; ++b) {
                const int32_t j = a.bseq[b];
                if (a.self_pairs && j <= i) continue;
                uint32_t h = slot_of((uint32_t)j, mask);
                for (uint32_t probe = 0; probe < cap; ++probe) {
                    const uint32_t cur = atomicCAS(&keys[h], kEmpty, (uint32_t)j);
                    if (cur == kEmpty || cur == (uint32_t)j) {
                        atomicAdd(&cnts[h], 1u);
                        break;
                    }
                    h = (h + 1) & mask;
                }
            }
        }
        __syncwarp();
        for (uint32_t t = lane; t < cap; t += 32) {
            const uint32_t j = keys[t];
            if (j != kEmpty && cnts[t] >= (uint32_t)a.min_shared) {
                const uint32_t e = atomicAdd(&s_n[w], 1u);
                if (WRITE || a.stash) list[e] = ((uint64_t)j << 32) | cnts[t];
            }
        }
        __syncwarp();
        const uint32_t m = s_n[w];
        if (!WRITE) {
            if (lane == 0) a.ccount[i] = m;
            if (!a.stash) continue;
        }
        if (m == 0) continue;
        // bitonic sort of list[0, P) by j (padding sorts last); P <= cap / 2
        const uint32_t P = m <= 1 ? 1 : 1u << (32 - __clz(m - 1));
        for (uint32_t t = m + lane; t < P; t += 32) list[t] = ~0ull;
        __syncwarp();
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t jj = k >> 1; jj > 0; jj >>= 1) {
                for (uint32_t t = lane; t < P; t += 32) {
                    const uint32_t u = t ^ jj;
                    if (u > t) {
                        const uint64_t x = list[t], y = list[u];
                        if ((x > y) == ((t & k) == 0)) {
                            list[t] = y;
                            list[u] = x;
                        }
                    }
                }
                __syncwarp();
            }
        }
        if (!WRITE) {
            // the counting pass stashes the sorted row
            int64_t off = 0;
            if (lane == 0) {
                off = (int64_t)atomicAdd(a.stash_ctr, (unsigned long long)m);
                if (off + m > a.stash_cap) off = -1;
                a.stash_off[i] = off;
            }
            off = __shfl_sync(0xffffffffu, off, 0);
            if (off >= 0)
                for (uint32_t t = lane; t < m; t += 32) a.stash[off + t] = list[t];
            __syncwarp();
            continue;
        }
        const int64_t base = (int64_t)a.coff[i];
        for (uint32_t t = lane; t < m; t += 32) {
            const int64_t d = base + t;
            if (d < a.capacity) {
                const uint64_t v = list[t];
                a.out_pairs[2 * d] = (int32_t)i;
                a.out_pairs[2 * d + 1] = (int32_t)(v >> 32);
                if (a.out_counts) a.out_counts[d] = (int32_t)(v & 0xffffffffu);
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Identity of alignment records
// ---------------------------------------------------------------------------
// The traceback of the span's global DP (diagonal first, then F, then E;
// inside a gap its opening first) makes only local choices, so the
// statistics (identical columns, diagonal steps) of the path it follows from
// any cell and state are those of the cell it steps to plus its own step:
//   SF(a,b) = F opens ? SH(a-1,b) : SF(a-1,b)
//   SE(a,b) = E opens ? SH(a,b-1) : SE(a,b-1)
//   SH(a,b) = H = H(a-1,b-1) + s ? SH(a-1,b-1) + ([q_a = r_b], 1)
//           : H = F(a,b) ? SF(a,b) : SE(a,b)
// with zero at the borders (gaps only); the answer is SH(n, m), and a path
// from (0, 0) to (n, m) with D diagonal steps has n + m - D columns.  The wavefront below computes H, E, F and these pairs
// forward, one warp per pair: lane k holds kIdR columns of a chunk of 32 kIdR
// columns and streams the span's query rows (row t - k + 1 at step t), the
// left inputs of its first column arriving from lane k - 1 by shuffle and,
// for lane 0 of a later chunk, from the boundary column the previous chunk
// left in global memory.
constexpr int kIdR = 8;                        // columns per lane
constexpr int kIdWarps = 4;                    // warps per block
constexpr int kIdSmallCols = 64;               // spans of up to 64 columns: 8-lane groups
constexpr int kIdMidCols = 128;                // up to 128 columns: 16-lane groups
constexpr int kIdClasses = 4;
constexpr int kIdCoopCols = 2048;              // spans of >= 8 chunks: one block per span
constexpr int kIdCoopColsSmall = 1024;         // >= 4 chunks, when the batch leaves warps idle
constexpr int kIdSmallBatchPerSM = 64;         // pairs per SM up to which a batch counts as small
constexpr int kIdSpinLimit = 1 << 25;          // bounded wait on the previous chunk's progress
// Work lists: the regular classes 0..3, then the cooperative spans of classes
// 2 and 3.  Each list is ordered by decreasing work (longest first, so that
// no long span starts near the end of its launch), through a counting sort
// over kIdBuckets buckets of a span's warp steps, four per doubling.
constexpr int kIdLists = kIdClasses + 2;
constexpr int kIdBuckets = 128;
constexpr int32_t kNegInf = -(1 << 28);

// A chunk's last column at one row: H, E and the (matches, columns) of H and
// E.  The scratch is sized in IdBnd entries (the widest form); a kernel keeps
// its boundary rows in its own statistics width (16 bytes when the pairs are
// packed 16 / 16 bits: one store and one load a row), in global memory and
// in the shared-memory stage.
struct IdBnd {
    int32_t h, e;
    uint64_t sh, se;
};
template <class St>
struct __align__(sizeof(St) == 4 ? 16 : 8) IdRow {
    int32_t h, e;
    St sh, se;
};
static_assert(sizeof(IdRow<uint32_t>) <= sizeof(IdBnd) && sizeof(IdRow<uint64_t>) <= sizeof(IdBnd),
              "a boundary row fits its scratch entry");

struct IdentArgs {
    SeqView q, r;
    const int32_t* pairs;
    const swgb_record* rec;
    int64_t n_pairs;
    int8_t mat[kAlpha * kAlpha];
    int32_t go, ge;
    int32_t id_num, id_den, cov_num, cov_den;
    int32_t coop_cols;         // spans of at least this many columns go cooperative
    int32_t* out;              // [n_pairs][3]: matches, columns, pass
    IdBnd* bnd;                // per-warp boundary columns, one entry per row
    int64_t bnd_stride;
    const int64_t* list;       // the pairs of this launch's list, longest first
    int64_t n_list;
    int64_t* lists;            // the kIdLists lists one after another (n_pairs entries)
    uint32_t* hist;            // [kIdLists][kIdBuckets] pair counts, then as many list cursors
    unsigned long long* ctr;   // [0] task counter, [1..kIdLists] list sizes
    int32_t* status;
};

// prmt.b32 in its default mode: a selector nibble with bit 3 set replicates
// the sign of the byte it selects (the C intrinsic __byte_perm ignores that bit)
__device__ __forceinline__ uint32_t prmt_sext(uint32_t a, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(a), "r"(sel));
    return d;
}

// (matches, diagonal steps): packed 16 / 16 bits in a uint32_t when the span
// has fewer than 65536 rows + columns, else 32 / 32 bits in a uint64_t.
template <class St>
struct Stat;
template <>
struct Stat<uint32_t> {
    __device__ static uint32_t make(uint32_t m, uint32_t c) { return (m << 16) | c; }
    __device__ static uint32_t inc(bool match) { return match ? 0x10001u : 1u; }
    __device__ static uint32_t matches(uint32_t s) { return s >> 16; }
    __device__ static uint32_t columns(uint32_t s) { return s & 0xffffu; }
};
template <>
struct Stat<uint64_t> {
    __device__ static uint64_t make(uint32_t m, uint32_t c) { return ((uint64_t)m << 32) | c; }
    __device__ static uint64_t inc(bool match) { return match ? 0x100000001ull : 1ull; }
    __device__ static uint32_t matches(uint64_t s) { return (uint32_t)(s >> 32); }
    __device__ static uint32_t columns(uint64_t s) { return (uint32_t)s; }
};

__device__ __forceinline__ void ident_write(const IdentArgs& a, int64_t p, int32_t mt, int32_t cols,
                                            int32_t pass) {
    a.out[3 * p] = mt;
    a.out[3 * p + 1] = cols;
    a.out[3 * p + 2] = pass;
}

// Classes (rows + columns < 65536): 0 = at most kIdSmallCols columns, 1 = at
// most kIdMidCols, 2 = more; 3 = rows + columns >= 65536.  ident_route gives
// pair p's list (its class, or 4 / 5 for the spans of classes 2 / 3 of at
// least coop_cols columns) and work bucket, or -1 for a pair answered at
// classification: a zero score (0, 0, fail) or a record outside its
// sequences (-1, -1, fail and status 3), written when ANSWER is set.
template <bool ANSWER>
__device__ int ident_route(const IdentArgs& a, int64_t p, int* bucket) {
    const swgb_record rc = a.rec[p];
    if (rc.score <= 0) {
        if (ANSWER) ident_write(a, p, 0, 0, 0);
        return -1;
    }
    const int32_t qi = a.pairs[2 * p], ri = a.pairs[2 * p + 1];
    const bool ok_idx = qi >= 0 && qi < a.q.n && ri >= 0 && ri < a.r.n;
    const int64_t lq = ok_idx ? a.q.off[qi + 1] - a.q.off[qi] : 0;
    const int64_t lr = ok_idx ? a.r.off[ri + 1] - a.r.off[ri] : 0;
    const int64_t n = (int64_t)rc.q_end - rc.q_start + 1, m = (int64_t)rc.r_end - rc.r_start + 1;
    if (!ok_idx || rc.q_start < 0 || rc.q_end >= lq || rc.r_start < 0 || rc.r_end >= lr ||
        n <= 0 || m <= 0 || n >= a.bnd_stride) {
        if (ANSWER) {
            atomicMax(a.status, 3);
            ident_write(a, p, -1, -1, 0);
        }
        return -1;
    }
    const int cls = n + m >= 65536 ? 3 : (m <= kIdSmallCols ? 0 : (m <= kIdMidCols ? 1 : 2));
    const bool coop = cls >= 2 && m >= a.coop_cols;
    // warp steps of the span: chunks (per warp when cooperative) x rows
    const int64_t chunk = cls == 0 ? 8 * kIdR : (cls == 1 ? 16 * kIdR : 32 * kIdR);
    int64_t nch = (m + chunk - 1) / chunk;
    if (coop) nch = (nch + kIdWarps - 1) / kIdWarps;
    const uint64_t work = (uint64_t)(nch * (n + 32));
    const int e = 63 - __clzll((long long)work);                 // work >= 33: e >= 5
    *bucket = min(4 * e + (int)((work >> (e - 2)) & 3u), kIdBuckets - 1);
    return coop ? kIdClasses + (cls - 2) : cls;
}

// Counting pass: answers what needs no alignment and counts the pairs of
// each (list, bucket).
__global__ void ident_classify_kernel(IdentArgs a) {
    __shared__ uint32_t s_hist[kIdLists * kIdBuckets];
    for (int i = threadIdx.x; i < kIdLists * kIdBuckets; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t base = (int64_t)blockIdx.x * blockDim.x;
    for (int64_t p0 = base; p0 < a.n_pairs; p0 += stride) {
        const int64_t p = p0 + threadIdx.x;
        int bucket = 0;
        const int list = p < a.n_pairs ? ident_route<true>(a, p, &bucket) : -1;
        const int key = list < 0 ? -1 : list * kIdBuckets + bucket;
        // one shared atomic per distinct key of the warp
        const unsigned same = __match_any_sync(0xffffffffu, key);
        if (key >= 0 && (threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&s_hist[key], (uint32_t)__popc(same));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kIdLists * kIdBuckets; i += blockDim.x)
        if (s_hist[i]) atomicAdd(&a.hist[i], s_hist[i]);
}

// One block: the lists one after another, each by decreasing bucket; the
// cursor of every (list, bucket) and the list sizes (ctr[1 + list]).
__global__ void ident_scan_kernel(IdentArgs a) {
    __shared__ uint32_t s_cnt[kIdLists * kIdBuckets];
    for (int i = threadIdx.x; i < kIdLists * kIdBuckets; i += blockDim.x) s_cnt[i] = a.hist[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t off = 0;
        for (int l = 0; l < kIdLists; ++l) {
            const uint32_t first = off;
            for (int b = kIdBuckets - 1; b >= 0; --b) {
                const uint32_t c = s_cnt[l * kIdBuckets + b];
                s_cnt[l * kIdBuckets + b] = off;
                off += c;
            }
            a.ctr[1 + l] = off - first;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kIdLists * kIdBuckets; i += blockDim.x)
        a.hist[kIdLists * kIdBuckets + i] = s_cnt[i];
}

// Placing pass: each routed pair at its (list, bucket) cursor.
__global__ void ident_place_kernel(IdentArgs a) {
    uint32_t* cursor = a.hist + kIdLists * kIdBuckets;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t base = (int64_t)blockIdx.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t p0 = base; p0 < a.n_pairs; p0 += stride) {
        const int64_t p = p0 + threadIdx.x;
        int bucket = 0;
        const int list = p < a.n_pairs ? ident_route<false>(a, p, &bucket) : -1;
        const int key = list < 0 ? -1 : list * kIdBuckets + bucket;
        // one global atomic per distinct key of the warp; ranks below it
        const unsigned same = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(same) - 1;
        uint32_t pos = 0;
        if (key >= 0 && lane == leader) pos = atomicAdd(&cursor[key], (uint32_t)__popc(same));
        pos = __shfl_sync(0xffffffffu, pos, leader);
        const uint64_t at = (uint64_t)pos + __popc(same & ((1u << lane) - 1u));
        if (key >= 0) {
            if (at < (uint64_t)a.n_pairs) a.lists[at] = p;
            else atomicMax(a.status, 5);   // the two passes routed differently
        }
    }
}

// The wavefront of groups of G lanes, one pair per group (G = 8: four pairs
// per warp, one chunk of 64 columns; G = 32: one pair per warp, chunks of 256
// columns).  PROF: lane-private substitution profile in shared memory
// (prof[letter] = the 8 scores of the lane's columns) instead of one lookup
// per cell.
// PF: the letter, its profile word and lane 0's boundary entry are fetched
// ahead of the step that uses them.  That takes their latency off the
// step's dependency chain, which bounds a warp that runs alone (small
// batches, cooperative spans); a full GPU hides it with other warps, and
// there the extra instructions would cost throughput.
// COOP (G = 32): the kIdWarps warps of a block share one span, warp w taking
// chunks w, w + kIdWarps, ...; a chunk's boundary column goes to its warp's
// buffer, and the next chunk's lane 0 waits (bounded) until the producing
// warp's progress counter in shared memory passes the row it needs.  Chunk
// c's progress is published as c (n + 1) + row, so the counters only grow.
template <int G, class St, bool PROF, bool COOP, bool PF>
__global__ void __launch_bounds__(kIdWarps * 32) ident_kernel(IdentArgs a) {
    static_assert(!COOP || G == 32, "cooperative spans use 32-lane chunks");
    constexpr int GROUPS = 32 / G;
    constexpr int CHUNK = G * kIdR;
    __shared__ int8_t s_mat[kAlpha * kAlpha];
    __shared__ __align__(8) uint2 s_prof[PROF ? kIdWarps * 32 * kAlpha : 1];
    __shared__ long long s_prog[COOP ? kIdWarps : 1];
    __shared__ IdRow<St> s_stage[G == 32 ? kIdWarps * 2 * 32 : 1];
    __shared__ int s_abort;    // COOP: a wait ran out; later waits return at once
    __shared__ int64_t s_task;
    for (int t = threadIdx.x; t < kAlpha * kAlpha; t += blockDim.x) s_mat[t] = a.mat[t];
    __syncthreads();
    using S = Stat<St>;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int grp = lane / G, gl = lane % G;
    const int64_t gw = (int64_t)blockIdx.x * kIdWarps + w;
    // boundary columns: one per warp (COOP: the block's kIdWarps, one per chunk residue)
    IdRow<St>* const bnd_base =
        reinterpret_cast<IdRow<St>*>(a.bnd) + (COOP ? (int64_t)blockIdx.x * kIdWarps : gw) * a.bnd_stride;
    uint2* prof = s_prof + (PROF ? (w * 32 + lane) * kAlpha : 0);
    const int32_t ge = a.ge, oe = a.go + a.ge;
    for (;;) {
        int64_t task = 0;
        if (COOP) {
            __syncthreads();
            if (threadIdx.x == 0) {
                s_task = (int64_t)atomicAdd(a.ctr, 1ull);
                for (int k = 0; k < kIdWarps; ++k) s_prog[k] = -1;
                s_abort = 0;
            }
            __syncthreads();
            task = s_task;
        } else {
            if (lane == 0) task = (int64_t)atomicAdd(a.ctr, 1ull);
            task = __shfl_sync(0xffffffffu, task, 0);
        }
        const int64_t first = task * GROUPS;
        if (first >= a.n_list) break;
        // this group's pair (groups past the list compute nothing)
        const int64_t li = first + grp;
        const bool live = li < a.n_list;
        const int64_t p = !live ? 0 : a.list[li];
        swgb_record rc{0, 0, 0, 0, 0};
        int n = 0, m = 0, lq = 0, lr = 0;
        const uint8_t *qs = nullptr, *rs = nullptr;
        if (live) {
            rc = a.rec[p];
            const int32_t qi = a.pairs[2 * p], ri = a.pairs[2 * p + 1];
            lq = (int)(a.q.off[qi + 1] - a.q.off[qi]);
            lr = (int)(a.r.off[ri + 1] - a.r.off[ri]);
            n = rc.q_end - rc.q_start + 1;
            m = rc.r_end - rc.r_start + 1;
            qs = a.q.res + a.q.off[qi] + rc.q_start;
            rs = a.r.res + a.r.off[ri] + rc.r_start;
        }
        // warp-uniform extents
        int n_w = n, nch_w = (m + CHUNK - 1) / CHUNK;
        for (int d = 16; d; d >>= 1) {
            n_w = max(n_w, __shfl_xor_sync(0xffffffffu, n_w, d));
            nch_w = max(nch_w, __shfl_xor_sync(0xffffffffu, nch_w, d));
        }
        int32_t hnm = kNegInf;
        St snm = 0;
        for (int c = COOP ? w : 0; c < nch_w; c += COOP ? kIdWarps : 1) {
            const int c0 = c * CHUNK + gl * kIdR;
            IdRow<St>* const wbuf = bnd_base + (COOP ? (c % kIdWarps) * a.bnd_stride : 0);
            IdRow<St>* const rbuf = bnd_base + (COOP ? ((c + kIdWarps - 1) % kIdWarps) * a.bnd_stride : 0);
            int rcode[kIdR];
            int32_t H[kIdR], F[kIdR];
            St SH[kIdR], SF[kIdR];
#pragma unroll
            for (int x = 0; x < kIdR; ++x) {
                const int b = c0 + x + 1;
                rcode[x] = b <= m ? rs[b - 1] : 0;
                H[x] = -(oe + ge * (b - 1));
                F[x] = kNegInf;
                SH[x] = 0;
                SF[x] = 0;
            }
            if (PROF) {
                __syncwarp();
                for (int l = 0; l < kAlpha; ++l) {
                    uint32_t lo = 0, hi = 0;
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        lo |= (uint32_t)(uint8_t)s_mat[l * kAlpha + rcode[x]] << (8 * x);
                        hi |= (uint32_t)(uint8_t)s_mat[l * kAlpha + rcode[x + 4]] << (8 * x);
                    }
                    prof[l] = make_uint2(lo, hi);
                }
                __syncwarp();
            }
            int32_t h_out = -(oe + ge * (c0 + kIdR - 1)), e_out = kNegInf;
            St sh_out = 0, se_out = 0;
            int32_t hd_next = c0 == 0 ? 0 : -(oe + ge * (c0 - 1));
            St sd_next = 0;
            const bool read_b = G == 32 && c > 0 && gl == 0;
            // the letter of span row `row` (any code outside the span: its
            // cells are not computed)
            auto letter = [&](int row) -> int { return row >= 1 && row <= n ? qs[row - 1] : 0; };
            // COOP: the whole warp waits (bounded) until the previous chunk's
            // warp has finished span row `row`
            auto wait_rows = [&](int row) {
                const long long want = (long long)(c - 1) * (n + 1) + row;
                volatile long long* prog = s_prog + (c - 1) % kIdWarps;
                volatile int* abort_flag = &s_abort;
                int spins = 0;
                while (*prog < want && !*abort_flag && ++spins < kIdSpinLimit) {
                }
                if (spins >= kIdSpinLimit) {
                    *abort_flag = 1;
                    atomicMax(a.status, 4);
                }
                __threadfence_block();
            };
            // G = 32: the previous chunk's boundary passes through a
            // two-batch stage in shared memory, batch k = rows 32 k + 1 ..
            // 32 k + 32: the warp loads batch k + 1 from global memory (one
            // row a lane) at step 32 k + 8 and stages it at the end of step
            // 32 k + 30, so that lane 0's read of a row never waits on a
            // global load.  (Without COOP the previous chunk is this warp's
            // own, finished before this one began; the rows a batch load
            // reads are past the ones lane 31 has overwritten by then.)
            IdRow<St>* const stage = s_stage + (G == 32 ? w * 64 : 0);
            const bool staged = G == 32 && c > 0;
            auto fetch = [&](int row) -> IdRow<St> { return rbuf[row]; };
            IdRow<St> next_row{kNegInf, kNegInf, 0, 0};
            if (staged) {
                if (COOP) wait_rows(min(32, n));
                if (lane + 1 <= n) stage[lane] = fetch(lane + 1);
                __syncwarp();
            }
            // lane 0 of a later chunk: the previous chunk's boundary at `row`
            auto boundary = [&](int row) -> IdRow<St> {
                return stage[(((row - 1) >> 5) & 1) * 32 + ((row - 1) & 31)];
            };
            // PF: the letter two rows on, its profile word and the boundary
            // entry one row on
            int qc_next = 0, qc_after = 0;
            uint2 pw_next = make_uint2(0u, 0u);
            IdRow<St> b_next{kNegInf, kNegInf, 0, 0};
            if constexpr (PF) {
                qc_next = letter(1 - gl);
                qc_after = letter(2 - gl);
                if (PROF) pw_next = prof[qc_next];
                if (read_b && n >= 1) b_next = boundary(1);
            }
            for (int t = 0; t < n_w + G - 1; ++t) {
                const int arow = t - gl + 1;
                const int32_t up_h = __shfl_up_sync(0xffffffffu, h_out, 1, G);
                const int32_t up_e = __shfl_up_sync(0xffffffffu, e_out, 1, G);
                const St up_sh = __shfl_up_sync(0xffffffffu, sh_out, 1, G);
                const St up_se = __shfl_up_sync(0xffffffffu, se_out, 1, G);
                int32_t hl = up_h, el = up_e;
                St shl = up_sh, sel = up_se;
                const int32_t hd = hd_next;
                const St sd = sd_next;
                int qc = 0;
                uint2 pw = make_uint2(0u, 0u);
                if constexpr (PF) {
                    qc = qc_next;
                    pw = pw_next;
                    qc_next = qc_after;
                    if (PROF) pw_next = prof[qc_next];
                    qc_after = letter(arow + 2);
                }
                if (gl == 0) {
                    if (!read_b) {
                        hl = -(oe + ge * (arow - 1));   // H(a, 0)
                        el = kNegInf;
                        shl = 0;
                        sel = 0;
                    } else if (arow >= 1 && arow <= n) {
                        IdRow<St> v;
                        if constexpr (PF) {
                            v = b_next;
                            if (arow + 1 <= n) b_next = boundary(arow + 1);
                        } else {
                            v = boundary(arow);
                        }
                        hl = v.h;
                        el = v.e;
                        shl = v.sh;
                        sel = v.se;
                    }
                }
                if (arow >= 1 && arow <= n && c0 < m) {
                    if constexpr (!PF) {
                        qc = qs[arow - 1];
                        if (PROF) pw = prof[qc];
                    }
                    int32_t hleft = hl, eleft = el, hdiag = hd;
                    St shleft = shl, seleft = sel, sdiag = sd;
#pragma unroll
                    for (int x = 0; x < kIdR; ++x) {
                        const int32_t eo = hleft - oe;
                        const int32_t e = __viaddmax_s32(eleft, -ge, eo);
                        const St se = e == eo ? shleft : seleft;
                        const int32_t fo = H[x] - oe;
                        const int32_t f = __viaddmax_s32(F[x], -ge, fo);
                        const St sf = f == fo ? SH[x] : SF[x];
                        // byte x % 4 of the profile word, sign-extended (one byte permute)
                        const uint32_t xb = (uint32_t)(x & 3);   // a constant once unrolled
                        const uint32_t sel8 = xb | ((xb | 8u) << 4) | ((xb | 8u) << 8) | ((xb | 8u) << 12);
                        const int32_t s = PROF ? (int32_t)prmt_sext(x < 4 ? pw.x : pw.y, sel8)
                                               : (int32_t)s_mat[qc * kAlpha + rcode[x]];
                        const int32_t d = hdiag + s;
                        const int32_t h = __vimax3_s32(d, e, f);
                        const St salt = h == f ? sf : se;
                        const St sh = h == d ? sdiag + S::inc(qc == rcode[x]) : salt;
                        hdiag = H[x];
                        sdiag = SH[x];
                        H[x] = h;
                        F[x] = f;
                        SH[x] = sh;
                        SF[x] = sf;
                        hleft = h;
                        eleft = e;
                        shleft = sh;
                        seleft = se;
                    }
                    h_out = hleft;
                    e_out = eleft;
                    sh_out = shleft;
                    se_out = seleft;
                    if (G == 32 && gl == 31 && c + 1 < nch_w) {
                        wbuf[arow] = IdRow<St>{hleft, eleft, shleft, seleft};
                        if (COOP) {
                            __threadfence_block();
                            *(volatile long long*)(s_prog + c % kIdWarps) = (long long)c * (n + 1) + arow;
                        }
                    }
                }
                hd_next = gl == 0 ? hl : up_h;
                sd_next = gl == 0 ? shl : up_sh;
                if (staged) {
                    const int row0 = 32 * ((t >> 5) + 1) + 1;   // the next batch's first row
                    if ((t & 31) == 8 && row0 <= n) {
                        if (COOP) wait_rows(min(row0 + 31, n));
                        if (row0 + lane <= n) next_row = fetch(row0 + lane);
                    } else if ((t & 31) == 30 && row0 <= n) {
                        stage[(((row0 - 1) >> 5) & 1) * 32 + lane] = next_row;
                        __syncwarp();
                    }
                }
            }
            // the lane owning column m: no row past n is computed, so its
            // columns hold row n once the steps are done
            if (n >= 1 && m > c0 && m <= c0 + kIdR) {
#pragma unroll
                for (int x = 0; x < kIdR; ++x)
                    if (c0 + x + 1 == m) {
                        hnm = H[x];
                        snm = SH[x];
                    }
            }
            __syncwarp();
        }
        // the lane owning (n, m) answers for its group
        if (live && hnm != kNegInf) {
            if (hnm != rc.score) {
                atomicMax(a.status, 2);
                ident_write(a, p, -1, -1, 0);
            } else {
                const int32_t mt = (int32_t)S::matches(snm);
                const int32_t cols = n + m - (int32_t)S::columns(snm);   // minus diagonal steps
                const bool pass = cols > 0 && (int64_t)mt * a.id_den >= (int64_t)a.id_num * cols &&
                                  (int64_t)n * a.cov_den >= (int64_t)a.cov_num * lq &&
                                  (int64_t)m * a.cov_den >= (int64_t)a.cov_num * lr;
                ident_write(a, p, mt, cols, pass ? 1 : 0);
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Pair features of the learned candidate filter
// ---------------------------------------------------------------------------
// For a pair (i of set A, j of set B), with K(s) the distinct k-mers of
// standard letters of s and p_s(x) their first positions (kmer_sets), the
// shared k-mers x give diagonals d = p_i(x) - p_j(x) and 24 bins
// floor(24 (d + lj - k) / D), D = li + lj - 2k + 1.  The 32 features are
// integer ratios num / den rounded through double to float (0 for den = 0):
//   0 c/(c+16), 1 min(l)/max(l), 2..25 hist[t]/c,
//   26 sum_y |nA(y) lj - nB(y) li| / (2 li lj), 27 li/(li+256), 28 lj/(lj+256),
//   29 max_t hist[t]/c, 30 c/min(|K(i)|, |K(j)|), 31 (max d - min d)/D (c >= 2).
constexpr int kFeat = 32;
constexpr int kFeatBins = 24;
constexpr int kFeatWarps = 8;
constexpr int kFeatWarpSlots = 1024;  // warp-private shared table of K(i): up to 512 k-mers
// Per warp, an 8192-bit filter of K(i) (one bit per k-mer, another
// multiplicative hash than the table's): a partner k-mer whose bit is clear is
// not in K(i), so most misses cost one shared load instead of a probe run.
constexpr int kFeatBitWords = 256;
constexpr int kFeatSmemBytes = kFeatWarps * (kFeatWarpSlots * 8 + kFeatBitWords * 4);
__device__ __forceinline__ uint32_t feat_bit_of(uint32_t key) { return (key * 0x85ebca6bu) >> 19; }
constexpr int64_t kJoinStashMax = int64_t(1) << 27;   // entries (8 B) of the joins' stash
constexpr int kFeatChunk = 32;        // consecutive pairs per warp task
constexpr int kFeatInFlight = 8;      // partner k-mers loaded at once per lane

struct FeatArgs {
    SeqView A, B;
    int k;
    const uint32_t *kmA, *posA, *cntA;     // kmer_sets of A
    const uint32_t *kmB, *posB, *cntB;     // kmer_sets of B
    const uint32_t *compA, *compB;         // [n][20] letter counts
    const int32_t* pairs;
    int64_t n_pairs;
    float* out;                            // [n_pairs][32]
    uint32_t* gtab;                        // per-warp global tables (keys, positions)
    uint32_t gslots;
    unsigned long long* ctr;
    int32_t* status;
};

__global__ void composition_kernel(SeqView s, uint32_t* comp) {
    __shared__ uint32_t cnt[8][kStdLetters];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < s.n; i += warps) {
        if (lane < kStdLetters) cnt[w][lane] = 0;
        __syncwarp();
        for (int64_t p = s.off[i] + lane; p < s.off[i + 1]; p += 32) {
            const uint32_t c = s.res[p];
            if (c < (uint32_t)kStdLetters) atomicAdd(&cnt[w][c], 1u);
        }
        __syncwarp();
        if (lane < kStdLetters) comp[i * kStdLetters + lane] = cnt[w][lane];
        __syncwarp();
    }
}

__device__ __forceinline__ float feat_ratio(int64_t num, int64_t den) {
    return den == 0 ? 0.0f : __double2float_rn((double)num / (double)den);
}

// One warp per task of kFeatChunk consecutive pairs; for each run of pairs
// with the same first index i it builds K(i) (k-mer -> first position) in a
// warp-private hash table and probes every partner's k-mers against it.
__global__ void __launch_bounds__(kFeatWarps * 32) features_kernel(FeatArgs a) {
    extern __shared__ __align__(16) uint32_t s_tab[];
    __shared__ uint32_t s_hist[kFeatWarps][kFeatBins];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* const s_keys = s_tab + w * 2 * kFeatWarpSlots;
    uint32_t* const s_bits = s_tab + kFeatWarps * 2 * kFeatWarpSlots + w * kFeatBitWords;
    uint32_t* const g_keys = a.gtab ? a.gtab + ((size_t)blockIdx.x * kFeatWarps + w) * 2 * a.gslots
                                    : nullptr;
    for (;;) {
        int64_t task = 0;
        if (lane == 0) task = (int64_t)atomicAdd(a.ctr, 1ull);
        const int64_t t0 = __shfl_sync(0xffffffffu, task, 0) * kFeatChunk;
        if (t0 >= a.n_pairs) break;
        const int64_t t1 = min(t0 + (int64_t)kFeatChunk, a.n_pairs);
        int64_t p0 = t0;
        while (p0 < t1) {
            const int32_t i = a.pairs[2 * p0];
            int64_t p1 = p0 + 1;
            while (p1 < t1 && a.pairs[2 * p1] == i) ++p1;
            const bool ok_i = i >= 0 && i < a.A.n;
            const uint32_t ni = ok_i ? a.cntA[i] : 0u;
            const uint32_t cap = pow2_at_least(2ull * ni);
            uint32_t* keys = s_keys;
            uint32_t* pos;
            uint32_t tcap = kFeatWarpSlots;
            if (cap > (uint32_t)kFeatWarpSlots) {
                keys = g_keys;
                tcap = a.gslots;
            }
            const bool table_ok = cap <= tcap && keys != nullptr;
            pos = keys + tcap;
            const uint32_t mask = cap - 1;
            __syncwarp();
            if (table_ok) {
                for (uint32_t s = lane; s < cap; s += 32) keys[s] = kEmpty;
                for (int s = lane; s < kFeatBitWords; s += 32) s_bits[s] = 0u;
                __syncwarp();
                const int64_t oi = a.A.off[i];
                // K(i)'s entries (k-mer, position) loaded four per lane ahead
                // of their inserts, so the loads overlap
                for (uint32_t e0 = lane; e0 < ni; e0 += 128) {
                    uint32_t xs[4], ps[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const bool in = e0 + 32 * u < ni;
                        xs[u] = in ? a.kmA[oi + e0 + 32 * u] : kEmpty;
                        ps[u] = in ? a.posA[oi + e0 + 32 * u] : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t x = xs[u];
                        if (x == kEmpty) continue;
                        const uint32_t hb = feat_bit_of(x);
                        atomicOr(&s_bits[hb >> 5], 1u << (hb & 31));
                        uint32_t h = slot_of(x, mask);
                        for (uint32_t probe = 0; probe < cap; ++probe) {
                            if (atomicCAS(&keys[h], kEmpty, x) == kEmpty) {
                                pos[h] = ps[u];
                                break;
                            }
                            h = (h + 1) & mask;
                        }
                    }
                }
                __syncwarp();
            }
            for (int64_t p = p0; p < p1; ++p) {
                const int32_t j = a.pairs[2 * p + 1];
                float* o = a.out + p * kFeat;
                if (!ok_i || j < 0 || j >= a.B.n || !table_ok) {
                    if (lane == 0) atomicMax(a.status, ok_i && j >= 0 && j < a.B.n ? 2 : 3);
                    o[lane] = 0.0f;
                    continue;
                }
                const int64_t li = a.A.off[i + 1] - a.A.off[i], lj = a.B.off[j + 1] - a.B.off[j];
                const uint32_t nj = a.cntB[j];
                const int64_t oj = a.B.off[j];
                const int64_t D = li + lj - 2 * (int64_t)a.k + 1;
                if (lane < kFeatBins) s_hist[w][lane] = 0;
                __syncwarp();
                int c = 0;
                int32_t dmin = INT32_MAX, dmax = INT32_MIN;
                const int32_t lj32 = (int32_t)lj, D32 = (int32_t)D;
                // kFeatInFlight partner k-mers loaded per lane at once
                for (uint32_t e0 = lane; e0 < nj; e0 += 32 * kFeatInFlight) {
                    uint32_t xs[kFeatInFlight];
#pragma unroll
                    for (int u = 0; u < kFeatInFlight; ++u)
                        xs[u] = e0 + 32 * u < nj ? a.kmB[oj + e0 + 32 * u] : kEmpty;
#pragma unroll
                    for (int u = 0; u < kFeatInFlight; ++u) {
                        const uint32_t x = xs[u];
                        if (x == kEmpty) continue;
                        const uint32_t hb = feat_bit_of(x);
                        if (((s_bits[hb >> 5] >> (hb & 31)) & 1u) == 0u) continue;   // not in K(i)
                        uint32_t h = slot_of(x, mask);
                        for (uint32_t probe = 0; probe < cap; ++probe) {
                            const uint32_t key = keys[h];
                            if (key == x) {
                                // 0 <= d + lj - k <= li + lj - 2k = D - 1 (both positions
                                // start a k-mer): the bin is an unsigned 32-bit quotient
                                const int32_t d = (int32_t)pos[h] - (int32_t)a.posB[oj + e0 + 32 * u];
                                atomicAdd(&s_hist[w][(uint32_t)(kFeatBins * (d + lj32 - a.k)) / (uint32_t)D32], 1u);
                                ++c;
                                dmin = min(dmin, d);
                                dmax = max(dmax, d);
                                break;
                            }
                            if (key == kEmpty) break;
                            h = (h + 1) & mask;
                        }
                    }
                }
                for (int s = 16; s; s >>= 1) {
                    c += __shfl_xor_sync(0xffffffffu, c, s);
                    dmin = min(dmin, __shfl_xor_sync(0xffffffffu, dmin, s));
                    dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, s));
                }
                __syncwarp();
                const uint32_t hmax =
                    __reduce_max_sync(0xffffffffu, lane < kFeatBins ? s_hist[w][lane] : 0u);
                // lanes 2..25 produce the histogram features
                const uint32_t hv = (lane >= 2 && lane < 2 + kFeatBins) ? s_hist[w][lane - 2] : 0u;
                int64_t cd = 0;
                if (lane < kStdLetters) {
                    const int64_t v = (int64_t)a.compA[(int64_t)i * kStdLetters + lane] * lj -
                                      (int64_t)a.compB[(int64_t)j * kStdLetters + lane] * li;
                    cd = v < 0 ? -v : v;
                }
                for (int s = 16; s; s >>= 1) cd += __shfl_xor_sync(0xffffffffu, (long long)cd, s);
                // lane f's numerator and denominator, then one division for all lanes
                int64_t num, den;
                if (lane == 0) { num = c; den = c + 16; }
                else if (lane == 1) { num = min(li, lj); den = max(li, lj); }
                else if (lane < 2 + kFeatBins) { num = hv; den = c; }
                else if (lane == 26) { num = cd; den = 2 * li * lj; }
                else if (lane == 27) { num = li; den = li + 256; }
                else if (lane == 28) { num = lj; den = lj + 256; }
                else if (lane == 29) { num = hmax; den = c; }
                else if (lane == 30) { num = c; den = min(ni, nj); }
                else { num = (int64_t)dmax - dmin; den = c >= 2 ? D : 0; }
                o[lane] = feat_ratio(num, den);
                __syncwarp();
            }
            p0 = p1;
        }
    }
}

// kept[p] = 1 when logit[p] >= threshold
__global__ void select_flags_kernel(const float* __restrict__ logits, int64_t n, float threshold,
                                    uint32_t* flags) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
        flags[p] = logits[p] >= threshold ? 1u : 0u;
}

__global__ void select_scatter_kernel(const int32_t* __restrict__ pairs, const uint32_t* __restrict__ flags,
                                      const uint64_t* __restrict__ pos, int64_t n, int32_t* out,
                                      int64_t* index_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        if (flags[p]) {
            const uint64_t d = pos[p];
            out[2 * d] = pairs[2 * p];
            out[2 * d + 1] = pairs[2 * p + 1];
            if (index_out) index_out[d] = p;
        }
    }
}

}  // namespace
}  // namespace swgb

// ===========================================================================
// Host side
// ===========================================================================
struct SearchStore {
    int device = 0;
    uint32_t* ent_kmer = nullptr; int64_t ent_cap = 0;
    uint32_t* ent_pos = nullptr;  int64_t entp_cap = 0;
    uint32_t* kcount = nullptr;   int64_t kcount_cap = 0;
    uint32_t* hist = nullptr;     int64_t hist_cap = 0;
    uint32_t* start = nullptr;    int64_t start_cap = 0;
    int32_t* bseq = nullptr;      int64_t bseq_cap = 0;
    uint32_t* need = nullptr;     int64_t need_cap = 0;
    uint32_t* ccount = nullptr;   int64_t ccount_cap = 0;
    uint64_t* coff = nullptr;     int64_t coff_cap = 0;
    uint64_t* part = nullptr;     int64_t part_cap = 0;
    uint32_t* gtab = nullptr;     int64_t gtab_cap = 0;
    IdBnd* bnd = nullptr;         int64_t bnd_cap = 0;
    int64_t* lists = nullptr;     int64_t lists_cap = 0;
    uint2* range = nullptr;       int64_t range_cap = 0;
    int32_t* large_rows = nullptr; int64_t large_rows_cap = 0;
    uint64_t* stash = nullptr;    int64_t stash_cap = 0;     // joins: the counting pass's rows
    int64_t* stash_off = nullptr; int64_t stash_off_cap = 0;
    // pair features: k-mer sets of a second set, letter counts of both
    uint32_t* ent2_kmer = nullptr; int64_t ent2_cap = 0;
    uint32_t* ent2_pos = nullptr;  int64_t ent2p_cap = 0;
    uint32_t* kcount2 = nullptr;   int64_t kcount2_cap = 0;
    uint32_t* comp = nullptr;      int64_t comp_cap = 0;
    uint32_t* comp2 = nullptr;     int64_t comp2_cap = 0;
    uint32_t* flags = nullptr;     int64_t flags_cap = 0;
    unsigned long long* ctr = nullptr;   // [16] work counters and statistics
    uint32_t* id_hist = nullptr;         // identity lists: bucket counts and cursors
    int32_t* status = nullptr;
};

void search_store_free(SearchStore* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    void* ptrs[] = {s->ent_kmer, s->ent_pos, s->kcount, s->hist, s->start, s->bseq,
                    s->need, s->ccount, s->coff, s->part, s->gtab, s->bnd, s->ctr,
                    s->status, s->large_rows, s->lists, s->range, s->ent2_kmer, s->ent2_pos, s->kcount2,
                    s->comp, s->comp2, s->flags, s->stash, s->stash_off, s->id_hist};
    for (void* p : ptrs) cudaFree(p);
    delete s;
}

namespace {

int search_store(swgb_ctx* ctx, SearchStore** out) {
    if (!ctx->search) {
        SearchStore* s = new (std::nothrow) SearchStore();
        if (!s) return fail(ctx, SWGB_ENOMEM, "search scratch: host allocation");
        s->device = ctx->device;
        cudaError_t e = cudaMalloc(&s->ctr, sizeof(unsigned long long) * 16);
        if (e == cudaSuccess) e = cudaMalloc(&s->status, sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&s->id_hist, sizeof(uint32_t) * 2 * kIdLists * kIdBuckets);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(join_kernel<false, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kJoinSmemBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(join_kernel<false, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kJoinSmemBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kFeatSmemBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(join_warp_kernel<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kWarpJoinSmemBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(join_warp_kernel<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kWarpJoinSmemBytes);
        // The identity launches run side by side; an SM holds blocks of
        // several kernels only under one split of its L1 / shared memory, so
        // all of them ask for the same (largest shared) split.
        {
            const void* ident_fns[] = {
                (const void*)ident_kernel<8, uint32_t, false, false, false>,
                (const void*)ident_kernel<16, uint32_t, true, false, false>,
                (const void*)ident_kernel<32, uint32_t, true, false, false>,
                (const void*)ident_kernel<32, uint64_t, true, false, false>,
                (const void*)ident_kernel<8, uint32_t, false, false, true>,
                (const void*)ident_kernel<16, uint32_t, true, false, true>,
                (const void*)ident_kernel<32, uint32_t, true, false, true>,
                (const void*)ident_kernel<32, uint64_t, true, false, true>,
                (const void*)ident_kernel<32, uint32_t, true, true, true>,
                (const void*)ident_kernel<32, uint64_t, true, true, true>};
            for (const void* fn : ident_fns)
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared);
        }
        if (e != cudaSuccess) {
            search_store_free(s);
            return cuda_fail(ctx, e, "search scratch");
        }
        ctx->search = s;
    }
    *out = ctx->search;
    return SWGB_OK;
}

// Exclusive scan of in[0, n) into out[0, n] on st.
template <class Out>
int device_scan(swgb_ctx* ctx, SearchStore* S, const uint32_t* in, int64_t n, Out* out,
                cudaStream_t st) {
    const int64_t nb = std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile);
    CK(grow(&S->part, &S->part_cap, nb + 1), "scan scratch");
    scan_reduce_kernel<<<(unsigned)nb, kScanT, 0, st>>>(in, n, S->part);
    scan_part_kernel<<<1, kScanT, 0, st>>>(S->part, nb);
    scan_apply_kernel<Out><<<(unsigned)nb, kScanT, 0, st>>>(in, n, S->part, nb, out);
    CK(cudaGetLastError(), "scan kernels");
    return SWGB_OK;
}

int64_t warp_grid(swgb_ctx* ctx, int64_t items, int threads) {
    const int64_t per = threads / 32;
    return std::max<int64_t>(1, std::min<int64_t>((items + per - 1) / per, (int64_t)ctx->sm_count * 32));
}

}  // namespace

namespace {

int64_t kmer_space(int k) {
    int64_t V = 1;
    for (int t = 0; t < k; ++t) V *= kStdLetters;
    return V;
}

// Global hash tables of sequences above the shared-memory class, for
// kmer_sets launches over a set of longest length max_len (reserved before
// any launch that may still run; grow() frees the old buffer).
int reserve_set_tables(swgb_ctx* ctx, SearchStore* S, int64_t max_len, uint32_t* gslots) {
    *gslots = pow2_at_least((uint64_t)std::max<int64_t>(max_len, 1) * 2);
    if (*gslots > (uint32_t)kSetSmemSlots)
        CK(grow(&S->gtab, &S->gtab_cap, (int64_t)ctx->sm_count * 4 * 2 * *gslots), "k-mer table scratch");
    return SWGB_OK;
}

// Distinct k-mers (with first positions) of every sequence of `set` into
// kmer / pos at the set's offsets, their numbers into cnt.
int build_sets(swgb_ctx* ctx, SearchStore* S, const swgb_seqset* set, int k, uint32_t* kmer,
               uint32_t* pos, uint32_t* cnt, uint32_t gslots, int32_t* launches, cudaStream_t st) {
    if (set->n == 0) return SWGB_OK;
    CK(cudaMemsetAsync(S->ctr, 0, sizeof(unsigned long long), st), "memset");
    SetArgs sa{view(set), k, kmer, pos, cnt, S->gtab, gslots, S->ctr, S->status};
    kmer_sets_kernel<<<ctx->sm_count * 4, kSearchThreads, 0, st>>>(sa);
    CK(cudaGetLastError(), "kmer_sets kernel");
    *launches += 1;
    return SWGB_OK;
}

// Buckets of the distinct k-mers of `set` (the columns of the sequence x
// k-mer matrix): start [V + 1], and per entry its sequence and position.
int build_buckets(swgb_ctx* ctx, SearchStore* S, const swgb_seqset* set, const uint32_t* kmer,
                  const uint32_t* cnt, int64_t V, uint32_t* start, int32_t* bseq,
                  int32_t* launches, cudaStream_t st) {
    CK(grow(&S->hist, &S->hist_cap, V), "bucket scratch");
    CK(cudaMemsetAsync(S->hist, 0, sizeof(uint32_t) * V, st), "memset");
    const int64_t wg = warp_grid(ctx, std::max<int64_t>(set->n, 1), 256);
    if (set->n > 0) {
        kmer_hist_kernel<<<(unsigned)wg, 256, 0, st>>>(view(set), kmer, cnt, S->hist);
        CK(cudaGetLastError(), "kmer_hist kernel");
        *launches += 1;
    }
    int rc = device_scan<uint32_t>(ctx, S, S->hist, V, start, st);
    if (rc) return rc;
    *launches += 3;
    // the histogram's array becomes the scatter's cursors: a copy of the starts
    CK(cudaMemcpyAsync(S->hist, start, sizeof(uint32_t) * V, cudaMemcpyDeviceToDevice, st), "cursor copy");
    if (set->n > 0) {
        kmer_scatter_kernel<<<(unsigned)wg, 256, 0, st>>>(view(set), kmer, cnt, S->hist, bseq);
        CK(cudaGetLastError(), "kmer_scatter kernel");
        *launches += 1;
    }
    return SWGB_OK;
}

// The join of the rows' k-mer sets with the columns' buckets: pairs (row i,
// column j) with >= min_shared common k-mers (j > i for one set), ordered by
// (i, j); *found receives their number, the first `capacity` are written.
int join_rows(swgb_ctx* ctx, SearchStore* S, const swgb_seqset* rows, const uint32_t* kmer,
              const uint32_t* cnt, const uint32_t* start, const int32_t* bseq, int64_t n_cols,
              bool self_pairs, int min_shared, int32_t* pairs, int32_t* counts, int64_t capacity,
              int64_t* found, int32_t* launches, cudaStream_t st) {
    const int64_t n = rows->n;
    *found = 0;
    if (n == 0) return SWGB_OK;
    CK(grow(&S->need, &S->need_cap, n), "join scratch");
    CK(grow(&S->ccount, &S->ccount_cap, n), "join scratch");
    CK(grow(&S->coff, &S->coff_cap, n + 1), "join scratch");
    CK(grow(&S->large_rows, &S->large_rows_cap, n), "join scratch");
    CK(grow(&S->range, &S->range_cap, std::max<int64_t>(rows->total, 1)), "join scratch");
    // the counting pass stashes each row's sorted list (room for the caller's
    // capacity, at most kJoinStashMax entries); if they all fit, a copy
    // replaces the writing pass
    const int64_t stash_cap = std::min<int64_t>(std::max<int64_t>(capacity, 1), kJoinStashMax);
    CK(grow(&S->stash, &S->stash_cap, stash_cap), "join scratch");
    CK(grow(&S->stash_off, &S->stash_off_cap, n), "join scratch");
    CK(cudaMemsetAsync(S->ctr + 1, 0, sizeof(unsigned long long) * 10, st), "memset");
    JoinArgs ja{};
    ja.s = view(rows);
    ja.ent_kmer = kmer;
    ja.kcount = cnt;
    ja.start = start;
    ja.bseq = bseq;
    ja.n_cols = n_cols;
    ja.self_pairs = self_pairs ? 1 : 0;
    ja.need = S->need;
    ja.ccount = S->ccount;
    ja.coff = S->coff;
    ja.out_pairs = pairs;
    ja.out_counts = counts;
    ja.capacity = capacity;
    ja.min_shared = min_shared;
    ja.stats = S->ctr + 4;
    ja.status = S->status;
    ja.large_rows = S->large_rows;
    ja.n_tasks = n;
    ja.range = S->range;
    ja.stash = S->stash;
    ja.stash_cap = stash_cap;
    ja.stash_off = S->stash_off;
    ja.stash_ctr = S->ctr + 10;
    const int64_t wg = warp_grid(ctx, n, 256);
    row_need_kernel<<<(unsigned)wg, 256, 0, st>>>(ja);
    CK(cudaGetLastError(), "row_need kernel");
    *launches += 1;
    unsigned long long stats[2] = {0, 0};
    CK(cudaMemcpyAsync(stats, S->ctr + 4, sizeof(stats), cudaMemcpyDeviceToHost, st), "stats D2H");
    CK(cudaStreamSynchronize(st), "stream sync");
    const uint64_t max_need = stats[0], n_large = stats[1];
    int large_blocks = 0;
    uint32_t join_gslots = 0;
    if (n_large > 0) {
        join_gslots = pow2_at_least(2 * max_need);
        const int64_t per_block = 3ll * join_gslots;   // words
        const int64_t budget = (int64_t)1 << 29;       // 2 GiB of words
        large_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(
            std::min<int64_t>((int64_t)n_large, (int64_t)ctx->sm_count * 2), budget / per_block));
        CK(grow(&S->gtab, &S->gtab_cap, (int64_t)large_blocks * per_block), "join scratch");
    }
    ja.gtab = S->gtab;
    ja.gslots = join_gslots;
    const int join_blocks = ctx->sm_count * 4;
    const int warp_blocks = ctx->sm_count * 4;
    for (int pass = 0; pass < 2; ++pass) {
        ja.ctr = S->ctr + 1 + pass;
        JoinArgs jl = ja;
        jl.ctr = S->ctr + 6 + pass;
        jl.n_tasks = (int64_t)n_large;
        JoinArgs jw = ja;
        jw.ctr = S->ctr + 8 + pass;
        if (pass == 0) {
            join_warp_kernel<false><<<warp_blocks, kWarpJoinWarps * 32, kWarpJoinSmemBytes, st>>>(jw);
            join_kernel<false, false><<<join_blocks, kSearchThreads, kJoinSmemBytes, st>>>(ja);
            if (large_blocks) join_kernel<true, false><<<large_blocks, kSearchThreads, 0, st>>>(jl);
            CK(cudaGetLastError(), "join kernel (count)");
            *launches += (large_blocks ? 3 : 2) + 3;
            int rc = device_scan<uint64_t>(ctx, S, S->ccount, n, S->coff, st);
            if (rc) return rc;
            unsigned long long stashed = 0;
            CK(cudaMemcpyAsync(&stashed, S->ctr + 10, sizeof(stashed), cudaMemcpyDeviceToHost, st), "stash D2H");
            CK(cudaStreamSynchronize(st), "stream sync");
            if ((int64_t)stashed <= stash_cap) {
                join_copy_kernel<<<(unsigned)wg, 256, 0, st>>>(ja);
                CK(cudaGetLastError(), "join copy kernel");
                *launches += 1;
                break;   // every row's list is in place: no writing pass
            }
        } else {
            join_warp_kernel<true><<<warp_blocks, kWarpJoinWarps * 32, kWarpJoinSmemBytes, st>>>(jw);
            join_kernel<false, true><<<join_blocks, kSearchThreads, kJoinSmemBytes, st>>>(ja);
            if (large_blocks) join_kernel<true, true><<<large_blocks, kSearchThreads, 0, st>>>(jl);
            CK(cudaGetLastError(), "join kernel (write)");
            *launches += large_blocks ? 3 : 2;
        }
    }
    uint64_t total = 0;
    int32_t status = 0;
    CK(cudaMemcpyAsync(&total, S->coff + n, sizeof(total), cudaMemcpyDeviceToHost, st), "count D2H");
    CK(cudaMemcpyAsync(&status, S->status, sizeof(status), cudaMemcpyDeviceToHost, st), "status D2H");
    CK(cudaStreamSynchronize(st), "stream sync");
    if (status) return fail(ctx, SWGB_EINTERNAL, "join: a hash table was smaller than its bound");
    *found = (int64_t)total;
    return SWGB_OK;
}

int check_discover_args(swgb_ctx* ctx, int k, int min_shared, int32_t* pairs, int64_t capacity,
                        int64_t* n_found) {
    if (!n_found) return fail(ctx, SWGB_EINVAL, "discover: n_found is NULL");
    *n_found = 0;
    if (k < 1 || k > 6) return fail(ctx, SWGB_EINVAL, "discover: k must be 1..6");
    if (min_shared < 1) return fail(ctx, SWGB_EINVAL, "discover: min_shared must be >= 1");
    if (capacity < 0 || (capacity > 0 && !pairs))
        return fail(ctx, SWGB_EINVAL, "discover: negative capacity or pairs is NULL");
    return SWGB_OK;
}

}  // namespace

SWGB_EXPORT int swgb_discover(swgb_ctx* ctx, const swgb_seqset* set, int k, int min_shared,
                              int32_t* pairs, int32_t* counts, int64_t capacity, int64_t* n_found,
                              void* stream) {
    if (!ctx) return SWGB_EINVAL;
    if (!set) return fail(ctx, SWGB_EINVAL, "discover: set is NULL");
    int rc = check_discover_args(ctx, k, min_shared, pairs, capacity, n_found);
    if (rc) return rc;
    if (set->device != ctx->device) return fail(ctx, SWGB_EINVAL, "discover: set on another device");
    if (set->total >= (int64_t)UINT32_MAX)
        return fail(ctx, SWGB_ETOOBIG, "discover: more than 2^32-1 residues in the set");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    ctx->last_search_launches = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (set->n < 2) return SWGB_OK;
    SearchStore* S = nullptr;
    rc = search_store(ctx, &S);
    if (rc) return rc;
    const int64_t V = kmer_space(k);
    const int64_t total = std::max<int64_t>(set->total, 1);
    CK(grow(&S->ent_kmer, &S->ent_cap, total), "discover scratch");
    CK(grow(&S->ent_pos, &S->entp_cap, total), "discover scratch");
    CK(grow(&S->bseq, &S->bseq_cap, total), "discover scratch");
    CK(grow(&S->kcount, &S->kcount_cap, set->n), "discover scratch");
    CK(grow(&S->start, &S->start_cap, V + 1), "discover scratch");
    uint32_t gslots = 0;
    rc = reserve_set_tables(ctx, S, set->max_len, &gslots);
    if (rc) return rc;
    int32_t launches = 0;
    CK(cudaMemsetAsync(S->status, 0, sizeof(int32_t), st), "memset");
    rc = build_sets(ctx, S, set, k, S->ent_kmer, S->ent_pos, S->kcount, gslots, &launches, st);
    if (!rc) rc = build_buckets(ctx, S, set, S->ent_kmer, S->kcount, V, S->start, S->bseq, &launches, st);
    if (!rc) rc = join_rows(ctx, S, set, S->ent_kmer, S->kcount, S->start, S->bseq, set->n, true,
                            min_shared, pairs, counts, capacity, n_found, &launches, st);
    ctx->last_search_launches = launches;
    return rc;
}

// ---------------------------------------------------------------------------
// Resident k-mer index of a reference set
// ---------------------------------------------------------------------------
struct swgb_index {
    swgb_ctx* ctx = nullptr;
    int device = 0;
    const swgb_seqset* refs = nullptr;
    int k = 6;
    int64_t V = 0;
    int64_t n = 0;
    uint32_t* kmer = nullptr;   // k-mer sets of the references (at their offsets)
    uint32_t* pos = nullptr;
    uint32_t* cnt = nullptr;
    uint32_t* comp = nullptr;   // [n][20] letter counts
    uint32_t* start = nullptr;  // [V + 1]
    int32_t* bseq = nullptr;
    int64_t bytes = 0;
};

SWGB_EXPORT void swgb_index_destroy(swgb_index* ix) {
    if (!ix) return;
    cudaSetDevice(ix->device);
    void* ptrs[] = {ix->kmer, ix->pos, ix->cnt, ix->comp, ix->start, ix->bseq};
    for (void* p : ptrs) cudaFree(p);
    delete ix;
}

SWGB_EXPORT int swgb_index_create(swgb_ctx* ctx, const swgb_seqset* refs, int k, void* stream,
                                  swgb_index** out) {
    if (!ctx) return SWGB_EINVAL;
    if (!refs || !out) return fail(ctx, SWGB_EINVAL, "index: refs or out is NULL");
    *out = nullptr;
    if (k < 1 || k > 6) return fail(ctx, SWGB_EINVAL, "index: k must be 1..6");
    if (refs->device != ctx->device) return fail(ctx, SWGB_EINVAL, "index: set on another device");
    if (refs->total >= (int64_t)UINT32_MAX)
        return fail(ctx, SWGB_ETOOBIG, "index: more than 2^32-1 residues in the set");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    SearchStore* S = nullptr;
    int rc = search_store(ctx, &S);
    if (rc) return rc;
    swgb_index* ix = new (std::nothrow) swgb_index();
    if (!ix) return fail(ctx, SWGB_ENOMEM, "index: host allocation");
    ix->ctx = ctx;
    ix->device = ctx->device;
    ix->refs = refs;
    ix->k = k;
    ix->V = kmer_space(k);
    ix->n = refs->n;
    const int64_t total = std::max<int64_t>(refs->total, 1), n = std::max<int64_t>(refs->n, 1);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](auto** p, int64_t count) {
        const size_t bytes = sizeof(**p) * (size_t)count;
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
        ix->bytes += (int64_t)bytes;
    };
    alloc(&ix->kmer, total);
    alloc(&ix->pos, total);
    alloc(&ix->bseq, total);
    alloc(&ix->cnt, n);
    alloc(&ix->comp, n * kStdLetters);
    alloc(&ix->start, ix->V + 1);
    if (e != cudaSuccess) {
        swgb_index_destroy(ix);
        return cuda_fail(ctx, e, "index allocation");
    }
    uint32_t gslots = 0;
    rc = reserve_set_tables(ctx, S, refs->max_len, &gslots);
    int32_t launches = 0;
    if (!rc) {
        e = cudaMemsetAsync(S->status, 0, sizeof(int32_t), st);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "memset");
    }
    if (!rc) rc = build_sets(ctx, S, refs, k, ix->kmer, ix->pos, ix->cnt, gslots, &launches, st);
    if (!rc && refs->n > 0) {
        composition_kernel<<<(unsigned)warp_grid(ctx, refs->n, 256), 256, 0, st>>>(view(refs), ix->comp);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "composition kernel");
        launches += 1;
    }
    if (!rc) rc = build_buckets(ctx, S, refs, ix->kmer, ix->cnt, ix->V, ix->start, ix->bseq, &launches, st);
    int32_t status = 0;
    if (!rc) {
        e = cudaMemcpyAsync(&status, S->status, sizeof(status), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "index build");
        else if (status) rc = fail(ctx, SWGB_EINTERNAL, "index: a k-mer table was smaller than its set");
    }
    ctx->last_search_launches = launches;
    if (rc) {
        swgb_index_destroy(ix);
        return rc;
    }
    *out = ix;
    return SWGB_OK;
}

SWGB_EXPORT int swgb_index_info(const swgb_index* ix, int64_t* n_refs, int* k, int64_t* bytes) {
    if (!ix) return SWGB_EINVAL;
    if (n_refs) *n_refs = ix->n;
    if (k) *k = ix->k;
    if (bytes) *bytes = ix->bytes;
    return SWGB_OK;
}

SWGB_EXPORT int swgb_index_query(swgb_ctx* ctx, const swgb_index* ix, const swgb_seqset* queries,
                                 int min_shared, int32_t* pairs, int32_t* counts, int64_t capacity,
                                 int64_t* n_found, void* stream) {
    if (!ctx) return SWGB_EINVAL;
    if (!ix || !queries) return fail(ctx, SWGB_EINVAL, "index_query: index or queries is NULL");
    int rc = check_discover_args(ctx, ix->k, min_shared, pairs, capacity, n_found);
    if (rc) return rc;
    if (queries->device != ctx->device || ix->device != ctx->device)
        return fail(ctx, SWGB_EINVAL, "index_query: set or index on another device");
    if (queries->total >= (int64_t)UINT32_MAX)
        return fail(ctx, SWGB_ETOOBIG, "index_query: more than 2^32-1 query residues");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    ctx->last_search_launches = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (queries->n == 0 || ix->n == 0) return SWGB_OK;
    SearchStore* S = nullptr;
    rc = search_store(ctx, &S);
    if (rc) return rc;
    const int64_t total = std::max<int64_t>(queries->total, 1);
    CK(grow(&S->ent_kmer, &S->ent_cap, total), "index_query scratch");
    CK(grow(&S->ent_pos, &S->entp_cap, total), "index_query scratch");
    CK(grow(&S->kcount, &S->kcount_cap, queries->n), "index_query scratch");
    uint32_t gslots = 0;
    rc = reserve_set_tables(ctx, S, queries->max_len, &gslots);
    if (rc) return rc;
    int32_t launches = 0;
    CK(cudaMemsetAsync(S->status, 0, sizeof(int32_t), st), "memset");
    rc = build_sets(ctx, S, queries, ix->k, S->ent_kmer, S->ent_pos, S->kcount, gslots, &launches, st);
    if (!rc) rc = join_rows(ctx, S, queries, S->ent_kmer, S->kcount, ix->start, ix->bseq, ix->n, false,
                            min_shared, pairs, counts, capacity, n_found, &launches, st);
    ctx->last_search_launches = launches;
    return rc;
}

SWGB_EXPORT int swgb_search_launches(const swgb_ctx* ctx) {
    return ctx ? ctx->last_search_launches : -1;
}

SWGB_EXPORT int swgb_identity(swgb_ctx* ctx, const swgb_seqset* queries, const swgb_seqset* refs,
                              const int32_t* pairs, const swgb_record* records, int64_t n_pairs,
                              const swgb_params* params, const swgb_thresholds* th,
                              swgb_identity_record* out, void* stream) {
    if (!ctx) return SWGB_EINVAL;
    if (!queries || !refs || !params || !params->matrix || !th)
        return fail(ctx, SWGB_EINVAL, "identity: NULL argument");
    if (n_pairs < 0) return fail(ctx, SWGB_EINVAL, "identity: negative pair count");
    if (n_pairs > 0 && (!pairs || !records || !out))
        return fail(ctx, SWGB_EINVAL, "identity: NULL buffer");
    if (params->gap_open < 0 || params->gap_extend < 1)
        return fail(ctx, SWGB_EINVAL, "gap_open must be >= 0 and gap_extend >= 1");
    if (th->id_num < 0 || th->id_den < 1 || th->cov_num < 0 || th->cov_den < 1)
        return fail(ctx, SWGB_EINVAL, "identity: thresholds need num >= 0, den >= 1");
    if (queries->device != ctx->device || refs->device != ctx->device)
        return fail(ctx, SWGB_EINVAL, "identity: set on another device");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    ctx->last_search_launches = 0;
    if (n_pairs == 0) return SWGB_OK;
    cudaStream_t st = (cudaStream_t)stream;
    SearchStore* S = nullptr;
    int rc = search_store(ctx, &S);
    if (rc) return rc;
    IdentArgs a{};
    a.q = view(queries);
    a.r = view(refs);
    a.pairs = pairs;
    a.rec = records;
    a.n_pairs = n_pairs;
    std::memcpy(a.mat, params->matrix, sizeof(a.mat));
    a.go = params->gap_open;
    a.ge = params->gap_extend;
    a.id_num = th->id_num;
    a.id_den = th->id_den;
    a.cov_num = th->cov_num;
    a.cov_den = th->cov_den;
    a.out = reinterpret_cast<int32_t*>(out);
    a.status = S->status;
    // A batch that leaves warps idle (serving batches of a few thousand
    // pairs) is bound by its longest spans, each walked by one warp: there
    // spans of 4+ chunks go cooperative, on up to 4 blocks per SM.  A large
    // batch fills the SMs anyway and keeps the cooperative launch for the
    // longest spans, beside the regular ones.
    const bool small_batch = n_pairs <= (int64_t)ctx->sm_count * kIdSmallBatchPerSM;
    a.coop_cols = small_batch ? kIdCoopColsSmall : kIdCoopCols;
    const int coop_blocks_per_sm = small_batch ? 4 : 2;
    // one boundary column per resident warp of the large classes (rows of the
    // longest query + 1)
    const int64_t max_rows = queries->max_len + 1;
    a.bnd_stride = max_rows;
    CK(grow(&S->lists, &S->lists_cap, n_pairs), "identity scratch");
    a.lists = S->lists;
    a.hist = S->id_hist;
    a.ctr = S->ctr;
    CK(cudaMemsetAsync(S->ctr, 0, sizeof(unsigned long long) * 8, st), "memset");
    CK(cudaMemsetAsync(S->id_hist, 0, sizeof(uint32_t) * kIdLists * kIdBuckets, st), "memset");
    CK(cudaMemsetAsync(S->status, 0, sizeof(int32_t), st), "memset");
    // the lists, each longest span first: count, scan, place
    const int64_t g = std::min<int64_t>((n_pairs + 255) / 256, (int64_t)ctx->sm_count * 16);
    ident_classify_kernel<<<(unsigned)g, 256, 0, st>>>(a);
    CK(cudaGetLastError(), "ident_classify kernel");
    ident_scan_kernel<<<1, 256, 0, st>>>(a);
    CK(cudaGetLastError(), "ident_scan kernel");
    ident_place_kernel<<<(unsigned)g, 256, 0, st>>>(a);
    CK(cudaGetLastError(), "ident_place kernel");
    unsigned long long cnt[kIdLists] = {0, 0, 0, 0, 0, 0};   // list sizes (long spans of 2, 3 apart)
    static_assert(kIdLists == 6, "four classes and two cooperative lists");
    CK(cudaMemcpyAsync(cnt, S->ctr + 1, sizeof(cnt), cudaMemcpyDeviceToHost, st), "sizes D2H");
    CK(cudaStreamSynchronize(st), "stream sync");
    int64_t list_base[kIdLists];
    int64_t listed = 0;
    for (int l = 0; l < kIdLists; ++l) {
        list_base[l] = listed;
        listed += (int64_t)cnt[l];
    }
    int32_t launches = 3;
    const int64_t resident_blocks = (int64_t)ctx->sm_count * 8;
    // classes 2 and 3 split: spans of >= coop_cols columns go to the
    // cooperative launches, the rest to the regular ones
    const int64_t coop_n[2] = {(int64_t)cnt[4], (int64_t)cnt[5]};
    const int64_t reg_n[kIdClasses] = {(int64_t)cnt[0], (int64_t)cnt[1], (int64_t)cnt[2], (int64_t)cnt[3]};
    const int pairs_per_warp[kIdClasses] = {4, 2, 1, 1};
    int blocks_of[kIdClasses] = {0, 0, 0, 0};
    int64_t bnd_warps = 0;
    for (int cls = 0; cls < kIdClasses; ++cls) {
        const int64_t tasks = (reg_n[cls] + pairs_per_warp[cls] - 1) / pairs_per_warp[cls];
        blocks_of[cls] = (int)std::min<int64_t>((tasks + kIdWarps - 1) / kIdWarps, resident_blocks);
        // every warp of a chunked (32-lane) launch owns a boundary column
        if (cls >= 2) bnd_warps = std::max<int64_t>(bnd_warps, (int64_t)blocks_of[cls] * kIdWarps);
    }
    int coop_blocks[2] = {0, 0};
    for (int k = 0; k < 2; ++k)
        coop_blocks[k] = (int)std::min<int64_t>(coop_n[k], (int64_t)ctx->sm_count * coop_blocks_per_sm);
    const int64_t coop_warps = (int64_t)std::max(coop_blocks[0], coop_blocks[1]) * kIdWarps;
    if (bnd_warps + coop_warps > 0)
        CK(grow(&S->bnd, &S->bnd_cap, (bnd_warps + coop_warps) * max_rows), "identity scratch");
    a.bnd = S->bnd;
    // The regular chunked classes (2, then 3: they share their boundary
    // columns) run on the caller's stream; the cooperative launches (the
    // longest spans, their own boundary region) on the stream of the
    // greatest priority, so that their blocks are resident from the start
    // (the regular launches are persistent and would otherwise hold every
    // SM's registers until their lists run out), and the short-span classes
    // (0, 1) on a side stream, all at once, so that the short spans fill the
    // SMs the long spans' tail leaves idle.  Each launch has its own work
    // counter.
    CK(cudaMemsetAsync(S->ctr + 8, 0, sizeof(unsigned long long) * 8, st), "memset");
    CK(cudaEventRecord(ctx->fork_ev, st), "event record");
    cudaStream_t side = ctx->side[0], side_coop = ctx->first;
    CK(cudaStreamWaitEvent(side, ctx->fork_ev, 0), "stream wait");
    CK(cudaStreamWaitEvent(side_coop, ctx->fork_ev, 0), "stream wait");
    for (int k = 0; k < 2; ++k) {
        if (coop_n[k] == 0) continue;
        IdentArgs b = a;
        b.list = S->lists + list_base[kIdClasses + k];
        b.n_list = coop_n[k];
        // the cooperative region starts after bnd_warps x max_rows 24-byte
        // entries: 16-byte aligned (its rows are 16-byte vectors) because
        // bnd_warps is a multiple of the (even) warps per block
        static_assert(kIdWarps % 2 == 0 && sizeof(IdBnd) == 24, "cooperative boundary region alignment");
        b.bnd = S->bnd + bnd_warps * max_rows;
        b.ctr = S->ctr + 12 + k;
        if (k == 0) ident_kernel<32, uint32_t, true, true, true><<<coop_blocks[k], kIdWarps * 32, 0, side_coop>>>(b);
        else ident_kernel<32, uint64_t, true, true, true><<<coop_blocks[k], kIdWarps * 32, 0, side_coop>>>(b);
        CK(cudaGetLastError(), "ident kernel (cooperative)");
        launches += 1;
    }
    const int order[kIdClasses] = {2, 3, 0, 1};
    for (int k = 0; k < kIdClasses; ++k) {
        const int cls = order[k];
        if (reg_n[cls] == 0) continue;
        IdentArgs b = a;
        b.list = S->lists + list_base[cls];
        b.n_list = reg_n[cls];
        b.ctr = S->ctr + 8 + cls;
        const int blocks = blocks_of[cls];
        cudaStream_t s = cls >= 2 ? st : side;
        if (small_batch) {
            if (cls == 0) ident_kernel<8, uint32_t, false, false, true><<<blocks, kIdWarps * 32, 0, s>>>(b);
            else if (cls == 1) ident_kernel<16, uint32_t, true, false, true><<<blocks, kIdWarps * 32, 0, s>>>(b);
            else if (cls == 2) ident_kernel<32, uint32_t, true, false, true><<<blocks, kIdWarps * 32, 0, s>>>(b);
            else ident_kernel<32, uint64_t, true, false, true><<<blocks, kIdWarps * 32, 0, s>>>(b);
        } else {
            if (cls == 0) ident_kernel<8, uint32_t, false, false, false><<<blocks, kIdWarps * 32, 0, s>>>(b);
            else if (cls == 1) ident_kernel<16, uint32_t, true, false, false><<<blocks, kIdWarps * 32, 0, s>>>(b);
            else if (cls == 2) ident_kernel<32, uint32_t, true, false, false><<<blocks, kIdWarps * 32, 0, s>>>(b);
            else ident_kernel<32, uint64_t, true, false, false><<<blocks, kIdWarps * 32, 0, s>>>(b);
        }
        CK(cudaGetLastError(), "ident kernel");
        launches += 1;
    }
    CK(cudaEventRecord(ctx->join_ev[1], side_coop), "event record");
    CK(cudaStreamWaitEvent(st, ctx->join_ev[1], 0), "stream wait");
    CK(cudaEventRecord(ctx->join_ev[0], side), "event record");
    CK(cudaStreamWaitEvent(st, ctx->join_ev[0], 0), "stream wait");
    int32_t status = 0;
    CK(cudaMemcpyAsync(&status, S->status, sizeof(status), cudaMemcpyDeviceToHost, st), "status D2H");
    CK(cudaStreamSynchronize(st), "stream sync");
    ctx->last_search_launches = launches;
    if (status == 3) return fail(ctx, SWGB_ERANGE, "identity: a pair index or record outside its sequences");
    if (status == 4) return fail(ctx, SWGB_EINTERNAL, "identity: a chunk waited too long for the previous one");
    if (status == 5) return fail(ctx, SWGB_EINTERNAL, "identity: a work list overflowed");
    if (status) return fail(ctx, SWGB_EINTERNAL, "identity: a span's global optimum differs from its record's score");
    return SWGB_OK;
}

namespace {

// Features of pairs (i of A, j of B) from both sets' k-mer tables; the tables
// of B come from the caller (another set's, or an index's).
int run_features(swgb_ctx* ctx, SearchStore* S, const swgb_seqset* set_a, const swgb_seqset* set_b,
                 const uint32_t* kmB, const uint32_t* posB, const uint32_t* cntB,
                 const uint32_t* compB, bool b_is_a, int k, const int32_t* pairs, int64_t n_pairs,
                 float* out, int32_t* launches, cudaStream_t st) {
    // global hash tables: the k-mer sets of A (and B) and the feature
    // kernel's table of K(i), reserved before any launch
    const int blocks = ctx->sm_count * 3;
    const int64_t longest = std::max<int64_t>(set_a->max_len, b_is_a ? 0 : set_b->max_len);
    uint32_t gslots = 0;
    int rc = reserve_set_tables(ctx, S, longest, &gslots);
    if (rc) return rc;
    // per-warp global tables of rows above the shared-memory class
    const uint32_t fslots = pow2_at_least((uint64_t)std::max<int64_t>(set_a->max_len, 1) * 2);
    if (fslots > (uint32_t)kFeatWarpSlots)
        CK(grow(&S->gtab, &S->gtab_cap,
                std::max<int64_t>((int64_t)blocks * kFeatWarps * 2 * fslots,
                                  (int64_t)ctx->sm_count * 4 * 2 * gslots)), "features scratch");
    const int64_t total = std::max<int64_t>(set_a->total, 1), n = std::max<int64_t>(set_a->n, 1);
    CK(grow(&S->ent_kmer, &S->ent_cap, total), "features scratch");
    CK(grow(&S->ent_pos, &S->entp_cap, total), "features scratch");
    CK(grow(&S->kcount, &S->kcount_cap, n), "features scratch");
    CK(grow(&S->comp, &S->comp_cap, n * kStdLetters), "features scratch");
    CK(cudaMemsetAsync(S->status, 0, sizeof(int32_t), st), "memset");
    rc = build_sets(ctx, S, set_a, k, S->ent_kmer, S->ent_pos, S->kcount, gslots, launches, st);
    if (rc) return rc;
    if (set_a->n > 0) {
        composition_kernel<<<(unsigned)warp_grid(ctx, set_a->n, 256), 256, 0, st>>>(view(set_a), S->comp);
        CK(cudaGetLastError(), "composition kernel");
        *launches += 1;
    }
    if (b_is_a) {
        kmB = S->ent_kmer;
        posB = S->ent_pos;
        cntB = S->kcount;
        compB = S->comp;
    } else if (!kmB) {
        const int64_t tb = std::max<int64_t>(set_b->total, 1), nb = std::max<int64_t>(set_b->n, 1);
        CK(grow(&S->ent2_kmer, &S->ent2_cap, tb), "features scratch");
        CK(grow(&S->ent2_pos, &S->ent2p_cap, tb), "features scratch");
        CK(grow(&S->kcount2, &S->kcount2_cap, nb), "features scratch");
        CK(grow(&S->comp2, &S->comp2_cap, nb * kStdLetters), "features scratch");
        rc = build_sets(ctx, S, set_b, k, S->ent2_kmer, S->ent2_pos, S->kcount2, gslots, launches, st);
        if (rc) return rc;
        if (set_b->n > 0) {
            composition_kernel<<<(unsigned)warp_grid(ctx, set_b->n, 256), 256, 0, st>>>(view(set_b), S->comp2);
            CK(cudaGetLastError(), "composition kernel");
            *launches += 1;
        }
        kmB = S->ent2_kmer;
        posB = S->ent2_pos;
        cntB = S->kcount2;
        compB = S->comp2;
    }
    CK(cudaMemsetAsync(S->ctr + 1, 0, sizeof(unsigned long long), st), "memset");
    FeatArgs fa{view(set_a), view(set_b), k, S->ent_kmer, S->ent_pos, S->kcount, kmB, posB, cntB,
                S->comp, compB, pairs, n_pairs, out,
                fslots > (uint32_t)kFeatWarpSlots ? S->gtab : nullptr, fslots, S->ctr + 1, S->status};
    features_kernel<<<blocks, kFeatWarps * 32, kFeatSmemBytes, st>>>(fa);
    CK(cudaGetLastError(), "features kernel");
    *launches += 1;
    int32_t status = 0;
    CK(cudaMemcpyAsync(&status, S->status, sizeof(status), cudaMemcpyDeviceToHost, st), "status D2H");
    CK(cudaStreamSynchronize(st), "stream sync");
    if (status == 3) return fail(ctx, SWGB_ERANGE, "features: a pair index outside its set");
    if (status) return fail(ctx, SWGB_EINTERNAL, "features: a k-mer table was smaller than its set");
    return SWGB_OK;
}

}  // namespace

SWGB_EXPORT int swgb_pair_features(swgb_ctx* ctx, const swgb_seqset* set_a, const swgb_seqset* set_b,
                                   const int32_t* pairs, int64_t n_pairs, int k, float* out,
                                   void* stream) {
    if (!ctx) return SWGB_EINVAL;
    if (!set_a || !set_b) return fail(ctx, SWGB_EINVAL, "features: set is NULL");
    if (k < 1 || k > 6) return fail(ctx, SWGB_EINVAL, "features: k must be 1..6");
    if (n_pairs < 0 || (n_pairs > 0 && (!pairs || !out)))
        return fail(ctx, SWGB_EINVAL, "features: negative count or NULL buffer");
    if (set_a->device != ctx->device || set_b->device != ctx->device)
        return fail(ctx, SWGB_EINVAL, "features: set on another device");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    ctx->last_search_launches = 0;
    if (n_pairs == 0) return SWGB_OK;
    SearchStore* S = nullptr;
    int rc = search_store(ctx, &S);
    if (rc) return rc;
    int32_t launches = 0;
    rc = run_features(ctx, S, set_a, set_b, nullptr, nullptr, nullptr, nullptr, set_b == set_a, k,
                      pairs, n_pairs, out, &launches, (cudaStream_t)stream);
    ctx->last_search_launches = launches;
    return rc;
}

SWGB_EXPORT int swgb_index_features(swgb_ctx* ctx, const swgb_index* ix, const swgb_seqset* queries,
                                    const int32_t* pairs, int64_t n_pairs, float* out, void* stream) {
    if (!ctx) return SWGB_EINVAL;
    if (!ix || !queries) return fail(ctx, SWGB_EINVAL, "index_features: index or queries is NULL");
    if (n_pairs < 0 || (n_pairs > 0 && (!pairs || !out)))
        return fail(ctx, SWGB_EINVAL, "index_features: negative count or NULL buffer");
    if (queries->device != ctx->device || ix->device != ctx->device)
        return fail(ctx, SWGB_EINVAL, "index_features: set or index on another device");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    ctx->last_search_launches = 0;
    if (n_pairs == 0) return SWGB_OK;
    SearchStore* S = nullptr;
    int rc = search_store(ctx, &S);
    if (rc) return rc;
    int32_t launches = 0;
    rc = run_features(ctx, S, queries, ix->refs, ix->kmer, ix->pos, ix->cnt, ix->comp, false, ix->k,
                      pairs, n_pairs, out, &launches, (cudaStream_t)stream);
    ctx->last_search_launches = launches;
    return rc;
}

SWGB_EXPORT int swgb_select_pairs(swgb_ctx* ctx, const int32_t* pairs, const float* logits,
                                  int64_t n_pairs, float threshold, int32_t* kept,
                                  int64_t* kept_index, int64_t* n_kept, void* stream) {
    if (!ctx) return SWGB_EINVAL;
    if (!n_kept) return fail(ctx, SWGB_EINVAL, "select: n_kept is NULL");
    *n_kept = 0;
    if (n_pairs < 0 || (n_pairs > 0 && (!pairs || !logits || !kept)))
        return fail(ctx, SWGB_EINVAL, "select: negative count or NULL buffer");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    ctx->last_search_launches = 0;
    if (n_pairs == 0) return SWGB_OK;
    cudaStream_t st = (cudaStream_t)stream;
    SearchStore* S = nullptr;
    int rc = search_store(ctx, &S);
    if (rc) return rc;
    CK(grow(&S->flags, &S->flags_cap, n_pairs), "select scratch");
    CK(grow(&S->coff, &S->coff_cap, n_pairs + 1), "select scratch");
    const int64_t g = std::min<int64_t>((n_pairs + 255) / 256, (int64_t)ctx->sm_count * 16);
    select_flags_kernel<<<(unsigned)g, 256, 0, st>>>(logits, n_pairs, threshold, S->flags);
    CK(cudaGetLastError(), "select kernel");
    rc = device_scan<uint64_t>(ctx, S, S->flags, n_pairs, S->coff, st);
    if (rc) return rc;
    select_scatter_kernel<<<(unsigned)g, 256, 0, st>>>(pairs, S->flags, S->coff, n_pairs, kept,
                                                       kept_index);
    CK(cudaGetLastError(), "select kernel");
    uint64_t found = 0;
    CK(cudaMemcpyAsync(&found, S->coff + n_pairs, sizeof(found), cudaMemcpyDeviceToHost, st), "count D2H");
    CK(cudaStreamSynchronize(st), "stream sync");
    ctx->last_search_launches = 5;
    *n_kept = (int64_t)found;
    return SWGB_OK;
}
