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
// the global affine alignment of a record's span is filled by a warp
// wavefront that stores four decision bits per cell, then traced back from
// the span's end under a fixed preference -- diagonal, then a gap in the
// reference (query residue against a gap), then a gap in the query; inside a
// gap its opening before its extension -- counting identical columns.
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

__global__ void kmer_scatter_kernel(SeqView s, const uint32_t* __restrict__ ent_kmer,
                                    const uint32_t* __restrict__ ent_pos,
                                    const uint32_t* __restrict__ kcount,
                                    const uint32_t* __restrict__ start, uint32_t* fill,
                                    int32_t* bseq, uint32_t* bpos) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < s.n; i += warps) {
        const int64_t o = s.off[i];
        const uint32_t c = kcount[i];
        for (uint32_t e = lane; e < c; e += 32) {
            const uint32_t x = ent_kmer[o + e];
            const uint32_t slot = start[x] + atomicAdd(&fill[x], 1u);
            bseq[slot] = (int32_t)i;
            bpos[slot] = ent_pos[o + e];
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
    SeqView s;
    const uint32_t* ent_kmer;
    const uint32_t* kcount;
    const uint32_t* start;     // bucket starts [V + 1]
    const int32_t* bseq;
    uint32_t* need;            // [n] min(incidences with j > i, n - 1 - i)
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
            for (uint32_t b = a.start[x]; b < a.start[x + 1]; ++b) inc += a.bseq[b] > i;
        }
        for (int d = 16; d; d >>= 1) inc += __shfl_xor_sync(0xffffffffu, inc, d);
        if (lane == 0) {
            const uint64_t lim = (uint64_t)(n - 1 - i);
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
    const int64_t n = a.s.n;
    for (;;) {
        int64_t i = next_task(a.ctr, &s_task);
        if (i >= (LARGE ? a.n_tasks : n)) break;
        if (LARGE) i = a.large_rows[i];
        const uint32_t need = a.need[i];
        const bool large = 2ull * need > (unsigned long long)kJoinSmemSlots;
        if (need == 0 || large != LARGE) {
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
            const uint32_t x = a.ent_kmer[o + e];
            const uint32_t b1 = a.start[x + 1];
            for (uint32_t b = a.start[x]; b < b1; ++b) {
                const int32_t j = a.bseq[b];
                if (j <= i) continue;
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
                if (WRITE) list[e] = ((uint64_t)j << 32) | cnts[t];
            }
        }
        __syncthreads();
        const uint32_t m = s_n;
        if (!WRITE) {
            if (threadIdx.x == 0) a.ccount[i] = m;
            continue;
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

// ---------------------------------------------------------------------------
// Identity of alignment records
// ---------------------------------------------------------------------------
// Decision bits of one cell (a, b) of the span's global DP, 4 per cell:
//   bits 0-1: source of H -- 0 diagonal, 1 F (query residue against a gap),
//             2 E (gap against a reference residue), by the preference order;
//   bit 2:    F(a, b) opens its gap (F = H(a-1, b) - o - e);
//   bit 3:    E(a, b) opens its gap (E = H(a, b-1) - o - e).
// Layout per pair: rows a = 1..n of words; a row holds nch * 32 words, lane k
// of chunk c writing word c * 32 + k for columns c*256 + k*8 + 1 .. +8.
constexpr int kIdR = 8;                        // columns per lane
constexpr int kIdChunk = 32 * kIdR;            // columns per chunk
constexpr int kIdWarps = 4;                    // warps per block
constexpr int32_t kNegInf = -(1 << 28);

struct IdentArgs {
    SeqView q, r;
    const int32_t* pairs;
    const swgb_record* rec;
    int64_t n_pairs;
    int8_t mat[kAlpha * kAlpha];
    int32_t go, ge;
    int32_t id_num, id_den, cov_num, cov_den;
    int32_t* out;              // [n_pairs][3]: matches, columns, pass
    uint32_t* dir;             // per-warp regions of region_words words
    int64_t region_words;
    int64_t min_words, max_words;   // this launch takes pairs with min < need <= max
    int2* bnd;                 // per-warp chunk-boundary rows, bnd_stride entries each
    int64_t bnd_stride;
    unsigned long long* ctr;
    unsigned long long* stats; // [0] max need (words), [1] pairs above the small class
    int32_t* status;
    int64_t* large;            // [n_pairs] the pairs above the small class
    int64_t n_tasks;           // large launch: tasks are large[0, n_tasks); else all pairs
};

// words of decision bits of a record's span (0 when there is nothing to trace)
__device__ __forceinline__ int64_t ident_need(const swgb_record& rc) {
    if (rc.score <= 0) return 0;
    const int64_t n = (int64_t)rc.q_end - rc.q_start + 1, m = (int64_t)rc.r_end - rc.r_start + 1;
    if (n <= 0 || m <= 0) return 0;
    return n * ((m + kIdChunk - 1) / kIdChunk) * 32;
}

// Largest need, and the pairs above the small class appended to a.large
// (their count in stats[1]).
__global__ void ident_need_kernel(IdentArgs a, int64_t small_words) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n_pairs; p += stride) {
        const int64_t w = ident_need(a.rec[p]);
        if (w > 0) {
            atomicMax(&a.stats[0], (unsigned long long)w);
            if (w > small_words) a.large[atomicAdd(&a.stats[1], 1ull)] = p;
        }
    }
}

__global__ void __launch_bounds__(kIdWarps * 32) ident_kernel(IdentArgs a) {
    __shared__ int8_t s_mat[kAlpha * kAlpha];
    for (int t = threadIdx.x; t < kAlpha * kAlpha; t += blockDim.x) s_mat[t] = a.mat[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * kIdWarps + (threadIdx.x >> 5);
    uint32_t* dir = a.dir + gw * a.region_words;
    int2* bnd = a.bnd + gw * a.bnd_stride;
    const int32_t go = a.go, ge = a.ge, oe = go + ge;
    for (;;) {
        int64_t p = 0;
        if (lane == 0) p = (int64_t)atomicAdd(a.ctr, 1ull);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= a.n_tasks) break;
        if (a.min_words > 0) p = a.large[p];
        const swgb_record rc = a.rec[p];
        const int64_t need = ident_need(rc);
        const bool mine = need > a.min_words && need <= a.max_words;
        if (need == 0) {
            // nothing to trace: the smallest class writes the zero result
            if (a.min_words == 0 && lane == 0) {
                a.out[3 * p] = 0;
                a.out[3 * p + 1] = 0;
                a.out[3 * p + 2] = 0;
            }
            continue;
        }
        if (!mine) continue;
        const int32_t qi = a.pairs[2 * p], ri = a.pairs[2 * p + 1];
        // a record must lie inside its pair's sequences
        const bool ok_idx = qi >= 0 && qi < a.q.n && ri >= 0 && ri < a.r.n;
        const int lq = ok_idx ? (int)(a.q.off[qi + 1] - a.q.off[qi]) : 0;
        const int lr = ok_idx ? (int)(a.r.off[ri + 1] - a.r.off[ri]) : 0;
        if (!ok_idx || rc.q_start < 0 || rc.q_end >= lq || rc.r_start < 0 || rc.r_end >= lr) {
            if (lane == 0) {
                atomicMax(a.status, 3);
                a.out[3 * p] = -1;
                a.out[3 * p + 1] = -1;
                a.out[3 * p + 2] = 0;
            }
            continue;
        }
        const uint8_t* qs = a.q.res + a.q.off[qi] + rc.q_start;
        const uint8_t* rs = a.r.res + a.r.off[ri] + rc.r_start;
        const int n = rc.q_end - rc.q_start + 1, m = rc.r_end - rc.r_start + 1;
        const int nch = (m + kIdChunk - 1) / kIdChunk;
        const int64_t row_words = (int64_t)nch * 32;
        int32_t hnm = kNegInf;   // H(n, m), held by the lane owning column m
        for (int c = 0; c < nch; ++c) {
            // this lane's columns b = c0 + 1 .. c0 + kIdR (1-based)
            const int c0 = c * kIdChunk + lane * kIdR;
            int rcode[kIdR];
            int32_t H[kIdR], F[kIdR];
#pragma unroll
            for (int x = 0; x < kIdR; ++x) {
                const int b = c0 + x + 1;
                rcode[x] = b <= m ? rs[b - 1] : 0;
                H[x] = -(oe + ge * (b - 1));     // H(0, b)
                F[x] = kNegInf;                  // F(0, b)
            }
            // This lane's outputs of the previous step (its last column's H and
            // E), before its first row: H(0, c0 + kIdR), the diagonal of lane
            // k+1's first row.
            int32_t h_out = -(oe + ge * (c0 + kIdR - 1)), e_out = kNegInf;
            // lanes > 0: what lane-1 sent one step ago (the next diagonal);
            // lane 0: H(a - 1, c * kIdChunk), from the border or the boundary row
            int32_t hd_next = c0 == 0 ? 0 : -(oe + ge * (c0 - 1));
            for (int t = 0; t < n + 31; ++t) {
                const int arow = t - lane + 1;   // row of this lane at step t
                // lane-1's last column of its row at step t-1, which is row arow
                const int32_t up_h = __shfl_up_sync(0xffffffffu, h_out, 1);
                const int32_t up_e = __shfl_up_sync(0xffffffffu, e_out, 1);
                int32_t hl = up_h, el = up_e;
                const int32_t hd = hd_next;
                if (lane == 0) {
                    if (c == 0) {
                        hl = -(oe + ge * (arow - 1));   // H(a, 0)
                        el = kNegInf;                   // E(a, 0)
                    } else if (arow >= 1 && arow <= n) {
                        const int2 v = bnd[arow];
                        hl = v.x;
                        el = v.y;
                    }
                }
                if (arow >= 1 && arow <= n) {
                    const int qc = qs[arow - 1];
                    const int8_t* srow = s_mat + qc * kAlpha;
                    uint32_t word = 0;
                    int32_t hleft = hl, eleft = el, hdiag = hd;
#pragma unroll
                    for (int x = 0; x < kIdR; ++x) {
                        const int32_t eo_v = hleft - oe, ee_v = eleft - ge;
                        const int32_t e = max(eo_v, ee_v);
                        const uint32_t eopen = eo_v >= ee_v;
                        const int32_t fo_v = H[x] - oe, fe_v = F[x] - ge;
                        const int32_t f = max(fo_v, fe_v);
                        const uint32_t fopen = fo_v >= fe_v;
                        const int32_t d = hdiag + srow[rcode[x]];
                        const int32_t h = max(d, max(e, f));
                        const uint32_t src = h == d ? 0u : (h == f ? 1u : 2u);
                        word |= (src | (fopen << 2) | (eopen << 3)) << (4 * x);
                        hdiag = H[x];
                        H[x] = h;
                        F[x] = f;
                        hleft = h;
                        eleft = e;
                    }
                    dir[(int64_t)(arow - 1) * row_words + c * 32 + lane] = word;
                    h_out = hleft;
                    e_out = eleft;
                    if (lane == 31 && c + 1 < nch) bnd[arow] = make_int2(hleft, eleft);
                    if (arow == n && m > c0 && m <= c0 + kIdR) {
#pragma unroll
                        for (int x = 0; x < kIdR; ++x)
                            if (c0 + x + 1 == m) hnm = H[x];
                    }
                }
                // the next row's diagonal: lane-1's value received now (row
                // arow), or for lane 0 this row's left input
                hd_next = lane == 0 ? hl : up_h;
            }
            // chunk c's boundary row must be complete before chunk c + 1 reads it
            __syncwarp();
        }
        // H(n, m) must equal the record's score
        const int32_t hv = __reduce_max_sync(0xffffffffu, hnm);
        if (hv != rc.score) {
            if (lane == 0) {
                atomicMax(a.status, 2);
                a.out[3 * p] = -1;
                a.out[3 * p + 1] = -1;
                a.out[3 * p + 2] = 0;
            }
            continue;
        }
        __syncwarp();
        if (lane == 0) {
            int ai = n, bi = m, state = 0;
            int32_t mt = 0, cols = 0;
            for (int guard = 0; guard < 2 * (n + m) + 2 && (ai > 0 || bi > 0); ++guard) {
                if (ai == 0) { cols += bi; bi = 0; break; }
                if (bi == 0) { cols += ai; ai = 0; break; }
                const uint32_t w = dir[(int64_t)(ai - 1) * row_words + (bi - 1) / kIdR];
                const uint32_t bits = (w >> (4 * ((bi - 1) % kIdR))) & 15u;
                if (state == 0) {
                    const uint32_t src = bits & 3u;
                    if (src == 0) {
                        mt += qs[ai - 1] == rs[bi - 1];
                        ++cols;
                        --ai;
                        --bi;
                    } else {
                        state = src == 1 ? 1 : 2;
                    }
                } else if (state == 1) {
                    ++cols;
                    state = (bits & 4u) ? 0 : 1;
                    --ai;
                } else {
                    ++cols;
                    state = (bits & 8u) ? 0 : 2;
                    --bi;
                }
            }
            const int64_t sq = n, sr = m;
            const bool pass = cols > 0 && (int64_t)mt * a.id_den >= (int64_t)a.id_num * cols &&
                              sq * a.cov_den >= (int64_t)a.cov_num * lq &&
                              sr * a.cov_den >= (int64_t)a.cov_num * lr;
            a.out[3 * p] = mt;
            a.out[3 * p + 1] = cols;
            a.out[3 * p + 2] = pass ? 1 : 0;
        }
        __syncwarp();
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
    uint32_t* bpos = nullptr;     int64_t bpos_cap = 0;
    uint32_t* need = nullptr;     int64_t need_cap = 0;
    uint32_t* ccount = nullptr;   int64_t ccount_cap = 0;
    uint64_t* coff = nullptr;     int64_t coff_cap = 0;
    uint64_t* part = nullptr;     int64_t part_cap = 0;
    uint32_t* gtab = nullptr;     int64_t gtab_cap = 0;
    uint32_t* dir = nullptr;      int64_t dir_cap = 0;
    int2* bnd = nullptr;          int64_t bnd_cap = 0;
    int64_t* large = nullptr;     int64_t large_cap = 0;
    int32_t* large_rows = nullptr; int64_t large_rows_cap = 0;
    unsigned long long* ctr = nullptr;   // [8] work counters and statistics
    int32_t* status = nullptr;
};

void search_store_free(SearchStore* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    void* ptrs[] = {s->ent_kmer, s->ent_pos, s->kcount, s->hist, s->start, s->bseq, s->bpos,
                    s->need, s->ccount, s->coff, s->part, s->gtab, s->dir, s->bnd, s->ctr,
                    s->status, s->large, s->large_rows};
    for (void* p : ptrs) cudaFree(p);
    delete s;
}

namespace {

int search_store(swgb_ctx* ctx, SearchStore** out) {
    if (!ctx->search) {
        SearchStore* s = new (std::nothrow) SearchStore();
        if (!s) return fail(ctx, SWGB_ENOMEM, "search scratch: host allocation");
        s->device = ctx->device;
        cudaError_t e = cudaMalloc(&s->ctr, sizeof(unsigned long long) * 8);
        if (e == cudaSuccess) e = cudaMalloc(&s->status, sizeof(int32_t));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(join_kernel<false, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kJoinSmemBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(join_kernel<false, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kJoinSmemBytes);
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

SWGB_EXPORT int swgb_discover(swgb_ctx* ctx, const swgb_seqset* set, int k, int min_shared,
                              int32_t* pairs, int32_t* counts, int64_t capacity, int64_t* n_found,
                              void* stream) {
    if (!ctx) return SWGB_EINVAL;
    if (!set || !n_found) return fail(ctx, SWGB_EINVAL, "discover: set or n_found is NULL");
    *n_found = 0;
    if (k < 1 || k > 6) return fail(ctx, SWGB_EINVAL, "discover: k must be 1..6");
    if (min_shared < 1) return fail(ctx, SWGB_EINVAL, "discover: min_shared must be >= 1");
    if (capacity < 0 || (capacity > 0 && !pairs))
        return fail(ctx, SWGB_EINVAL, "discover: negative capacity or pairs is NULL");
    if (set->device != ctx->device) return fail(ctx, SWGB_EINVAL, "discover: set on another device");
    if (set->total >= (int64_t)UINT32_MAX)
        return fail(ctx, SWGB_ETOOBIG, "discover: more than 2^32-1 residues in the set");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = set->n;
    if (n < 2) return SWGB_OK;
    SearchStore* S = nullptr;
    int rc = search_store(ctx, &S);
    if (rc) return rc;
    int64_t V = 1;
    for (int t = 0; t < k; ++t) V *= kStdLetters;
    const int64_t total = std::max<int64_t>(set->total, 1);
    CK(grow(&S->ent_kmer, &S->ent_cap, total), "discover scratch");
    CK(grow(&S->ent_pos, &S->entp_cap, total), "discover scratch");
    CK(grow(&S->bseq, &S->bseq_cap, total), "discover scratch");
    CK(grow(&S->bpos, &S->bpos_cap, total), "discover scratch");
    CK(grow(&S->kcount, &S->kcount_cap, n), "discover scratch");
    CK(grow(&S->need, &S->need_cap, n), "discover scratch");
    CK(grow(&S->ccount, &S->ccount_cap, n), "discover scratch");
    CK(grow(&S->coff, &S->coff_cap, n + 1), "discover scratch");
    CK(grow(&S->hist, &S->hist_cap, V), "discover scratch");
    CK(grow(&S->start, &S->start_cap, V + 1), "discover scratch");

    const int set_blocks = ctx->sm_count * 4;
    const uint32_t set_gslots = pow2_at_least((uint64_t)std::max<int64_t>(set->max_len, 1) * 2);
    if (set_gslots > (uint32_t)kSetSmemSlots)
        CK(grow(&S->gtab, &S->gtab_cap, (int64_t)set_blocks * 2 * set_gslots), "discover scratch");

    ctx->last_search_launches = 0;
    int32_t launches = 0;
    CK(cudaMemsetAsync(S->ctr, 0, sizeof(unsigned long long) * 8, st), "memset");
    CK(cudaMemsetAsync(S->status, 0, sizeof(int32_t), st), "memset");
    SetArgs sa{view(set), k, S->ent_kmer, S->ent_pos, S->kcount, S->gtab, set_gslots, S->ctr + 0,
               S->status};
    kmer_sets_kernel<<<set_blocks, kSearchThreads, 0, st>>>(sa);
    CK(cudaGetLastError(), "kmer_sets kernel");
    CK(cudaMemsetAsync(S->hist, 0, sizeof(uint32_t) * V, st), "memset");
    const int64_t wg = warp_grid(ctx, n, 256);
    kmer_hist_kernel<<<(unsigned)wg, 256, 0, st>>>(view(set), S->ent_kmer, S->kcount, S->hist);
    CK(cudaGetLastError(), "kmer_hist kernel");
    rc = device_scan<uint32_t>(ctx, S, S->hist, V, S->start, st);
    if (rc) return rc;
    CK(cudaMemsetAsync(S->hist, 0, sizeof(uint32_t) * V, st), "memset");
    kmer_scatter_kernel<<<(unsigned)wg, 256, 0, st>>>(view(set), S->ent_kmer, S->ent_pos, S->kcount,
                                                      S->start, S->hist, S->bseq, S->bpos);
    CK(cudaGetLastError(), "kmer_scatter kernel");
    launches += 3 + 3;   // sets, histogram, scatter + the scan

    JoinArgs ja{};
    ja.s = view(set);
    ja.ent_kmer = S->ent_kmer;
    ja.kcount = S->kcount;
    ja.start = S->start;
    ja.bseq = S->bseq;
    ja.need = S->need;
    ja.ccount = S->ccount;
    ja.coff = S->coff;
    ja.out_pairs = pairs;
    ja.out_counts = counts;
    ja.capacity = capacity;
    ja.min_shared = min_shared;
    ja.stats = S->ctr + 4;
    ja.status = S->status;
    CK(grow(&S->large_rows, &S->large_rows_cap, n), "discover scratch");
    ja.large_rows = S->large_rows;
    ja.n_tasks = n;
    row_need_kernel<<<(unsigned)wg, 256, 0, st>>>(ja);
    CK(cudaGetLastError(), "row_need kernel");
    launches += 1;
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
        CK(grow(&S->gtab, &S->gtab_cap, (int64_t)large_blocks * per_block), "discover scratch");
    }
    ja.gtab = S->gtab;
    ja.gslots = join_gslots;
    const int join_blocks = ctx->sm_count * 4;
    for (int pass = 0; pass < 2; ++pass) {
        ja.ctr = S->ctr + 1 + pass;
        unsigned long long* lctr = S->ctr + 6 + pass;
        if (pass == 0) {
            join_kernel<false, false><<<join_blocks, kSearchThreads, kJoinSmemBytes, st>>>(ja);
            if (large_blocks) {
                JoinArgs jl = ja;
                jl.ctr = lctr;
                jl.n_tasks = (int64_t)n_large;
                join_kernel<true, false><<<large_blocks, kSearchThreads, 0, st>>>(jl);
            }
            CK(cudaGetLastError(), "join kernel (count)");
            launches += (large_blocks ? 2 : 1) + 3;
            rc = device_scan<uint64_t>(ctx, S, S->ccount, n, S->coff, st);
            if (rc) return rc;
        } else {
            join_kernel<false, true><<<join_blocks, kSearchThreads, kJoinSmemBytes, st>>>(ja);
            if (large_blocks) {
                JoinArgs jl = ja;
                jl.ctr = lctr;
                jl.n_tasks = (int64_t)n_large;
                join_kernel<true, true><<<large_blocks, kSearchThreads, 0, st>>>(jl);
            }
            CK(cudaGetLastError(), "join kernel (write)");
            launches += large_blocks ? 2 : 1;
        }
    }
    uint64_t found = 0;
    int32_t status = 0;
    CK(cudaMemcpyAsync(&found, S->coff + n, sizeof(found), cudaMemcpyDeviceToHost, st), "count D2H");
    CK(cudaMemcpyAsync(&status, S->status, sizeof(status), cudaMemcpyDeviceToHost, st), "status D2H");
    CK(cudaStreamSynchronize(st), "stream sync");
    ctx->last_search_launches = launches;
    if (status) return fail(ctx, SWGB_EINTERNAL, "discover: a hash table was smaller than its bound");
    *n_found = (int64_t)found;
    return SWGB_OK;
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
    a.stats = S->ctr + 4;
    // small class: spans of up to kSmallWords words per warp
    constexpr int64_t kSmallWords = 1 << 16;   // e.g. 512 x 1024 cells
    CK(grow(&S->large, &S->large_cap, n_pairs), "identity scratch");
    a.large = S->large;
    a.n_tasks = n_pairs;
    CK(cudaMemsetAsync(S->ctr, 0, sizeof(unsigned long long) * 8, st), "memset");
    CK(cudaMemsetAsync(S->status, 0, sizeof(int32_t), st), "memset");
    const int64_t g = std::min<int64_t>((n_pairs + 255) / 256, (int64_t)ctx->sm_count * 16);
    ident_need_kernel<<<(unsigned)g, 256, 0, st>>>(a, kSmallWords);
    CK(cudaGetLastError(), "ident_need kernel");
    unsigned long long stats[2] = {0, 0};
    CK(cudaMemcpyAsync(stats, S->ctr + 4, sizeof(stats), cudaMemcpyDeviceToHost, st), "stats D2H");
    CK(cudaStreamSynchronize(st), "stream sync");
    const int64_t max_need = (int64_t)stats[0], n_large = (int64_t)stats[1];
    const int64_t max_rows = std::max(queries->max_len, refs->max_len) + 1;
    const int small_blocks = ctx->sm_count * 8;
    int large_blocks = 0;
    int64_t large_words = 0;
    if (n_large > 0) {
        large_words = max_need;
        const int64_t budget = (int64_t)1 << 31;   // 8 GiB of words
        const int64_t warps = std::max<int64_t>(1, std::min<int64_t>(
            std::min<int64_t>(n_large, (int64_t)ctx->sm_count * kIdWarps), budget / large_words));
        large_blocks = (int)((warps + kIdWarps - 1) / kIdWarps);
    }
    const int64_t small_warps = (int64_t)small_blocks * kIdWarps;
    const int64_t large_warps = (int64_t)large_blocks * kIdWarps;
    CK(grow(&S->dir, &S->dir_cap, small_warps * kSmallWords + large_warps * large_words), "identity scratch");
    CK(grow(&S->bnd, &S->bnd_cap, (small_warps + large_warps) * max_rows), "identity scratch");
    a.bnd_stride = max_rows;
    a.dir = S->dir;
    a.bnd = S->bnd;
    a.region_words = kSmallWords;
    a.min_words = 0;
    a.max_words = kSmallWords;
    a.ctr = S->ctr + 0;
    ident_kernel<<<small_blocks, kIdWarps * 32, 0, st>>>(a);
    CK(cudaGetLastError(), "ident kernel");
    if (large_blocks) {
        IdentArgs b = a;
        b.dir = S->dir + small_warps * kSmallWords;
        b.bnd = S->bnd + small_warps * max_rows;
        b.region_words = large_words;
        b.min_words = kSmallWords;
        b.max_words = large_words;
        b.n_tasks = n_large;
        b.ctr = S->ctr + 1;
        ident_kernel<<<large_blocks, kIdWarps * 32, 0, st>>>(b);
        CK(cudaGetLastError(), "ident kernel (large spans)");
    }
    int32_t status = 0;
    CK(cudaMemcpyAsync(&status, S->status, sizeof(status), cudaMemcpyDeviceToHost, st), "status D2H");
    CK(cudaStreamSynchronize(st), "stream sync");
    ctx->last_search_launches = 2 + (large_blocks ? 1 : 0);
    if (status == 3) return fail(ctx, SWGB_ERANGE, "identity: a pair index or record outside its sequences");
    if (status) return fail(ctx, SWGB_EINTERNAL, "identity: a span's global optimum differs from its record's score");
    return SWGB_OK;
}
