// swgb_band.cu -- the banded reverse pass with its exactness certificate.
//
// The reverse pass finds the start of a scored pair: the first cell, in
// row-major order over the reversed prefixes q[q_end..0] x r[r_end..0], whose
// local-DP value is the score S (include/swgb.h).  Every such cell starts an
// optimal alignment that ends at the reversed origin, so the anchored DP
// (H = 0 only at the origin's virtual predecessor, minus infinity elsewhere
// on the border, values floored at kFloorH <= 0) has exactly the same cells of
// value S; a floor at or below zero neither creates nor removes them (a path
// from a floored cell would score above S).
//
// band_kernel evaluates that anchored DP only over a staircase band D around
// the diagonals the alignment can use (a pair's end diagonal lr - lq gives
// the drift; the band covers band_width whole diagonals centred on it), and
// keeps the result only when no alignment ending at the origin with score S
// can leave D.  Such an alignment would leave D through an exit: a cell n of
// D with a neighbour c outside D that the alignment enters next (in reverse
// order).  Its score is at most
//     H_D(n)            the band's value at n (the part from the origin to n
//                       lies in D: n is the alignment's first exit), plus
//     Hf(c)             the forward pass's value at c (the rest is an
//                       alignment of the forward prefixes ending at c), plus
//     o                 one gap opening charged twice when n and c lie in
//                       the same gap,
// and Hf(c) is at most the forward pass's maximum over c's block of reference
// rows (the fmax slots the forward kernels record).  An alignment through an
// exit n can only start at or after n's streamed position, so only exits at
// or before the position a* of the first cell of value S found in D matter.
// If for every such exit
//     H_D(n) + fmax(c) + o < S
// no alignment of score S ending at the origin leaves D through one, every
// cell of value S at or before a* lies in D, and the first one found is the
// pair's start.  Otherwise (or with no cell of value S in D) the pair is
// marked (q_start = kBandFallback) and re-run over the whole rectangle.  The
// kernel keeps, per pair, the smallest streamed position of an exit whose
// bound reaches S and certifies when it lies after a*.
//
// Layout: the reversed reference is held, the reversed query streamed, as in
// dp_kernel, but the G lanes of a group form a ring.  Virtual lane V holds rows
// [V R, V R + R) for the streamed positions [V R - khi, V R - khi + WV), WV =
// (G - 1)(R + 1), at time t = position + V + khi; the physical lane V mod G then
// spends R + 1 steps idle and moves on to V + G.  Lane V takes the row above
// it from lane V - 1 (the previous lane of the ring) one step later; for the
// last R positions of its window that lane has moved on, and the input is
// minus infinity (those cells lie outside D).  The exits of D are the cells
// at the last position of each lane's window (right edge) and the bottom row
// of each lane at the first R positions of its window, before the next lane
// starts (the staircase); lane V + 1 sees the latter arrive while it idles and
// keeps their maximum.
//
// Profiles prof[letter][row] = s + o + e of both pairs of a group live in the
// warp's slice of global scratch (built once per task), so a lane moving on to
// new rows only moves its pointer.
#include <climits>
#include <cstdint>

#include "swgb_internal.cuh"
#include "swgb_lane.cuh"

namespace swgb {

namespace {

constexpr int kFloorH = -8192;          // anchored DP floor (H units)
// resident blocks per SM the register budget is sized for
__host__ __device__ constexpr int band_min_blocks(int R) { return R > 12 ? 6 : 8; }

template <int G, int R>
__global__ void __launch_bounds__(kBandThreads, band_min_blocks(R)) band_kernel(const BandArgs a) {
    using L = Lane<true>;
    constexpr int PACK = 2;
    constexpr int GROUPS = 32 / G;
    constexpr int LS = (R + 3) / 4 * 4;
    constexpr int R1 = R + 1;
    constexpr int CYC = G * R1;           // steps between two moves of a lane
    constexpr int WV = (G - 1) * R1;      // steps of a lane's window
    constexpr int W = G * R1 - 2 * R;     // whole diagonals the band covers
    static_assert(WV - R - 1 > 0 && CYC - 5 > WV - 1, "event order");

    __shared__ __align__(16) uint8_t tabT[kSmatRegion];
    const int prows = a.sc.prof_rows;
    const int pad_row = prows - 1;
    for (int k = threadIdx.x; k < kTabTBytes; k += blockDim.x) {
        const int y = k / kTabTStride, x = k % kTabTStride;
        tabT[k] = x >= prows ? (uint8_t)0 : a.sc.profu[x == pad_row ? kPadCode : x][y];
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int g = lane / G;
    const int gl = lane % G;
    const int64_t wslot = (int64_t)blockIdx.x * (kBandThreads / 32) + warp;
    if (wslot >= a.slots) {   // a grid wider than the scratch: a host error
        if (lane == 0) set_status(a.status, SWGB_EINTERNAL);
        return;
    }
    const int64_t rstride = a.rstride;
    // per pair: prows profile rows, then one row of reversed query codes
    const int64_t pair_bytes = (int64_t)(prows + 1) * rstride;
    uint8_t* const wprof = a.prof + wslot * a.prof_stride + (int64_t)g * PACK * pair_bytes;

    const int64_t begin = a.scan[(int64_t)a.bucket * kQBins];
    const int64_t end = a.scan[(int64_t)(a.bucket + 1) * kQBins];
    const int oe = a.sc.go + a.sc.ge;
    const int zero_h = kBias - oe;                            // Hop at H = 0
    const uint32_t NOE = L::splat(-oe);
    const uint32_t NE = L::splat(-a.sc.ge);
    const uint32_t HNEG = L::splat(kBias + kFloorH - oe);     // Hop, E, F at H = floor
    const uint32_t HZERO = L::splat(zero_h);
    const uint32_t BF = L::splat(kBias + kFloorH);            // the floor in phase 1
    const uint32_t one = (uint32_t)a.sc.one;
    const uint32_t C_UOP = (uint32_t)(-(oe * 65537));
    const int ring_src = (gl + G - 1) & (G - 1);

    for (;;) {
        uint32_t task = 0;
        if (lane == 0) task = atomicAdd(a.task_ctr, 1u);
        task = __shfl_sync(kFull, task, 0);
        const int64_t first = begin + (int64_t)task * (GROUPS * PACK);
        if (first >= end) break;

        // ---- the (up to) two pairs of this group
        int pid[PACK], lq[PACK], lr[PACK], S[PACK], khi[PACK], sb[PACK], tnat[PACK];
        const uint8_t* qp[PACK];
        const uint8_t* rp[PACK];
        const int32_t* fm[PACK];
        int tend = 0;
#pragma unroll
        for (int h = 0; h < PACK; ++h) {
            const int64_t pos = first + g * PACK + h;
            pid[h] = -1;
            lq[h] = lr[h] = S[h] = khi[h] = tnat[h] = 0;
            sb[h] = 16;
            qp[h] = rp[h] = nullptr;
            fm[h] = nullptr;
            if (pos < end) {
                const int p = a.order[pos];
                const swgb_record rec = a.out[p];
                const int32_t qi = a.pairs[2 * (int64_t)p], ri = a.pairs[2 * (int64_t)p + 1];
                pid[h] = p;
                qp[h] = a.q.res + a.q.off[qi];
                rp[h] = a.r.res + a.r.off[ri];
                lq[h] = rec.q_end + 1;
                lr[h] = rec.r_end + 1;
                S[h] = rec.score;
                const int delta = lr[h] - lq[h];
                const int ad = delta < 0 ? -delta : delta;
                khi[h] = (delta > 0 ? delta : 0) + (ad < W ? (W - ad) / 2 : 0);
                fm[h] = a.fmax + (int64_t)p * kFmaxSlots;
                sb[h] = fm[h][0];   // block height (the reverse keys checked it is recorded)
                // the last virtual lane with a cell of the matrix in its window
                const int v_rows = (lr[h] + R - 1) / R;
                const int v_cols = (lq[h] - 1 + khi[h]) / R + 1;
                const int v_end = v_rows < v_cols ? v_rows : v_cols;
                tnat[h] = (v_end - 1) * R1 + WV;
            }
            tend = max(tend, tnat[h]);
        }
        int lr_w = max(lr[0], lr[1]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            tend = max(tend, __shfl_xor_sync(kFull, tend, off));
            lr_w = max(lr_w, __shfl_xor_sync(kFull, lr_w, off));
        }
        // rows any lane can reach before tend (+ one group of steps), and at
        // least 16 pad rows past every reference of the warp; warp-uniform
        int64_t rows_used = ((int64_t)(tend + 4) / R1 + G + 1) * R + LS;
        if (rows_used < (int64_t)lr_w + 16) rows_used = (int64_t)lr_w + 16;
        const int64_t rows_built = (rows_used + 15) / 16 * 16;
        if (rows_built > rstride) {   // scratch rows sized by the host for the longest reference
            if (lane == 0) set_status(a.status, SWGB_EINTERNAL);
            continue;
        }
        // a lane without rows of its own (before its first window) reads this
        // all-pad stretch of its profile rows
        const int64_t pad_off = rows_built - 16;
        // streamed positions any lane reads a letter of: p = t - V(t) - khi with
        // t <= tend + 7 and V(t) >= t / (R + 1) - G, so p < tend + 8 - tend / (R + 1)
        // + G; and p >= -khi >= -W.  The query row holds code(p) at p + W.
        const int64_t qlen = ((int64_t)tend + 8 - tend / R1 + G + W + 4 + 3) / 4 * 4;
        if (qlen > rstride) {
            if (lane == 0) set_status(a.status, SWGB_EINTERNAL);
            continue;
        }

        // ---- profiles: prof_h[x][b] = s(x, r[r_end - b]) + o + e for b < lr, 0
        // past it; four rows x at a time by 4 x 4 byte transposes of the table
        __syncwarp();
#pragma unroll
        for (int h = 0; h < PACK; ++h) {
            uint8_t* base = wprof + (int64_t)h * pair_bytes;
            for (int64_t w = gl; 4 * w < rows_built; w += G) {
                const int b0 = (int)(4 * w);
                int y[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) y[j] = b0 + j < lr[h] ? rp[h][lr[h] - 1 - (b0 + j)] : kPadCode;
                for (int xq = 0; 4 * xq < prows; ++xq) {
                    uint32_t wv[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        wv[j] = *reinterpret_cast<const uint32_t*>(tabT + y[j] * kTabTStride + 4 * xq);
                    const uint32_t t0 = prmt(wv[0], wv[1], 0x5140u), t1 = prmt(wv[0], wv[1], 0x7362u);
                    const uint32_t t2 = prmt(wv[2], wv[3], 0x5140u), t3 = prmt(wv[2], wv[3], 0x7362u);
                    const uint32_t o4[4] = {prmt(t0, t2, 0x5410u), prmt(t0, t2, 0x7632u), prmt(t1, t3, 0x5410u),
                                            prmt(t1, t3, 0x7632u)};
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        if (4 * xq + m < prows)
                            *reinterpret_cast<uint32_t*>(base + (int64_t)(4 * xq + m) * rstride + b0) = o4[m];
                }
            }
            // the reversed query's profile rows, pad_row outside [0, lq)
            uint8_t* qrow = base + (int64_t)prows * rstride;
            for (int64_t w = gl; 4 * w < qlen; w += G) {
                uint32_t v = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int pq = (int)(4 * w) + j - W;
                    const uint32_t c = (pq < 0 || pq >= lq[h]) ? (uint32_t)pad_row : qp[h][lq[h] - 1 - pq];
                    v |= c << (8 * j);
                }
                *reinterpret_cast<uint32_t*>(qrow + 4 * w) = v;
            }
        }
        __syncwarp();

        // largest forward maximum over reference rows j in [j_lo, j_hi] of half
        // h (blocks of sb rows, sb >= 8: at most three blocks for R + 1 rows)
        auto fmax_rows = [&](int h, int j_lo, int j_hi) -> int {
            j_lo = max(j_lo, 0);
            j_hi = min(j_hi, lr[h] - 1);
            if (pid[h] < 0 || j_hi < j_lo) return INT_MIN / 2;
            int v = INT_MIN / 2;
            for (int k = j_lo / sb[h]; k <= j_hi / sb[h]; ++k) v = max(v, fm[h][1 + k]);
            return v;
        };

        // ---- per-lane ring state
        const int t0 = gl * R1;                       // first step of this lane's first window
        int V = gl == 0 ? 0 : gl - G;                 // virtual lane (rows V R ..)
        const uint8_t* pb[PACK];                      // profile of this lane's rows, letter 0
        auto set_rows = [&](int v) {
#pragma unroll
            for (int h = 0; h < PACK; ++h)
                pb[h] = wprof + (int64_t)h * pair_bytes + (v >= 0 ? (int64_t)v * R : pad_off);
        };
        set_rows(V);
        int vq = V;                                   // virtual lane of the letters loaded
        const uint8_t* qb[PACK];                      // query row, shifted so qb[t] is step t's letter
        auto set_letters = [&](int v) {
#pragma unroll
            for (int h = 0; h < PACK; ++h)
                qb[h] = wprof + (int64_t)h * pair_bytes + (int64_t)prows * rstride + W - v - khi[h];
        };
        set_letters(vq);
        uint32_t Hop[R], F[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            Hop[r] = HNEG;
            F[r] = HNEG;
        }
        // origin: H = 0 diagonally before (0, 0), i.e. above row 0 at streamed
        // position -1; minus infinity above row 0 from position 0 on
        uint32_t fill = HNEG;
#pragma unroll
        for (int h = 0; h < PACK; ++h)
            if (khi[h] > 0) fill = (fill & (h ? 0x0000ffffu : 0xffff0000u)) | (HZERO & (h ? 0xffff0000u : 0x0000ffffu));
        uint32_t hin_prev = gl == 0 ? HZERO : HNEG;
        uint32_t ein = gl == 0 ? fill : HNEG, hin = ein;
        // input mask (x * mm + ma), staircase accumulation mask, window flag
        const int k0 = (CYC - t0) % CYC;              // cycle step of step 0
        uint32_t mm, ma, am;
        bool live_v = gl == 0;
        if (gl == 0) {
            mm = 0u;
            ma = fill;
            am = 0u;
        } else {
            const bool masked = k0 >= WV - R && k0 < WV;
            mm = masked ? 0u : one;
            ma = masked ? HNEG : 0u;
            am = (k0 >= WV && k0 <= CYC - 2) ? one : 0u;
        }
        uint32_t exacc = 0;                           // staircase exits seen while idle (Hop)
        // vmin: smallest streamed position of an exit whose bound reaches S (only
        // exits at or before the first S position found matter)
        int fm_right[PACK], fm_stair[PACK], vmin[PACK], best_a[PACK], best_b[PACK];
        auto prefetch = [&](int v) {
#pragma unroll
            for (int h = 0; h < PACK; ++h) {
                const int re = lr[h] - 1;
                fm_right[h] = v >= 0 ? fmax_rows(h, re - v * R - R, re - v * R) : INT_MIN / 2;
                const int bn = (v + G) * R;
                fm_stair[h] = fmax_rows(h, re - bn, re - bn + 1);
            }
        };
        prefetch(V);
#pragma unroll
        for (int h = 0; h < PACK; ++h) {
            vmin[h] = INT_MAX;
            best_a[h] = INT_MAX;
            best_b[h] = INT_MAX;
        }
        // S in Hop units per half (an absent pair can never be met)
        uint32_t TSm1 = 0;
#pragma unroll
        for (int h = 0; h < PACK; ++h) {
            const uint32_t ts = pid[h] >= 0 ? (uint32_t)(S[h] + zero_h - 1) : 0xfffeu;
            TSm1 |= ts << (16 * h);
        }
        // Phase changes of this lane: at the end of steps tc + ev_off(ei), tc the
        // first step of the lane's current cycle (lanes 1.. start in a pre-start
        // cycle that ends at their first window), ei the next change in cycle
        // order; and, for lane 0, the step khi_h - 1 after which the origin's
        // H = 0 above row 0 of pair h gives way to minus infinity.
        auto ev_off = [&](int e) -> int {
            return e == 0 ? WV - R - 1 : e == 1 ? WV - 1 : e == 2 ? CYC - 5 : e == 3 ? CYC - 3 : e == 4 ? CYC - 2 : CYC - 1;
        };
        int tc = gl == 0 ? 0 : t0 - CYC;
        int ei = 0;
        while (ei < 5 && tc + ev_off(ei) < 0) ++ei;
        int ft[PACK];
#pragma unroll
        for (int h = 0; h < PACK; ++h) ft[h] = (gl == 0 && khi[h] > 0) ? khi[h] - 1 : INT_MAX;
        int next_ev = min(tc + ev_off(ei), min(ft[0], ft[PACK - 1]));
        // fires at the end of step t; inputs for step t + 1 follow
        auto on_event = [&](int t) {
#pragma unroll
            for (int h = 0; h < PACK; ++h) {
                if (t == ft[h]) {   // lane 0, first window only (khi < WV - R)
                    fill = (fill & (h ? 0x0000ffffu : 0xffff0000u)) | (HNEG & (h ? 0xffff0000u : 0x0000ffffu));
                    ma = fill;
                    ft[h] = INT_MAX;
                }
            }
            if (t == tc + ev_off(ei)) {
                if (ei == 0) {   // the lane above has moved on: minus infinity from above
                    mm = 0u;
                    ma = HNEG;
                } else if (ei == 1) {   // last step of the window: right-edge exits
                    if (V >= 0) {
                        uint32_t m = Hop[0];
#pragma unroll
                        for (int r = 1; r < R; ++r) m = L::max3(m, Hop[r], Hop[r]);
#pragma unroll
                        for (int h = 0; h < PACK; ++h) {
                            const int a_last = t - V - khi[h];
                            if (pid[h] >= 0 && V * R < lr[h] && a_last + 1 < lq[h] &&
                                L::get(m, h) - zero_h + fm_right[h] + a.sc.go >= S[h])
                                vmin[h] = min(vmin[h], a_last);
                        }
                    }
                    live_v = false;
                    mm = one;
                    ma = 0u;
                    am = one;
                } else if (ei == 2) {   // letters loaded from the next step on are the new rows'
                    vq = V + G;
                    set_letters(vq);
                } else if (ei == 3) {   // profiles loaded from the next step on are the new rows'
                    set_rows(V + G);
                } else if (ei == 4) {   // the last staircase value has arrived
                    am = 0u;
                } else {   // move on to rows G R further up
                    const int bn = (V + G) * R;
#pragma unroll
                    for (int h = 0; h < PACK; ++h) {
                        const int x = (int)L::get(exacc, h);
                        // the lane above's first R positions, from bn - R - khi on
                        if (pid[h] >= 0 && x > 0 && bn < lr[h] && x - zero_h + fm_stair[h] + a.sc.go >= S[h])
                            vmin[h] = min(vmin[h], bn - R - khi[h]);
                    }
                    exacc = 0u;
                    V += G;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        Hop[r] = HNEG;
                        F[r] = HNEG;
                    }
                    live_v = true;
                    mm = one;
                    ma = 0u;
                    prefetch(V);
                }
                if (++ei == 6) {
                    ei = 0;
                    tc += CYC;
                }
            }
            next_ev = min(tc + ev_off(ei), min(ft[0], ft[PACK - 1]));
        };

        // ---- letters: each lane reads its own from the pair's query row, four
        // steps ahead (a lane moving on to new rows jumps back G - 1 positions,
        // so letters cannot be handed down the ring); profile words two steps
        // ahead, in three rotating sets
        ProfWords<LS> pwA[PACK], pwB[PACK], pwC[PACK];
        int x2[PACK], x3[PACK];
#pragma unroll
        for (int h = 0; h < PACK; ++h) {
            pwA[h] = load_prof<LS>(reinterpret_cast<const int8_t*>(pb[h]) + (int64_t)qb[h][0] * rstride);
            pwB[h] = load_prof<LS>(reinterpret_cast<const int8_t*>(pb[h]) + (int64_t)qb[h][1] * rstride);
            x2[h] = qb[h][2];
            x3[h] = qb[h][3];
        }
        int stop_w = tend - 1;
        int chk = 0;   // steps since the last end test

        auto step = [&](int t, const ProfWords<LS> (&pw)[PACK], ProfWords<LS> (&pwn)[PACK], bool last) {
            // pwn receives the profile words of step t + 2
#pragma unroll
            for (int h = 0; h < PACK; ++h) {
                pwn[h] = load_prof<LS>(reinterpret_cast<const int8_t*>(pb[h]) + (int64_t)x2[h] * rstride);
                x2[h] = x3[h];
                x3[h] = qb[h][t + 4];
            }
            // phase 1, rows high to low in place: U = max(Hdiag + s, F, floor) - (o + e)
#pragma unroll
            for (int r = R - 1; r >= 0; --r) {
                const uint32_t s = L::widen(pw[0].w[r >> 2], pw[PACK - 1].w[r >> 2], r & 3);
                const uint32_t hd = r == 0 ? hin_prev : Hop[r - 1];
                Hop[r] = L::max3(s * one + hd, F[r], BF) * one + C_UOP;
            }
            // phase 2, the chain along the rows
            uint32_t e = ein;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t hn = L::addmax(e, NOE, Hop[r]);
                e = L::addmax(e, NE, Hop[r]);
                Hop[r] = hn;
            }
            // phase 3, F of the next position
#pragma unroll
            for (int r = 0; r < R; ++r) F[r] = L::addmax(F[r], NE, Hop[r]);
            hin_prev = hin;
            const uint32_t e_next = __shfl_sync(kFull, e, ring_src, G);
            const uint32_t h_next = __shfl_sync(kFull, Hop[R - 1], ring_src, G);
            // a cell of value S (rare): the first row holding it, per half
            const uint32_t smax = tree_max<true, R>(Hop, 0u);
            if (L::max3(smax, TSm1, TSm1) != TSm1 && live_v) {
#pragma unroll
                for (int h = 0; h < PACK; ++h) {
                    const uint32_t ts = L::get(TSm1, h) + 1u;
                    if ((uint32_t)L::get(smax, h) == ts) {
                        int row = R - 1;
#pragma unroll
                        for (int r = R - 1; r >= 0; --r)
                            if ((uint32_t)L::get(Hop[r], h) == ts) row = r;
                        const int ai = t - V - khi[h], bi = V * R + row;
                        if (ai < best_a[h] || (ai == best_a[h] && bi < best_b[h])) {
                            best_a[h] = ai;
                            best_b[h] = bi;
                        }
                    }
                }
            }
            // staircase exits: the lane above's first outputs while this lane idles
            const uint32_t x = h_next * am;
            exacc = L::max3(exacc, x, x);
            if (t >= next_ev) on_event(t);
            ein = e_next * mm + ma;
            hin = h_next * mm + ma;
            if (last && (chk += 3) >= 32) {
                chk = 0;
                // stop once every cell at or before the first S position found
                // has been computed (all lanes whose windows reach it)
                int stop = 0;
#pragma unroll
                for (int h = 0; h < PACK; ++h) {
                    const int fa = group_min<G>(best_a[h]);
                    int sh = tnat[h] - 1;
                    if (fa != INT_MAX) sh = min(sh, fa + khi[h] + (fa + khi[h]) / R);
                    stop = max(stop, pid[h] >= 0 ? sh : 0);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) stop = max(stop, __shfl_xor_sync(kFull, stop, off));
                stop_w = stop;
            }
        };

        // steps in threes (step t computes with one profile set and loads the
        // set of step t + 2 into the one step t - 1 used); the third step of a
        // group tests for the end every 32 steps or so
        int t = 0;
        while (t <= stop_w) {
            step(t, pwA, pwC, false);
            step(t + 1, pwB, pwA, false);
            step(t + 2, pwC, pwB, true);
            t += 3;
        }
        // staircase exits still held by lanes that have not moved on
        {
            const int bn = (V + G) * R;
#pragma unroll
            for (int h = 0; h < PACK; ++h) {
                const int x = (int)L::get(exacc, h);
                if (pid[h] >= 0 && x > 0 && bn < lr[h] && x - zero_h + fm_stair[h] + a.sc.go >= S[h])
                    vmin[h] = min(vmin[h], bn - R - khi[h]);
            }
        }

        // ---- reduce over the group and write
#pragma unroll
        for (int h = 0; h < PACK; ++h) {
            int ba = best_a[h], bb = best_b[h], vm = vmin[h];
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                const int oa = __shfl_xor_sync(kFull, ba, off, G);
                const int ob = __shfl_xor_sync(kFull, bb, off, G);
                vm = min(vm, __shfl_xor_sync(kFull, vm, off, G));
                if (oa < ba || (oa == ba && ob < bb)) {
                    ba = oa;
                    bb = ob;
                }
            }
            if (gl == 0 && pid[h] >= 0) {
                swgb_record* rec = &a.out[pid[h]];
                if (ba >= 0 && ba < lq[h] && bb >= 0 && bb < lr[h] && vm > ba) {
                    rec->q_start = lq[h] - 1 - ba;
                    rec->r_start = lr[h] - 1 - bb;
                    atomicAdd(&a.counters[kCtrBandCertified], 1ull);
                } else {
                    rec->q_start = kBandFallback;
                }
            }
        }
        __syncwarp();
    }
}

using BandFn = void (*)(const BandArgs);

BandFn band_lookup(int cfg) {
    return cfg == 0 ? &band_kernel<band_G(0), band_R(0)> : &band_kernel<band_G(1), band_R(1)>;
}

}  // namespace

cudaError_t launch_band(int cfg, const BandArgs& a, int grid_blocks, cudaStream_t st) {
    band_lookup(cfg)<<<grid_blocks, kBandThreads, 0, st>>>(a);
    return cudaGetLastError();
}

int band_blocks_per_sm(int cfg) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, band_lookup(cfg), kBandThreads, 0) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t band_configure(int cfg) {
    return cudaFuncSetAttribute(band_lookup(cfg), cudaFuncAttributePreferredSharedMemoryCarveout,
                                10);   // percent: room for the blocks' tables, the rest L1
}

int64_t band_rstride(int64_t max_len) {
    // profile rows a lane can reach: the reference plus about two rings
    // (2 G R + R + LS); query positions read: the query plus about two band
    // widths and a window (2 W + WV + G + 12); 4 G (R + 1) + 64 covers both
    int64_t extra = 0;
    for (int c = 0; c < kBandConfigs; ++c) {
        const int64_t e = 4 * (int64_t)band_G(c) * (band_R(c) + 1) + 64;
        extra = e > extra ? e : extra;
    }
    return (max_len + extra + 15) / 16 * 16;
}

int64_t band_prof_bytes_per_warp(int64_t rstride, int prof_rows) {
    // the larger of the configs' needs: groups per warp x 2 pairs x (profile
    // rows + the query row)
    int64_t groups = 0;
    for (int c = 0; c < kBandConfigs; ++c) groups = groups > 32 / band_G(c) ? groups : 32 / band_G(c);
    return groups * 2 * (prof_rows + 1) * rstride;
}

}  // namespace swgb
