"""The exactness certificate of the banded reverse pass, checked on the CPU.

A plain numpy model of the band's geometry and bound, written from their
definition (it shares nothing with the CUDA kernel): the anchored DP over the
reversed prefixes restricted to the computed region D -- on a tile of G lanes
x R rows, chunk c of the reversed reference streams the window
[c G R - khi, (c + 1) G R + W - khi), and lane g of the chunk computes its rows
at the positions [w0 - g, w0 - g + steps), steps = the window plus the G - 1
steps of wavefront fill, rounded up to four -- the exits of D (cells of D with
a successor inside the matrix but outside D) at positions up to a0, the first
position holding S in D, and the bound region value + forward maximum of the
successor's rows + gap open < S at each of them.  The claims pinned here:
whenever the bound holds, the region's first cell of value S gives exactly
the oracle's start; a region that a planted optimal alignment must leave
never certifies; and a region covering the whole matrix always certifies.
"""
import numpy as np
import pytest

FLOOR = -8192
NEG = -10 ** 6


def forward_local(q, r, m, go, ge):
    """H of the local forward DP (rows = query, columns = reference)."""
    lq, lr = len(q), len(r)
    H = np.zeros((lq, lr), np.int64)
    Hp = np.zeros(lr + 1, np.int64)
    F = np.full(lr, NEG, np.int64)
    k = np.arange(lr)
    for i in range(lq):
        s = m[q[i], r]
        F = np.maximum(F - ge, Hp[1:] - go - ge)
        part = np.maximum(np.maximum(Hp[:-1] + s, F), 0)
        run = np.maximum.accumulate(part + ge * k)
        E = np.full(lr, NEG, np.int64)
        E[1:] = run[:-1] - go - ge * k[1:]
        H[i] = np.maximum(part, E)
        Hp = np.concatenate([[0], H[i]])
    return H


def band_geometry(la, lb, margin):
    d = lb - la
    return abs(d) + 2 * margin, max(d, 0) + margin


def region(la, lb, G, R, W, khi):
    """Mask [a, b] of the computed region D (a = position, b = row)."""
    rows = G * R
    D = np.zeros((la, lb), bool)
    for c in range(-(-lb // rows)):
        w0 = max(0, c * rows - khi)
        w1 = min(la, (c + 1) * rows + W - khi)
        if w1 <= w0:
            continue
        steps = 4 * (-(-(w1 - w0 + G - 1) // 4))
        for g in range(G):
            b0 = c * rows + g * R
            if b0 >= lb:
                break
            D[max(0, w0 - g):max(0, min(la, w0 - g + steps)), b0:min(b0 + R, lb)] = True
    return D


def anchored_in_region(qr, rr, m, go, ge, inD):
    """Anchored DP over the reversed prefixes, H = 0 only before the origin,
    cells outside D at the floor."""
    la, lb = len(qr), len(rr)
    A = np.full((la, lb), FLOOR, np.int64)
    Hp = np.full(lb + 1, FLOOR, np.int64)
    Hp[0] = 0
    F = np.full(lb, NEG, np.int64)
    k = np.arange(lb)
    for a in range(la):
        s = m[qr[a], rr]
        F = np.where(inD[a], np.maximum(F - ge, Hp[1:] - go - ge), NEG)
        part = np.where(inD[a], np.maximum(np.maximum(Hp[:-1] + s, F), FLOOR), FLOOR)
        run = np.maximum.accumulate(part + ge * k)
        E = np.full(lb, NEG, np.int64)
        E[1:] = run[:-1] - go - ge * k[1:]
        A[a] = np.where(inD[a], np.maximum(part, E), FLOOR)
        Hp = np.concatenate([[FLOOR], A[a]])
    return A


def banded_start(q, r, rec, m, go, ge, G, R, margin, lane_rows):
    """(certified, start or None) of the band model for the record rec;
    lane_rows = rows per entry of the forward maxima."""
    S, qs, qe, rs, re_ = rec
    qr, rr = q[:qe + 1][::-1], r[:re_ + 1][::-1]
    la, lb = len(qr), len(rr)
    W, khi = band_geometry(la, lb, margin)
    D = region(la, lb, G, R, W, khi)
    A = anchored_in_region(qr, rr, m, go, ge, D)
    hits = np.argwhere(A == S)
    if len(hits) == 0:
        return False, None
    a0, b0 = hits[0]
    Hf = forward_local(q, r, m, go, ge)
    blk = np.array([Hf[:, j:j + lane_rows].max() for j in range(0, len(r), lane_rows)])
    fm = blk[(re_ - np.arange(lb)) // lane_rows]          # reversed row -> its block
    fm_next = np.concatenate([fm[1:], [NEG]])
    Dp = np.zeros((la + 1, lb + 1), bool)
    Dp[:la, :lb] = D
    inm = np.zeros((la + 1, lb + 1), bool)
    inm[:la, :lb] = True
    right = D & inm[1:, :lb] & ~Dp[1:, :lb]
    down_or_diag = D & ((inm[:la, 1:] & ~Dp[:la, 1:]) | (inm[1:, 1:] & ~Dp[1:, 1:]))
    early = (np.arange(la) <= a0)[:, None]
    if (right & early & (A + fm[None, :] + go >= S)).any():
        return False, None
    if (down_or_diag & early & (A + fm_next[None, :] + go >= S)).any():
        return False, None
    return True, (qe - a0, re_ - b0)


def homologous(rng, L, mut=0.3, indel=0.04):
    q = rng.integers(0, 20, size=L)
    r = []
    for x in q:
        u = rng.random()
        if u < indel / 2:
            continue
        if u < indel:
            r.extend(rng.integers(0, 20, size=int(rng.integers(1, 4))))
        r.append(int(rng.integers(0, 20)) if rng.random() < mut else int(x))
    return q.astype(np.uint8), np.asarray(r, np.uint8)


@pytest.mark.parametrize("G,R,margin,lane_rows", [(8, 4, 12, 4), (8, 3, 16, 8), (4, 5, 10, 2)])
def test_a_certified_band_gives_the_oracle_start(oracle_mod, G, R, margin, lane_rows):
    mat = oracle_mod.blosum62()
    m = mat.astype(np.int64)
    rng = np.random.default_rng(G * 100 + R)
    certified = 0
    for trial in range(60):
        if trial % 3 == 2:
            q = rng.integers(0, 20, size=int(rng.integers(60, 150))).astype(np.uint8)
            r = rng.integers(0, 20, size=int(rng.integers(60, 150))).astype(np.uint8)
        else:
            q, r = homologous(rng, int(rng.integers(100, 250)))
        rec = oracle_mod.align_pair(q, r, mat, 11, 1)
        if rec[0] == 0:
            continue
        ok, start = banded_start(q, r, rec, m, 11, 1, G, R, margin, lane_rows)
        if ok:
            certified += 1
            assert start == (rec[1], rec[3]), (trial, rec, start)
    assert certified >= 15


def test_an_alignment_leaving_the_band_is_refused(oracle_mod):
    """q = A X B C, r = A B Y C with |X| = |Y| = 40 and B identical: the optimal
    alignment runs 40 diagonals off the end diagonal, more than the band's
    margin of 8."""
    mat = oracle_mod.blosum62()
    m = mat.astype(np.int64)
    rng = np.random.default_rng(7)
    for _ in range(10):
        A, B, C = (rng.integers(0, 20, size=n) for n in (20, 60, 20))
        X, Y = rng.integers(0, 20, size=40), rng.integers(0, 20, size=40)
        q = np.concatenate([A, X, B, C]).astype(np.uint8)
        r = np.concatenate([A, B, Y, C]).astype(np.uint8)
        rec = oracle_mod.align_pair(q, r, mat, 11, 1)
        assert rec[1] < 20 and rec[2] > 119            # the planted alignment is the optimum
        ok, _ = banded_start(q, r, rec, m, 11, 1, 4, 4, 8, 4)
        assert not ok


def test_a_band_over_the_whole_matrix_always_certifies(oracle_mod):
    mat = oracle_mod.blosum62()
    m = mat.astype(np.int64)
    rng = np.random.default_rng(8)
    for _ in range(20):
        q, r = homologous(rng, int(rng.integers(20, 60)))
        rec = oracle_mod.align_pair(q, r, mat, 11, 1)
        if rec[0] == 0:
            continue
        ok, start = banded_start(q, r, rec, m, 11, 1, 8, 4, 80, 4)   # margin wider than the pair
        assert ok and start == (rec[1], rec[3])


def test_the_region_is_the_stated_staircase():
    """Row b of chunk c, lane g: exactly the positions [w0 - g, w0 - g + steps)
    inside the matrix; the origin's cell is in D, and D holds every diagonal
    of the band for every row."""
    la, lb, G, R = 90, 70, 4, 3
    W, khi = band_geometry(la, lb, 6)
    D = region(la, lb, G, R, W, khi)
    assert D[0, 0]
    rows = G * R
    for b in range(lb):
        c, g = divmod(b, rows)
        g //= R
        w0 = max(0, c * rows - khi)
        w1 = min(la, (c + 1) * rows + W - khi)
        steps = 4 * (-(-(w1 - w0 + G - 1) // 4))
        want = np.zeros(la, bool)
        want[max(0, w0 - g):max(0, min(la, w0 - g + steps))] = True
        assert (D[:, b] == want).all(), b
        for a in range(max(0, b - khi), min(la, b - khi + W)):
            assert D[a, b], (a, b)
