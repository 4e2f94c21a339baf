"""The exactness certificate of the banded reverse pass, checked on the CPU.

A plain numpy model of the band's geometry and bound, written from their
definition (it shares nothing with the CUDA kernel): the anchored reverse DP
restricted to the staircase band of a ring of G lanes x R rows, the band's
exits at or before the first position a0 holding S in the band, and the
bound band value + forward maximum of the successor's rows + gap open < S at
each of them.  The claim pinned here: whenever the bound holds, the band's
row-major-first cell of value S gives exactly the oracle's start; a band that a planted optimal alignment must leave never certifies;
and a band covering the whole matrix always certifies.
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


def band_mask(la, lb, G, R, khi):
    """Cells (a, b) of the band: virtual lane V = b // R holds positions
    [V R - khi, V R - khi + (G - 1)(R + 1))."""
    a = np.arange(la)[:, None]
    V = np.arange(lb)[None, :] // R
    return (a >= V * R - khi) & (a < V * R - khi + (G - 1) * (R + 1))


def anchored_in_band(qr, rr, m, go, ge, inD):
    """Anchored DP over the reversed prefixes, H = 0 only before the origin,
    cells outside the band at the floor."""
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


def banded_start(q, r, rec, m, go, ge, G, R, slot_rows):
    """(certified, start or None) of the band model for the record rec."""
    S, qs, qe, rs, re_ = rec
    qr, rr = q[:qe + 1][::-1], r[:re_ + 1][::-1]
    la, lb = len(qr), len(rr)
    W = G * (R + 1) - 2 * R
    d = lb - la
    khi = max(0, d) + max(W - abs(d), 0) // 2
    inD = band_mask(la, lb, G, R, khi)
    A = anchored_in_band(qr, rr, m, go, ge, inD)
    hits = np.argwhere(A == S)
    if len(hits) == 0:
        return False, None
    a0, b0 = hits[0]
    Hf = forward_local(q, r, m, go, ge)
    slot = np.array([Hf[:, j:j + slot_rows].max() for j in range(0, len(r), slot_rows)])

    def fmax(j_lo, j_hi):
        j_lo, j_hi = max(j_lo, 0), min(j_hi, re_)
        return slot[j_lo // slot_rows: j_hi // slot_rows + 1].max() if j_hi >= j_lo else NEG

    # exits at or before the first S position a0 whose bound reaches S: an
    # alignment through an exit starts at or after the exit's position
    WV = (G - 1) * (R + 1)
    for V in range(-(-lb // R)):
        b_lo, b_hi = V * R, min(V * R + R, lb)
        a_last = V * R - khi + WV - 1
        if 0 <= a_last < la - 1 and a_last <= a0:     # right edge, successor inside the matrix
            if A[a_last, b_lo:b_hi].max() + fmax(re_ - b_hi, re_ - b_lo) + go >= S:
                return False, None
        if b_hi < lb:                                 # staircase: bottom row before lane V + 1 starts
            a_s, a_e = max(V * R - khi, 0), min(V * R - khi + R, la)
            a_e = min(a_e, a0 + 1)
            if a_e > a_s and A[a_s:a_e, b_hi - 1].max() + fmax(re_ - b_hi, re_ - b_hi + 1) + go >= S:
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


@pytest.mark.parametrize("G,R,slot_rows", [(16, 4, 4), (16, 6, 8), (32, 3, 2)])
def test_a_certified_band_gives_the_oracle_start(oracle_mod, G, R, slot_rows):
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
        ok, start = banded_start(q, r, rec, m, 11, 1, G, R, slot_rows)
        if ok:
            certified += 1
            assert start == (rec[1], rec[3]), (trial, rec, start)
    assert certified >= 15


def test_an_alignment_leaving_the_band_is_refused(oracle_mod):
    """q = A X B C, r = A B Y C with |X| = |Y| = 40 and B identical: the optimal
    alignment runs 40 diagonals off the end diagonal, wider than the band."""
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
        ok, _ = banded_start(q, r, rec, m, 11, 1, 4, 4, 4)   # a band of 12 diagonals
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
        ok, start = banded_start(q, r, rec, m, 11, 1, 32, 8, 4)   # 272 diagonals
        assert ok and start == (rec[1], rec[3])
