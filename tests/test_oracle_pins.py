"""Pins the CPU oracle to facts that do not come from the oracle itself.

* brute-force enumeration of every local alignment of tiny sequences, under
  an asymmetric toy matrix (catches transposed operands), BLOSUM62 and several
  gap penalties;
* the gap-cost convention: (open o, extend e) with cost o + e*L equals the
  other convention o' + e*(L-1) with o' = o + e, checked by enumeration;
* the closed-form self-alignment score (sum of the BLOSUM62 diagonal with the
  full-length span), whose premise is checked on the table;
* homopolymers, single residues, sequences with no positive score;
* invariants: S >= 0, S <= max_s * min(lq, lr), swap symmetry, coordinate
  bounds, and the reported span re-scored by an independent global programme;
* the BLOSUM62 transcription against its published Karlin-Altschul lambda and
  relative entropy.
"""
import os
import random

import numpy as np
import pytest

from brute_force import brute_record, global_affine

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

STD20 = "ARNDCQEGHILKMFPSTWYV"


def toy_matrix():
    """Asymmetric 4-letter matrix (codes 0..3) embedded in a 24 x 24 table."""
    m = np.full((24, 24), -3, dtype=np.int8)
    toy = np.array([[3, -1, -2, 1],
                    [-2, 4, 0, -1],
                    [1, -3, 2, -2],
                    [0, 2, -1, 5]], dtype=np.int8)
    m[:4, :4] = toy
    return m


def gap_linear(o, e):
    return lambda L: o + e * L


def check_against_brute(oracle_mod, q, r, mat, o, e):
    got = oracle_mod.align_pair(np.array(q, np.uint8), np.array(r, np.uint8), mat, o, e)
    want, _ = brute_record(q, r, lambda a, b: int(mat[a, b]), gap_linear(o, e))
    assert got == want, (q, r, o, e, got, want)


def test_brute_force_toy_matrix(oracle_mod):
    rng = random.Random(1)
    mat = toy_matrix()
    for _ in range(400):
        lq, lr = rng.randint(0, 5), rng.randint(0, 5)
        q = [rng.randrange(4) for _ in range(lq)]
        r = [rng.randrange(4) for _ in range(lr)]
        o, e = rng.choice([(0, 1), (1, 1), (2, 1), (3, 2), (11, 1), (1, 3)])
        check_against_brute(oracle_mod, q, r, mat, o, e)


def test_brute_force_ties(oracle_mod):
    """Match +1 / mismatch -1 on two letters: many equal-scoring alignments."""
    rng = random.Random(2)
    mat = np.full((24, 24), -1, dtype=np.int8)
    mat[0, 0] = mat[1, 1] = 1
    for _ in range(300):
        q = [rng.randrange(2) for _ in range(rng.randint(1, 6))]
        r = [rng.randrange(2) for _ in range(rng.randint(1, 6))]
        o, e = rng.choice([(0, 1), (1, 1), (2, 1)])
        check_against_brute(oracle_mod, q, r, mat, o, e)


def test_brute_force_blosum62(oracle_mod):
    rng = random.Random(3)
    mat = oracle_mod.blosum62()
    for _ in range(150):
        q = [rng.randrange(24) for _ in range(rng.randint(1, 6))]
        r = [rng.randrange(24) for _ in range(rng.randint(1, 6))]
        o, e = rng.choice([(11, 1), (11, 2), (5, 2), (0, 1)])
        check_against_brute(oracle_mod, q, r, mat, o, e)


def test_brute_force_length7(oracle_mod):
    rng = random.Random(4)
    mat = toy_matrix()
    for _ in range(6):
        q = [rng.randrange(4) for _ in range(7)]
        r = [rng.randrange(4) for _ in range(7)]
        check_against_brute(oracle_mod, q, r, mat, 2, 1)


def long_gap_cases():
    """Two runs of a high-scoring letter split by k inserted letters, in either
    sequence: the optimum bridges the insertion with one gap of length k."""
    for k in range(1, 5):
        for left, right in [(3, 3), (2, 4), (4, 1)]:
            a = [3] * left + [3] * right
            b = [3] * left + [2] * k + [3] * right
            for o, e in [(1, 1), (2, 1), (1, 2)]:
                yield a, b, o, e
                yield b, a, o, e


def test_brute_force_long_gaps(oracle_mod):
    mat = toy_matrix()
    for q, r, o, e in long_gap_cases():
        check_against_brute(oracle_mod, q, r, mat, o, e)


def test_gap_convention_equivalence(oracle_mod):
    """Cost o + e*L (the oracle's) equals o' + e*(L-1) with o' = o + e."""
    rng = random.Random(5)
    mat = toy_matrix()
    for _ in range(150):
        q = [rng.randrange(4) for _ in range(rng.randint(1, 6))]
        r = [rng.randrange(4) for _ in range(rng.randint(1, 6))]
        o, e = rng.choice([(1, 1), (3, 2), (11, 1)])
        got = oracle_mod.align_pair(np.array(q, np.uint8), np.array(r, np.uint8), mat, o, e)
        want, _ = brute_record(q, r, lambda a, b: int(mat[a, b]),
                               lambda L, o2=o + e: o2 + e * (L - 1))
        assert got == want


def test_end_and_start_belong_to_one_optimal_alignment(oracle_mod):
    """The start found by the reverse pass and the end of the forward pass are
    the two ends of a single optimal alignment (the property that makes the
    reverse pass on the reversed prefixes exact)."""
    rng = random.Random(6)
    mat = toy_matrix()
    for _ in range(200):
        q = [rng.randrange(4) for _ in range(rng.randint(1, 6))]
        r = [rng.randrange(4) for _ in range(rng.randint(1, 6))]
        rec = oracle_mod.align_pair(np.array(q, np.uint8), np.array(r, np.uint8), mat, 1, 1)
        _, opt = brute_record(q, r, lambda a, b: int(mat[a, b]), gap_linear(1, 1))
        if rec[0] > 0:
            assert (rec[1], rec[2], rec[3], rec[4]) in opt


def test_blosum62_published_statistics(oracle_mod):
    """lambda and relative entropy of the transcribed table under the Robinson
    background match the published BLAST values to 4 digits."""
    from scipy.optimize import brentq
    params, freq = {}, {}
    for line in open(os.path.join(GOLDEN, "blosum62_karlin_altschul.txt")):
        if line.startswith("#") or not line.strip():
            continue
        kind, k, v = line.split()
        (params if kind == "param" else freq)[k] = float(v)
    alpha = oracle_mod.ALPHABET
    idx = [alpha.index(c) for c in STD20]
    s = oracle_mod.blosum62().astype(np.float64)[np.ix_(idx, idx)]
    p = np.array([freq[c] for c in STD20])
    f = lambda lam: float((p[:, None] * p[None, :] * np.exp(lam * s)).sum() - 1.0)
    lam = brentq(f, 1e-3, 2.0)
    qab = p[:, None] * p[None, :] * np.exp(lam * s)
    ent = lam * float((qab * s).sum())
    assert abs(lam - params["lambda"]) < 1e-4
    assert abs(ent - params["entropy"]) < 1e-4


def test_blosum62_shape_facts(oracle_mod):
    m = oracle_mod.blosum62().astype(int)
    assert (m == m.T).all()
    star = oracle_mod.ALPHABET.index("*")
    assert m[star, star] == 1
    assert (np.delete(m[star], star) == -4).all()
    w = oracle_mod.ALPHABET.index("W")
    assert m.max() == 11 == m[w, w]


def test_blosum62_ambiguity_rows(oracle_mod):
    """The B, Z and X rows of the NCBI BLOSUM62 file (the 24-letter table BLAST
    distributes with B = N or D, Z = Q or E, X = any, * = stop), pinned by what
    their construction fixes rather than by a second transcription.

    B and Z are log-odds rows of pooled letters: the pooled ratio
    (q_Nx + q_Dx) / ((p_N + p_D) p_x) is a weighted mean of the ratios of N and
    D, so before rounding s(B, x) lies between s(N, x) and s(D, x), and half-bit
    rounding is monotone, so the published integers do too (B against B, Z
    and Z against Z pool four cells each).  X is the score of an unknown
    residue: the published row is within one unit of the background-expected
    score sum_y p_y s(y, x) of each standard letter (Robinson & Robinson
    frequencies; the NCBI table was built with the BLOCKS background, so the
    rounding can differ by one), and -1 against itself and the ambiguity
    codes."""
    a = oracle_mod.ALPHABET
    m = oracle_mod.blosum62().astype(int)
    ix = {c: a.index(c) for c in a}
    std = [ix[c] for c in STD20]

    def between(v, xs):
        return min(xs) <= v <= max(xs)

    for amb, (u, w) in (("B", ("N", "D")), ("Z", ("Q", "E"))):
        for x in std:
            assert between(m[ix[amb], x], (m[ix[u], x], m[ix[w], x])), (amb, a[x])
        assert between(m[ix[amb], ix[amb]], [m[ix[s], ix[t]] for s in (u, w) for t in (u, w)])
    assert between(m[ix["B"], ix["Z"]], [m[ix[s], ix[t]] for s in "ND" for t in "QE"])
    freq = {}
    for line in open(os.path.join(GOLDEN, "blosum62_karlin_altschul.txt")):
        if line.startswith("freq"):
            _, k, v = line.split()
            freq[k] = float(v)
    p = np.array([freq[c] for c in STD20])
    p /= p.sum()
    expected = p @ m[np.ix_(std, std)]
    got = m[ix["X"], std]
    assert (np.abs(got - expected) < 1.0).all(), (got, np.round(expected, 2))
    assert (np.abs(got - np.round(expected)) <= 1).all()
    assert m[ix["X"], ix["X"]] == m[ix["X"], ix["B"]] == m[ix["X"], ix["Z"]] == -1
    # the stop code: the table's minimum against everything, +1 against itself
    assert m[ix["*"], ix["*"]] == 1 and (np.delete(m[ix["*"]], ix["*"]) == m.min()).all()


def test_self_alignment_closed_form(oracle_mod):
    """In the 20 x 20 standard block every off-diagonal entry is below both
    diagonal entries of its row and column, so a sequence aligned to itself
    has the full diagonal as its unique optimum: S = sum of s(q_i, q_i) and
    the span is the whole sequence (lengths past 2978 exceed 11 * n > 32767)."""
    m = oracle_mod.blosum62().astype(int)
    idx = [oracle_mod.ALPHABET.index(c) for c in STD20]
    sub = m[np.ix_(idx, idx)]
    diag = np.diag(sub)
    off_diag = ~np.eye(20, dtype=bool)
    assert (sub[off_diag] < np.minimum.outer(diag, diag)[off_diag]).all()
    rng = np.random.default_rng(7)
    for n in [1, 2, 3, 17, 250, 1000, 2979, 5000]:
        q = rng.choice(np.array(idx, np.uint8), size=n)
        got = oracle_mod.align_pair(q, q, m.astype(np.int8), 11, 1)
        assert got == (int(m[q, q].sum()), 0, n - 1, 0, n - 1)


def test_homopolymers(oracle_mod):
    a = oracle_mod.ALPHABET.index("A")
    for n in range(1, 9):
        for k in range(1, 9):
            got = oracle_mod.align_pair(np.full(n, a, np.uint8), np.full(k, a, np.uint8))
            t = min(n, k)
            assert got == (4 * t, 0, t - 1, 0, t - 1)


def test_single_residues(oracle_mod):
    m = oracle_mod.blosum62().astype(int)
    for x in range(24):
        for y in range(24):
            got = oracle_mod.align_pair(np.array([x], np.uint8), np.array([y], np.uint8))
            if m[x, y] > 0:
                assert got == (m[x, y], 0, 0, 0, 0)
            else:
                assert got == (0, -1, -1, -1, -1)


def test_no_positive_substitution(oracle_mod):
    assert oracle_mod.align_pair("WWWWW", "PPPPPPP") == (0, -1, -1, -1, -1)
    assert oracle_mod.align_pair("", "ACDE") == (0, -1, -1, -1, -1)
    assert oracle_mod.align_pair("ACDE", "") == (0, -1, -1, -1, -1)
    assert oracle_mod.align_pair("", "") == (0, -1, -1, -1, -1)


def _mutate(rng, seq, rate):
    out = []
    for c in seq:
        u = rng.random()
        if u < rate:
            out.append(rng.randrange(20))
        elif u < rate + 0.03:
            continue
        elif u < rate + 0.06:
            out.extend([c, rng.randrange(20)])
        else:
            out.append(c)
    return out


def test_invariants_and_span_rescore(oracle_mod):
    rng = random.Random(8)
    m = oracle_mod.blosum62()
    score = lambda a, b: int(m[a, b])
    for t in range(40):
        lq = rng.randint(1, 90)
        q = [rng.randrange(20) for _ in range(lq)]
        r = _mutate(rng, q, 0.4) if t % 2 == 0 else [rng.randrange(20) for _ in range(rng.randint(1, 90))]
        if not r:
            r = [0]
        o, e = rng.choice([(11, 1), (11, 2), (10, 1)])
        rec = oracle_mod.align_pair(np.array(q, np.uint8), np.array(r, np.uint8), m, o, e)
        swp = oracle_mod.align_pair(np.array(r, np.uint8), np.array(q, np.uint8), m, o, e)
        S, qs, qe, rs, re = rec
        assert S >= 0
        assert S <= 11 * min(len(q), len(r))
        assert swp[0] == S
        if S == 0:
            assert rec == (0, -1, -1, -1, -1)
            continue
        assert 0 <= qs <= qe < len(q) and 0 <= rs <= re < len(r)
        # a zero or negative first/last column could be dropped without
        # lowering the score, giving an earlier end or a later start
        assert score(q[qe], r[re]) > 0 and score(q[qs], r[rs]) > 0
        assert global_affine(q[qs:qe + 1], r[rs:re + 1], score, o, e) == S


def test_batch_matches_single(oracle_mod):
    rng = np.random.default_rng(9)
    seqs = [rng.integers(0, 20, size=rng.integers(0, 60)).astype(np.uint8) for _ in range(30)]
    res = np.concatenate(seqs) if seqs else np.zeros(0, np.uint8)
    off = np.zeros(len(seqs) + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in seqs])
    pairs = rng.integers(0, len(seqs), size=(100, 2)).astype(np.int32)
    out = oracle_mod.align_batch(res, off, res, off, pairs, n_threads=4)
    for p in range(len(pairs)):
        assert tuple(out[p]) == oracle_mod.align_pair(seqs[pairs[p, 0]], seqs[pairs[p, 1]])
