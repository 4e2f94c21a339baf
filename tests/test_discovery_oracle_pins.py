"""Pins of the discovery and identity oracle (CPU only).

Shared k-mers: closed forms (homopolymers, distinct-letter sequences, a
common block between sequences over disjoint alphabets, repeats counted once,
k-mers broken by non-standard letters), symmetry, and the one-vs-all and
all-pairs entry points agreeing with each other.  Identity: identical and
singly-substituted sequences, a planted gap of known length, and, on tiny
inputs, exhaustive enumeration of global alignments: the traced alignment
must be optimal (its score is the record's), and its (identical columns,
columns) must be exactly those of the one optimal alignment that the stated
traceback preference selects, the selection made by brute force over the
enumerated alignments (tests/brute_force.py), on tie-rich matrices.
"""
import itertools

import numpy as np
import pytest

from brute_force import (enumerate_global, enumerate_global_columns, global_affine,
                         identity_of, preferred_alignment)

K = 6


def codes(seq):
    return np.asarray(seq, dtype=np.uint8)


def test_homopolymers_have_one_kmer(oracle_mod):
    for n, m in [(6, 6), (10, 30), (6, 100)]:
        assert oracle_mod.shared_kmers(codes([4] * n), codes([4] * m), K) == 1
    assert oracle_mod.shared_kmers(codes([4] * 5), codes([4] * 50), K) == 0
    assert oracle_mod.shared_kmers(codes([4] * 10), codes([5] * 10), K) == 0


def test_distinct_letter_sequence_shares_every_window(oracle_mod):
    rng = np.random.default_rng(1)
    for L in [6, 7, 13, 20]:
        s = codes(rng.permutation(20)[:L])
        assert oracle_mod.shared_kmers(s, s, K) == L - K + 1
        # a prefix of length P shares exactly its own P - K + 1 windows
        for P in range(K, L + 1):
            assert oracle_mod.shared_kmers(s[:P], s, K) == P - K + 1


def test_common_block_between_disjoint_alphabets(oracle_mod):
    """a over letters 0..5, b over 6..11, both containing the block c of 8
    distinct letters 12..19: every common 6-mer lies inside c (a junction
    k-mer holds a letter of one side only), so exactly 8 - 6 + 1 = 3."""
    rng = np.random.default_rng(2)
    for trial in range(20):
        c = list(12 + rng.permutation(8))
        a = list(rng.integers(0, 6, size=rng.integers(0, 30))) + c + list(rng.integers(0, 6, size=rng.integers(0, 30)))
        b = list(rng.integers(6, 12, size=rng.integers(0, 30))) + c + list(rng.integers(6, 12, size=rng.integers(0, 30)))
        assert oracle_mod.shared_kmers(codes(a), codes(b), K) == 3
        assert oracle_mod.shared_kmers(codes(b), codes(a), K) == 3


def test_repeats_count_once_and_nonstandard_letters_break_kmers(oracle_mod):
    x = list(range(6))
    assert oracle_mod.shared_kmers(codes(x + x + x), codes(x), K) == 1
    # X (code 22) inside every window of the second sequence: nothing formed
    y = list(range(12))
    broken = y[:5] + [22] + y[5:10] + [22]
    assert oracle_mod.shared_kmers(codes(y), codes(broken), K) == 0
    # B, Z, X, * each break k-mers; the standard-letter windows still count
    assert oracle_mod.shared_kmers(codes(y + [20] + y), codes(y), K) == 7
    for bad in (20, 21, 22, 23):
        z = codes(y[:5] + [bad] + y[5:10])
        assert oracle_mod.shared_kmers(z, z, K) == 0


def test_candidates_agree_between_entry_points(oracle_mod):
    rng = np.random.default_rng(3)
    seqs = []
    for f in range(40):   # families of 4 near-copies plus unrelated sequences
        root = rng.integers(0, 20, size=rng.integers(8, 60))
        for c in range(4):
            s = root.copy()
            flip = rng.random(len(s)) < 0.15
            s[flip] = rng.integers(0, 20, size=int(flip.sum()))
            seqs.append(s)
    for _ in range(40):
        seqs.append(rng.integers(0, 20, size=rng.integers(1, 60)))
    off = np.zeros(len(seqs) + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in seqs])
    res = np.concatenate(seqs).astype(np.uint8)
    ix = oracle_mod.KmerIndex(res, off, K)
    pairs, counts = ix.all_candidates(2, n_threads=3)
    assert len(pairs) > 20
    got = {(int(i), int(j)): int(c) for (i, j), c in zip(pairs, counts)}
    assert all(i < j for i, j in got)
    want = {}
    for i in range(len(seqs)):
        js, cs = ix.candidates_of(i, 2)
        for j, c in zip(js, cs):
            assert oracle_mod.shared_kmers(seqs[i], seqs[int(j)], K) == c
            if i < j:
                want[(i, int(j))] = int(c)
    assert got == want
    ix.close()


def test_identity_of_identical_and_substituted_sequences(oracle_mod):
    mat = oracle_mod.blosum62()
    rng = np.random.default_rng(4)
    s = codes(rng.integers(0, 20, size=120))
    rec = oracle_mod.align_pair(s, s, mat, 11, 1)
    assert rec == (int(mat[s, s].sum()), 0, 119, 0, 119)
    assert oracle_mod.span_identity(s, s, rec, mat, 11, 1) == (120, 120)
    t = s.copy()
    t[60] = (t[60] + 1) % 20
    rec = oracle_mod.align_pair(s, t, mat, 11, 1)
    assert rec[1:] == (0, 119, 0, 119)
    assert oracle_mod.span_identity(s, t, rec, mat, 11, 1) == (119, 120)


def test_identity_of_a_planted_gap(oracle_mod):
    """q = A + B, r = A + 3 tryptophans + B with A, B identical 40-mers: the
    optimum keeps both blocks and opens one 3-long gap, so 80 identical
    columns out of 83, score = diag(A) + diag(B) - (11 + 3)."""
    mat = oracle_mod.blosum62()
    rng = np.random.default_rng(5)
    for trial in range(10):
        A = rng.integers(0, 20, size=40)
        B = rng.integers(0, 20, size=40)
        q = codes(np.concatenate([A, B]))
        r = codes(np.concatenate([A, [17, 17, 17], B]))
        rec = oracle_mod.align_pair(q, r, mat, 11, 1)
        assert rec == (int(mat[A, A].sum() + mat[B, B].sum()) - 14, 0, 79, 0, 82)
        assert oracle_mod.span_identity(q, r, rec, mat, 11, 1) == (80, 83)
        # the same gap with the roles swapped: query residues against gaps
        rec = oracle_mod.align_pair(r, q, mat, 11, 1)
        assert rec == (int(mat[A, A].sum() + mat[B, B].sum()) - 14, 0, 82, 0, 79)
        assert oracle_mod.span_identity(r, q, rec, mat, 11, 1) == (80, 83)


@pytest.mark.parametrize("go,ge", [(11, 1), (3, 1), (0, 1), (2, 2)])
def test_identity_is_that_of_an_optimal_alignment(oracle_mod, go, ge):
    mat = oracle_mod.blosum62()
    score = lambda a, b: int(mat[a, b])
    rng = np.random.default_rng(6 + go)
    checked = 0
    for trial in range(300):
        q = codes(rng.integers(0, 6, size=rng.integers(1, 7)))
        r = codes(rng.integers(0, 6, size=rng.integers(1, 7)))
        rec = oracle_mod.align_pair(q, r, mat, go, ge)
        if rec[0] == 0:
            assert oracle_mod.span_identity(q, r, rec, mat, go, ge) == (0, 0)
            continue
        qs, qe, rs, re_ = rec[1:]
        span_q, span_r = list(q[qs:qe + 1]), list(r[rs:re_ + 1])
        alns = list(enumerate_global(span_q, span_r, score, go, ge))
        best = max(t for t, _, _ in alns)
        assert best == rec[0]
        optimal = {(same, cols) for t, same, cols in alns if t == best}
        assert oracle_mod.span_identity(q, r, rec, mat, go, ge) in optimal
        checked += 1
    assert checked > 100


def test_pass_fail_is_decided_exactly(oracle_mod):
    # identity exactly 3/10 and coverage exactly 7/10 pass; one less fails
    assert oracle_mod.passes((5, 0, 6, 0, 6), 3, 10, 10, 10)
    assert not oracle_mod.passes((5, 0, 6, 0, 6), 2, 10, 10, 10)
    assert not oracle_mod.passes((5, 0, 5, 0, 6), 3, 10, 10, 10)
    assert not oracle_mod.passes((5, 0, 6, 0, 5), 3, 10, 10, 10)
    assert not oracle_mod.passes((0, -1, -1, -1, -1), 0, 0, 10, 10)


def tie_rich_matrices():
    """24 x 24 int8 matrices on which many alignments tie: +1 / -1 over four
    letters, and a small asymmetric one."""
    pm = np.full((24, 24), -1, np.int8)
    np.fill_diagonal(pm, 1)
    rng = np.random.default_rng(31)
    asym = rng.integers(-2, 3, size=(24, 24)).astype(np.int8)
    np.fill_diagonal(asym, 3)
    return {"plus_minus_one": pm, "asymmetric": asym}


@pytest.mark.parametrize("name", ["plus_minus_one", "asymmetric"])
@pytest.mark.parametrize("go,ge", [(0, 1), (1, 1), (2, 1), (3, 2), (11, 1)])
def test_identity_follows_the_stated_traceback_preference(oracle_mod, name, go, ge):
    """Equality, not membership: over every global alignment of the whole
    (tiny) span, the preference -- diagonal, then a query residue against a
    gap, then a gap in the query, and a gap run opened as late as possible
    walking back -- selects one alignment; the oracle's (identical columns,
    columns) must be that alignment's."""
    mat = tie_rich_matrices()[name]
    score = lambda a, b: int(mat[a, b])
    rng = np.random.default_rng(100 * go + ge + len(name))
    checked = differ = 0
    for trial in range(400):
        q = codes(rng.integers(0, 4, size=rng.integers(1, 6)))
        r = codes(rng.integers(0, 4, size=rng.integers(1, 6)))
        total = global_affine(list(q), list(r), score, go, ge)
        if total == 0:
            continue   # a zero score is reported as no alignment
        alns = list(enumerate_global_columns(list(q), list(r), score, go, ge))
        best = max(t for t, _ in alns)
        assert best == total
        optimal = [c for t, c in alns if t == best]
        want = identity_of(list(q), list(r), preferred_alignment(optimal))
        rec = (total, 0, len(q) - 1, 0, len(r) - 1)
        assert oracle_mod.span_identity(q, r, rec, mat, go, ge) == want, (q, r, optimal)
        checked += 1
        differ += len({identity_of(list(q), list(r), c) for c in optimal}) > 1
    # the draw must hold many spans whose optimal alignments disagree
    assert checked > 250, checked
    if go <= 2:
        # small gap costs: many spans whose optimal alignments disagree
        assert differ > 3, differ
