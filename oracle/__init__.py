"""CPU oracle for batched Smith-Waterman with affine gaps, candidate
discovery by shared k-mers, alignment identity, and the learned candidate
filter (pair features here; the network in ``mlp_oracle``).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this package; the product path never
does, and the oracle imports nothing from the product.

The arithmetic lives in ``sw_oracle.c`` (plain int32 Gotoh, forward pass for
score and end, reverse pass on the reversed prefixes for the start) and
``discovery_oracle.c`` (distinct k-mer sets intersected by merging; global
Gotoh of an alignment's span traced back for its identity) and
``filter_oracle.c`` (the 32 features of a candidate pair); this module only
marshals arguments through ctypes.  Conventions (the paper states
none of them):

* rows are query residues, columns reference residues;
* a gap of length L costs ``gap_open + gap_extend * L``;
* the end is the row-major-first cell holding the maximum score;
* the start is the row-major-first cell holding that score in the local DP of
  the reversed prefixes q[q_end..0], r[r_end..0];
* coordinates are 0-based and inclusive; a zero score reports -1 for all four.
"""
import ctypes
import os

import numpy as np

from . import build as _build

ALPHABET = "ARNDCQEGHILKMFPSTWYVBZX*"
RECORD_DTYPE = np.dtype([("score", np.int32), ("q_start", np.int32),
                         ("q_end", np.int32), ("r_start", np.int32),
                         ("r_end", np.int32)])

_lib = None


def load():
    """Builds (if needed) and loads liboracle.so."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    lib = ctypes.CDLL(path)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i8p = ctypes.POINTER(ctypes.c_int8)
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_blosum62.argtypes = [i8p]
    lib.oracle_blosum62.restype = None
    lib.oracle_align_pair.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, i8p,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    lib.oracle_align_pair.restype = ctypes.c_int
    lib.oracle_forward_pair.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, i8p,
                                        ctypes.c_int32, ctypes.c_int32, i32p, i64p, i64p]
    lib.oracle_forward_pair.restype = ctypes.c_int
    lib.oracle_align_batch.argtypes = [u8p, i64p, u8p, i64p, i32p, ctypes.c_int64, i8p,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_int]
    lib.oracle_align_batch.restype = ctypes.c_int
    vp = ctypes.c_void_p
    lib.oracle_shared_kmers.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, ctypes.c_int]
    lib.oracle_shared_kmers.restype = ctypes.c_int64
    lib.oracle_kmer_index.argtypes = [u8p, i64p, ctypes.c_int64, ctypes.c_int]
    lib.oracle_kmer_index.restype = vp
    lib.oracle_kmer_index_free.argtypes = [vp]
    lib.oracle_kmer_index_free.restype = None
    lib.oracle_candidates_of.argtypes = [vp, ctypes.c_int64, ctypes.c_int, i32p, i32p, ctypes.c_int64]
    lib.oracle_candidates_of.restype = ctypes.c_int64
    lib.oracle_all_candidates.argtypes = [vp, ctypes.c_int, i32p, i32p, ctypes.c_int64, ctypes.c_int]
    lib.oracle_all_candidates.restype = ctypes.c_int64
    lib.oracle_span_identity.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, i32p, i8p,
                                         ctypes.c_int32, ctypes.c_int32, i32p, i32p]
    lib.oracle_span_identity.restype = ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    lib.oracle_pair_features.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, ctypes.c_int, fp]
    lib.oracle_pair_features.restype = ctypes.c_int
    lib.oracle_pair_features_batch.argtypes = [u8p, i64p, u8p, i64p, i32p, ctypes.c_int64,
                                               ctypes.c_int, fp]
    lib.oracle_pair_features_batch.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def blosum62():
    """The oracle's own BLOSUM62 transcription, int8 [24, 24] (row = query)."""
    out = np.zeros((24, 24), dtype=np.int8)
    load().oracle_blosum62(_ptr(out, ctypes.c_int8))
    return out


def encode(text):
    """ASCII protein string -> uint8 codes in ALPHABET order (upper case only)."""
    return np.array([ALPHABET.index(c) for c in text], dtype=np.uint8)


def _codes(x):
    if isinstance(x, str):
        return encode(x)
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint8))


def _matrix(mat):
    m = np.ascontiguousarray(np.asarray(mat, dtype=np.int8))
    if m.shape != (24, 24):
        raise ValueError("matrix must be 24 x 24")
    return m


def align_pair(q, r, mat=None, gap_open=11, gap_extend=1):
    """One pair -> (score, q_start, q_end, r_start, r_end)."""
    lib = load()
    qc, rc = _codes(q), _codes(r)
    m = _matrix(blosum62() if mat is None else mat)
    rec = np.zeros(1, dtype=RECORD_DTYPE)
    st = lib.oracle_align_pair(_ptr(qc, ctypes.c_uint8), len(qc), _ptr(rc, ctypes.c_uint8),
                               len(rc), _ptr(m, ctypes.c_int8), gap_open, gap_extend,
                               rec.ctypes.data)
    if st != 0:
        raise RuntimeError("oracle_align_pair failed: %d" % st)
    return tuple(int(v) for v in rec[0])


def forward_pair(q, r, mat=None, gap_open=11, gap_extend=1):
    """Forward pass only -> (score, q_end, r_end)."""
    lib = load()
    qc, rc = _codes(q), _codes(r)
    m = _matrix(blosum62() if mat is None else mat)
    s = ctypes.c_int32()
    qe = ctypes.c_int64()
    re_ = ctypes.c_int64()
    st = lib.oracle_forward_pair(_ptr(qc, ctypes.c_uint8), len(qc), _ptr(rc, ctypes.c_uint8),
                                 len(rc), _ptr(m, ctypes.c_int8), gap_open, gap_extend,
                                 ctypes.byref(s), ctypes.byref(qe), ctypes.byref(re_))
    if st != 0:
        raise RuntimeError("oracle_forward_pair failed: %d" % st)
    return s.value, qe.value, re_.value


def align_batch(q_res, q_off, r_res, r_off, pairs, mat=None, gap_open=11, gap_extend=1,
                n_threads=None):
    """Aligns pairs[p] = (q index, r index) over concatenated code buffers.

    Returns an int32 array [P, 5] of (score, q_start, q_end, r_start, r_end).
    """
    lib = load()
    q_res = np.ascontiguousarray(q_res, dtype=np.uint8)
    r_res = np.ascontiguousarray(r_res, dtype=np.uint8)
    q_off = np.ascontiguousarray(q_off, dtype=np.int64)
    r_off = np.ascontiguousarray(r_off, dtype=np.int64)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    n = pairs.shape[0]
    if n and (pairs[:, 0].min() < 0 or pairs[:, 0].max() >= len(q_off) - 1
              or pairs[:, 1].min() < 0 or pairs[:, 1].max() >= len(r_off) - 1):
        raise IndexError("pair index out of range")
    m = _matrix(blosum62() if mat is None else mat)
    out = np.zeros((n, 5), dtype=np.int32)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    st = lib.oracle_align_batch(_ptr(q_res, ctypes.c_uint8), _ptr(q_off, ctypes.c_int64),
                                _ptr(r_res, ctypes.c_uint8), _ptr(r_off, ctypes.c_int64),
                                _ptr(pairs, ctypes.c_int32), n, _ptr(m, ctypes.c_int8),
                                gap_open, gap_extend, out.ctypes.data, int(n_threads))
    if st != 0:
        raise RuntimeError("oracle_align_batch failed: %d" % st)
    return out


def shared_kmers(a, b, k=6):
    """|K(a) & K(b)|: distinct k-mers of standard letters common to a and b."""
    ac, bc = _codes(a), _codes(b)
    c = load().oracle_shared_kmers(_ptr(ac, ctypes.c_uint8), len(ac), _ptr(bc, ctypes.c_uint8),
                                   len(bc), k)
    if c < 0:
        raise ValueError("bad k or out of memory")
    return int(c)


class KmerIndex:
    """The distinct k-mer sets of every sequence of a set (res, off)."""

    def __init__(self, res, off, k=6):
        self._res = np.ascontiguousarray(res, dtype=np.uint8)
        self._off = np.ascontiguousarray(off, dtype=np.int64)
        self.n = len(self._off) - 1
        self._h = load().oracle_kmer_index(_ptr(self._res, ctypes.c_uint8),
                                           _ptr(self._off, ctypes.c_int64), self.n, k)
        if not self._h:
            raise RuntimeError("oracle_kmer_index failed")

    def close(self):
        if self._h:
            load().oracle_kmer_index_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def candidates_of(self, i, min_shared=2):
        """(js, counts): every j != i sharing >= min_shared k-mers with i."""
        lib = load()
        cap = 1024
        while True:
            js = np.zeros(cap, np.int32)
            cs = np.zeros(cap, np.int32)
            n = lib.oracle_candidates_of(self._h, int(i), min_shared, _ptr(js, ctypes.c_int32),
                                         _ptr(cs, ctypes.c_int32), cap)
            if n < 0:
                raise RuntimeError("oracle_candidates_of failed")
            if n <= cap:
                return js[:n], cs[:n]
            cap = int(n)

    def all_candidates(self, min_shared=2, n_threads=None):
        """(pairs [P, 2] with i < j ordered by (i, j), counts [P])."""
        lib = load()
        threads = n_threads or min(os.cpu_count() or 1, 64)
        cap = 1 << 16
        while True:
            pairs = np.zeros((cap, 2), np.int32)
            cs = np.zeros(cap, np.int32)
            n = lib.oracle_all_candidates(self._h, min_shared, _ptr(pairs, ctypes.c_int32),
                                          _ptr(cs, ctypes.c_int32), cap, threads)
            if n < 0:
                raise RuntimeError("oracle_all_candidates failed")
            if n <= cap:
                order = np.lexsort((pairs[:n, 1], pairs[:n, 0]))
                return pairs[:n][order], cs[:n][order]
            cap = int(n)


def span_identity(q, r, record, mat=None, gap_open=11, gap_extend=1):
    """(identical columns, columns) of the traced alignment of a record's span;
    (0, 0) for a zero score."""
    qc, rc = _codes(q), _codes(r)
    m = _matrix(blosum62() if mat is None else mat)
    rec = np.ascontiguousarray(np.asarray(record, dtype=np.int32).reshape(5))
    mt = ctypes.c_int32()
    cols = ctypes.c_int32()
    st = load().oracle_span_identity(_ptr(qc, ctypes.c_uint8), len(qc), _ptr(rc, ctypes.c_uint8),
                                     len(rc), _ptr(rec, ctypes.c_int32), _ptr(m, ctypes.c_int8),
                                     gap_open, gap_extend, ctypes.byref(mt), ctypes.byref(cols))
    if st < 0:
        raise RuntimeError("oracle_span_identity failed: %d" % st)
    return mt.value, cols.value


def passes(record, matches, columns, lq, lr, min_identity=(3, 10), min_coverage=(7, 10)):
    """Pass/fail at identity >= a/b and coverage >= c/d, decided exactly in
    integers: matches * b >= a * columns and, for both sequences,
    span * d >= c * length."""
    score, qs, qe, rs, re_ = (int(v) for v in record)
    if score <= 0 or columns <= 0:
        return False
    a, b = min_identity
    c, d = min_coverage
    return (matches * b >= a * columns and (qe - qs + 1) * d >= c * lq
            and (re_ - rs + 1) * d >= c * lr)


N_FEATURES = 32


def pair_features(a, b, k=6):
    """The 32 float32 features of the candidate pair (a, b)."""
    ac, bc = _codes(a), _codes(b)
    out = np.zeros(N_FEATURES, np.float32)
    rc = load().oracle_pair_features(_ptr(ac, ctypes.c_uint8), len(ac), _ptr(bc, ctypes.c_uint8),
                                     len(bc), k, _ptr(out, ctypes.c_float))
    if rc:
        raise ValueError("bad k or out of memory")
    return out


def pair_features_batch(res_a, off_a, res_b, off_b, pairs, k=6):
    """Features of pairs[p] = (index into set a, index into set b): float32 [P, 32]."""
    res_a = np.ascontiguousarray(res_a, dtype=np.uint8)
    res_b = np.ascontiguousarray(res_b, dtype=np.uint8)
    off_a = np.ascontiguousarray(off_a, dtype=np.int64)
    off_b = np.ascontiguousarray(off_b, dtype=np.int64)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    out = np.zeros((len(pairs), N_FEATURES), np.float32)
    rc = load().oracle_pair_features_batch(_ptr(res_a, ctypes.c_uint8), _ptr(off_a, ctypes.c_int64),
                                           _ptr(res_b, ctypes.c_uint8), _ptr(off_b, ctypes.c_int64),
                                           _ptr(pairs, ctypes.c_int32), len(pairs), k,
                                           _ptr(out, ctypes.c_float))
    if rc:
        raise ValueError("bad k or out of memory")
    return out
