"""Seeded synthetic workloads of protein pairs.

They stand in for the paper's Metaclust input, which is not available here:
sequences over the 20 standard amino acids at background frequencies, half of
the pairs homologous (reference = query mutated by substitution weighted by
the scoring matrix, plus geometric-length indels), half unrelated.

This module holds none of the alignment arithmetic.  It builds the 16-bit
sampling tables (background letters; per-letter substitution targets b != a
with weight p_b * exp(lambda * s(a, b)), lambda solving
sum_ab p_a p_b exp(lambda s_ab) = 1), then lets the C core in
``csrc/workload_gen.c`` draw every pair from its own splitmix64 stream.

Named workloads (sizes from the benchmark definitions):

* ``plain_10k``: 10,000 pairs, lengths uniform in [50, 500];
* ``batched_2m``: 2,000,000 pairs, log-normal lengths (median 250, sigma 0.7)
  clipped to [20, 5000];

both with substitution rate 0.40 and indel rate 0.05 (mean length 3).
"""
import ctypes
import dataclasses
import os

import numpy as np

from . import build as _build

# The 24-letter code order used by every buffer in this package.
ALPHABET = "ARNDCQEGHILKMFPSTWYVBZX*"

# Background amino-acid frequencies (Robinson & Robinson, PNAS 88:8880, 1991),
# for the 20 standard letters; codes 0..19 of ALPHABET.
ROBINSON_FREQ = {
    "A": 0.07805, "C": 0.01925, "D": 0.05364, "E": 0.06295, "F": 0.03856,
    "G": 0.07377, "H": 0.02199, "I": 0.05142, "K": 0.05744, "L": 0.09019,
    "M": 0.02243, "N": 0.04487, "P": 0.05203, "Q": 0.04264, "R": 0.05129,
    "S": 0.07120, "T": 0.05841, "V": 0.06441, "W": 0.01330, "Y": 0.03216,
}


class _Params(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int64), ("n_homologous", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("length_model", ctypes.c_int32),
                ("lmin", ctypes.c_int32), ("lmax", ctypes.c_int32),
                ("median", ctypes.c_double), ("sigma", ctypes.c_double),
                ("subst_rate", ctypes.c_double), ("indel_rate", ctypes.c_double),
                ("indel_mean", ctypes.c_double)]


@dataclasses.dataclass
class Spec:
    """What to draw.  ``length_model`` is "uniform" or "lognormal"."""
    name: str
    n_pairs: int
    length_model: str
    lmin: int
    lmax: int
    median: float = 0.0
    sigma: float = 0.0
    homologous_fraction: float = 0.5
    subst_rate: float = 0.40
    indel_rate: float = 0.05
    indel_mean: float = 3.0
    seed: int = 1


SPECS = {
    "plain_10k": Spec("plain_10k", 10_000, "uniform", 50, 500),
    "batched_2m": Spec("batched_2m", 2_000_000, "lognormal", 20, 5000, median=250.0, sigma=0.7),
}


@dataclasses.dataclass
class FamilySpec:
    """A sequence set of ``n_families`` x ``copies`` sequences: each family's
    root has a drawn length, every copy is mutate(root)."""
    name: str
    n_families: int
    copies: int
    length_model: str
    lmin: int
    lmax: int
    median: float = 0.0
    sigma: float = 0.0
    subst_rate: float = 0.40
    indel_rate: float = 0.05
    indel_mean: float = 3.0
    seed: int = 3


FAMILY_SPECS = {
    # the many-against-many block: 200,000 sequences in 20,000 families of 10
    "families_200k": FamilySpec("families_200k", 20_000, 10, "lognormal", 20, 5000,
                                median=250.0, sigma=0.7),
    # the same recipe at a size the all-pairs oracle finishes in seconds
    "families_2k": FamilySpec("families_2k", 200, 10, "lognormal", 20, 5000,
                              median=250.0, sigma=0.7),
}


@dataclasses.dataclass
class SequenceSet:
    """Concatenated residue codes with offsets, and each sequence's family."""
    spec: FamilySpec
    res: np.ndarray     # uint8 codes
    off: np.ndarray     # int64 [n + 1]
    family: np.ndarray  # int32 [n]

    @property
    def lengths(self):
        return np.diff(self.off)

    def __len__(self):
        return len(self.off) - 1

    def seq(self, i):
        return self.res[self.off[i]:self.off[i + 1]]


@dataclasses.dataclass
class Workload:
    """Concatenated residue codes with offsets; pair p = (query p, reference p)."""
    spec: Spec
    q_res: np.ndarray   # uint8 codes
    q_off: np.ndarray   # int64 [n + 1]
    r_res: np.ndarray
    r_off: np.ndarray
    pairs: np.ndarray   # int32 [P, 2]

    @property
    def q_len(self):
        return np.diff(self.q_off)

    @property
    def r_len(self):
        return np.diff(self.r_off)

    def cells(self):
        """Forward-pass cells sum(lq * lr) over the pairs."""
        ql = self.q_len[self.pairs[:, 0]].astype(np.int64)
        rl = self.r_len[self.pairs[:, 1]].astype(np.int64)
        return int((ql * rl).sum())

    def subset(self, idx):
        """The same sequences with only pairs[idx]."""
        return dataclasses.replace(self, pairs=np.ascontiguousarray(self.pairs[idx]))


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build_workload())
        vp = ctypes.c_void_p
        lib.wl_lengths.argtypes = [ctypes.POINTER(_Params), vp, vp, vp, vp, ctypes.c_int]
        lib.wl_lengths.restype = ctypes.c_int
        lib.wl_fill.argtypes = [ctypes.POINTER(_Params), vp, vp, vp, vp, vp, vp, ctypes.c_int]
        lib.wl_fill.restype = ctypes.c_int
        lib.wl_family_lengths.argtypes = [ctypes.POINTER(_Params), ctypes.c_int64, vp, vp, vp, ctypes.c_int]
        lib.wl_family_lengths.restype = ctypes.c_int
        lib.wl_family_fill.argtypes = [ctypes.POINTER(_Params), ctypes.c_int64, vp, vp, vp, vp, ctypes.c_int]
        lib.wl_family_fill.restype = ctypes.c_int
        _lib = lib
    return _lib


def background():
    """Background probabilities of codes 0..19."""
    p = np.array([ROBINSON_FREQ[c] for c in ALPHABET[:20]], dtype=np.float64)
    return p / p.sum()


def solve_lambda(mat, p):
    """lambda > 0 with sum_ab p_a p_b exp(lambda s_ab) = 1 (bisection)."""
    s = np.asarray(mat, dtype=np.float64)[:20, :20]
    pp = p[:, None] * p[None, :]
    f = lambda lam: float((pp * np.exp(lam * s)).sum() - 1.0)
    lo, hi = 1e-6, 1.0
    while f(hi) < 0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _table16(prob):
    """65536-entry inverse-CDF table: entry k = letter whose CDF bin holds
    (k + 0.5) / 65536."""
    cdf = np.cumsum(prob / prob.sum())
    u = (np.arange(65536, dtype=np.float64) + 0.5) / 65536.0
    return np.minimum(np.searchsorted(cdf, u, side="right"), len(prob) - 1).astype(np.uint8)


def sampling_tables(mat):
    """(background table [65536], substitution tables [20, 65536])."""
    p = background()
    lam = solve_lambda(mat, p)
    s = np.asarray(mat, dtype=np.float64)[:20, :20]
    sub = np.zeros((20, 65536), dtype=np.uint8)
    for a in range(20):
        w = p * np.exp(lam * s[a])
        w[a] = 0.0
        sub[a] = _table16(w)
    return _table16(p), np.ascontiguousarray(sub)


def generate(spec, mat, n_threads=None):
    """Draws the workload ``spec`` (a Spec or a name in SPECS).

    ``mat`` is the 24 x 24 substitution matrix that weights substitutions.
    """
    if isinstance(spec, str):
        spec = SPECS[spec]
    lib = _load()
    bg, sub = sampling_tables(mat)
    P = _Params(n_pairs=spec.n_pairs,
                n_homologous=int(round(spec.homologous_fraction * spec.n_pairs)),
                seed=spec.seed & 0xFFFFFFFFFFFFFFFF,
                length_model=0 if spec.length_model == "uniform" else 1,
                lmin=spec.lmin, lmax=spec.lmax, median=spec.median, sigma=spec.sigma,
                subst_rate=spec.subst_rate, indel_rate=spec.indel_rate,
                indel_mean=spec.indel_mean)
    n = spec.n_pairs
    threads = n_threads or min(os.cpu_count() or 1, 64)
    q_len = np.zeros(n, np.int64)
    r_len = np.zeros(n, np.int64)
    st = lib.wl_lengths(ctypes.byref(P), bg.ctypes.data, sub.ctypes.data,
                        q_len.ctypes.data, r_len.ctypes.data, threads)
    if st:
        raise RuntimeError("workload length pass failed: %d" % st)
    q_off = np.zeros(n + 1, np.int64)
    r_off = np.zeros(n + 1, np.int64)
    np.cumsum(q_len, out=q_off[1:])
    np.cumsum(r_len, out=r_off[1:])
    q_res = np.empty(int(q_off[-1]), np.uint8)
    r_res = np.empty(int(r_off[-1]), np.uint8)
    st = lib.wl_fill(ctypes.byref(P), bg.ctypes.data, sub.ctypes.data, q_off.ctypes.data,
                     r_off.ctypes.data, q_res.ctypes.data, r_res.ctypes.data, threads)
    if st:
        raise RuntimeError("workload fill pass failed: %d" % st)
    idx = np.arange(n, dtype=np.int32)
    pairs = np.ascontiguousarray(np.stack([idx, idx], axis=1))
    return Workload(spec, q_res, q_off, r_res, r_off, pairs)


def from_sequences(queries, references, pairs):
    """Workload from lists of code arrays and an explicit pair list."""
    def pack(seqs):
        lens = np.array([len(s) for s in seqs], dtype=np.int64)
        off = np.zeros(len(seqs) + 1, np.int64)
        np.cumsum(lens, out=off[1:])
        res = (np.concatenate([np.asarray(s, np.uint8) for s in seqs])
               if len(seqs) and off[-1] > 0 else np.zeros(0, np.uint8))
        return res, off
    q_res, q_off = pack(queries)
    r_res, r_off = pack(references)
    spec = Spec("explicit", len(pairs), "uniform", 0, 0)
    return Workload(spec, q_res, q_off, r_res, r_off,
                    np.ascontiguousarray(np.asarray(pairs, np.int32).reshape(-1, 2)))


def generate_families(spec, mat, n_threads=None):
    """Draws the family set ``spec`` (a FamilySpec or a name in FAMILY_SPECS)."""
    if isinstance(spec, str):
        spec = FAMILY_SPECS[spec]
    lib = _load()
    bg, sub = sampling_tables(mat)
    P = _Params(n_pairs=spec.n_families, n_homologous=0, seed=spec.seed & 0xFFFFFFFFFFFFFFFF,
                length_model=0 if spec.length_model == "uniform" else 1,
                lmin=spec.lmin, lmax=spec.lmax, median=spec.median, sigma=spec.sigma,
                subst_rate=spec.subst_rate, indel_rate=spec.indel_rate,
                indel_mean=spec.indel_mean)
    n = spec.n_families * spec.copies
    threads = n_threads or min(os.cpu_count() or 1, 64)
    lengths = np.zeros(n, np.int64)
    st = lib.wl_family_lengths(ctypes.byref(P), spec.copies, bg.ctypes.data, sub.ctypes.data,
                               lengths.ctypes.data, threads)
    if st:
        raise RuntimeError("family length pass failed: %d" % st)
    off = np.zeros(n + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    res = np.empty(int(off[-1]), np.uint8)
    st = lib.wl_family_fill(ctypes.byref(P), spec.copies, bg.ctypes.data, sub.ctypes.data,
                            off.ctypes.data, res.ctypes.data, threads)
    if st:
        raise RuntimeError("family fill pass failed: %d" % st)
    family = (np.arange(n, dtype=np.int64) // spec.copies).astype(np.int32)
    return SequenceSet(spec, res, off, family)
