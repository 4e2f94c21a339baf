"""Planted-mistake check of the discovery and identity pins.

Each case copies discovery_oracle.c, plants one plausible mistake, compiles
the copy on the CPU and runs a reduced battery of the pins against it; the
battery must reject every mutant and accept the unmodified source.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from brute_force import (enumerate_global, enumerate_global_columns, global_affine,
                         identity_of, preferred_alignment)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "discovery_oracle.c")

MUTANTS = {
    "repeats_counted": ("if (u == 0 || out[u - 1] != out[x]) out[u++] = out[x];", "out[u++] = out[x];"),
    "nonstandard_letters_form_kmers": ("if (s[p + t] >= STD_LETTERS) { ok = 0; break; }",
                                       "if (s[p + t] >= 24) { ok = 0; break; }"),
    "last_window_dropped": ("for (int64_t p = 0; p + k <= n; ++p) {", "for (int64_t p = 0; p + k < n; ++p) {"),
    "kmer_value_collides": ("v = v * STD_LETTERS + s[p + t];", "v = v + s[p + t];"),
    "gap_columns_uncounted": ("} else if (state == 1) {\n                ++cols;", "} else if (state == 1) {\n"),
    "mismatch_counted_identical": ("mt += q[qs + a - 1] == r[rs + b - 1];", "mt += 1;"),
    "span_gap_without_open": ("AT(E, a, b) = imax(AT(E, a, b - 1) - ge, AT(H, a, b - 1) - oe);",
                              "AT(E, a, b) = imax(AT(E, a, b - 1) - ge, AT(H, a, b - 1) - ge);"),
    # traceback preference swaps: each still traces an optimal alignment
    "gap_in_query_before_gap_in_reference": (
        "} else if (a > 0 && AT(H, a, b) == AT(F, a, b)) {\n                    state = 1;\n"
        "                } else {\n                    state = 2;\n                }",
        "} else if (b > 0 && AT(H, a, b) == AT(E, a, b)) {\n                    state = 2;\n"
        "                } else {\n                    state = 1;\n                }"),
    "query_gap_extension_before_opening": (
        "const int open = AT(F, a, b) == AT(H, a - 1, b) - oe;",
        "const int open = AT(F, a, b) != AT(F, a - 1, b) - ge;"),
    "reference_gap_extension_before_opening": (
        "const int open = AT(E, a, b) == AT(H, a, b - 1) - oe;",
        "const int open = AT(E, a, b) != AT(E, a, b - 1) - ge;"),
    "gap_before_diagonal": (
        "if (a > 0 && b > 0 &&\n                    AT(H, a, b) == AT(H, a - 1, b - 1) + mat[q[qs + a - 1] * 24 + r[rs + b - 1]]) {",
        "if (a > 0 && b > 0 && AT(H, a, b) != AT(F, a, b) && AT(H, a, b) != AT(E, a, b) &&\n"
        "                    AT(H, a, b) == AT(H, a - 1, b - 1) + mat[q[qs + a - 1] * 24 + r[rs + b - 1]]) {"),
}


def _compile(text, tmp_path, name):
    c = tmp_path / (name + ".c")
    so = tmp_path / (name + ".so")
    c.write_text(text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", str(so), str(c)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_shared_kmers.restype = ctypes.c_int64
    lib.oracle_shared_kmers.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_int]
    lib.oracle_span_identity.restype = ctypes.c_int
    lib.oracle_span_identity.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p]
    return lib


def _shared(lib, a, b):
    a = np.ascontiguousarray(a, np.uint8)
    b = np.ascontiguousarray(b, np.uint8)
    return lib.oracle_shared_kmers(a.ctypes.data, len(a), b.ctypes.data, len(b), 6)


def _identity(lib, q, r, rec, mat, go, ge):
    q = np.ascontiguousarray(q, np.uint8)
    r = np.ascontiguousarray(r, np.uint8)
    rec = np.ascontiguousarray(rec, np.int32)
    m = np.ascontiguousarray(mat, np.int8)
    mt = ctypes.c_int32()
    cols = ctypes.c_int32()
    st = lib.oracle_span_identity(q.ctypes.data, len(q), r.ctypes.data, len(r), rec.ctypes.data,
                                  m.ctypes.data, go, ge, ctypes.byref(mt), ctypes.byref(cols))
    return st, (mt.value, cols.value)


def _battery(lib, oracle_mod):
    rng = np.random.default_rng(21)
    if _shared(lib, [4] * 10, [4] * 30) != 1 or _shared(lib, [4] * 5, [4] * 50) != 0:
        return False
    s = rng.permutation(20)
    if _shared(lib, s, s) != 15 or _shared(lib, s[:9], s) != 4:
        return False
    x = list(range(6))
    if _shared(lib, x + x + x, x) != 1:
        return False
    y = list(range(12))
    if _shared(lib, y + [20] + y, y) != 7 or _shared(lib, y[:5] + [22] + y[5:10] + [22], y) != 0:
        return False
    z = y[:5] + [20] + y[5:10]
    if _shared(lib, z, z) != 0:
        return False
    for _ in range(10):
        c = list(12 + rng.permutation(8))
        a = list(rng.integers(0, 6, size=10)) + c
        b = c + list(rng.integers(6, 12, size=10))
        if _shared(lib, a, b) != 3:
            return False
    mat = oracle_mod.blosum62()
    q = rng.integers(0, 20, size=80)
    t = q.copy()
    t[40] = (t[40] + 1) % 20
    rec = oracle_mod.align_pair(q, t, mat, 11, 1)
    if _identity(lib, q, t, rec, mat, 11, 1) != (0, (79, 80)):
        return False
    A, B = rng.integers(0, 20, size=40), rng.integers(0, 20, size=40)
    q = np.concatenate([A, B])
    r = np.concatenate([A, [17, 17, 17], B])
    rec = oracle_mod.align_pair(q, r, mat, 11, 1)
    if _identity(lib, q, r, rec, mat, 11, 1) != (0, (80, 83)):
        return False
    rec = oracle_mod.align_pair(r, q, mat, 11, 1)   # the gap on the other side
    if _identity(lib, r, q, rec, mat, 11, 1) != (0, (80, 83)):
        return False
    score = lambda u, v: int(mat[u, v])
    for _ in range(60):
        q = rng.integers(0, 6, size=rng.integers(1, 7))
        r = rng.integers(0, 6, size=rng.integers(1, 7))
        rec = oracle_mod.align_pair(q, r, mat, 3, 1)
        if rec[0] == 0:
            continue
        alns = list(enumerate_global(list(q[rec[1]:rec[2] + 1]), list(r[rec[3]:rec[4] + 1]), score, 3, 1))
        best = max(a for a, _, _ in alns)
        st, got = _identity(lib, q, r, rec, mat, 3, 1)
        if st != 0 or got not in {(m_, c_) for a, m_, c_ in alns if a == best}:
            return False
    # the traceback preference, selected by brute force, on tie-rich matrices
    pm = np.full((24, 24), -1, np.int8)
    np.fill_diagonal(pm, 1)
    asym = np.random.default_rng(31).integers(-2, 3, size=(24, 24)).astype(np.int8)
    np.fill_diagonal(asym, 3)
    for m24, go, ge in ((pm, 1, 1), (pm, 2, 1), (asym, 0, 1), (asym, 1, 1), (asym, 1, 2)):
        score = lambda u, v: int(m24[u, v])
        for _ in range(300):
            q = list(rng.integers(0, 4, size=rng.integers(1, 7)))
            r = list(rng.integers(0, 4, size=rng.integers(1, 7)))
            total = global_affine(q, r, score, go, ge)
            if total == 0:
                continue
            alns = list(enumerate_global_columns(q, r, score, go, ge))
            best = max(t for t, _ in alns)
            want = identity_of(q, r, preferred_alignment([c for t, c in alns if t == best]))
            st, got = _identity(lib, q, r, (total, 0, len(q) - 1, 0, len(r) - 1), m24, go, ge)
            if st != 0 or got != want:
                return False
    return True


def test_unmodified_source_passes(tmp_path, oracle_mod):
    assert _battery(_compile(open(SRC).read(), tmp_path, "orig"), oracle_mod)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_rejected(tmp_path, oracle_mod, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert old in text, name
    assert not _battery(_compile(text.replace(old, new), tmp_path, name), oracle_mod)
