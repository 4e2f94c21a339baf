"""Planted-mistake check of the oracle pins.

Each case copies the oracle source, plants one plausible mistake (a dropped
term, a wrong sign, index or operand, a wrong tie-break), compiles the copy on
the CPU and runs a reduced battery of the pins against it.  The battery must
reject every mutant, and accept the unmodified source.
"""
import ctypes
import os
import random
import subprocess

import numpy as np
import pytest

from brute_force import brute_record
from test_oracle_pins import long_gap_cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sw_oracle.c")

MUTANTS = {
    "no_zero_floor": ("max2(max2(0, D), max2(E, F))", "max2(D, max2(E, F))"),
    "E_open_without_extend": ("Hcur[j - 1] - go - ge", "Hcur[j - 1] - go"),
    "F_open_without_extend": ("Hprev[j] - go - ge", "Hprev[j] - go"),
    "E_no_extension_cost": ("max2(E - ge,", "max2(E,"),
    "transposed_matrix": ("mat[a[i - 1] * ORACLE_ALPHA + b[j - 1]]",
                          "mat[b[j - 1] * ORACLE_ALPHA + a[i - 1]]"),
    "diagonal_from_above": ("Hprev[j - 1] + (int32_t)", "Hprev[j] + (int32_t)"),
    "F_from_diagonal": ("Hprev[j] - go - ge", "Hprev[j - 1] - go - ge"),
    "last_cell_tie_break": ("if (H > best)", "if (H >= best)"),
    "start_wrong_axis": ("out->q_start = (int32_t)(qe - a);", "out->q_start = (int32_t)(qe - b);"),
    "start_not_reversed": ("qrev[k] = q[qe - k];", "qrev[k] = q[k];"),
}


def _compile(src_text, tmp_path, name):
    c = tmp_path / (name + ".c")
    so = tmp_path / (name + ".so")
    c.write_text(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", str(so), str(c)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_align_pair.restype = ctypes.c_int
    lib.oracle_align_pair.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_void_p]
    return lib


def _align(lib, q, r, mat, o, e):
    q = np.array(q, np.uint8)
    r = np.array(r, np.uint8)
    m = np.ascontiguousarray(mat, np.int8)
    rec = np.zeros(5, np.int32)
    lib.oracle_align_pair(q.ctypes.data, len(q), r.ctypes.data, len(r), m.ctypes.data,
                          o, e, rec.ctypes.data)
    return tuple(int(v) for v in rec)


def _battery(lib, blosum):
    """True if every reduced pin holds."""
    toy = np.full((24, 24), -3, np.int8)
    toy[:4, :4] = [[3, -1, -2, 1], [-2, 4, 0, -1], [1, -3, 2, -2], [0, 2, -1, 5]]
    rng = random.Random(11)
    for _ in range(150):
        q = [rng.randrange(4) for _ in range(rng.randint(1, 5))]
        r = [rng.randrange(4) for _ in range(rng.randint(1, 5))]
        o, e = rng.choice([(1, 1), (2, 1), (3, 2)])
        want, _ = brute_record(q, r, lambda a, b: int(toy[a, b]), lambda L: o + e * L)
        if _align(lib, q, r, toy, o, e) != want:
            return False
    for q, r, o, e in long_gap_cases():
        want, _ = brute_record(q, r, lambda a, b: int(toy[a, b]), lambda L: o + e * L)
        if _align(lib, q, r, toy, o, e) != want:
            return False
    a = 0
    for n in range(1, 6):
        for k in range(1, 6):
            t = min(n, k)
            if _align(lib, [a] * n, [a] * k, blosum, 11, 1) != (4 * t, 0, t - 1, 0, t - 1):
                return False
    return True


@pytest.fixture(scope="module")
def blosum(oracle_mod):
    return oracle_mod.blosum62()


def test_unmodified_source_passes(tmp_path, blosum):
    lib = _compile(open(SRC).read(), tmp_path, "orig")
    assert _battery(lib, blosum)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_rejected(tmp_path, blosum, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert old in text, "mutation site not found: %s" % name
    lib = _compile(text.replace(old, new, 1), tmp_path, name)
    assert not _battery(lib, blosum)
