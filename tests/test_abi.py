"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU,
exports every function include/swgb.h declares, and its host-side pieces that
need no device behave (BLOSUM62 table, argument errors)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swgb.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(swgb_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2303_01845_gb300 import swgb
    return swgb.load()


def test_header_declares_the_api():
    names = declared_functions()
    for n in ["swgb_create", "swgb_destroy", "swgb_seqset_create", "swgb_align",
              "swgb_align_host", "swgb_sync", "swgb_last_stats", "swgb_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2303_01845_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.SWGB_LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # nothing but the declared API leaks out of the library
    ours = {n for n in exported if n.startswith("swgb")}
    assert ours == set(declared_functions())


def test_binding_covers_every_declared_symbol():
    from paper_2303_01845_gb300 import swgb
    bound = {name for name, _, _ in swgb._SIGS}
    assert bound == set(declared_functions())


def test_library_is_built_for_sm_103a(lib):
    from paper_2303_01845_gb300 import build
    out = subprocess.run(["cuobjdump", "--list-elf", build.SWGB_LIB], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_blosum62_matches_the_oracle_transcription(lib, oracle_mod):
    """Two independent transcriptions of the published matrix agree."""
    from paper_2303_01845_gb300 import swgb
    assert (swgb.swgb_blosum62() == oracle_mod.blosum62()).all()


def test_create_without_a_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2303_01845_gb300 import swgb
    with pytest.raises(swgb.SwgbError) as ei:
        swgb.swgb_create(0)
    assert ei.value.code == swgb.SWGB_ECUDA


def test_null_arguments_are_rejected(lib):
    from paper_2303_01845_gb300 import swgb
    assert lib.swgb_create(0, None) == swgb.SWGB_EINVAL
    assert lib.swgb_align(None, None, None, None, 0, None, None, None) == swgb.SWGB_EINVAL
    assert lib.swgb_sync(None, None) == swgb.SWGB_EINVAL
    assert lib.swgb_seqset_info(None, None, None) == swgb.SWGB_EINVAL
    lib.swgb_destroy(None)
    lib.swgb_seqset_destroy(None)


def header_constants():
    """The header's integer #defines (error codes, flags, sizes), evaluated."""
    out = {}
    for name, value in re.findall(r"^#define (SWGB_[A-Z_0-9]+)[ \t]+([^/\n]+)", open(HEADER).read(), flags=re.M):
        expr = re.sub(r"\b(0x[0-9a-fA-F]+|[0-9]+)[uU]\b", r"\1", value.strip())
        if re.fullmatch(r"[0-9a-fA-FxX()<> +\-]+", expr):
            out[name] = eval(expr, {"__builtins__": {}})   # integer literals, shifts and signs only
    return out


def test_binding_constants_match_the_header():
    """Every integer constant the binding mirrors has the header's value, and
    the binding mirrors every error code and flag."""
    from paper_2303_01845_gb300 import swgb
    consts = header_constants()
    assert consts["SWGB_SEQ_COPY"] == 0x4 and consts["SWGB_EINVAL"] == -1
    mirrored = {n: v for n, v in consts.items() if hasattr(swgb, n)}
    assert mirrored == {n: getattr(swgb, n) for n in mirrored}
    must = [n for n in consts if n.startswith(("SWGB_E", "SWGB_SEQ_")) or n in ("SWGB_OK", "SWGB_FORCE_INT32", "SWGB_TIMING")]
    assert all(hasattr(swgb, n) for n in must), [n for n in must if not hasattr(swgb, n)]
