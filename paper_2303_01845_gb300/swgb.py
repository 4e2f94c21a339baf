"""ctypes binding of libswgb (include/swgb.h): argument marshalling only.

Every step of the alignment runs in the CUDA library; this module converts
torch tensors / numpy arrays to pointers and raises ``SwgbError`` on a
non-zero status.  There is no fallback: importing it without a built
``libswgb.so`` raises.

Names follow the C ABI (``swgb_create``, ``swgb_align``, ...).  PyTorch is used
for device memory and streams only.
"""
import ctypes
import os

import numpy as np

from . import build as _build

SWGB_OK = 0
SWGB_EINVAL = -1
SWGB_ERANGE = -2
SWGB_EBADRES = -3
SWGB_ENOMEM = -4
SWGB_ECUDA = -5
SWGB_EINTERNAL = -6
SWGB_ETOOBIG = -7
SWGB_ETIMEDOUT = -8

SWGB_ALPHABET_SIZE = 24
SWGB_MAX_LENGTH = 65536
SWGB_SEQ_ASCII = 0x1
SWGB_SEQ_DEVICE = 0x2
SWGB_SEQ_COPY = 0x4
SWGB_FORCE_INT32 = 0x1
SWGB_TIMING = 0x2
SWGB_NOALLOC_SCRATCH_BYTES = 32 << 20
SWGB_NOALLOC_MAX_PAIRS = 1 << 19
SWGB_NOALLOC_MAX_QUERY_LENGTH = 4096
SWGB_MLP_PARAMS = 10561
SWGB_FEATURES = 32

ALPHABET = "ARNDCQEGHILKMFPSTWYVBZX*"

_NAMES = {SWGB_EINVAL: "EINVAL", SWGB_ERANGE: "ERANGE", SWGB_EBADRES: "EBADRES",
          SWGB_ENOMEM: "ENOMEM", SWGB_ECUDA: "ECUDA", SWGB_EINTERNAL: "EINTERNAL",
          SWGB_ETOOBIG: "ETOOBIG", SWGB_ETIMEDOUT: "ETIMEDOUT"}


class SwgbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_NAMES.get(code, "?"), code, msg))
        self.code = code


class swgb_record(ctypes.Structure):
    _fields_ = [("score", ctypes.c_int32), ("q_start", ctypes.c_int32),
                ("q_end", ctypes.c_int32), ("r_start", ctypes.c_int32),
                ("r_end", ctypes.c_int32)]


class swgb_params(ctypes.Structure):
    _fields_ = [("matrix", ctypes.POINTER(ctypes.c_int8)), ("gap_open", ctypes.c_int32),
                ("gap_extend", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class swgb_stats(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int64), ("n_int16_pairs", ctypes.c_int64),
                ("n_int32_pairs", ctypes.c_int64), ("n_reverse_pairs", ctypes.c_int64),
                ("forward_cells", ctypes.c_int64), ("reverse_cells", ctypes.c_int64),
                ("forward_ms", ctypes.c_float), ("reverse_ms", ctypes.c_float),
                ("total_ms", ctypes.c_float), ("kernel_launches", ctypes.c_int32),
                ("n_band_pairs", ctypes.c_int64), ("n_band_certified", ctypes.c_int64),
                ("forward_slots", ctypes.c_int64), ("reverse_slots", ctypes.c_int64)]


class swgb_tuning(ctypes.Structure):
    _fields_ = [("tile_overhead", ctypes.c_int32), ("band_min", ctypes.c_int32),
                ("best_ms", ctypes.c_float), ("runner_up_ms", ctypes.c_float),
                ("runner_up_overhead", ctypes.c_int32), ("band_off_ms", ctypes.c_float),
                ("candidates", ctypes.c_int32)]


class swgb_thresholds(ctypes.Structure):
    _fields_ = [("id_num", ctypes.c_int32), ("id_den", ctypes.c_int32),
                ("cov_num", ctypes.c_int32), ("cov_den", ctypes.c_int32)]


class swgb_identity_record(ctypes.Structure):
    _fields_ = [("matches", ctypes.c_int32), ("columns", ctypes.c_int32), ("pass_", ctypes.c_int32)]


class swgb_server_config(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch_queries", ctypes.c_int32),
                ("max_batch_residues", ctypes.c_int64), ("max_inflight_bytes", ctypes.c_int64),
                ("candidates_per_query", ctypes.c_int32), ("min_shared", ctypes.c_int32),
                ("threshold", ctypes.c_float), ("identity", swgb_thresholds)]


class swgb_server_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_pairs", ctypes.c_int64),
                ("n_candidates", ctypes.c_int64), ("pairs", ctypes.POINTER(ctypes.c_int32)),
                ("counts", ctypes.POINTER(ctypes.c_int32)), ("records", ctypes.POINTER(ctypes.c_int32)),
                ("identity", ctypes.POINTER(ctypes.c_int32)), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("batch_id", ctypes.c_int64), ("slot", ctypes.c_int32),
                ("error", ctypes.c_char_p), ("stage_ms", ctypes.c_double * 5)]


# (name, restype, argtypes) of every exported function
_VP = ctypes.c_void_p
_SIGS = [
    ("swgb_create", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_VP)]),
    ("swgb_destroy", None, [_VP]),
    ("swgb_last_error", ctypes.c_char_p, [_VP]),
    ("swgb_blosum62", None, [_VP]),
    ("swgb_seqset_create", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_uint32, _VP,
                                          ctypes.POINTER(_VP)]),
    ("swgb_seqset_load", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_uint32, _VP]),
    ("swgb_seqset_info", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64)]),
    ("swgb_seqset_destroy", None, [_VP]),
    ("swgb_align", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64,
                                  ctypes.POINTER(swgb_params), _VP, _VP]),
    ("swgb_align_host", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64,
                                       ctypes.POINTER(swgb_params), _VP, _VP]),
    ("swgb_sync", ctypes.c_int, [_VP, _VP]),
    ("swgb_last_stats", ctypes.c_int, [_VP, ctypes.POINTER(swgb_stats)]),
    ("swgb_probe_addmax_rate", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_int)]),
    ("swgb_set_tile_overhead", ctypes.c_int, [_VP, ctypes.c_int]),
    ("swgb_get_tile_overhead", ctypes.c_int, [_VP]),
    ("swgb_set_band_min", ctypes.c_int, [_VP, ctypes.c_int]),
    ("swgb_get_band_min", ctypes.c_int, [_VP]),
    ("swgb_last_tuning", ctypes.c_int, [_VP, ctypes.POINTER(swgb_tuning)]),
    ("swgb_autotune", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.POINTER(swgb_params),
                                     _VP, _VP, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_float)]),
    ("swgb_plan_create", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64,
                                        ctypes.POINTER(swgb_params), _VP, ctypes.POINTER(_VP)]),
    ("swgb_plan_launch", ctypes.c_int, [_VP, _VP]),
    ("swgb_plan_destroy", None, [_VP]),
    ("swgb_discover", ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, _VP, _VP, ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_int64), _VP]),
    ("swgb_identity", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int64,
                                     ctypes.POINTER(swgb_params), ctypes.POINTER(swgb_thresholds),
                                     _VP, _VP]),
    ("swgb_search_launches", ctypes.c_int, [_VP]),
    ("swgb_index_create", ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, ctypes.POINTER(_VP)]),
    ("swgb_index_destroy", None, [_VP]),
    ("swgb_index_info", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int64)]),
    ("swgb_index_query", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_int64), _VP]),
    ("swgb_index_features", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64, _VP, _VP]),
    ("swgb_pair_features", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_int, _VP, _VP]),
    ("swgb_mlp_create", ctypes.c_int, [_VP, _VP, ctypes.POINTER(_VP)]),
    ("swgb_mlp_destroy", None, [_VP]),
    ("swgb_mlp_set", ctypes.c_int, [_VP, _VP]),
    ("swgb_mlp_get", ctypes.c_int, [_VP, _VP]),
    ("swgb_mlp_forward", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP]),
    ("swgb_mlp_grad", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_float, _VP, _VP, _VP]),
    ("swgb_mlp_train", ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_float, ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                                      _VP]),
    ("swgb_mlp_fit", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_uint64,
                                    ctypes.POINTER(ctypes.c_float), _VP]),
    ("swgb_mlp_calibrate", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_float,
                                          ctypes.POINTER(ctypes.c_float), _VP]),
    ("swgb_select_pairs", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_float, _VP, _VP,
                                         ctypes.POINTER(ctypes.c_int64), _VP]),
    ("swgb_server_default_config", None, [ctypes.POINTER(swgb_server_config)]),
    ("swgb_server_create", ctypes.c_int, [ctypes.c_int, _VP, _VP, _VP, ctypes.POINTER(swgb_params),
                                          ctypes.POINTER(swgb_server_config), ctypes.POINTER(_VP)]),
    ("swgb_server_destroy", None, [_VP]),
    ("swgb_server_submit", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    ("swgb_server_wait", ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.POINTER(swgb_server_result)]),
    ("swgb_server_release", ctypes.c_int, [_VP, ctypes.c_int64]),
    ("swgb_server_stats", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    ("swgb_align_noalloc", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP, ctypes.c_int64,
                                          _VP, ctypes.c_int64, ctypes.POINTER(swgb_params), _VP,
                                          _VP]),
]

_lib = None


def library_path():
    return _build.SWGB_LIB


def load(build_if_missing=True):
    """Loads libswgb.so (building it in-tree if missing).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.SWGB_LIB
    if build_if_missing:
        path = _build.build_swgb()
    if not os.path.exists(path):
        raise ImportError("libswgb.so is not built (%s); run paper_2303_01845_gb300.build.build_all()" % path)
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(ctx, rc):
    if rc != SWGB_OK:
        msg = load().swgb_last_error(ctx)
        raise SwgbError(rc, msg.decode(errors="replace") if msg else "")


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x):
    """Data pointer of a torch tensor or numpy array (must be contiguous)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(x))


def swgb_blosum62():
    """The library's BLOSUM62, int8 [24, 24] (row = query letter)."""
    out = np.zeros((24, 24), dtype=np.int8)
    load().swgb_blosum62(out.ctypes.data)
    return out


def swgb_create(device=0):
    h = _VP()
    rc = load().swgb_create(int(device), ctypes.byref(h))
    if rc != SWGB_OK:
        raise SwgbError(rc, "swgb_create(device=%d) failed" % device)
    return h


def swgb_destroy(ctx):
    load().swgb_destroy(ctx)


def _seq_args(residues, offsets, flags):
    on_dev = hasattr(residues, "is_cuda") and residues.is_cuda
    if on_dev:
        flags |= SWGB_SEQ_DEVICE
        if not (hasattr(offsets, "is_cuda") and offsets.is_cuda):
            raise ValueError("residues and offsets must live on the same side")
    if hasattr(offsets, "dtype") and str(offsets.dtype) not in ("int64", "torch.int64"):
        raise TypeError("offsets must be int64")
    n = (offsets.shape[0] if hasattr(offsets, "shape") else len(offsets)) - 1
    return flags, max(n, 0)


def swgb_seqset_create(ctx, residues, offsets, ascii=False, stream=None, copy=False):
    """residues: uint8 codes (or ASCII with ascii=True); offsets: int64 [n+1].
    Host (numpy / CPU tensor) or device (CUDA tensor) buffers.  copy: pinned
    host residues go through the copy engines (SWGB_SEQ_COPY)."""
    flags, n = _seq_args(residues, offsets, (SWGB_SEQ_ASCII if ascii else 0) | (SWGB_SEQ_COPY if copy else 0))
    h = _VP()
    rc = load().swgb_seqset_create(ctx, _ptr(residues), _ptr(offsets), n, flags,
                                   _stream_handle(stream), ctypes.byref(h))
    _check(ctx, rc)
    return h


def swgb_seqset_load(ctx, seqset, residues, offsets, ascii=False, stream=None, copy=False):
    flags, n = _seq_args(residues, offsets, (SWGB_SEQ_ASCII if ascii else 0) | (SWGB_SEQ_COPY if copy else 0))
    rc = load().swgb_seqset_load(seqset, _ptr(residues), _ptr(offsets), n, flags,
                                 _stream_handle(stream))
    _check(ctx, rc)


def swgb_seqset_info(seqset):
    n = ctypes.c_int64()
    m = ctypes.c_int64()
    rc = load().swgb_seqset_info(seqset, ctypes.byref(n), ctypes.byref(m))
    if rc != SWGB_OK:
        raise SwgbError(rc, "swgb_seqset_info")
    return n.value, m.value


def swgb_seqset_destroy(seqset):
    load().swgb_seqset_destroy(seqset)


def make_params(matrix=None, gap_open=11, gap_extend=1, force_int32=False, timing=False):
    """swgb_params (keeps a reference to the matrix buffer)."""
    m = swgb_blosum62() if matrix is None else np.ascontiguousarray(matrix, dtype=np.int8)
    if m.shape != (24, 24):
        raise ValueError("matrix must be 24 x 24")
    p = swgb_params(m.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), int(gap_open),
                    int(gap_extend),
                    (SWGB_FORCE_INT32 if force_int32 else 0) | (SWGB_TIMING if timing else 0))
    p._matrix_ref = m
    return p


def swgb_align(ctx, queries, refs, pairs, params, out=None, stream=None):
    """pairs: CUDA int32 tensor [P, 2]; returns (and fills) CUDA int32 [P, 5].
    Asynchronous on `stream` (default: torch's current stream)."""
    import torch
    if not pairs.is_cuda or pairs.dtype != torch.int32:
        raise TypeError("pairs must be a CUDA int32 tensor")
    n = pairs.shape[0]
    if out is None:
        out = torch.empty((n, 5), dtype=torch.int32, device=pairs.device)
    if not out.is_cuda or out.dtype != torch.int32 or out.numel() < 5 * n:
        raise TypeError("out must be a CUDA int32 tensor with P x 5 elements")
    rc = load().swgb_align(ctx, queries, refs, _ptr(pairs), n, ctypes.byref(params), _ptr(out),
                           _stream_handle(stream))
    _check(ctx, rc)
    return out


def swgb_align_host(ctx, queries, refs, pairs, params, out=None, stream=None):
    """Host pairs int32 [P, 2] (numpy or CPU tensor, pinned for async copies)
    -> host records int32 [P, 5]; synchronous."""
    n = pairs.shape[0]
    if out is None:
        out = np.empty((n, 5), dtype=np.int32)
    rc = load().swgb_align_host(ctx, queries, refs, _ptr(pairs), n, ctypes.byref(params),
                                _ptr(out), _stream_handle(stream))
    _check(ctx, rc)
    return out


def swgb_sync(ctx, stream=None):
    _check(ctx, load().swgb_sync(ctx, _stream_handle(stream)))


def swgb_last_stats(ctx):
    s = swgb_stats()
    _check(ctx, load().swgb_last_stats(ctx, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in swgb_stats._fields_}


def swgb_probe_addmax_rate(ctx):
    """(lane-level add-max instructions per SM clock per SM, SM count)."""
    r = ctypes.c_double()
    n = ctypes.c_int()
    _check(ctx, load().swgb_probe_addmax_rate(ctx, ctypes.byref(r), ctypes.byref(n)))
    return r.value, n.value


def swgb_set_tile_overhead(ctx, overhead):
    _check(ctx, load().swgb_set_tile_overhead(ctx, int(overhead)))


def swgb_get_tile_overhead(ctx):
    return load().swgb_get_tile_overhead(ctx)


def swgb_set_band_min(ctx, band_min):
    _check(ctx, load().swgb_set_band_min(ctx, int(band_min)))


def swgb_get_band_min(ctx):
    return load().swgb_get_band_min(ctx)


def swgb_last_tuning(ctx):
    t = swgb_tuning()
    _check(ctx, load().swgb_last_tuning(ctx, ctypes.byref(t)))
    return {name: getattr(t, name) for name, _ in swgb_tuning._fields_}


def swgb_autotune(ctx, queries, refs, pairs, params, out, stream=None):
    """Times the tile-cost overhead and band threshold candidates on this batch
    (CUDA buffers), keeps the fastest in the context; returns (overhead, ms);
    swgb_last_tuning gives the rest."""
    best = ctypes.c_int()
    ms = ctypes.c_float()
    rc = load().swgb_autotune(ctx, queries, refs, _ptr(pairs), pairs.shape[0], ctypes.byref(params),
                              _ptr(out), _stream_handle(stream), ctypes.byref(best), ctypes.byref(ms))
    _check(ctx, rc)
    return best.value, ms.value


def swgb_plan_create(ctx, queries, refs, pairs, params, out):
    """Captures the pipeline for these CUDA buffers into a CUDA graph."""
    h = _VP()
    rc = load().swgb_plan_create(ctx, queries, refs, _ptr(pairs), pairs.shape[0],
                                 ctypes.byref(params), _ptr(out), ctypes.byref(h))
    _check(ctx, rc)
    return h


def swgb_plan_launch(ctx, plan, stream=None):
    _check(ctx, load().swgb_plan_launch(plan, _stream_handle(stream)))


def swgb_plan_destroy(plan):
    load().swgb_plan_destroy(plan)


def swgb_discover(ctx, seqset, k=6, min_shared=2, capacity=None, stream=None):
    """Candidate pairs i < j of one set sharing >= min_shared distinct k-mers.

    Returns (pairs CUDA int32 [P, 2] ordered by (i, j), counts CUDA int32 [P]).
    With capacity=None the call runs twice when the first guess is too small.
    """
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    cap = 1 << 16 if capacity is None else int(capacity)
    while True:
        pairs = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=dev)
        counts = torch.empty((max(cap, 1),), dtype=torch.int32, device=dev)
        found = ctypes.c_int64()
        rc = load().swgb_discover(ctx, seqset, int(k), int(min_shared), _ptr(pairs), _ptr(counts),
                                  cap, ctypes.byref(found), _stream_handle(stream))
        _check(ctx, rc)
        n = found.value
        if n <= cap or capacity is not None:
            m = min(n, cap)
            return pairs[:m], counts[:m]
        cap = n


def make_thresholds(min_identity=(3, 10), min_coverage=(7, 10)):
    return swgb_thresholds(int(min_identity[0]), int(min_identity[1]),
                           int(min_coverage[0]), int(min_coverage[1]))


def swgb_identity(ctx, queries, refs, pairs, records, params, thresholds=None, out=None,
                  stream=None):
    """Identity and pass/fail of alignment records (CUDA tensors): returns CUDA
    int32 [P, 3] = (identical columns, columns, pass).  Synchronous."""
    import torch
    n = pairs.shape[0]
    if out is None:
        out = torch.empty((n, 3), dtype=torch.int32, device=pairs.device)
    for t_ in (pairs, records, out):
        if not t_.is_cuda or t_.dtype != torch.int32 or not t_.is_contiguous():
            raise TypeError("pairs, records and out must be contiguous CUDA int32 tensors")
    if records.numel() < 5 * n or out.numel() < 3 * n:
        raise ValueError("records must hold P x 5 and out P x 3 int32")
    th = thresholds or make_thresholds()
    rc = load().swgb_identity(ctx, queries, refs, _ptr(pairs), _ptr(records), n,
                              ctypes.byref(params), ctypes.byref(th), _ptr(out),
                              _stream_handle(stream))
    _check(ctx, rc)
    return out


def _cuda(t_, dtype, what):
    import torch
    if not t_.is_cuda or t_.dtype != dtype or not t_.is_contiguous():
        raise TypeError("%s must be a contiguous CUDA %s tensor" % (what, dtype))


def swgb_pair_features(ctx, set_a, set_b, pairs, k=6, out=None, stream=None):
    """Features of the learned filter for CUDA int32 pairs [P, 2] (index into
    set_a, index into set_b): CUDA float32 [P, 32].  Synchronous."""
    import torch
    _cuda(pairs, torch.int32, "pairs")
    n = pairs.shape[0]
    if out is None:
        out = torch.empty((n, SWGB_FEATURES), dtype=torch.float32, device=pairs.device)
    _cuda(out, torch.float32, "out")
    rc = load().swgb_pair_features(ctx, set_a, set_b, _ptr(pairs), n, int(k), _ptr(out),
                                   _stream_handle(stream))
    _check(ctx, rc)
    return out


def swgb_select_pairs(ctx, pairs, logits, threshold, stream=None):
    """(kept pairs CUDA int32 [K, 2], their positions CUDA int64 [K]) of the
    pairs whose logit is >= threshold, in order.  Synchronous."""
    import torch
    _cuda(pairs, torch.int32, "pairs")
    _cuda(logits, torch.float32, "logits")
    n = pairs.shape[0]
    kept = torch.empty((max(n, 1), 2), dtype=torch.int32, device=pairs.device)
    index = torch.empty((max(n, 1),), dtype=torch.int64, device=pairs.device)
    nk = ctypes.c_int64()
    rc = load().swgb_select_pairs(ctx, _ptr(pairs), _ptr(logits), n, float(threshold), _ptr(kept),
                                  _ptr(index), ctypes.byref(nk), _stream_handle(stream))
    _check(ctx, rc)
    return kept[:nk.value], index[:nk.value]


class Index:
    """A resident k-mer index of a reference SeqSet (swgb_index_*)."""

    def __init__(self, aligner, refs, k=6, stream=None):
        self.aligner = aligner
        self.refs = refs          # kept alive: the index reads the set
        h = _VP()
        _check(aligner.ctx, load().swgb_index_create(aligner.ctx, refs.handle, int(k),
                                                     _stream_handle(stream), ctypes.byref(h)))
        self.handle = h

    def info(self):
        n = ctypes.c_int64()
        k = ctypes.c_int()
        b = ctypes.c_int64()
        load().swgb_index_info(self.handle, ctypes.byref(n), ctypes.byref(k), ctypes.byref(b))
        return {"n_refs": n.value, "k": k.value, "bytes": b.value}

    def query(self, queries, min_shared=2, capacity=None, stream=None, ctx=None):
        """(pairs CUDA int32 [P, 2] = (query, reference), counts CUDA int32 [P])."""
        import torch
        ctx = ctx or self.aligner.ctx
        dev = torch.device("cuda", torch.cuda.current_device())
        cap = 1 << 16 if capacity is None else int(capacity)
        while True:
            pairs = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=dev)
            counts = torch.empty((max(cap, 1),), dtype=torch.int32, device=dev)
            found = ctypes.c_int64()
            _check(ctx, load().swgb_index_query(ctx, self.handle, queries.handle, int(min_shared),
                                                _ptr(pairs), _ptr(counts), cap, ctypes.byref(found),
                                                _stream_handle(stream)))
            if found.value <= cap or capacity is not None:
                m = min(found.value, cap)
                return pairs[:m], counts[:m]
            cap = found.value

    def features(self, queries, pairs, out=None, stream=None, ctx=None):
        import torch
        ctx = ctx or self.aligner.ctx
        _cuda(pairs, torch.int32, "pairs")
        n = pairs.shape[0]
        if out is None:
            out = torch.empty((n, SWGB_FEATURES), dtype=torch.float32, device=pairs.device)
        _check(ctx, load().swgb_index_features(ctx, self.handle, queries.handle, _ptr(pairs), n,
                                               _ptr(out), _stream_handle(stream)))
        return out

    def close(self):
        if self.handle:
            load().swgb_index_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The learned filter's network (swgb_mlp_*), parameters on the device."""

    def __init__(self, ctx, init):
        init = np.ascontiguousarray(init, dtype=np.float32).reshape(-1)
        if init.size != SWGB_MLP_PARAMS:
            raise ValueError("expected %d parameters" % SWGB_MLP_PARAMS)
        self.ctx = ctx
        h = _VP()
        _check(ctx, load().swgb_mlp_create(ctx, init.ctypes.data, ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            load().swgb_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        _check(self.ctx, load().swgb_mlp_set(self.handle, params.ctypes.data))

    def get(self):
        out = np.zeros(SWGB_MLP_PARAMS, np.float32)
        _check(self.ctx, load().swgb_mlp_get(self.handle, out.ctypes.data))
        return out

    def forward(self, features, out=None, stream=None):
        import torch
        _cuda(features, torch.float32, "features")
        n = features.shape[0]
        if out is None:
            out = torch.empty((n,), dtype=torch.float32, device=features.device)
        _check(self.ctx, load().swgb_mlp_forward(self.handle, _ptr(features), n, _ptr(out),
                                                 _stream_handle(stream)))
        return out

    def grad(self, features, labels, pos_weight=1.0, stream=None):
        """(gradient CUDA float32 [SWGB_MLP_PARAMS], loss CUDA float32 [1])."""
        import torch
        _cuda(features, torch.float32, "features")
        _cuda(labels, torch.float32, "labels")
        g = torch.empty((SWGB_MLP_PARAMS,), dtype=torch.float32, device=features.device)
        loss = torch.empty((1,), dtype=torch.float32, device=features.device)
        _check(self.ctx, load().swgb_mlp_grad(self.handle, _ptr(features), _ptr(labels),
                                              features.shape[0], float(pos_weight), _ptr(g),
                                              _ptr(loss), _stream_handle(stream)))
        return g, loss

    def train(self, features, labels, order=None, batch=8192, lr=1e-3, pos_weight=1.0,
              stream=None):
        """One pass in minibatches (order: CUDA int32 permutation or None);
        returns the mean minibatch loss."""
        import torch
        _cuda(features, torch.float32, "features")
        _cuda(labels, torch.float32, "labels")
        if order is not None:
            _cuda(order, torch.int32, "order")
        ml = ctypes.c_float()
        _check(self.ctx, load().swgb_mlp_train(self.handle, _ptr(features), _ptr(labels),
                                               _ptr(order), features.shape[0], int(batch),
                                               float(lr), float(pos_weight), ctypes.byref(ml),
                                               _stream_handle(stream)))
        return ml.value

    def fit(self, features, labels, epochs, batch=8192, lr=3e-3, pos_weight=0.0, seed=1, stream=None):
        """swgb_mlp_fit: `epochs` seeded passes; pos_weight <= 0 means the
        library's default; returns the per-epoch mean losses."""
        import torch
        _cuda(features, torch.float32, "features")
        _cuda(labels, torch.float32, "labels")
        losses = (ctypes.c_float * max(int(epochs), 1))()
        _check(self.ctx, load().swgb_mlp_fit(self.handle, _ptr(features), _ptr(labels), features.shape[0],
                                             int(epochs), int(batch), float(lr), float(pos_weight),
                                             ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), losses,
                                             _stream_handle(stream)))
        return [losses[k] for k in range(int(epochs))]

    def calibrate(self, features, labels, recall, stream=None):
        """swgb_mlp_calibrate: the logit threshold keeping `recall` of the positives."""
        import torch
        _cuda(features, torch.float32, "features")
        _cuda(labels, torch.float32, "labels")
        t = ctypes.c_float()
        _check(self.ctx, load().swgb_mlp_calibrate(self.handle, _ptr(features), _ptr(labels),
                                                   features.shape[0], float(recall), ctypes.byref(t),
                                                   _stream_handle(stream)))
        return t.value


def server_config(**kw):
    """swgb_server_config with the library's defaults, overridden by kw
    (identity=(num, den, num, den))."""
    cfg = swgb_server_config()
    load().swgb_server_default_config(ctypes.byref(cfg))
    for k, v in kw.items():
        if k == "identity":
            cfg.identity = swgb_thresholds(*[int(x) for x in v])
        else:
            setattr(cfg, k, v)
    return cfg


class Server:
    """A query server over a resident reference set (swgb_server_*)."""

    def __init__(self, refs, index, params, mlp_params=None, device=0, **cfg):
        self.refs, self.index, self.params = refs, index, params   # kept alive
        self.cfg = server_config(**cfg)
        mp = None
        if mlp_params is not None:
            self._mlp = np.ascontiguousarray(mlp_params, dtype=np.float32).reshape(-1)
            mp = self._mlp.ctypes.data
        h = _VP()
        rc = load().swgb_server_create(int(device), refs.handle, index.handle, mp, ctypes.byref(params),
                                       ctypes.byref(self.cfg), ctypes.byref(h))
        if rc != SWGB_OK:
            raise SwgbError(rc, "swgb_server_create failed")
        self.handle = h

    def submit(self, codes, offsets):
        codes = np.ascontiguousarray(codes, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        t = ctypes.c_int64()
        rc = load().swgb_server_submit(self.handle, codes.ctypes.data if codes.size else None,
                                       offsets.ctypes.data, len(offsets) - 1, ctypes.byref(t))
        if rc != SWGB_OK:
            raise SwgbError(rc, "swgb_server_submit failed")
        return t.value

    def wait(self, ticket, timeout_ms=-1, release=True):
        """Results of a request as numpy copies: pairs [P, 2], counts [P],
        records [P, 5], identity [P, 3], plus candidates, latency_ms,
        queue_ms, batch_id, slot and stage_ms (host wall time of the batch's
        stages: queries loaded, candidates, filter, alignment + identity,
        results back)."""
        r = swgb_server_result()
        rc = load().swgb_server_wait(self.handle, int(ticket), int(timeout_ms), ctypes.byref(r))
        if rc != SWGB_OK:
            raise SwgbError(rc, "swgb_server_wait failed")
        if r.status != SWGB_OK:
            msg = r.error.decode(errors="replace") if r.error else ""
            raise SwgbError(r.status, "request %d failed: %s" % (ticket, msg))
        n = r.n_pairs

        def arr(ptr, shape):
            if n == 0:
                return np.zeros(shape, np.int32)
            return np.ctypeslib.as_array(ptr, shape=shape).copy()
        out = {"pairs": arr(r.pairs, (n, 2)), "counts": arr(r.counts, (n,)),
               "records": arr(r.records, (n, 5)), "identity": arr(r.identity, (n, 3)),
               "candidates": r.n_candidates, "latency_ms": r.latency_ms, "queue_ms": r.queue_ms,
               "batch_id": r.batch_id, "slot": r.slot, "stage_ms": list(r.stage_ms)}
        if release:
            load().swgb_server_release(self.handle, int(ticket))
        return out

    def stats(self):
        mo = ctypes.c_int32()
        pend = ctypes.c_int64()
        b = ctypes.c_int64()
        load().swgb_server_stats(self.handle, ctypes.byref(mo), ctypes.byref(pend), ctypes.byref(b))
        return {"max_overlap": mo.value, "pending": pend.value, "inflight_bytes": b.value}

    def close(self):
        if getattr(self, "handle", None):
            load().swgb_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def swgb_align_noalloc(q_codes, q_offsets, r_codes, r_offsets, pairs, params, out, stream=None):
    """Allocation-free alignment for callers that cannot allocate device memory
    while they align (a pool or arena owns the device, or the footprint must
    stay fixed): every argument is a caller-owned CUDA tensor (codes uint8,
    offsets int64, pairs int32 [P, 2], out int32 [P, 5]) and the library's
    scratch is a fixed array compiled into it.  Synchronous.  Limits:
    SWGB_NOALLOC_MAX_PAIRS pairs per call, queries up to
    SWGB_NOALLOC_MAX_QUERY_LENGTH residues; larger inputs raise ETOOBIG."""
    import torch
    _cuda(q_codes, torch.uint8, "q_codes")
    _cuda(q_offsets, torch.int64, "q_offsets")
    _cuda(r_codes, torch.uint8, "r_codes")
    _cuda(r_offsets, torch.int64, "r_offsets")
    _cuda(pairs, torch.int32, "pairs")
    _cuda(out, torch.int32, "out")
    if q_offsets.dim() != 1 or r_offsets.dim() != 1 or q_offsets.numel() < 1 or r_offsets.numel() < 1:
        raise ValueError("offsets must be 1-D with n + 1 entries")
    if pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must be int32 [P, 2]")
    n = pairs.shape[0]
    if out.numel() < 5 * n:
        raise ValueError("out must hold P x 5 int32")
    dev = pairs.device
    if any(t.device != dev for t in (q_codes, q_offsets, r_codes, r_offsets, out)):
        raise ValueError("swgb_align_noalloc: every tensor must be on one device")
    # the C call runs on the calling thread's current device
    with torch.cuda.device(dev):
        rc = load().swgb_align_noalloc(_ptr(q_codes), _ptr(q_offsets), q_offsets.shape[0] - 1,
                                       _ptr(r_codes), _ptr(r_offsets), r_offsets.shape[0] - 1,
                                       _ptr(pairs), n, ctypes.byref(params), _ptr(out),
                                       _stream_handle(stream))
    if rc != SWGB_OK:
        extra = ""
        if rc == SWGB_ETOOBIG:
            extra = ("a size exceeds the fixed limits: at most %d pairs per call and %d residues "
                     "per query" % (SWGB_NOALLOC_MAX_PAIRS, SWGB_NOALLOC_MAX_QUERY_LENGTH))
        raise SwgbError(rc, "swgb_align_noalloc failed" + (": " + extra if extra else ""))
    return out


class Aligner:
    """Owns a context; convenience wrapper over the functions above."""

    def __init__(self, device=0):
        self.ctx = swgb_create(device)
        self.device = device

    def close(self):
        if self.ctx:
            swgb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def seqset(self, residues, offsets, ascii=False, stream=None, copy=False):
        return SeqSet(self, swgb_seqset_create(self.ctx, residues, offsets, ascii, stream, copy))

    def align(self, queries, refs, pairs, params=None, out=None, stream=None, sync=True):
        params = params or make_params()
        out = swgb_align(self.ctx, queries.handle, refs.handle, pairs, params, out, stream)
        if sync:
            swgb_sync(self.ctx, stream)
        return out

    def align_host(self, queries, refs, pairs, params=None, out=None, stream=None):
        params = params or make_params()
        return swgb_align_host(self.ctx, queries.handle, refs.handle, pairs, params, out, stream)

    def stats(self):
        return swgb_last_stats(self.ctx)

    def discover(self, seqset, k=6, min_shared=2, capacity=None, stream=None):
        return swgb_discover(self.ctx, seqset.handle, k, min_shared, capacity, stream)

    def features(self, set_a, set_b, pairs, k=6, out=None, stream=None):
        return swgb_pair_features(self.ctx, set_a.handle, set_b.handle, pairs, k, out, stream)

    def identity(self, queries, refs, pairs, records, params=None, thresholds=None, out=None,
                 stream=None):
        params = params or make_params()
        return swgb_identity(self.ctx, queries.handle, refs.handle, pairs, records, params,
                             thresholds, out, stream)


class SeqSet:
    def __init__(self, aligner, handle):
        self.aligner = aligner
        self.handle = handle

    def info(self):
        return swgb_seqset_info(self.handle)

    def load(self, residues, offsets, ascii=False, stream=None, copy=False):
        swgb_seqset_load(self.aligner.ctx, self.handle, residues, offsets, ascii, stream, copy)

    def close(self):
        if self.handle:
            swgb_seqset_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
