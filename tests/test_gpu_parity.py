"""GPU parity: every record from the CUDA library (called through the C ABI)
equals the CPU oracle's, bit for bit.

Sizes: the whole 10,000-pair uniform-length workload; ragged length grids that
cross every tile shape, the 512-row chunk boundary and the 16-bit/32-bit
switch; edge cases (empty sequences, single residues, no positive score,
out-of-range pairs); and, in the benchmark's launch configuration, the
2,000,000-pair log-normal workload checked on a seeded sample plus every
pair on the 32-bit path.
"""
import numpy as np
import pytest

from gpu_helpers import assert_same, device_sets, gpu_records, oracle_records

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def aligner(torch_cuda):
    from paper_2303_01845_gb300 import swgb
    a = swgb.Aligner(0)
    yield a
    a.close()


@pytest.fixture(scope="module")
def blosum(oracle_mod):
    return oracle_mod.blosum62()


@pytest.fixture(scope="module")
def plain10k(blosum):
    from paper_2303_01845_gb300 import workload
    return workload.generate("plain_10k", blosum)


def params(mat, go=11, ge=1, **kw):
    from paper_2303_01845_gb300 import swgb
    return swgb.make_params(mat, go, ge, **kw)


def test_plain_10k_bit_exact(aligner, oracle_mod, blosum, plain10k):
    got = gpu_records(aligner, plain10k, params(blosum))
    want = oracle_records(oracle_mod, plain10k, blosum, 11, 1)
    assert_same(got, want, plain10k)
    st = aligner.stats()
    assert st["forward_cells"] == plain10k.cells()
    assert st["n_int16_pairs"] == len(plain10k.pairs)
    assert st["n_reverse_pairs"] == int((want[:, 0] > 0).sum())
    # cell updates computed: every forward cell at least once, fill and
    # padding on top; the reverse pass computes some
    assert st["forward_slots"] >= st["forward_cells"]
    assert st["forward_slots"] < 2 * st["forward_cells"]
    assert 0 < st["reverse_slots"] <= st["forward_slots"]


def test_plain_10k_forced_int32_path(aligner, oracle_mod, blosum, plain10k):
    sub = plain10k.subset(np.arange(0, 10000, 7))
    got = gpu_records(aligner, sub, params(blosum, force_int32=True))
    want = oracle_records(oracle_mod, sub, blosum, 11, 1)
    assert_same(got, want, sub)
    assert aligner.stats()["n_int32_pairs"] == len(sub.pairs)


def test_gap_settings_and_asymmetric_matrix(aligner, oracle_mod, blosum, plain10k):
    sub = plain10k.subset(np.arange(3, 10000, 13))
    for go, ge in [(11, 2), (0, 1), (5, 3), (20, 4)]:
        assert_same(gpu_records(aligner, sub, params(blosum, go, ge)),
                    oracle_records(oracle_mod, sub, blosum, go, ge), sub)
    rng = np.random.default_rng(5)
    asym = rng.integers(-6, 7, size=(24, 24)).astype(np.int8)
    assert_same(gpu_records(aligner, sub, params(asym, 7, 2)),
                oracle_records(oracle_mod, sub, asym, 7, 2), sub)


def test_matrices_at_the_packed_score_range(aligner, oracle_mod, plain10k):
    """The packed path holds s + o + e in a byte of 0..127: a matrix reaching
    both ends of that range stays packed; one entry with s + o + e < 0 moves
    every pair to the 32-bit path, with the same records."""
    sub = plain10k.subset(np.arange(5, 10000, 17))
    go, ge = 40, 3
    lo, hi = -(go + ge), 127 - (go + ge)
    rng = np.random.default_rng(11)
    wide = rng.integers(lo, hi + 1, size=(24, 24)).astype(np.int8)
    wide[0, 0], wide[1, 2] = hi, lo
    np.fill_diagonal(wide[4:], 40)
    want = oracle_records(oracle_mod, sub, wide, go, ge)
    assert_same(gpu_records(aligner, sub, params(wide, go, ge)), want, sub)
    st = aligner.stats()
    assert st["n_int16_pairs"] + st["n_int32_pairs"] == len(sub.pairs)
    assert st["n_int16_pairs"] > 0
    out = wide.copy()
    out[3, 3] = lo - 1
    want = oracle_records(oracle_mod, sub, out, go, ge)
    assert_same(gpu_records(aligner, sub, params(out, go, ge)), want, sub)
    assert aligner.stats()["n_int16_pairs"] == 0


HELD_LENGTHS = [1, 2, 7, 8, 9, 31, 32, 33, 47, 48, 49, 63, 64, 65, 95, 96, 97, 127, 128, 129,
                143, 144, 145, 159, 160, 161, 175, 176, 177, 191, 192, 193, 207, 208, 209,
                223, 224, 225, 239, 240, 241, 255, 256, 257, 287, 288, 289, 319, 320, 321,
                351, 352, 353, 383, 384, 385, 415, 416, 417, 447, 448, 449, 479, 480, 481,
                511, 512, 513, 767, 768, 769, 1023, 1024, 1025,
                1537, 2999]
STREAM_LENGTHS = [1, 2, 3, 30, 31, 32, 33, 100, 257, 512, 513, 1200]

TILE_SHAPES = [(4, 8), (4, 12), (8, 8), (8, 12)] + [(16, r) for r in range(8, 17)] + \
    [(32, r) for r in range(9, 17)]
FIRST_CHUNKABLE = 13


def tile_of(lq, lr):
    """(shape, chunks) the library's cost model gives a pair: (G lanes, R rows)
    from TILE_SHAPES, the 32-lane ones also tiling longer references in
    chunks; cost (lq + G - 1) * chunks * G * (R + 4)."""
    best = None
    for s, (G, R) in enumerate(TILE_SHAPES):
        rows = G * R
        n = 1
        if lr > rows:
            if s < FIRST_CHUNKABLE:
                continue
            n = -(-lr // rows)
        cost = (lq + G - 1) * n * G * (R + 4)
        if best is None or cost < best[0]:
            best = (cost, s, n)
    return best[1], best[2]


def ragged_workload(seed, mat, held=HELD_LENGTHS, stream=STREAM_LENGTHS):
    """Queries of every streamed length against references of every held
    length; half of the references derived from a query (mutated), half
    unrelated."""
    from paper_2303_01845_gb300 import workload
    rng = np.random.default_rng(seed)
    p = workload.background()
    queries = [rng.choice(20, size=n, p=p).astype(np.uint8) for n in stream]
    refs, pairs = [], []
    for qi, q in enumerate(queries):
        for L in held:
            # homologous: a window of the query (repeated to length L), mutated
            base = np.resize(q, L).copy()
            mask = rng.random(L) < 0.3
            base[mask] = rng.choice(20, size=int(mask.sum()), p=p)
            refs.append(base)
            pairs.append((qi, len(refs) - 1))
            refs.append(rng.choice(20, size=L, p=p).astype(np.uint8))
            pairs.append((qi, len(refs) - 1))
    return workload.from_sequences(queries, refs, pairs)


def test_ragged_lengths_all_shapes(aligner, oracle_mod, blosum):
    wl = ragged_workload(11, blosum)
    tiles = {tile_of(wl.q_len[q], wl.r_len[r]) for q, r in wl.pairs}
    assert {s for s, _ in tiles} == set(range(len(TILE_SHAPES)))
    chunked = {s for s, n in tiles if n >= 2}
    assert chunked <= set(range(FIRST_CHUNKABLE, len(TILE_SHAPES))) and len(chunked) >= 3
    assert_same(gpu_records(aligner, wl, params(blosum)),
                oracle_records(oracle_mod, wl, blosum, 11, 1), wl)


def test_ragged_lengths_int32(aligner, oracle_mod, blosum):
    wl = ragged_workload(12, blosum, held=[1, 33, 257, 513, 1537], stream=[1, 40, 600])
    assert_same(gpu_records(aligner, wl, params(blosum, force_int32=True)),
                oracle_records(oracle_mod, wl, blosum, 11, 1), wl)


def int32_expected(mat, q, r):
    """A pair needs the 32-bit path iff its score bound passes 32767: the
    bound is min(sum of the best score of each query letter, sum of the best
    score of each reference letter), checked only when 11 * min(lq, lr) does."""
    m = np.asarray(mat, np.int64)
    if max(0, int(m.max())) * min(len(q), len(r)) <= 32767:
        return False
    rowmax = np.maximum(m.max(axis=1), 0)
    colmax = np.maximum(m.max(axis=0), 0)
    return min(int(rowmax[q].sum()), int(colmax[r].sum())) > 32767


def test_self_alignment_closed_form_across_the_int16_limit(aligner, blosum):
    """Self-alignments have S = sum of the diagonal over the full length; the
    longest ones pass 32767 and take the 32-bit path."""
    from paper_2303_01845_gb300 import workload
    rng = np.random.default_rng(13)
    lens = [1, 5, 64, 300, 2978, 2979, 3500, 5000, 9000]
    seqs = [rng.integers(0, 20, size=n).astype(np.uint8) for n in lens]
    wl = workload.from_sequences(seqs, seqs, [(k, k) for k in range(len(seqs))])
    got = gpu_records(aligner, wl, params(blosum))
    m = blosum.astype(np.int64)
    for k, s in enumerate(seqs):
        n = len(s)
        assert tuple(got[k]) == (int(m[s, s].sum()), 0, n - 1, 0, n - 1)
    st = aligner.stats()
    assert st["n_int32_pairs"] == sum(1 for s in seqs if int32_expected(blosum, s, s))
    assert st["n_int32_pairs"] >= 1


def test_tryptophan_runs_at_the_int16_limit(aligner, oracle_mod, blosum):
    """W-W scores 11: W runs long enough to pass 32767 must not wrap."""
    from paper_2303_01845_gb300 import workload
    w = workload.ALPHABET.index("W")
    rng = np.random.default_rng(14)
    seqs = []
    for n in [2970, 2978, 2979, 2990, 3100]:
        s = np.full(n, w, np.uint8)
        s[rng.integers(0, n, size=5)] = rng.integers(0, 20, size=5)
        seqs.append(s)
    pairs = [(a, b) for a in range(len(seqs)) for b in range(len(seqs))]
    wl = workload.from_sequences(seqs, seqs, pairs)
    want = oracle_records(oracle_mod, wl, blosum, 11, 1)
    assert_same(gpu_records(aligner, wl, params(blosum)), want, wl)
    # scores right at the 16-bit limit are exercised on both paths
    n32 = sum(int32_expected(blosum, seqs[a], seqs[b]) for a, b in pairs)
    assert aligner.stats()["n_int32_pairs"] == n32
    assert 0 < n32 < len(pairs)
    assert want[:, 0].max() > 32767 and (want[:, 0] > 32000).sum() > n32


def test_edge_cases(aligner, oracle_mod, blosum):
    from paper_2303_01845_gb300 import workload
    A = workload.ALPHABET
    enc = lambda s: np.array([A.index(c) for c in s], np.uint8)
    seqs = [enc(s) for s in ["", "A", "W", "WWWWW", "PPPPPPP", "AAAA", "AAAAAAA",
                             "HEAGAWGHEE", "PAWHEAE", "*", "BZX*", "C" * 40]]
    n = len(seqs)
    pairs = [(a, b) for a in range(n) for b in range(n)]
    wl = workload.from_sequences(seqs, seqs, pairs)
    got = gpu_records(aligner, wl, params(blosum))
    assert_same(got, oracle_records(oracle_mod, wl, blosum, 11, 1), wl)
    # empty sequences report a zero record
    for p, (a, b) in enumerate(pairs):
        if len(seqs[a]) == 0 or len(seqs[b]) == 0:
            assert tuple(got[p]) == (0, -1, -1, -1, -1)


def test_one_set_against_itself_and_repeated_pairs(aligner, oracle_mod, blosum, plain10k, torch_cuda):
    torch = torch_cuda
    q, _ = device_sets(aligner, plain10k)
    rng = np.random.default_rng(15)
    pairs = rng.integers(0, 300, size=(2000, 2)).astype(np.int32)
    pairs[:50] = pairs[50:100]
    out = aligner.align(q, q, torch.from_numpy(pairs).cuda(), params(blosum)).cpu().numpy()
    want = oracle_mod.align_batch(plain10k.q_res, plain10k.q_off, plain10k.q_res, plain10k.q_off,
                                  pairs, blosum, 11, 1)
    assert_same(out, want)


def test_record_is_independent_of_the_batch(aligner, blosum, plain10k, torch_cuda):
    """A pair's record is the same alone, in a small batch and in the full one
    (different buckets, partners in the packed register, launch grids)."""
    torch = torch_cuda
    q, r = device_sets(aligner, plain10k)
    full = gpu_records(aligner, plain10k, params(blosum), sets=(q, r))
    rng = np.random.default_rng(16)
    pick = rng.choice(10000, size=40, replace=False)
    for k in pick[:10]:
        one = aligner.align(q, r, torch.from_numpy(plain10k.pairs[k:k + 1].copy()).cuda(),
                            params(blosum)).cpu().numpy()
        assert (one[0] == full[k]).all()
    few = aligner.align(q, r, torch.from_numpy(plain10k.pairs[pick].copy()).cuda(),
                        params(blosum)).cpu().numpy()
    assert (few == full[pick]).all()


def test_ascii_and_host_paths(aligner, oracle_mod, blosum, plain10k, torch_cuda):
    from paper_2303_01845_gb300 import workload
    sub = plain10k.subset(np.arange(0, 600))
    alpha = np.frombuffer(workload.ALPHABET.encode(), np.uint8)
    q_ascii = alpha[sub.q_res]
    # mixed case is accepted
    q_ascii = np.where(np.arange(len(q_ascii)) % 2 == 0, q_ascii, q_ascii + 32 * (q_ascii >= 65))
    qs = aligner.seqset(q_ascii.astype(np.uint8), sub.q_off, ascii=True)
    rs = aligner.seqset(sub.r_res, sub.r_off)
    got = aligner.align_host(qs, rs, np.ascontiguousarray(sub.pairs), params(blosum))
    assert_same(got, oracle_records(oracle_mod, sub, blosum, 11, 1), sub)


def test_seqset_offsets_checked_and_rebased_on_device(aligner, oracle_mod, blosum, plain10k, torch_cuda):
    """Sequence-set offsets are checked, measured and rebased on the device:
    offsets that start past 0 (host and device buffers) give the same records
    as the same sets starting at 0, the longest length is measured, and
    offsets that decrease in the middle are refused with ERANGE."""
    torch = torch_cuda
    from paper_2303_01845_gb300 import swgb
    sub = plain10k.subset(np.arange(0, 10000, 97))
    want = oracle_records(oracle_mod, sub, blosum, 11, 1)
    convs = {"host": lambda a: a, "pinned": lambda a: torch.from_numpy(a).pin_memory(),
             "device": lambda a: torch.from_numpy(a).cuda()}
    for shift in (0, 7):   # residues read 16 bytes at a time, or byte by byte
        pad = np.full(shift, 3, np.uint8)
        q_res = np.concatenate([pad, sub.q_res]); q_off = sub.q_off + shift
        r_res = np.concatenate([pad, sub.r_res]); r_off = sub.r_off + shift
        for kind, conv in convs.items():
            q = aligner.seqset(conv(q_res), conv(q_off))
            r = aligner.seqset(conv(r_res), conv(r_off))
            assert swgb.swgb_seqset_info(q.handle) == (len(sub.q_off) - 1, int(np.diff(sub.q_off).max()))
            got = gpu_records(aligner, sub, params(blosum), sets=(q, r))
            assert_same(got, want, sub)
            q.close()
            r.close()
    bad = np.array([0, 3, 2, 5], np.int64)   # total >= 0, decreasing in the middle
    for kind, conv in convs.items():
        res = np.zeros(5, np.uint8)
        with pytest.raises(swgb.SwgbError) as ei:
            aligner.seqset(conv(res), conv(bad))
        assert ei.value.code == swgb.SWGB_ERANGE
    # a code of 24 or more anywhere in a long set (the 16-byte pass) is refused
    long_res = np.random.default_rng(4).integers(0, 20, size=4000).astype(np.uint8)
    long_off = np.array([0, 1000, 4000], np.int64)
    for pos, code in ((0, 24), (1999, 255), (3999, 30)):
        res = long_res.copy()
        res[pos] = code
        for kind, conv in convs.items():
            with pytest.raises(swgb.SwgbError) as ei:
                aligner.seqset(conv(res), conv(long_off))
            assert ei.value.code == swgb.SWGB_EBADRES
    ok = aligner.seqset(convs["pinned"](long_res), convs["pinned"](long_off))
    assert swgb.swgb_seqset_info(ok.handle) == (2, 3000)
    ok.close()


def test_sets_uploaded_by_copy_engines_on_another_context(aligner, oracle_mod, blosum, plain10k, torch_cuda):
    """SWGB_SEQ_COPY sends pinned host residues through the copy engines
    instead of the encode kernel's in-place read: the same records, also from
    offsets that start past 0.  Sets of a second context, loaded on a helper
    thread while the first context aligns the other buffer (the pipelined
    end-to-end pattern), align identically."""
    torch = torch_cuda
    import concurrent.futures
    from paper_2303_01845_gb300 import swgb
    sub = plain10k.subset(np.arange(0, 10000, 53))
    want = oracle_records(oracle_mod, sub, blosum, 11, 1)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    pad = np.full(7, 3, np.uint8)
    q = aligner.seqset(pin(np.concatenate([pad, sub.q_res])), pin(sub.q_off + 7), copy=True)
    r = aligner.seqset(pin(np.concatenate([pad, sub.r_res])), pin(sub.r_off + 7), copy=True)
    assert swgb.swgb_seqset_info(q.handle) == (len(sub.q_off) - 1, int(np.diff(sub.q_off).max()))
    assert_same(gpu_records(aligner, sub, params(blosum), sets=(q, r)), want, sub)
    q.close()
    r.close()
    q_res, q_off, r_res, r_off = pin(sub.q_res), pin(sub.q_off), pin(sub.r_res), pin(sub.r_off)
    loader = swgb.Aligner(0)
    stream = torch.cuda.Stream()
    bufs = []
    try:
        bufs = [(loader.seqset(q_res, q_off, stream=stream, copy=True),
                 loader.seqset(r_res, r_off, stream=stream, copy=True)) for _ in range(2)]

        def load(k):
            bufs[k][0].load(q_res, q_off, stream=stream, copy=True)
            bufs[k][1].load(r_res, r_off, stream=stream, copy=True)

        with concurrent.futures.ThreadPoolExecutor(1) as ex:
            pending = ex.submit(load, 0)
            for i in range(4):
                pending.result()
                if i + 1 < 4:
                    pending = ex.submit(load, (i + 1) % 2)
                assert_same(gpu_records(aligner, sub, params(blosum), sets=bufs[i % 2]), want, sub)
    finally:
        for bq, br in bufs:
            bq.close()
            br.close()
        loader.close()


def test_errors_are_reported(aligner, blosum, plain10k, torch_cuda):
    torch = torch_cuda
    from paper_2303_01845_gb300 import swgb
    q, r = device_sets(aligner, plain10k)
    pairs = torch.tensor([[0, 0], [5, 10**6], [-1, 3], [7, 7]], dtype=torch.int32).cuda()
    with pytest.raises(swgb.SwgbError) as ei:
        aligner.align(q, r, pairs, params(blosum))
    assert ei.value.code == swgb.SWGB_ERANGE
    out = swgb.swgb_align(aligner.ctx, q.handle, r.handle, pairs, params(blosum))
    with pytest.raises(swgb.SwgbError):
        swgb.swgb_sync(aligner.ctx)
    got = out.cpu().numpy()
    assert tuple(got[1]) == (0, -1, -1, -1, -1) and tuple(got[2]) == (0, -1, -1, -1, -1)
    assert got[0, 0] > 0 and got[3, 0] > 0
    # the context stays usable
    ok = aligner.align(q, r, pairs[[0, 3]].contiguous(), params(blosum)).cpu().numpy()
    assert (ok == got[[0, 3]]).all()
    # bad residues
    with pytest.raises(swgb.SwgbError) as ei:
        aligner.seqset(np.array([0, 1, 30], np.uint8), np.array([0, 3], np.int64))
    assert ei.value.code == swgb.SWGB_EBADRES
    with pytest.raises(swgb.SwgbError) as ei:
        aligner.seqset(np.frombuffer(b"AC1D", np.uint8).copy(), np.array([0, 4], np.int64), ascii=True)
    assert ei.value.code == swgb.SWGB_EBADRES
    # too long
    with pytest.raises(swgb.SwgbError) as ei:
        aligner.seqset(np.zeros(swgb.SWGB_MAX_LENGTH + 1, np.uint8),
                       np.array([0, swgb.SWGB_MAX_LENGTH + 1], np.int64))
    assert ei.value.code == swgb.SWGB_ERANGE
    # bad penalties
    for go, ge in [(-1, 1), (11, 0), (120, 1)]:
        with pytest.raises(swgb.SwgbError) as ei:
            aligner.align(q, r, pairs[[0]].contiguous(), params(blosum, go, ge))
        assert ei.value.code == swgb.SWGB_EINVAL
    # empty batch
    empty = torch.zeros((0, 2), dtype=torch.int32).cuda()
    assert aligner.align(q, r, empty, params(blosum)).shape == (0, 5)


@pytest.fixture(scope="module")
def batched2m(blosum):
    from paper_2303_01845_gb300 import workload
    return workload.generate("batched_2m", blosum)


def test_batched_2m_sampled_parity(aligner, oracle_mod, blosum, batched2m, torch_cuda):
    """The full 2,000,000-pair workload in one call (the benchmark's launch
    configuration); a seeded sample of 20,000 pairs plus every 32-bit pair is
    compared with the oracle, and every record is checked for the properties
    that hold at any size."""
    torch = torch_cuda
    wl = batched2m
    q, r = device_sets(aligner, wl)
    pairs = torch.from_numpy(wl.pairs).cuda()
    out = aligner.align(q, r, pairs, params(blosum)).cpu().numpy()
    st = aligner.stats()
    assert st["forward_cells"] == wl.cells()
    ql = wl.q_len[wl.pairs[:, 0]]
    rl = wl.r_len[wl.pairs[:, 1]]
    s, qs, qe, rs, re_ = out.T
    assert (s >= 0).all() and (s <= 11 * np.minimum(ql, rl)).all()
    pos = s > 0
    assert (out[~pos] == [0, -1, -1, -1, -1]).all()
    assert ((0 <= qs) & (qs <= qe) & (qe < ql))[pos].all()
    assert ((0 <= rs) & (rs <= re_) & (re_ < rl))[pos].all()
    long_pairs = np.nonzero(11 * np.minimum(ql, rl) > 32767)[0]
    int32_pairs = np.array([p for p in long_pairs if int32_expected(
        blosum, wl.q_res[wl.q_off[p]:wl.q_off[p + 1]], wl.r_res[wl.r_off[p]:wl.r_off[p + 1]])],
        dtype=np.int64)
    assert st["n_int32_pairs"] == len(int32_pairs)
    rng = np.random.default_rng(17)
    sample = np.union1d(rng.choice(len(wl.pairs), size=20000, replace=False), long_pairs)
    sub = wl.subset(sample)
    assert_same(out[sample], oracle_records(oracle_mod, sub, blosum, 11, 1), sub)


def test_plan_replays_the_pipeline(aligner, blosum, plain10k, torch_cuda):
    """A plan captured into a CUDA graph gives the records swgb_align gives,
    and replays new pair lists written into the same buffer."""
    torch = torch_cuda
    from paper_2303_01845_gb300 import swgb
    q, r = device_sets(aligner, plain10k)
    prm = params(blosum)
    rng = np.random.default_rng(18)
    pick1 = rng.choice(10000, size=3000, replace=False)
    pick2 = rng.choice(10000, size=3000, replace=False)
    pairs = torch.from_numpy(plain10k.pairs[pick1].copy()).cuda()
    out = torch.zeros((3000, 5), dtype=torch.int32, device="cuda")
    plan = swgb.swgb_plan_create(aligner.ctx, q.handle, r.handle, pairs, prm, out)
    try:
        want1 = aligner.align(q, r, pairs.clone(), prm).cpu().numpy()
        swgb.swgb_plan_launch(aligner.ctx, plan)
        swgb.swgb_sync(aligner.ctx)
        assert (out.cpu().numpy() == want1).all()
        assert aligner.stats()["forward_cells"] == int(
            (plain10k.q_len[plain10k.pairs[pick1, 0]] * plain10k.r_len[plain10k.pairs[pick1, 1]]).sum())
        pairs.copy_(torch.from_numpy(plain10k.pairs[pick2].copy()))
        want2 = aligner.align(q, r, pairs.clone(), prm).cpu().numpy()
        out.zero_()
        swgb.swgb_plan_launch(aligner.ctx, plan)
        swgb.swgb_sync(aligner.ctx)
        assert (out.cpu().numpy() == want2).all()
    finally:
        swgb.swgb_plan_destroy(plan)
    # a plan captured with timing records its kernel times at every replay
    tprm = swgb.make_params(blosum, 11, 1, timing=True)
    plan = swgb.swgb_plan_create(aligner.ctx, q.handle, r.handle, pairs, tprm, out)
    try:
        for _ in range(2):
            swgb.swgb_plan_launch(aligner.ctx, plan)
            swgb.swgb_sync(aligner.ctx)
            st = aligner.stats()
            assert st["forward_ms"] > 0 and st["reverse_ms"] > 0
            assert st["total_ms"] >= st["forward_ms"] + st["reverse_ms"]
        assert (out.cpu().numpy() == want2).all()
    finally:
        swgb.swgb_plan_destroy(plan)


def test_plan_refuses_a_query_set_reloaded_with_other_letters(aligner, blosum, plain10k, torch_cuda):
    """A plan captured over queries of the 20 standard letters stages 21
    profile rows; once its query set is reloaded with B / Z / X / * codes the
    replay is refused (nothing is launched), and a new plan aligns the set."""
    torch = torch_cuda
    from paper_2303_01845_gb300 import swgb
    q, r = device_sets(aligner, plain10k)
    prm = params(blosum)
    pairs = torch.from_numpy(plain10k.pairs[:500].copy()).cuda()
    out = torch.zeros((500, 5), dtype=torch.int32, device="cuda")
    plan = swgb.swgb_plan_create(aligner.ctx, q.handle, r.handle, pairs, prm, out)
    try:
        res = plain10k.q_res.copy()
        res[::7] = 22   # X
        q.load(torch.from_numpy(res).cuda(), torch.from_numpy(plain10k.q_off).cuda())
        with pytest.raises(swgb.SwgbError) as ei:
            swgb.swgb_plan_launch(aligner.ctx, plan)
        assert ei.value.code == swgb.SWGB_EINVAL
    finally:
        swgb.swgb_plan_destroy(plan)
    want = aligner.align(q, r, pairs.clone(), prm).cpu().numpy()
    plan = swgb.swgb_plan_create(aligner.ctx, q.handle, r.handle, pairs, prm, out)
    try:
        out.zero_()
        swgb.swgb_plan_launch(aligner.ctx, plan)
        swgb.swgb_sync(aligner.ctx)
        assert (out.cpu().numpy() == want).all()
    finally:
        swgb.swgb_plan_destroy(plan)
    q.close()
    r.close()


def test_tile_selection_does_not_change_records(aligner, blosum, plain10k, torch_cuda):
    """Records are identical under every tile-cost setting, and the autotuner
    keeps one of its candidates."""
    torch = torch_cuda
    from paper_2303_01845_gb300 import swgb
    q, r = device_sets(aligner, plain10k)
    prm = params(blosum)
    pairs = torch.from_numpy(plain10k.pairs[::3].copy()).cuda()
    saved = swgb.swgb_get_tile_overhead(aligner.ctx)
    try:
        ref = None
        for c in [0, 3, 6, 12, 64]:
            swgb.swgb_set_tile_overhead(aligner.ctx, c)
            assert swgb.swgb_get_tile_overhead(aligner.ctx) == c
            got = aligner.align(q, r, pairs, prm).cpu().numpy()
            if ref is None:
                ref = got
            assert (got == ref).all()
        with pytest.raises(swgb.SwgbError):
            swgb.swgb_set_tile_overhead(aligner.ctx, 65)
        out = torch.zeros((pairs.shape[0], 5), dtype=torch.int32, device="cuda")
        best, ms = swgb.swgb_autotune(aligner.ctx, q.handle, r.handle, pairs, prm, out)
        assert best in (2, 4, 6, 8, 10, 12, 14, 17, 20, 24, 28, 32, 40) and ms > 0
        assert swgb.swgb_get_tile_overhead(aligner.ctx) == best
        assert (out.cpu().numpy() == ref).all()
    finally:
        swgb.swgb_set_tile_overhead(aligner.ctx, saved)
