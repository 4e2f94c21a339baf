"""GPU parity of candidate discovery (shared k-mers) and of alignment identity
/ pass-fail, through the C ABI, against the CPU oracle on the same seeded
inputs.  Candidate lists and counts must be identical (bit-exact integers);
identity records (identical columns, columns, pass) likewise."""
import numpy as np
import pytest

from paper_2303_01845_gb300 import workload

pytestmark = pytest.mark.gpu

K = 6


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch


@pytest.fixture(scope="module")
def aligner(torch_mod):
    from paper_2303_01845_gb300 import swgb
    al = swgb.Aligner(0)
    yield al
    al.close()


@pytest.fixture(scope="module")
def mat():
    from paper_2303_01845_gb300 import swgb
    return swgb.swgb_blosum62()


def pack(seqs):
    lens = np.array([len(s) for s in seqs], dtype=np.int64)
    off = np.zeros(len(seqs) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    res = (np.concatenate([np.asarray(s, np.uint8) for s in seqs]) if off[-1] > 0
           else np.zeros(0, np.uint8))
    return res, off


def gpu_set(aligner, torch_mod, res, off):
    return aligner.seqset(torch_mod.from_numpy(res).cuda(), torch_mod.from_numpy(off).cuda())


def gpu_discover(aligner, torch_mod, res, off, k=K, min_shared=2, capacity=None):
    s = gpu_set(aligner, torch_mod, res, off)
    pairs, counts = aligner.discover(s, k, min_shared, capacity)
    out = pairs.cpu().numpy(), counts.cpu().numpy()
    s.close()
    return out


def oracle_candidates(oracle_mod, res, off, k=K, min_shared=2):
    ix = oracle_mod.KmerIndex(res, off, k)
    try:
        return ix.all_candidates(min_shared)
    finally:
        ix.close()


def assert_same_candidates(got, want):
    gp, gc = got
    wp, wc = want
    assert gp.shape == wp.shape, (gp.shape, wp.shape)
    np.testing.assert_array_equal(gp, wp)
    np.testing.assert_array_equal(gc, wc)


# ---------------------------------------------------------------------------
# discovery
# ---------------------------------------------------------------------------
def test_discover_family_block_matches_oracle(aligner, torch_mod, oracle_mod, mat):
    fs = workload.generate_families("families_2k", mat)
    got = gpu_discover(aligner, torch_mod, fs.res, fs.off)
    want = oracle_candidates(oracle_mod, fs.res, fs.off)
    assert len(want[0]) > 1000
    assert_same_candidates(got, want)


@pytest.mark.parametrize("k,min_shared", [(1, 1), (2, 3), (3, 2), (4, 1), (5, 2), (6, 1)])
def test_discover_every_k_and_threshold(aligner, torch_mod, oracle_mod, k, min_shared):
    rng = np.random.default_rng(100 + 10 * k + min_shared)
    seqs = []
    for _ in range(300):
        L = int(rng.integers(0, 60))
        seqs.append(rng.integers(0, 24 if rng.random() < 0.2 else 20, L))
    res, off = pack(seqs)
    got = gpu_discover(aligner, torch_mod, res, off, k, min_shared)
    want = oracle_candidates(oracle_mod, res, off, k, min_shared)
    assert_same_candidates(got, want)


def test_discover_edge_sets(aligner, torch_mod, oracle_mod):
    A, L, W, X, STAR = 0, 10, 17, 22, 23
    seqs = [
        [],                                  # empty
        [A] * 5,                             # shorter than k
        [A] * 40,                            # homopolymer: one distinct k-mer
        [A] * 7,                             # shares that one k-mer
        [L, W] * 20,                         # period-2 repeat: two distinct k-mers
        [W, L] * 3,                          # both of them
        list(range(20)) + list(range(20)),   # 15 distinct k-mers, twice
        list(range(20)),                     # shares all 15
        list(range(10)) + [X] + list(range(10, 20)),   # X breaks windows
        list(range(6)) + [STAR] + list(range(6)),       # * breaks windows
        list(range(20)),                     # identical to an earlier sequence
    ]
    res, off = pack(seqs)
    for ms in (1, 2, 3):
        got = gpu_discover(aligner, torch_mod, res, off, K, ms)
        want = oracle_candidates(oracle_mod, res, off, K, ms)
        assert_same_candidates(got, want)
    # fewer than two sequences: nothing to find
    r1, o1 = pack([list(range(20))])
    p, c = gpu_discover(aligner, torch_mod, r1, o1)
    assert p.shape == (0, 2) and c.shape == (0,)


def test_discover_long_sequences_and_crowded_rows(aligner, torch_mod, oracle_mod):
    """A sequence of > 2048 k-mers takes the global-memory k-mer table, and rows
    with more than 2048 partner incidences the global-memory join table."""
    rng = np.random.default_rng(7)
    core = rng.integers(0, 20, 12)
    seqs = [np.concatenate([core, rng.integers(0, 20, int(rng.integers(0, 30)))])
            for _ in range(2600)]
    long_seq = rng.integers(0, 20, 9000)
    seqs[5] = np.concatenate([long_seq, core])
    seqs[6] = long_seq[1000:6000].copy()
    res, off = pack(seqs)
    got = gpu_discover(aligner, torch_mod, res, off)
    want = oracle_candidates(oracle_mod, res, off)
    assert len(want[0]) > 2599 * 2598 // 2
    assert_same_candidates(got, want)


def test_discover_capacity_reports_the_total(aligner, torch_mod, oracle_mod, mat):
    fs = workload.generate_families("families_2k", mat)
    full = gpu_discover(aligner, torch_mod, fs.res, fs.off)
    cap = len(full[0]) // 3
    from paper_2303_01845_gb300 import swgb
    s = gpu_set(aligner, torch_mod, fs.res, fs.off)
    pairs = torch_mod.zeros((cap, 2), dtype=torch_mod.int32, device="cuda")
    counts = torch_mod.zeros((cap,), dtype=torch_mod.int32, device="cuda")
    import ctypes
    found = ctypes.c_int64()
    rc = swgb.load().swgb_discover(aligner.ctx, s.handle, 6, 2, pairs.data_ptr(),
                                   counts.data_ptr(), cap, ctypes.byref(found),
                                   torch_mod.cuda.current_stream().cuda_stream)
    assert rc == 0
    assert found.value == len(full[0])
    np.testing.assert_array_equal(pairs.cpu().numpy(), full[0][:cap])
    np.testing.assert_array_equal(counts.cpu().numpy(), full[1][:cap])
    s.close()


def test_discover_rejects_bad_arguments(aligner, torch_mod):
    from paper_2303_01845_gb300 import swgb
    res, off = pack([list(range(20))] * 3)
    s = gpu_set(aligner, torch_mod, res, off)
    for k, ms in ((0, 2), (7, 2), (6, 0)):
        with pytest.raises(swgb.SwgbError) as e:
            aligner.discover(s, k, ms)
        assert e.value.code == swgb.SWGB_EINVAL
    s.close()


@pytest.mark.slow
def test_discover_full_block_sampled_rows(aligner, torch_mod, oracle_mod, mat):
    """The 200,000-sequence block: every candidate of 24 sampled sequences (as
    the first or the second member of a pair) against the oracle's merge of
    that sequence's k-mer set with every other set."""
    fs = workload.generate_families("families_200k", mat)
    pairs, counts = gpu_discover(aligner, torch_mod, fs.res, fs.off)
    assert (pairs[:, 0] < pairs[:, 1]).all()
    key = pairs[:, 0].astype(np.int64) * len(fs) + pairs[:, 1]
    assert (np.diff(key) > 0).all()       # ordered by (i, j), no duplicates
    ix = oracle_mod.KmerIndex(fs.res, fs.off, K)
    rng = np.random.default_rng(11)
    try:
        for i in rng.choice(len(fs), 24, replace=False):
            js, cs = ix.candidates_of(int(i), 2)
            sel1 = pairs[:, 0] == i
            sel2 = pairs[:, 1] == i
            gj = np.concatenate([pairs[sel2, 0], pairs[sel1, 1]])
            gc = np.concatenate([counts[sel2], counts[sel1]])
            o = np.argsort(gj, kind="stable")
            np.testing.assert_array_equal(gj[o], js)
            np.testing.assert_array_equal(gc[o], cs)
    finally:
        ix.close()


# ---------------------------------------------------------------------------
# identity and pass/fail
# ---------------------------------------------------------------------------
def identity_case(aligner, torch_mod, oracle_mod, mat, res_q, off_q, res_r, off_r, pairs, go=11,
                  ge=1, th=((3, 10), (7, 10))):
    from paper_2303_01845_gb300 import swgb
    q = gpu_set(aligner, torch_mod, res_q, off_q)
    r = gpu_set(aligner, torch_mod, res_r, off_r)
    params = swgb.make_params(mat, go, ge)
    dp = torch_mod.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).cuda()
    rec = aligner.align(q, r, dp, params)
    ident = aligner.identity(q, r, dp, rec, params, swgb.make_thresholds(*th)).cpu().numpy()
    rec = rec.cpu().numpy()
    q.close()
    r.close()
    want_rec = oracle_mod.align_batch(res_q, off_q, res_r, off_r, pairs, mat, go, ge)
    np.testing.assert_array_equal(rec, want_rec)
    want = np.zeros((len(pairs), 3), np.int32)
    for p, (qi, ri) in enumerate(pairs):
        qs = res_q[off_q[qi]:off_q[qi + 1]]
        rs = res_r[off_r[ri]:off_r[ri + 1]]
        mt, cols = oracle_mod.span_identity(qs, rs, want_rec[p], mat, go, ge)
        want[p] = (mt, cols, oracle_mod.passes(want_rec[p], mt, cols, len(qs), len(rs), *th))
    bad = np.nonzero((ident != want).any(axis=1))[0]
    assert not len(bad), "%d of %d differ; first pair %d gpu %s oracle %s record %s" % (
        len(bad), len(pairs), bad[0], ident[bad[0]].tolist(), want[bad[0]].tolist(),
        want_rec[bad[0]].tolist())
    return ident, want_rec


def test_identity_of_family_candidates(aligner, torch_mod, oracle_mod, mat):
    fs = workload.generate_families("families_2k", mat)
    pairs, _ = oracle_candidates(oracle_mod, fs.res, fs.off)
    ident, rec = identity_case(aligner, torch_mod, oracle_mod, mat, fs.res, fs.off, fs.res, fs.off,
                               pairs)
    assert ident[:, 2].sum() > 0 and (ident[:, 2] == 0).sum() > 0


@pytest.mark.parametrize("go,ge", [(11, 1), (11, 2), (5, 3), (0, 1)])
def test_identity_homologous_pairs_and_gap_settings(aligner, torch_mod, oracle_mod, mat, go, ge):
    wl = workload.generate(workload.Spec("id", 400, "uniform", 20, 700, seed=5 + go + ge), mat)
    identity_case(aligner, torch_mod, oracle_mod, mat, wl.q_res, wl.q_off, wl.r_res, wl.r_off,
                  wl.pairs, go, ge)


def test_identity_long_spans_take_the_large_class(aligner, torch_mod, oracle_mod, mat):
    """Spans above 65,536 words of decision bits (e.g. 1,500 x 1,500) run in
    the second launch with per-warp regions sized to the largest span."""
    wl = workload.generate(workload.Spec("idlong", 24, "uniform", 1200, 2600, seed=9,
                                         homologous_fraction=1.0), mat)
    ident, rec = identity_case(aligner, torch_mod, oracle_mod, mat, wl.q_res, wl.q_off, wl.r_res,
                               wl.r_off, wl.pairs)
    spans = (rec[:, 2] - rec[:, 1] + 1) * (rec[:, 4] - rec[:, 3] + 1)
    assert spans.max() > 1_000_000


def test_identity_edge_cases(aligner, torch_mod, oracle_mod, mat):
    W, P, A, L = 17, 14, 0, 10
    qs = [[W] * 30, [P, P], [], [A] * 10 + [W] * 20 + [A] * 10, list(range(20)), [L] * 300]
    rs = [[W] * 30, [W, W], [A, A], [W] * 10 + [P] * 5 + [W] * 10, list(range(19, -1, -1)),
          [L] * 299 + [W]]
    pairs = np.array([[k, k] for k in range(len(qs))], np.int32)
    rq, oq = pack(qs)
    rr, orr = pack(rs)
    ident, rec = identity_case(aligner, torch_mod, oracle_mod, mat, rq, oq, rr, orr, pairs)
    assert ident[0].tolist() == [30, 30, 1]       # identical: identity 1, coverage 1
    assert ident[1].tolist() == [0, 0, 0]         # P vs W: no positive score
    assert ident[2].tolist() == [0, 0, 0]         # empty query


def test_identity_thresholds(aligner, torch_mod, oracle_mod, mat):
    wl = workload.generate(workload.Spec("idth", 200, "uniform", 30, 300, seed=21), mat)
    for th in (((1, 2), (1, 2)), ((0, 1), (0, 1)), ((9, 10), (9, 10))):
        identity_case(aligner, torch_mod, oracle_mod, mat, wl.q_res, wl.q_off, wl.r_res, wl.r_off,
                      wl.pairs, th=th)


def test_identity_few_large_spans_among_small_ones(aligner, torch_mod, oracle_mod, mat):
    """Five long homologous pairs among many short ones: the large-span launch
    starts more warps than it has pairs, every warp with its own boundary
    column."""
    long_wl = workload.generate(workload.Spec("idfew", 5, "uniform", 600, 900, seed=31,
                                              homologous_fraction=1.0), mat)
    short_wl = workload.generate(workload.Spec("idmany", 300, "uniform", 20, 60, seed=32), mat)
    qs = [long_wl.q_res[long_wl.q_off[i]:long_wl.q_off[i + 1]] for i in range(5)] + \
         [short_wl.q_res[short_wl.q_off[i]:short_wl.q_off[i + 1]] for i in range(300)]
    rs = [long_wl.r_res[long_wl.r_off[i]:long_wl.r_off[i + 1]] for i in range(5)] + \
         [short_wl.r_res[short_wl.r_off[i]:short_wl.r_off[i + 1]] for i in range(300)]
    rq, oq = pack(qs)
    rr, orr = pack(rs)
    pairs = np.array([[k, k] for k in range(len(qs))], np.int32)
    ident, rec = identity_case(aligner, torch_mod, oracle_mod, mat, rq, oq, rr, orr, pairs)
    assert ((rec[:5, 4] - rec[:5, 3] + 1) > 256).all()


def test_identity_cooperative_spans_match_oracle(aligner, torch_mod, oracle_mod, mat):
    """Spans of more than 2,048 columns run on one block of four warps that
    pipeline the span's chunks."""
    wl = workload.generate(workload.Spec("idcoop", 6, "uniform", 2600, 4200, seed=41,
                                         homologous_fraction=1.0), mat)
    ident, rec = identity_case(aligner, torch_mod, oracle_mod, mat, wl.q_res, wl.q_off, wl.r_res,
                               wl.r_off, wl.pairs)
    assert ((rec[:, 4] - rec[:, 3] + 1) >= 2048).sum() >= 3


def test_identity_large_batch_keeps_mid_spans_regular(aligner, torch_mod, oracle_mod, mat):
    """A batch of more than 64 pairs per SM fills the GPU: there only spans of
    2,048+ columns go cooperative, those of 1,024..2,047 columns stay on one
    warp each (in a small batch both go cooperative)."""
    n_small = torch_mod.cuda.get_device_properties(0).multi_processor_count * 64 + 500
    long_wl = workload.generate(workload.Spec("idbig", 4, "uniform", 2300, 2600, seed=51,
                                              homologous_fraction=1.0), mat)
    mid_wl = workload.generate(workload.Spec("idmid", 4, "uniform", 1100, 1500, seed=52,
                                             homologous_fraction=1.0), mat)
    short_wl = workload.generate(workload.Spec("idshort", n_small, "uniform", 20, 60, seed=53), mat)
    parts = [(long_wl, 4), (mid_wl, 4), (short_wl, n_small)]
    qs = [w.q_res[w.q_off[i]:w.q_off[i + 1]] for w, n in parts for i in range(n)]
    rs = [w.r_res[w.r_off[i]:w.r_off[i + 1]] for w, n in parts for i in range(n)]
    rq, oq = pack(qs)
    rr, orr = pack(rs)
    pairs = np.array([[k, k] for k in range(len(qs))], np.int32)
    ident, rec = identity_case(aligner, torch_mod, oracle_mod, mat, rq, oq, rr, orr, pairs)
    cols = rec[:8, 4] - rec[:8, 3] + 1
    assert (cols[:4] >= 2048).sum() >= 2 and ((cols[4:] >= 1024) & (cols[4:] < 2048)).sum() >= 2


def test_identity_of_very_long_self_alignments(aligner, torch_mod, mat):
    """Closed form where the oracle's traceback matrix would not fit: a
    sequence of standard letters aligned with itself scores the sum of its
    diagonal over the whole length (every off-diagonal BLOSUM62 entry is below
    both diagonal ones), so its identity record is (n, n, pass).  Lengths
    33,000 (rows + columns >= 65,536: 64-bit statistics) and 6,000."""
    from paper_2303_01845_gb300 import swgb
    rng = np.random.default_rng(43)
    seqs = [rng.integers(0, 20, 33000).astype(np.uint8), rng.integers(0, 20, 6000).astype(np.uint8)]
    res, off = pack(seqs)
    s = aligner.seqset(torch_mod.from_numpy(res).cuda(), torch_mod.from_numpy(off).cuda())
    pairs = torch_mod.tensor([[0, 0], [1, 1]], dtype=torch_mod.int32, device="cuda")
    params = swgb.make_params(mat, 11, 1)
    rec = aligner.align(s, s, pairs, params)
    ident = aligner.identity(s, s, pairs, rec, params).cpu().numpy()
    rec = rec.cpu().numpy()
    for k, q in enumerate(seqs):
        n = len(q)
        assert rec[k].tolist() == [int(mat[q, q].astype(np.int64).sum()), 0, n - 1, 0, n - 1]
        assert ident[k].tolist() == [n, n, 1]
    s.close()
