"""The allocation-free entry point (swgb_align_noalloc) against swgb_align.

swgb_align_noalloc serves callers that cannot allocate device memory while
they align; its scratch is one fixed array inside the library, shared by every
call.  Two calls in a row (different batches, so the second starts from the
first one's leftovers) must each give exactly the records swgb_align gives.
The first call's records are also compared with the CPU oracle's.  The file
is collected last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _workload(seed):
    from paper_2303_01845_gb300 import swgb, workload
    mat = swgb.swgb_blosum62()
    wl = workload.generate(workload.Spec("na", 3000, "uniform", 20, 700, seed=seed), mat)
    # append long pairs: queries up to the 4096 limit, references past one
    # 512-row chunk, some on the 32-bit path
    rng = np.random.default_rng(seed)
    extra_q = [rng.integers(0, 20, size=n).astype(np.uint8) for n in (4096, 3000, 1500, 40)]
    extra_r = [np.resize(extra_q[0], 5000), extra_q[1].copy(), rng.integers(0, 20, size=2600).astype(np.uint8),
               rng.integers(0, 20, size=9000).astype(np.uint8)]
    qs = [wl.q_res[wl.q_off[k]:wl.q_off[k + 1]] for k in range(len(wl.q_off) - 1)] + extra_q
    rs = [wl.r_res[wl.r_off[k]:wl.r_off[k + 1]] for k in range(len(wl.r_off) - 1)] + extra_r
    n0 = len(wl.q_off) - 1
    pairs = np.concatenate([wl.pairs, [[n0 + k, n0 + k] for k in range(4)], [[n0, n0 + 3], [7, n0]]])
    return workload.from_sequences(qs, rs, pairs.astype(np.int32)), mat


def _tensors(wl):
    import torch
    return (torch.from_numpy(wl.q_res).cuda(), torch.from_numpy(wl.q_off).cuda(),
            torch.from_numpy(wl.r_res).cuda(), torch.from_numpy(wl.r_off).cuda())


def test_noalloc_matches_swgb_align_on_two_calls_in_a_row():
    import torch
    from paper_2303_01845_gb300 import swgb
    assert torch.cuda.is_available()
    al = swgb.Aligner(0)
    params = swgb.make_params(swgb.swgb_blosum62(), 11, 1)
    for call, seed in enumerate([21, 22]):
        wl, mat = _workload(seed)
        if call == 0:
            import oracle
            oracle_rec = oracle.align_batch(wl.q_res, wl.q_off, wl.r_res, wl.r_off, wl.pairs, mat, 11, 1)
        qc, qo, rc, ro = _tensors(wl)
        pairs = torch.from_numpy(wl.pairs).cuda()
        if call == 1:
            pairs = pairs[torch.randperm(len(pairs), generator=torch.Generator().manual_seed(3))
                          .cuda()].contiguous()
        qs = al.seqset(qc, qo)
        rs = al.seqset(rc, ro)
        want = al.align(qs, rs, pairs, params).cpu().numpy()
        out = torch.full((len(pairs), 5), -7, dtype=torch.int32, device="cuda")
        swgb.swgb_align_noalloc(qc, qo, rc, ro, pairs, params, out)
        got = out.cpu().numpy()
        bad = np.nonzero((got != want).any(axis=1))[0]
        assert len(bad) == 0, "call %d: %d records differ, first %s vs %s" % (
            call, len(bad), got[bad[0]].tolist(), want[bad[0]].tolist())
        assert (got[:, 0] > 0).sum() > len(got) // 2
        if call == 0:
            # and both against the oracle, record by record
            assert np.array_equal(got, oracle_rec)
        qs.close()
        rs.close()
    al.close()


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch
    from paper_2303_01845_gb300 import swgb
    params = swgb.make_params(swgb.swgb_blosum62(), 11, 1)
    long_q = torch.zeros(swgb.SWGB_NOALLOC_MAX_QUERY_LENGTH + 1, dtype=torch.uint8, device="cuda")
    off = torch.tensor([0, long_q.numel()], dtype=torch.int64, device="cuda")
    pairs = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    out = torch.zeros((1, 5), dtype=torch.int32, device="cuda")
    with pytest.raises(swgb.SwgbError) as ei:
        swgb.swgb_align_noalloc(long_q, off, long_q, off, pairs, params, out)
    assert ei.value.code == swgb.SWGB_ETOOBIG
    many = torch.zeros((swgb.SWGB_NOALLOC_MAX_PAIRS + 1, 2), dtype=torch.int32, device="cuda")
    out2 = torch.zeros((many.shape[0], 5), dtype=torch.int32, device="cuda")
    short = torch.zeros(10, dtype=torch.uint8, device="cuda")
    off2 = torch.tensor([0, 10], dtype=torch.int64, device="cuda")
    with pytest.raises(swgb.SwgbError) as ei:
        swgb.swgb_align_noalloc(short, off2, short, off2, many, params, out2)
    assert ei.value.code == swgb.SWGB_ETOOBIG


def test_noalloc_rejects_bad_offsets_and_tensors():
    """Negative or decreasing offsets are refused before any alignment kernel
    runs (no residue is read through them); tensors of the wrong type or
    shape are refused by the binding."""
    import torch
    from paper_2303_01845_gb300 import swgb
    params = swgb.make_params(swgb.swgb_blosum62(), 11, 1)
    codes = torch.zeros(64, dtype=torch.uint8, device="cuda")
    good = torch.tensor([0, 32, 64], dtype=torch.int64, device="cuda")
    pairs = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    out = torch.zeros((1, 5), dtype=torch.int32, device="cuda")
    for bad in ([-8, 32, 64], [0, 40, 32]):
        off = torch.tensor(bad, dtype=torch.int64, device="cuda")
        with pytest.raises(swgb.SwgbError) as ei:
            swgb.swgb_align_noalloc(codes, off, codes, good, pairs, params, out)
        assert ei.value.code == swgb.SWGB_ERANGE
    with pytest.raises(TypeError):
        swgb.swgb_align_noalloc(codes, good.to(torch.int32), codes, good, pairs, params, out)
    with pytest.raises(ValueError):
        swgb.swgb_align_noalloc(codes, good, codes, good, pairs.view(-1), params, out)
    # a good call after the refused ones
    swgb.swgb_align_noalloc(codes, good, codes, good, pairs, params, out)
    torch.cuda.synchronize()
