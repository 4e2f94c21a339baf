"""GPU tests of the query server (swgb_server_*) and the resident k-mer index
(swgb_index_*) through the C ABI: index candidates against the oracle's
k-mer-set merges, server results against the same steps called directly,
each request's results the same alone and in the mix, and admission by
memory."""
import threading

import numpy as np
import pytest

from paper_2303_01845_gb300 import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch


@pytest.fixture(scope="module")
def mat():
    from paper_2303_01845_gb300 import swgb
    return swgb.swgb_blosum62()


def split_families(fs, copies):
    """References = the first copies - 1 members of every family, queries =
    the last member."""
    n = len(fs)
    last = np.arange(copies - 1, n, copies)
    is_q = np.zeros(n, bool)
    is_q[last] = True

    def pack(idx):
        lens = (fs.off[idx + 1] - fs.off[idx]).astype(np.int64)
        off = np.zeros(len(idx) + 1, np.int64)
        np.cumsum(lens, out=off[1:])
        res = np.concatenate([fs.res[fs.off[i]:fs.off[i + 1]] for i in idx]).astype(np.uint8)
        return res, off
    return pack(np.nonzero(~is_q)[0]), pack(last)


@pytest.fixture(scope="module")
def setup(torch_mod, mat):
    from paper_2303_01845_gb300 import swgb
    spec = workload.FamilySpec("serve_test", 600, 11, "lognormal", 20, 3000, median=250.0, sigma=0.7,
                               seed=21)
    fs = workload.generate_families(spec, mat)
    (rr, ro), (qr, qo) = split_families(fs, 11)
    al = swgb.Aligner(0)
    refs = al.seqset(torch_mod.from_numpy(rr).cuda(), torch_mod.from_numpy(ro).cuda())
    index = swgb.Index(al, refs, 6)
    yield al, refs, index, (rr, ro), (qr, qo)
    index.close()
    refs.close()
    al.close()


def requests_of(qr, qo, sizes):
    """Consecutive query ranges of the given sizes as (codes, offsets)."""
    out, q = [], 0
    for s in sizes:
        off = qo[q:q + s + 1] - qo[q]
        out.append((qr[qo[q]:qo[q + s]], off))
        q += s
    return out


def direct(al, index, refs, codes, offsets, params, torch_mod, net=None, threshold=0.0):
    """The server's steps called one by one on one request."""
    from paper_2303_01845_gb300 import swgb
    q = al.seqset(torch_mod.from_numpy(codes).cuda(), torch_mod.from_numpy(offsets).cuda())
    cand, counts = index.query(q, 2)
    n_cand = cand.shape[0]
    if net is not None and n_cand:
        feats = index.features(q, cand)
        kept, kidx = swgb.swgb_select_pairs(al.ctx, cand, net.forward(feats), threshold)
        counts = counts[kidx]
        cand = kept.contiguous()
    rec = swgb.swgb_align(al.ctx, q.handle, refs.handle, cand, params)
    ident = swgb.swgb_identity(al.ctx, q.handle, refs.handle, cand, rec, params)
    swgb.swgb_sync(al.ctx)
    out = {"pairs": cand.cpu().numpy(), "counts": counts.cpu().numpy(), "records": rec.cpu().numpy(),
           "identity": ident.cpu().numpy(), "candidates": n_cand}
    q.close()
    return out


def same(a, b):
    for k in ("pairs", "counts", "records", "identity"):
        np.testing.assert_array_equal(np.asarray(a[k]).reshape(-1), np.asarray(b[k]).reshape(-1), err_msg=k)
    assert a["candidates"] == b["candidates"]


def test_index_query_matches_oracle(setup, torch_mod, oracle_mod):
    al, refs, index, (rr, ro), (qr, qo) = setup
    q = al.seqset(torch_mod.from_numpy(qr).cuda(), torch_mod.from_numpy(qo).cuda())
    pairs, counts = index.query(q, 2)
    pairs, counts = pairs.cpu().numpy(), counts.cpu().numpy()
    q.close()
    # the oracle: every query's k-mer set merged with every reference's
    allres = np.concatenate([qr, rr])
    alloff = np.concatenate([qo, qo[-1] + ro[1:]])
    ix = oracle_mod.KmerIndex(allres, alloff, 6)
    nq = len(qo) - 1
    want_p, want_c = [], []
    try:
        for i in range(nq):
            js, cs = ix.candidates_of(i, 2)
            sel = js >= nq
            want_p += [(i, j - nq) for j in js[sel]]
            want_c += list(cs[sel])
    finally:
        ix.close()
    assert len(want_p) > 100
    np.testing.assert_array_equal(pairs, np.array(want_p, np.int32).reshape(-1, 2))
    np.testing.assert_array_equal(counts, np.array(want_c, np.int32))


def test_index_features_match_pair_features(setup, torch_mod):
    from paper_2303_01845_gb300 import swgb
    al, refs, index, _, (qr, qo) = setup
    q = al.seqset(torch_mod.from_numpy(qr).cuda(), torch_mod.from_numpy(qo).cuda())
    pairs, _ = index.query(q, 2)
    a = index.features(q, pairs).cpu().numpy()
    b = swgb.swgb_pair_features(al.ctx, q.handle, refs.handle, pairs).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    q.close()


@pytest.mark.parametrize("with_filter", [False, True])
def test_results_alone_and_in_the_mix(setup, torch_mod, mat, with_filter):
    """Twenty requests submitted at once by four client threads run in
    overlapping batches; each request's results equal those of the same
    request run alone on a one-slot server and those of the library calls
    made one by one."""
    from paper_2303_01845_gb300 import filter as F
    from paper_2303_01845_gb300 import swgb
    al, refs, index, _, (qr, qo) = setup
    params = swgb.make_params(mat, 11, 1)
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in rng.integers(1, 50, 20)]
    reqs = requests_of(qr, qo, sizes)
    mlp = F.init_params(3) if with_filter else None
    net = swgb.MLP(al.ctx, mlp) if with_filter else None
    thr = -0.05
    mixed = Server_run(refs, index, params, mlp, thr, reqs, slots=3, threads=4)
    res_mix, overlap = mixed
    assert overlap >= 2, "the batches never overlapped"
    alone, _ = Server_run(refs, index, params, mlp, thr, reqs, slots=1, threads=1, one_at_a_time=True)
    for k, (codes, offs) in enumerate(reqs):
        same(res_mix[k], alone[k])
        same(res_mix[k], direct(al, index, refs, codes, offs, params, torch_mod, net, thr))
    if net is not None:
        net.close()


def Server_run(refs, index, params, mlp, thr, reqs, slots, threads, one_at_a_time=False):
    from paper_2303_01845_gb300 import swgb
    srv = swgb.Server(refs, index, params, mlp, slots=slots, threshold=thr, max_batch_queries=64)
    results = [None] * len(reqs)
    if one_at_a_time:
        for k, (c, o) in enumerate(reqs):
            results[k] = srv.wait(srv.submit(c, o))
    else:
        tickets = [None] * len(reqs)

        def client(w):
            for k in range(w, len(reqs), threads):
                tickets[k] = srv.submit(*reqs[k])
        th = [threading.Thread(target=client, args=(w,)) for w in range(threads)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for k, t in enumerate(tickets):
            results[k] = srv.wait(t)
    overlap = srv.stats()["max_overlap"]
    srv.close()
    return results, overlap


def test_admission_by_memory(setup, torch_mod, mat):
    """A budget that holds one request at a time serialises the batches; a
    request above the budget is refused at submission."""
    from paper_2303_01845_gb300 import swgb
    al, refs, index, _, (qr, qo) = setup
    params = swgb.make_params(mat, 11, 1)
    reqs = requests_of(qr, qo, [10] * 6)
    one = max(24 * len(c) + 10 * 256 * 192 for c, _ in reqs)
    srv = swgb.Server(refs, index, params, None, slots=3, max_inflight_bytes=one,
                      max_batch_queries=10)
    tickets = [srv.submit(c, o) for c, o in reqs]
    for t in tickets:
        srv.wait(t)
    assert srv.stats()["max_overlap"] == 1
    big_q = requests_of(qr, qo, [40])[0]
    with pytest.raises(swgb.SwgbError) as e:
        srv.submit(*big_q)
    assert e.value.code == swgb.SWGB_ETOOBIG
    srv.close()


def test_server_rejects_bad_requests(setup, torch_mod, mat):
    """Host-side failures reach the caller as status codes, and the server
    keeps serving good requests after them."""
    from paper_2303_01845_gb300 import swgb
    al, refs, index, _, (qr, qo) = setup
    srv = swgb.Server(refs, index, swgb.make_params(mat, 11, 1), None, slots=2)
    codes, offs = requests_of(qr, qo, [3])[0]
    bad_code = codes.copy()
    bad_code[5] = 30
    with pytest.raises(swgb.SwgbError) as e:
        srv.submit(bad_code, offs)
    assert e.value.code == swgb.SWGB_EBADRES
    bad_off = offs.copy()
    bad_off[2] = bad_off[1] - 1
    with pytest.raises(swgb.SwgbError) as e:
        srv.submit(codes, bad_off)
    assert e.value.code == swgb.SWGB_ERANGE
    with pytest.raises(swgb.SwgbError) as e:
        srv.wait(123456789)
    assert e.value.code == swgb.SWGB_EINVAL
    res = srv.wait(srv.submit(codes, offs))
    assert res["candidates"] >= len(res["records"])
    # the batch's stage times are host wall times inside the request's latency
    assert len(res["stage_ms"]) == 5 and min(res["stage_ms"]) >= 0.0
    assert sum(res["stage_ms"]) <= res["latency_ms"] + 1e-3
    srv.close()
