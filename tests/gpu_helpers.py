"""Shared helpers of the GPU parity tests: run a workload through the C ABI and
through the oracle on identical inputs."""
import numpy as np


def device_sets(aligner, wl):
    import torch
    q = aligner.seqset(torch.from_numpy(wl.q_res).cuda(), torch.from_numpy(wl.q_off).cuda())
    r = aligner.seqset(torch.from_numpy(wl.r_res).cuda(), torch.from_numpy(wl.r_off).cuda())
    return q, r


def gpu_records(aligner, wl, params, sets=None):
    import torch
    from paper_2303_01845_gb300 import swgb
    q, r = sets if sets is not None else device_sets(aligner, wl)
    pairs = torch.from_numpy(np.ascontiguousarray(wl.pairs)).cuda()
    out = aligner.align(q, r, pairs, params)
    return out.cpu().numpy()


def oracle_records(oracle_mod, wl, mat, go, ge):
    return oracle_mod.align_batch(wl.q_res, wl.q_off, wl.r_res, wl.r_off, wl.pairs, mat, go, ge)


def assert_same(got, want, wl=None):
    got = np.asarray(got).reshape(-1, 5)
    want = np.asarray(want).reshape(-1, 5)
    assert got.shape == want.shape
    bad = np.nonzero((got != want).any(axis=1))[0]
    if len(bad):
        lines = []
        for p in bad[:10]:
            extra = ""
            if wl is not None:
                qi, ri = wl.pairs[p]
                extra = " lq=%d lr=%d" % (wl.q_off[qi + 1] - wl.q_off[qi], wl.r_off[ri + 1] - wl.r_off[ri])
            lines.append("pair %d: gpu %s oracle %s%s" % (p, got[p].tolist(), want[p].tolist(), extra))
        raise AssertionError("%d of %d records differ:\n%s" % (len(bad), len(got), "\n".join(lines)))
