"""The banded reverse pass (the band variant of dp_kernel) against the oracle.

A scored pair whose prefixes are long enough may find its start over a band of
diagonals instead of the whole rectangle; its result is kept only under the
exactness certificate, else the pair is re-run over the rectangle.  Either way
every record must equal the oracle's.  The cases: long homologous pairs of the
batched workload's recipe (most of them certified), pairs built so that their
optimal alignment leaves any band around the end diagonal through a long
excursion (the certificate must refuse them), pairs whose end drift is wide,
and the same batch with the band switched off.
"""
import numpy as np
import pytest

from gpu_helpers import assert_same, device_sets, oracle_records

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch


@pytest.fixture(scope="module")
def aligner(torch_cuda):
    from paper_2303_01845_gb300 import swgb
    al = swgb.Aligner(0)
    yield al
    al.close()


@pytest.fixture(scope="module")
def blosum(oracle_mod):
    return oracle_mod.blosum62()


def params(mat, go=11, ge=1):
    from paper_2303_01845_gb300 import swgb
    return swgb.make_params(mat, go, ge)


def long_homologous(mat, n, lmin, lmax, seed):
    from paper_2303_01845_gb300 import workload
    spec = workload.Spec("band_long", n, "uniform", lmin, lmax, homologous_fraction=1.0, seed=seed)
    return workload.generate(spec, mat)


def excursion_pairs(seed, n):
    """q = A X B Y C, r = A B C with |X| = |Y| = 200 and B, C long and
    identical: the best alignment matches B after a 200-column gap and C after
    another, so it runs 200 diagonals off the end diagonal and back."""
    from paper_2303_01845_gb300 import workload
    rng = np.random.default_rng(seed)
    qs, rs = [], []
    for _ in range(n):
        A = rng.integers(0, 20, size=int(rng.integers(100, 200)))
        B = rng.integers(0, 20, size=int(rng.integers(300, 500)))
        C = rng.integers(0, 20, size=int(rng.integers(100, 300)))
        X = rng.integers(0, 20, size=200)
        Y = rng.integers(0, 20, size=200)
        qs.append(np.concatenate([A, X, B, C]).astype(np.uint8))
        rs.append(np.concatenate([A, B, Y, C]).astype(np.uint8))
    pairs = np.stack([np.arange(n), np.arange(n)], axis=1).astype(np.int32)
    return workload.from_sequences(qs, rs, pairs)


def run(aligner, wl, prm, band_min):
    from paper_2303_01845_gb300 import swgb
    import torch
    saved = swgb.swgb_get_band_min(aligner.ctx)
    swgb.swgb_set_band_min(aligner.ctx, band_min)
    try:
        q, r = device_sets(aligner, wl)
        got = aligner.align(q, r, torch.from_numpy(wl.pairs).cuda(), prm).cpu().numpy()
        st = aligner.stats()
        q.close()
        r.close()
    finally:
        swgb.swgb_set_band_min(aligner.ctx, saved)
    return got, st


def test_long_homologous_pairs_bit_exact_and_mostly_certified(aligner, oracle_mod, blosum):
    """Homologous pairs of 900..1500 residues take the band and nearly all
    certify; pairs of 300..3000 mix band and rectangle; every record exact."""
    prm = params(blosum)
    wl = long_homologous(blosum, 1500, 900, 1500, seed=40)
    got, st = run(aligner, wl, prm, 256)
    assert_same(got, oracle_records(oracle_mod, wl, blosum, 11, 1), wl)
    assert st["n_band_pairs"] > 1400, st
    assert st["n_band_certified"] >= 0.9 * st["n_band_pairs"], st
    wl = long_homologous(blosum, 2000, 300, 3000, seed=41)
    got, st = run(aligner, wl, prm, 256)
    assert_same(got, oracle_records(oracle_mod, wl, blosum, 11, 1), wl)
    assert st["n_band_pairs"] > 600, st
    assert st["n_band_certified"] >= 0.8 * st["n_band_pairs"], st


def test_band_off_and_on_give_the_same_records(aligner, blosum):
    wl = long_homologous(blosum, 1500, 200, 1500, seed=42)
    prm = params(blosum)
    off, st0 = run(aligner, wl, prm, 0)
    assert st0["n_band_pairs"] == 0
    for band_min in (64, 384):
        on, st = run(aligner, wl, prm, band_min)
        assert st["n_band_pairs"] > 0
        assert (on == off).all(), band_min


def test_alignment_leaving_every_band_is_refused_by_the_certificate(aligner, oracle_mod, blosum):
    wl = excursion_pairs(43, 64)
    prm = params(blosum)
    got, st = run(aligner, wl, prm, 64)
    want = oracle_records(oracle_mod, wl, blosum, 11, 1)
    assert_same(got, want, wl)
    # the planted alignment: starts in A, ends in C
    assert (want[:, 1] < 200).all() and (want[:, 0] > 1500).all()
    assert st["n_band_pairs"] > 0
    assert st["n_band_certified"] < st["n_band_pairs"], st


def test_mixed_batch_with_gap_settings(aligner, oracle_mod, blosum):
    """Band and rectangle pairs, drift wider than the bands, short pairs and
    unrelated pairs in one batch, under several gap settings."""
    from paper_2303_01845_gb300 import workload
    a = long_homologous(blosum, 400, 300, 2500, seed=44)
    b = excursion_pairs(45, 20)
    rng = np.random.default_rng(46)
    qs = [a.q_res[a.q_off[k]:a.q_off[k + 1]] for k in range(len(a.q_off) - 1)]
    rs = [a.r_res[a.r_off[k]:a.r_off[k + 1]] for k in range(len(a.r_off) - 1)]
    qs += [b.q_res[b.q_off[k]:b.q_off[k + 1]] for k in range(len(b.q_off) - 1)]
    rs += [b.r_res[b.r_off[k]:b.r_off[k + 1]] for k in range(len(b.r_off) - 1)]
    for _ in range(40):   # drift of 300..900 residues: wider than any band
        core = rng.integers(0, 20, size=int(rng.integers(400, 800))).astype(np.uint8)
        qs.append(core)
        rs.append(np.concatenate([rng.integers(0, 20, size=int(rng.integers(300, 900))), core]).astype(np.uint8))
    for _ in range(40):   # unrelated long pairs
        qs.append(rng.integers(0, 20, size=int(rng.integers(400, 1500))).astype(np.uint8))
        rs.append(rng.integers(0, 20, size=int(rng.integers(400, 1500))).astype(np.uint8))
    n = len(qs)
    pairs = np.stack([np.arange(n), np.arange(n)], axis=1).astype(np.int32)
    pairs = pairs[rng.permutation(n)]
    wl = workload.from_sequences(qs, rs, pairs)
    for go, ge in ((11, 1), (11, 2), (5, 1)):
        got, st = run(aligner, wl, params(blosum, go, ge), 128)
        assert_same(got, oracle_records(oracle_mod, wl, blosum, go, ge), wl)
        assert st["n_band_pairs"] > 0


def test_band_setting_changes_between_calls_of_one_context(torch_cuda, oracle_mod, blosum):
    """A context whose workspace was grown for a small banded call, then set
    back to no band, aligns a larger batch (its maxima arrays hold the small
    call's pairs only and must not be touched), then a larger banded one."""
    from paper_2303_01845_gb300 import swgb
    al = swgb.Aligner(0)
    try:
        prm = params(blosum)
        small = long_homologous(blosum, 300, 900, 1400, seed=47)
        got, st = run(al, small, prm, 256)
        assert st["n_band_pairs"] > 0
        assert_same(got, oracle_records(oracle_mod, small, blosum, 11, 1), small)
        big = long_homologous(blosum, 4000, 50, 1200, seed=48)
        want = oracle_records(oracle_mod, big, blosum, 11, 1)
        got, st = run(al, big, prm, 0)
        assert st["n_band_pairs"] == 0
        assert_same(got, want, big)
        got, st = run(al, big, prm, 256)
        assert st["n_band_pairs"] > 0
        assert_same(got, want, big)
    finally:
        al.close()


def test_band_with_an_asymmetric_matrix_and_the_32_bit_path(aligner, oracle_mod, blosum):
    """The certificate does not depend on the matrix: BLOSUM62 with an
    asymmetric perturbation of -1..1 (homologous pairs still score high, so
    long ones take the band) gives the oracle's records; with the 32-bit path
    forced no pair takes the band (it needs the packed path)."""
    from paper_2303_01845_gb300 import swgb
    wl = long_homologous(blosum, 600, 700, 1600, seed=49)
    rng = np.random.default_rng(50)
    asym = (blosum.astype(np.int16) + rng.integers(-1, 2, size=blosum.shape)).astype(np.int8)
    assert not np.array_equal(asym, asym.T)
    got, st = run(aligner, wl, params(asym, 10, 1), 256)
    assert_same(got, oracle_records(oracle_mod, wl, asym, 10, 1), wl)
    assert st["n_band_pairs"] > 0
    got, st = run(aligner, wl, swgb.make_params(blosum, 11, 1, force_int32=True), 256)
    assert_same(got, oracle_records(oracle_mod, wl, blosum, 11, 1), wl)
    assert st["n_band_pairs"] == 0 and st["n_int32_pairs"] == len(wl.pairs)
