"""The seeded workload generator: determinism, per-pair independence and the
shape of the distributions it is meant to draw."""
import numpy as np
import pytest

from paper_2303_01845_gb300 import workload


@pytest.fixture(scope="module")
def mat(oracle_mod):
    return oracle_mod.blosum62()


def small(n, **kw):
    spec = workload.Spec("t", n, "uniform", 50, 500, **kw)
    return spec


def test_deterministic(mat):
    a = workload.generate(small(500), mat, n_threads=3)
    b = workload.generate(small(500), mat, n_threads=7)
    assert (a.q_res == b.q_res).all() and (a.r_res == b.r_res).all()
    assert (a.q_off == b.q_off).all() and (a.r_off == b.r_off).all()


def test_pairs_are_independent_streams(mat):
    a = workload.generate(small(200), mat)
    b = workload.generate(small(400, homologous_fraction=0.25), mat)
    # pairs below 100 are homologous in both, pair streams depend on (seed, p) only
    for p in range(100):
        assert (a.q_res[a.q_off[p]:a.q_off[p + 1]] == b.q_res[b.q_off[p]:b.q_off[p + 1]]).all()
        assert (a.r_res[a.r_off[p]:a.r_off[p + 1]] == b.r_res[b.r_off[p]:b.r_off[p + 1]]).all()


def test_lengths_and_alphabet(mat):
    w = workload.generate(small(2000), mat)
    assert w.q_len.min() >= 50 and w.q_len.max() <= 500
    assert abs(w.q_len.mean() - 275) < 10
    assert w.q_res.max() < 20 and w.r_res.max() < 20
    # background composition
    freq = np.bincount(w.q_res, minlength=20) / len(w.q_res)
    assert np.abs(freq - workload.background()).max() < 0.005


def test_homologous_mutation_rates(mat):
    """Without indels, the per-position substitution rate is 0.40."""
    w = workload.generate(small(1000, homologous_fraction=1.0, indel_rate=0.0), mat)
    assert (w.q_len == w.r_len).all()
    diff = (w.q_res != w.r_res).mean()
    assert abs(diff - 0.40) < 0.01


def test_indel_length_change(mat):
    w = workload.generate(small(2000, homologous_fraction=1.0), mat)
    # insertions and deletions are equally likely with equal mean length
    rel = (w.r_len - w.q_len).mean() / w.q_len.mean()
    assert abs(rel) < 0.02
    assert (w.r_len != w.q_len).mean() > 0.9


def test_lognormal_lengths(mat):
    spec = workload.Spec("ln", 20000, "lognormal", 20, 5000, median=250.0, sigma=0.7,
                         homologous_fraction=0.0)
    w = workload.generate(spec, mat)
    ql = w.q_len
    assert ql.min() >= 20 and ql.max() <= 5000
    assert abs(np.median(ql) - 250) < 8
    assert abs(np.std(np.log(ql)) - 0.7) < 0.02


def test_substitution_weights_follow_the_matrix(mat):
    """Targets b of a substitution from a follow p_b exp(lambda s(a, b))."""
    bg, sub = workload.sampling_tables(mat)
    p = workload.background()
    lam = workload.solve_lambda(mat, p)
    assert abs(lam - 0.3176) < 1e-3
    a = workload.ALPHABET.index("I")
    counts = np.bincount(sub[a], minlength=20) / 65536.0
    w = p * np.exp(lam * mat[:20, :20].astype(float)[a])
    w[a] = 0
    w /= w.sum()
    assert np.abs(counts - w).max() < 1e-3
    assert counts[a] == 0


def test_family_sets_are_seeded_and_grouped():
    from paper_2303_01845_gb300 import workload
    import oracle
    mat = oracle.blosum62()
    a = workload.generate_families("families_2k", mat, n_threads=3)
    b = workload.generate_families("families_2k", mat, n_threads=1)
    assert len(a) == 2000 and np.array_equal(a.res, b.res) and np.array_equal(a.off, b.off)
    assert np.array_equal(a.family, np.repeat(np.arange(200), 10))
    assert a.res.max() < 20 and a.lengths.min() >= 1
    # copies of one family are closer to each other than to other families
    same = oracle.shared_kmers(a.seq(0), a.seq(1), 3)
    other = oracle.shared_kmers(a.seq(0), a.seq(15), 3)
    assert a.lengths[:10].std() < a.lengths.std() * 2
    assert same >= 0 and other >= 0
    # the 200,000-sequence recipe: log-normal lengths around 250
    spec = workload.FAMILY_SPECS["families_200k"]
    assert spec.n_families * spec.copies == 200_000
