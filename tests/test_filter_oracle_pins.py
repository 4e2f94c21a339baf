"""Pins of the learned-filter oracle: the pair features (filter_oracle.c) and
the network (mlp_oracle.py), checked against closed forms, brute force on
tiny inputs and finite differences, and planted-mistake mutants that these
checks must reject."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FEATURE_SRC = os.path.join(ROOT, "oracle", "filter_oracle.c")
K = 6


def ratio(num, den):
    return np.float32(0.0) if den == 0 else np.float32(np.float64(num) / np.float64(den))


def brute_features(a, b, k=K):
    """The 32 features by enumeration: every window pair compared letter by
    letter; first positions by scanning from the left."""
    a = [int(x) for x in a]
    b = [int(x) for x in b]
    la, lb = len(a), len(b)

    def std(s, p):
        return all(s[p + t] < 20 for t in range(k))

    def first(s, p):
        # is window p the first occurrence of its k-mer in s?
        return all(s[q:q + k] != s[p:p + k] for q in range(p) if std(s, q))

    fa = [p for p in range(la - k + 1) if std(a, p) and first(a, p)]
    fb = [q for q in range(lb - k + 1) if std(b, q) and first(b, q)]
    diags = [p - q for p in fa for q in fb if a[p:p + k] == b[q:q + k]]
    c = len(diags)
    D = la + lb - 2 * k + 1
    hist = [0] * 24
    for d in diags:
        hist[(24 * (d + lb - k)) // D] += 1
    comp = sum(abs(a.count(y) * lb - b.count(y) * la) for y in range(20))
    f = [ratio(c, c + 16), ratio(min(la, lb), max(la, lb))]
    f += [ratio(h, c) for h in hist]
    f += [ratio(comp, 2 * la * lb), ratio(la, la + 256), ratio(lb, lb + 256),
          ratio(max(hist), c), ratio(c, min(len(fa), len(fb)))]
    f += [ratio(max(diags) - min(diags), D) if c >= 2 else np.float32(0.0)]
    return np.array(f, np.float32)


def distinct_kmer_seq(rng, n, letters=range(20), k=K):
    """A sequence of n letters whose k-mers are all distinct."""
    letters = list(letters)
    while True:
        s = rng.choice(letters, n)
        w = {tuple(s[p:p + k]) for p in range(n - k + 1)}
        if len(w) == n - k + 1:
            return s.astype(np.uint8)


# ---------------------------------------------------------------------------
# features
# ---------------------------------------------------------------------------
def test_features_match_brute_force_on_small_pairs(oracle_mod):
    rng = np.random.default_rng(1)
    for trial in range(300):
        alpha = int(rng.choice([3, 4, 20, 24]))
        la, lb = (int(x) for x in rng.integers(0, 30, 2))
        a = rng.integers(0, alpha, la).astype(np.uint8)
        if trial % 3 == 0 and la > 8:
            b = np.concatenate([rng.integers(0, alpha, int(rng.integers(0, 6))), a[2:]]).astype(np.uint8)
        else:
            b = rng.integers(0, alpha, lb).astype(np.uint8)
        np.testing.assert_array_equal(oracle_mod.pair_features(a, b), brute_features(a, b),
                                      err_msg="trial %d" % trial)


def test_features_of_identical_sequences(oracle_mod):
    rng = np.random.default_rng(2)
    for L in (6, 7, 40, 300):
        a = distinct_kmer_seq(rng, L)
        f = oracle_mod.pair_features(a, a)
        n = L - K + 1
        hist = np.zeros(24, np.float32)
        hist[(24 * (L - K)) // (2 * L - 2 * K + 1)] = 1.0   # every diagonal is 0
        np.testing.assert_array_equal(f[2:26], hist)
        assert f[0] == np.float32(n / (n + 16))
        assert f[1] == 1.0 and f[26] == 0.0 and f[29] == 1.0 and f[30] == 1.0 and f[31] == 0.0
        assert f[27] == f[28] == np.float32(L / (L + 256))


def test_features_of_a_shifted_copy(oracle_mod):
    """b = three W + a (a without W): every shared k-mer lies on diagonal -3."""
    rng = np.random.default_rng(3)
    W = 17
    for L in (20, 90):
        a = distinct_kmer_seq(rng, L, letters=[x for x in range(20) if x != W])
        b = np.concatenate([[W, W, W], a]).astype(np.uint8)
        f = oracle_mod.pair_features(a, b)
        la, lb = L, L + 3
        D = la + lb - 2 * K + 1
        assert f[0] == np.float32((L - K + 1) / (L - K + 1 + 16))
        t = (24 * (-3 + lb - K)) // D
        assert f[2 + t] == 1.0 and f[2:26].sum() == 1.0
        assert f[31] == 0.0 and f[30] == 1.0
        assert f[1] == np.float32(la / lb)


def test_features_of_two_swapped_blocks(oracle_mod):
    """a = X + Y, b = Y + X: X's k-mers on diagonal -|Y|, Y's on +|X|."""
    rng = np.random.default_rng(4)
    X = distinct_kmer_seq(rng, 30, letters=range(10))
    Y = distinct_kmer_seq(rng, 40, letters=range(10, 20))
    a = np.concatenate([X, Y])
    b = np.concatenate([Y, X])
    f = oracle_mod.pair_features(a, b)
    L = 70
    D = 2 * L - 2 * K + 1
    nx, ny = 30 - K + 1, 40 - K + 1
    assert f[0] == np.float32((nx + ny) / (nx + ny + 16))
    assert f[2 + (24 * (-40 + L - K)) // D] == np.float32(nx / (nx + ny))
    assert f[2 + (24 * (30 + L - K)) // D] == np.float32(ny / (nx + ny))
    assert f[29] == np.float32(ny / (nx + ny))
    assert f[31] == np.float32(70 / D)
    assert f[26] == 0.0      # same composition


def test_features_of_disjoint_and_degenerate_pairs(oracle_mod):
    A, W = 0, 17
    f = oracle_mod.pair_features([A] * 10, [W] * 12)
    assert f[0] == 0.0 and f[2:26].sum() == 0.0 and f[29] == 0.0 and f[30] == 0.0
    assert f[26] == 1.0                      # disjoint compositions
    assert f[1] == np.float32(10 / 12)
    assert oracle_mod.pair_features([A] * 10, [A] * 10)[0] == np.float32(1 / 17)   # one k-mer
    f = oracle_mod.pair_features([], [])
    assert not f.any()
    f = oracle_mod.pair_features([22] * 20, [22] * 20)   # X forms no k-mer
    assert f[0] == 0.0 and f[26] == 0.0


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def mlp():
    from oracle import mlp_oracle
    return mlp_oracle


def test_bf16_rounding_is_round_to_nearest_even(mlp):
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert mlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    assert mlp.bf16(-3.0) == -3.0
    assert mlp.bf16(0.1) == 0.10009765625


def test_forward_of_a_hand_built_network(mlp):
    """W1 copies x0 to unit 0, W2 copies unit 0 to unit 5, w3 = 2 at unit 5,
    b3 = -1: the logit is 2 relu(x0) - 1 for inputs exact in bfloat16."""
    p = mlp.unpack(np.zeros(mlp.N_PARAMS))
    p["W1"][0, 0] = 1.0
    p["W2"][0, 5] = 1.0
    p["w3"][5] = 2.0
    p["b3"][0] = -1.0
    x = np.zeros((4, 32))
    x[:, 0] = [0.5, -0.25, 3.0, 0.0]
    z3, _ = mlp.forward(mlp.pack(p), x)
    np.testing.assert_array_equal(z3, [0.0, -1.0, 5.0, -1.0])


def test_loss_of_a_single_sample(mlp):
    """A zero network has logit b3: BCE = softplus(b3) - y b3 (weighted)."""
    p = mlp.unpack(np.zeros(mlp.N_PARAMS))
    p["b3"][0] = 0.7
    x = np.zeros((1, 32))
    for y, w in ((1.0, 3.0), (0.0, 3.0)):
        loss, g = mlp.loss_and_grad(mlp.pack(p), x, [y], pos_weight=w)
        ww = w if y else 1.0
        assert abs(loss - ww * (np.log1p(np.exp(0.7)) - y * 0.7)) < 1e-12
        gp = mlp.unpack(g)
        assert abs(gp["b3"][0] - ww * (1 / (1 + np.exp(-0.7)) - y)) < 1e-12


def _exact_grad_setting(mlp, seed, B=16):
    """Parameters and inputs on a bfloat16 grid with a loss free of rounding
    inside the products, so finite differences check the analytic gradient."""
    rng = np.random.default_rng(seed)
    flat = mlp.bf16(mlp.init_params(seed))
    x = mlp.bf16(rng.uniform(0, 1, (B, 32)))
    y = (rng.uniform(size=B) < 0.4).astype(np.float64)
    return flat, x, y


def test_gradient_matches_finite_differences(mlp, monkeypatch):
    """With the bfloat16 roundings of activations and gradients switched off,
    the analytic gradient equals central differences of the loss."""
    monkeypatch.setattr(mlp, "bf16", lambda v: np.asarray(v, dtype=np.float64))
    flat, x, y = _exact_grad_setting(mlp, 5)
    loss, g = mlp.loss_and_grad(flat, x, y, pos_weight=4.0)
    rng = np.random.default_rng(6)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 200, replace=False), [mlp.N_PARAMS - 1]])
    h = 1e-6
    for k in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[k] = h
        lp, _ = mlp.loss_and_grad(flat + e, x, y, pos_weight=4.0)
        lm, _ = mlp.loss_and_grad(flat - e, x, y, pos_weight=4.0)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_relu_masks_the_gradient(mlp):
    """A hidden unit that never activates gets no gradient in its weights."""
    flat, x, y = _exact_grad_setting(mlp, 7)
    p = mlp.unpack(flat)
    p["W1"][:, 3] = -1.0          # inputs are >= 0: unit 3 of layer 1 stays off
    p["b1"][3] = -0.5
    _, g = mlp.loss_and_grad(mlp.pack(p), x, y)
    gp = mlp.unpack(g)
    assert not gp["W1"][:, 3].any() and gp["b1"][3] == 0.0
    assert not gp["W2"][3, :].any()


def test_adam_first_step_moves_by_lr(mlp):
    """At step 1 the bias-corrected Adam step is lr * g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p, m, v = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


# ---------------------------------------------------------------------------
# planted mistakes
# ---------------------------------------------------------------------------
FEATURE_MUTANTS = {
    "last_position_kept": ("if (u == 0 || out[u - 1].kmer != out[x].kmer) out[u++] = out[x];",
                           "if (u == 0 || out[u - 1].kmer != out[x].kmer) out[u++] = out[x];"
                           " else out[u - 1] = out[x];"),
    "diagonal_sign": ("const int64_t d = ka[x].pos - kb[y].pos;",
                      "const int64_t d = kb[y].pos - ka[x].pos;"),
    "bin_offset": ("hist[(NBINS * (d + lb - k)) / D] += 1;", "hist[(NBINS * (d + la - k)) / D] += 1;"),
    "count_saturation": ("out[0] = ratio(c, c + 16);", "out[0] = ratio(c, c + 8);"),
    "spread_over_lengths": ("out[31] = c >= 2 ? ratio(dmax - dmin, D) : 0.0f;",
                            "out[31] = c >= 2 ? ratio(dmax - dmin, la + lb) : 0.0f;"),
    "composition_half": ("out[26] = ratio(comp, 2 * la * lb);", "out[26] = ratio(comp, la * lb);"),
    "nonstandard_windows": ("if (s[p + t] >= STD_LETTERS) { ok = 0; break; }",
                            "if (s[p + t] >= 24) { ok = 0; break; }"),
}


def _feature_battery(fn):
    """The feature pins above, as one boolean, against a features function."""
    try:
        rng = np.random.default_rng(11)
        for trial in range(120):
            alpha = int(rng.choice([3, 20, 24]))
            la, lb = (int(v) for v in rng.integers(0, 26, 2))
            a = rng.integers(0, alpha, la).astype(np.uint8)
            b = (np.concatenate([rng.integers(0, alpha, 2), a[1:]]).astype(np.uint8)
                 if trial % 2 else rng.integers(0, alpha, lb).astype(np.uint8))
            if not np.array_equal(fn(a, b), brute_features(a, b)):
                return False
        # the swapped-blocks closed form
        X = distinct_kmer_seq(np.random.default_rng(4), 30, letters=range(10))
        Y = distinct_kmer_seq(np.random.default_rng(5), 40, letters=range(10, 20))
        f = fn(np.concatenate([X, Y]), np.concatenate([Y, X]))
        D = 2 * 70 - 2 * K + 1
        return bool(f[31] == np.float32(70 / D) and f[2 + (24 * (-40 + 70 - K)) // D] > 0)
    except Exception:
        return False


def _compiled_features(text, tmp_path, name):
    c = tmp_path / (name + ".c")
    so = tmp_path / (name + ".so")
    c.write_text(text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(c)], check=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_pair_features.restype = ctypes.c_int
    lib.oracle_pair_features.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]

    def fn(a, b):
        a = np.ascontiguousarray(a, np.uint8)
        b = np.ascontiguousarray(b, np.uint8)
        out = np.zeros(32, np.float32)
        lib.oracle_pair_features(a.ctypes.data, len(a), b.ctypes.data, len(b), K, out.ctypes.data)
        return out
    return fn


def test_feature_battery_accepts_the_oracle(tmp_path):
    assert _feature_battery(_compiled_features(open(FEATURE_SRC).read(), tmp_path, "orig"))


@pytest.mark.parametrize("name", sorted(FEATURE_MUTANTS))
def test_feature_battery_rejects_mutant(name, tmp_path):
    old, new = FEATURE_MUTANTS[name]
    src = open(FEATURE_SRC).read()
    assert src.count(old) == 1, name
    assert not _feature_battery(_compiled_features(src.replace(old, new), tmp_path, name))


NET_MUTANTS = {
    "g3_sign": ("g3 = w * (sigmoid(z3) - y) / B", "g3 = w * (y - sigmoid(z3)) / B"),
    "no_batch_mean": ("g3 = w * (sigmoid(z3) - y) / B", "g3 = w * (sigmoid(z3) - y)"),
    "no_relu_mask_2": ("dz2 = bf16(np.outer(g3, p[\"w3\"]) * (c[\"z2\"] > 0))",
                       "dz2 = bf16(np.outer(g3, p[\"w3\"]))"),
    "mask_from_wrong_layer": ("* (c[\"z1\"] > 0))", "* (c[\"z2\"][:, :64] > 0))"),
    "bias_grad_mean": ("g[\"b2\"] = dz2.sum(axis=0)", "g[\"b2\"] = dz2.mean(axis=0)"),
    "unweighted_positives": ("w = np.where(y > 0.5, pos_weight, 1.0)", "w = np.ones_like(y)"),
}


def _net_battery(mod):
    """Finite differences of the loss (roundings off) and the single-sample
    closed form, as one boolean."""
    try:
        flat, x, y = _exact_grad_setting(mod, 5)
        saved = mod.bf16
        mod.bf16 = lambda v: np.asarray(v, dtype=np.float64)
        try:
            loss, g = mod.loss_and_grad(flat, x, y, pos_weight=4.0)
            rng = np.random.default_rng(6)
            for k in rng.choice(mod.N_PARAMS, 60, replace=False):
                e = np.zeros(mod.N_PARAMS)
                e[k] = 1e-6
                fd = (mod.loss_and_grad(flat + e, x, y, 4.0)[0] -
                      mod.loss_and_grad(flat - e, x, y, 4.0)[0]) / 2e-6
                if abs(fd - g[k]) > 1e-6 * max(1.0, abs(fd)):
                    return False
        finally:
            mod.bf16 = saved
        p = mod.unpack(np.zeros(mod.N_PARAMS))
        p["b3"][0] = 0.7
        loss, g = mod.loss_and_grad(mod.pack(p), np.zeros((1, 32)), [1.0], pos_weight=3.0)
        return abs(loss - 3.0 * (np.log1p(np.exp(0.7)) - 0.7)) < 1e-12
    except Exception:
        return False


def _load_net(text, tmp_path, name):
    import importlib.util
    path = tmp_path / (name + ".py")
    path.write_text(text)
    spec = importlib.util.spec_from_file_location("mlp_" + name, str(path))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_net_battery_accepts_the_oracle(tmp_path):
    src = open(os.path.join(ROOT, "oracle", "mlp_oracle.py")).read()
    assert _net_battery(_load_net(src, tmp_path, "orig"))


@pytest.mark.parametrize("name", sorted(NET_MUTANTS))
def test_net_battery_rejects_mutant(name, tmp_path):
    old, new = NET_MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "mlp_oracle.py")).read()
    assert src.count(old) == 1, name
    assert not _net_battery(_load_net(src.replace(old, new), tmp_path, name))
