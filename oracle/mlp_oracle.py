"""CPU oracle of the learned candidate filter's network: a 32 -> 64 -> 128 -> 1
multilayer perceptron with ReLU, BF16 weights and activations, FP32
accumulation, trained on a weighted binary cross-entropy with Adam.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports it.  The arithmetic is plain numpy in float64; the points where the
device rounds a value to bfloat16 (the operands of its matrix products) are
rounded here the same way (float64 -> float32 -> bfloat16, round to nearest
even), so that the two differ only by accumulation order and precision.

The paper has no learned filter (its only candidate filter is the common
k-mer threshold, program-parameters table); the network, its loss and its
optimiser are this library's definitions:

  x   = bf16(features)                    [B, 32]
  z1  = x W1 + b1,  a1 = bf16(relu(z1))   [B, 64]
  z2  = a1 W2 + b2, a2 = bf16(relu(z2))   [B, 128]
  z3  = a2 w3 + b3                        [B]      (the logit)
  L   = (1/B) sum_n w_n (softplus(z3_n) - y_n z3_n),  w_n = pos_weight if y_n else 1
  g3  = w (sigmoid(z3) - y) / B
  dw3 = a2^T g3,               db3 = sum g3
  dz2 = bf16(g3 w3^T * [z2 > 0]), dW2 = a1^T dz2, db2 = sum_n dz2
  dz1 = bf16(dz2 W2^T * [z1 > 0]), dW1 = x^T dz1,  db1 = sum_n dz1
  (W1, W2 in the products are their bfloat16 copies.)

Parameters are packed in this order (10,561 floats):
  W1 [32, 64] (row = input), b1 [64], W2 [64, 128], b2 [128], w3 [128], b3 [1].
"""
import numpy as np

N_IN, N_H1, N_H2 = 32, 64, 128
SHAPES = [("W1", (N_IN, N_H1)), ("b1", (N_H1,)), ("W2", (N_H1, N_H2)), ("b2", (N_H2,)),
          ("w3", (N_H2,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    """Packed parameter vector -> dict of float64 arrays."""
    flat = np.asarray(flat, dtype=np.float64).reshape(-1)
    if flat.size != N_PARAMS:
        raise ValueError("expected %d parameters" % N_PARAMS)
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[k:k + n].reshape(shape).copy()
        k += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(x):
    """Round to bfloat16 (via float32, round to nearest even), as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, drawn
    with numpy's PCG64 from `seed` (the device path receives these values)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.startswith("b"):
            p[name] = np.zeros(shape)
        else:
            fan_in = shape[0]
            lim = 1.0 / np.sqrt(fan_in)
            p[name] = rng.uniform(-lim, lim, size=shape)
    return pack(p).astype(np.float32).astype(np.float64)


def forward(flat, x):
    """Logits z3 [B] and the intermediate values (float64)."""
    p = unpack(flat)
    xb = bf16(x)
    z1 = xb @ bf16(p["W1"]) + p["b1"]
    a1 = bf16(np.maximum(z1, 0.0))
    z2 = a1 @ bf16(p["W2"]) + p["b2"]
    a2 = bf16(np.maximum(z2, 0.0))
    z3 = a2 @ p["w3"] + p["b3"][0]
    return z3, {"x": xb, "z1": z1, "a1": a1, "z2": z2, "a2": a2}


def softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def loss_and_grad(flat, x, y, pos_weight=1.0):
    """Weighted mean BCE over the batch and its gradient (packed)."""
    p = unpack(flat)
    z3, c = forward(flat, x)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    B = len(y)
    w = np.where(y > 0.5, pos_weight, 1.0)
    loss = float(np.sum(w * (softplus(z3) - y * z3)) / B)
    g3 = w * (sigmoid(z3) - y) / B
    g = {}
    g["w3"] = c["a2"].T @ g3
    g["b3"] = np.array([g3.sum()])
    dz2 = bf16(np.outer(g3, p["w3"]) * (c["z2"] > 0))
    g["W2"] = c["a1"].T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = bf16((dz2 @ bf16(p["W2"]).T) * (c["z1"] > 0))
    g["W1"] = c["x"].T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def adam_step(flat, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return flat - lr * mhat / (np.sqrt(vhat) + eps), m, v
