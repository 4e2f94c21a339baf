"""The learned candidate filter end to end: exact labels from the aligner,
features, training on the device, threshold calibration, and the filtered
many-against-many search.

Orchestration only: every step runs in libswgb (discovery, features,
alignment, identity, the network's forward and backward passes, Adam, the
seeded training loop, threshold calibration, selection); this module passes
the sizes, seeds and recall target through.

The paper's own filter is the common-k-mer threshold (program-parameters
table); the learned one is trained on pass/fail labels of exact alignments
(identity >= 30 %, coverage >= 70 %) and keeps a candidate when its logit
reaches a threshold set for a target recall of the training positives.
"""
import numpy as np

from . import swgb


def exact_labels(al, s, cand, params, thresholds=None):
    """Aligns every candidate of set s against s and returns (records, identity
    records [P, 3] = matches, columns, pass) as CUDA tensors."""
    rec = swgb.swgb_align(al.ctx, s.handle, s.handle, cand, params)
    ident = swgb.swgb_identity(al.ctx, s.handle, s.handle, cand, rec, params, thresholds)
    return rec, ident


def train(al, features, labels, epochs=20, batch=2048, lr=3e-3, seed=1, pos_weight=None,
          init=None):
    """Trains a network on CUDA features [P, 32] / labels [P] (0 or 1) with
    swgb_mlp_fit: epochs of minibatch Adam in sample orders the library draws
    from `seed`; pos_weight None means the library's sqrt(negatives /
    positives).  Returns (MLP, per-epoch mean losses)."""
    import torch
    y = labels.to(torch.float32).contiguous()
    if init is None:
        init = init_params(seed)
    net = swgb.MLP(al.ctx, init)
    losses = net.fit(features, y, epochs, batch=batch, lr=lr,
                     pos_weight=0.0 if pos_weight is None else pos_weight, seed=seed)
    return net, losses


def init_params(seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and zero biases drawn
    with numpy's PCG64 from `seed`, float32, packed in the library's order
    (W1 [32][64], b1 [64], W2 [64][128], b2 [128], w3 [128], b3 [1])."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape, weight in (((32, 64), True), ((64,), False), ((64, 128), True), ((128,), False),
                          ((128,), True), ((1,), False)):
        if weight:
            lim = 1.0 / np.sqrt(shape[0])
            parts.append(rng.uniform(-lim, lim, size=shape).reshape(-1))
        else:
            parts.append(np.zeros(int(np.prod(shape))))
    return np.concatenate(parts).astype(np.float32)


def calibrate(net, features, labels, recall=0.995):
    """The largest threshold keeping at least `recall` of the positives of
    (features, labels) (swgb_mlp_calibrate)."""
    import torch
    return net.calibrate(features, labels.to(torch.float32).contiguous(), recall)


def filtered_search(al, s, net, threshold, params, k=6, min_shared=2, thresholds=None):
    """Discovery -> features -> network -> selection -> alignment and identity
    of the kept candidates.  Returns a dict of CUDA tensors: candidates,
    counts, logits, kept (pairs), kept_index, records, identity."""
    cand, counts = al.discover(s, k, min_shared)
    feats = swgb.swgb_pair_features(al.ctx, s.handle, s.handle, cand, k)
    logits = net.forward(feats)
    kept, index = swgb.swgb_select_pairs(al.ctx, cand, logits, threshold)
    rec, ident = exact_labels(al, s, kept.contiguous(), params, thresholds)
    return {"candidates": cand, "counts": counts, "logits": logits, "kept": kept,
            "kept_index": index, "records": rec, "identity": ident}
