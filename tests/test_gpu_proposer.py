"""The learned proposer on the GPU against its FP64 oracle: features, forward pass and
gradients; training lowers the loss; and the trained net's recall and work saving."""
import os

import numpy as np
import pytest

from oracle import net as on
from synth import workloads

pytestmark = pytest.mark.gpu

NS = (1 << 16) + 16          # 16 x 4096 feature samples plus the largest feature lag


def oracle_params(flat):
    """Flat FP32 vector (W1 b1 ... W4 b4) -> [(W, b)] in FP64."""
    ps, o = [], 0
    for ci, co in zip(on.CH[:-1], on.CH[1:]):
        W = flat[o:o + co * ci * on.K].reshape(co, ci, on.K).astype(np.float64)
        o += co * ci * on.K
        b = flat[o:o + co].astype(np.float64)
        o += co
        ps.append((W, b))
    return ps


@pytest.fixture(scope="module")
def signals():
    return np.stack([workloads.mix_stream(i, NS, seed_base=0xC7C1_F004) for i in range(4)]).astype(np.complex64)


def gpu_features(cyc, xs):
    import torch
    n = xs.shape[0]
    xd = torch.from_numpy(xs.view(np.float32)).cuda()
    f = torch.empty((n, 11, 4096), dtype=torch.float16, device="cuda")
    cyc.cyc_features(xd, NS, n, f)
    return f


def test_features_match_oracle(cyc, signals):
    f = gpu_features(cyc, signals).float().cpu().numpy()
    for i, x in enumerate(signals):
        ref = on.features(x)
        assert np.max(np.abs(f[i] - ref)) < 2e-2, i


def test_forward_and_gradients_match_oracle(cyc, signals):
    import torch
    f = gpu_features(cyc, signals[:2])
    net = cyc.cyc_net_create(None, 7)
    try:
        flat = cyc.cyc_net_get_params(net)
        # the kernels use FP16 weights and features: give the oracle the same inputs
        ps = oracle_params(flat.astype(np.float16).astype(np.float32))
        feats = f.float().cpu().numpy().astype(np.float64)
        logits = torch.empty((2, 2, 512), dtype=torch.float32, device="cuda")
        cyc.cyc_net_forward(net, f, 2, logits)
        lg = logits.cpu().numpy()
        rng = np.random.default_rng(3)
        labels = (rng.uniform(size=(2, 2, 512)) < 0.02).astype(np.float32)
        for i in range(2):
            ref, _ = on.forward(ps, feats[i])
            scale = np.max(np.abs(ref)) + 1e-3
            assert np.max(np.abs(lg[i] - ref)) / scale < 2e-2, i
        g, loss = cyc.cyc_net_gradients(net, f, torch.from_numpy(labels).cuda(), 2, 5.0)
        lref, gref = on.batch_loss_and_grads(ps, list(feats), list(labels), pos_weight=5.0)
        assert abs(loss - lref) / lref < 1e-2
        # element by element, each tensor against a tolerance scaled by its largest entry
        # (FP16 activations and weights; a wrong gradient at a few positions, e.g. at the
        # circular wrap of a convolution, is an error of the order of those entries)
        go = oracle_params(g)
        for li, ((gW, gb), (rW, rb)) in enumerate(zip(go, gref)):
            errW = np.max(np.abs(gW - rW)) / np.max(np.abs(rW))
            errb = np.max(np.abs(gb - rb)) / np.max(np.abs(rb))
            assert errW < 3e-2, (li, errW)
            assert errb < 3e-2, (li, errb)
    finally:
        cyc.cyc_net_destroy(net)


def test_training_lowers_the_loss(cyc, signals):
    import torch
    f = gpu_features(cyc, signals)
    rng = np.random.default_rng(4)
    labels = torch.from_numpy((rng.uniform(size=(4, 2, 512)) < 0.02).astype(np.float32)).cuda()
    net = cyc.cyc_net_create(None, 9)
    try:
        first = cyc.cyc_net_train_step(net, f, labels, 4, 3e-3, 5.0)
        for _ in range(100):
            last = cyc.cyc_net_train_step(net, f, labels, 4, 3e-3, 5.0)
        assert last < 0.7 * first
    finally:
        cyc.cyc_net_destroy(net)


def test_trained_proposer_recall_and_gain(cyc):
    """The committed weights against full-grid detections on 1024 held-out signals of the mix:
    recall >= 99% of the detected cycle frequencies while running the estimator on 32 per
    form (or the full grid when the proposer falls back), i.e. with more than 4x less
    projection work than the full 512-point grid."""
    from paper_2405_16911_gb300 import proposer_train as pt
    import torch
    if not os.path.exists(pt.WEIGHTS):
        pytest.skip("no trained weights committed")
    n = 1024
    xs = pt.make_signals(n, pt.SEED_TEST)
    xd = torch.from_numpy(xs.view(np.float32)).cuda().view(n, NS * 2)
    labels = pt.label(cyc, xd, n)
    net = cyc.cyc_net_create(np.load(pt.WEIGHTS), 0)
    try:
        r = pt.recall_and_gain(cyc, net, xd, labels)
    finally:
        cyc.cyc_net_destroy(net)
    assert r["detections"] >= 100, r
    assert r["recall"] >= 0.99, r
    assert r["work_ratio"] > 4.0, r


def test_propose_path_equals_the_batch_path(cyc, signals):
    """cyc_propose computes one signal's features with a CTA per (channel, segment); its
    proposals must be the top-k of the logits that the batch path (cyc_features, one CTA per
    channel, then cyc_net_forward) gives for the same signal."""
    import torch
    net = cyc.cyc_net_create(None, 21)
    try:
        f = gpu_features(cyc, signals[:1])
        logits = torch.empty((1, 2, 512), dtype=torch.float32, device="cuda")
        cyc.cyc_net_forward(net, f, 1, logits)
        lg = logits.cpu().numpy()[0]
        xd = torch.from_numpy(signals[0].view(np.float32).copy()).cuda()
        ac, aj, conf, fb = cyc.cyc_propose(net, xd, NS, k=16, tau=0.0)
        for form, al in ((0, ac), (1, aj)):
            got = set(np.round((np.asarray(al) + 0.5) * 512).astype(int).tolist())
            order = np.argsort(-lg[form], kind="stable")
            assert got == set(order[:16].tolist()), form
    finally:
        cyc.cyc_net_destroy(net)
