"""Training and evaluation of the learned cycle-frequency proposer (the net of include/cyc.h).

Signals come from the serving mix (GMSK BT 0.3/0.5, RRC(0.35) BPSK/QPSK, 2-16 samples per
symbol, carrier offset U(-1/4, 1/4), SNR U(-5, 20) dB), 65552 samples each.  Each signal is
labelled by the full-grid estimator itself (lags 0..63, a = -1/2 + k/512, both forms, BF16x3)
with a constant-false-alarm detection rule per form that judges every cycle frequency
against the estimator's noise around it (that noise is not flat in a: the spectrum of each
lag product piles variance near a = 0 for CONV and near twice the carrier for CONJ):

    s(a)  = max_m |R^a(m)|^2                        (the conventional a = 0 line excluded)
    nu(a) = median of s over the grid bins a +- 2..16
    detected  <=>  s(a) > kappa nu(a)  and  s(a) is the largest of its neighbours
    kappa = ln(A L F / P_fa) / (ln L + 0.5772)      (A = 512, L = 64, F = 2, P_fa = 1e-3)

For complex Gaussian estimator noise of variance sigma^2 per entry, the maximum over L lags
has median close to sigma^2 (ln L + Euler's constant) and exceeds sigma^2 ln(A L F / P_fa)
with probability P_fa / (A F), so kappa nu(a) is the false-alarm threshold with sigma^2
estimated locally; for white noise it is the fixed threshold ln(A L F / P_fa) R^0(0)^2/N_eff.
and the net is trained with the library's own forward, backward and Adam kernels.

    python -m paper_2405_16911_gb300.proposer_train --train 4096 --test 512 --out weights.npy
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np

NS = (1 << 16) + 16          # 16 x 4096 feature samples plus the largest feature lag
LAGS = np.arange(64, dtype=np.int32)
GRID = -0.5 + np.arange(512) / 512.0
P_FA = 1e-3
SEED_TRAIN, SEED_TEST = 0xC7C1_0004, 0xC7C1_8004
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "proposer_weights.npy")


def _gen(args):
    from synth import workloads
    sid, base = args
    return workloads.mix_stream(sid, NS, seed_base=base)


def make_signals(n: int, seed_base: int, workers: int = 0) -> np.ndarray:
    """[n][NS] complex64, generated in a spawn pool (safe before or after CUDA use)."""
    import multiprocessing as mp
    workers = workers or min(16, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        sigs = pool.map(_gen, [(i, seed_base) for i in range(n)], chunksize=16)
    return np.stack(sigs).astype(np.complex64)


WIN = 16
KAPPA = math.log(len(GRID) * len(LAGS) * 2 / P_FA) / (math.log(len(LAGS)) + 0.5772156649)


def detect(R: np.ndarray, n_eff: int) -> np.ndarray:
    """Labels [2][512] from a full-grid estimate R [2][512][64] (see module doc)."""
    s2 = (np.abs(R) ** 2).max(axis=2)
    s2[0, 256] = 0.0                                # the conventional a = 0 line is always there
    A = s2.shape[1]
    offs = np.array([d for d in range(-WIN, WIN + 1) if abs(d) > 1])
    idx = (np.arange(A)[:, None] + offs[None, :]) % A
    nu = np.median(s2[:, idx], axis=2)
    left, right = np.roll(s2, 1, axis=1), np.roll(s2, -1, axis=1)
    return ((s2 > KAPPA * nu) & (s2 >= left) & (s2 >= right)).astype(np.float32)


def label(pkg, xs_dev, n: int, precision: str = "bf16x3"):
    """Full-grid estimates of n signals already on the device -> labels [n][2][512]."""
    labels = np.zeros((n, 2, 512), dtype=np.float32)
    with pkg.Stream(LAGS, GRID, pkg.CYC_BOTH, precision=precision, max_chunk=NS) as s:
        for i in range(n):
            s.reset()
            s.push(xs_dev[i])
            R, n_eff = s.read()
            labels[i] = detect(R, n_eff)
    return labels


def features(pkg, xs_dev, n: int):
    import torch
    f = torch.empty((n, 11, 4096), dtype=torch.float16, device="cuda")
    step = 256
    for i in range(0, n, step):
        m = min(step, n - i)
        pkg.cyc_features(xs_dev[i], NS, m, f[i])
    return f


def recall_and_gain(pkg, net, xs_dev, labels, k: int = 32, tau: float = 0.9):
    """Share of the full-grid detections within +-1 bin of a proposal (proposals count as
    the full grid when the proposer falls back), and the projection work saved."""
    hit = hit_topk = tot = 0
    fallbacks = 0
    work = 0
    for i in range(len(labels)):
        ac, aj, conf, fb = pkg.cyc_propose(net, xs_dev[i], NS, k=k, tau=tau)
        fallbacks += fb
        work += 2 * 512 if fb else 2 * k
        for f, al in ((0, ac), (1, aj)):
            det = np.nonzero(labels[i, f] > 0.5)[0]
            tot += det.size
            prop = np.round((al + 0.5) * 512).astype(int) % 512
            found = sum(1 for d in det if np.any(np.abs(((prop - d + 256) % 512) - 256) <= 1))
            hit_topk += found
            hit += det.size if fb else found
    n = len(labels)
    return {"recall": hit / max(tot, 1), "recall_topk_only": hit_topk / max(tot, 1), "detections": tot,
            "signals": n, "fallback_rate": fallbacks / n, "work_ratio": (2 * 512 * n) / max(work, 1)}


def train(pkg, feats, labels, epochs: int = 30, batch: int = 32, lr: float = 2e-3, pos_weight: float = 4.0,
          seed: int = 1, log=print):
    import torch
    net = pkg.cyc_net_create(None, seed)
    lab = torch.from_numpy(labels).cuda()
    n = feats.shape[0]
    rng = np.random.default_rng(seed)
    for ep in range(epochs):
        order = rng.permutation(n)
        tot = 0.0
        t0 = time.perf_counter()
        lr_ep = lr * (0.5 ** (ep // 10))
        for s in range(0, n - batch + 1, batch):
            idx = torch.from_numpy(order[s:s + batch]).cuda()
            fb = feats.index_select(0, idx).contiguous()
            lb = lab.index_select(0, idx).contiguous()
            tot += pkg.cyc_net_train_step(net, fb, lb, batch, lr_ep, pos_weight)
        torch.cuda.synchronize()
        log("epoch %d loss %.5f (%.1f s)" % (ep, tot / max(1, n // batch), time.perf_counter() - t0))
    return net


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=4096)
    ap.add_argument("--test", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--tau", type=float, default=0.9)
    ap.add_argument("--out", default=WEIGHTS)
    args = ap.parse_args()
    t0 = time.perf_counter()
    xtr = make_signals(args.train, SEED_TRAIN)
    xte = make_signals(args.test, SEED_TEST)
    print("signals generated in %.1f s" % (time.perf_counter() - t0))
    import torch

    import paper_2405_16911_gb300 as pkg
    pkg.load()
    dtr = torch.from_numpy(xtr.view(np.float32)).cuda().view(args.train, NS * 2)
    dte = torch.from_numpy(xte.view(np.float32)).cuda().view(args.test, NS * 2)
    t0 = time.perf_counter()
    ltr = label(pkg, dtr, args.train)
    lte = label(pkg, dte, args.test)
    print("labelled in %.1f s: %.2f CONV + %.2f CONJ detections per signal" % (
        time.perf_counter() - t0, ltr[:, 0].sum() / args.train, ltr[:, 1].sum() / args.train))
    from synth import workloads
    kinds = np.array([workloads.mix_stream_params(i, SEED_TRAIN)["kind"] for i in range(args.train)])
    for kd, name in enumerate(("GMSK 0.3", "GMSK 0.5", "RRC BPSK", "RRC QPSK")):
        m = kinds == kd
        print("  %-8s %5d signals: %.2f CONV, %.2f CONJ detections" % (
            name, m.sum(), ltr[m, 0].sum() / max(m.sum(), 1), ltr[m, 1].sum() / max(m.sum(), 1)))
    ftr = features(pkg, dtr, args.train)
    net = train(pkg, ftr, ltr, epochs=args.epochs)
    np.save(args.out, pkg.cyc_net_get_params(net))
    for tau in (args.tau, 0.8, 0.7, 0.5, 0.0):
        print("test tau=%.2f:" % tau, recall_and_gain(pkg, net, dte, lte, tau=tau))
    pkg.cyc_net_destroy(net)


if __name__ == "__main__":
    main()
