"""Learned activation proposer: activation traces of the progressive mesh,
training of the network with the library's own GPU kernels (lbm_mlp_*),
and the trained parameters.

A trace records, every few steps of a progressive-mesh run, the frontier
blocks with their features (lbm_frontier_features); the label of a block
is 1 when the criterion creates it within the next HORIZON steps (from
lbm_activation_steps at the end of the run).  Training minimises the mean
binary cross-entropy with Adam on mini-batches; inputs are standardised
with the training set's mean and standard deviation, which are stored
with the parameters.

    python -m paper_1510_03560_gb300.proposer --out proposer_weights.npz
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import workloads as W

PKG = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(PKG, "proposer_weights.npz")
HORIZON = 16
TRAIN_SEEDS = tuple(range(1510035610, 1510035618))
VALID_SEEDS = (1510035618, 1510035619)


def trace_case(seed: int, n: int = 128):
    """The 256^3 injection recipe at n^3 (inlet n/4 square) with another
    sphere seed."""
    return W.porous_injection(n=(n, n, n), seed=seed, inlet=n // 4, x_free=max(n // 16, 4))


def collect(L, seed: int, n: int = 128, steps: int = 1500, every: int = 4):
    """Features and labels of one run: X [m][34], Y [m]."""
    sim = L.from_case(trace_case(seed, n))
    rows = []
    for t in range(0, steps, every):
        ids, feat = sim.frontier_features()
        rows.append((t, ids, feat))
        sim.step(every)
    act = sim.activation_steps()
    sim.close()
    X = np.concatenate([f for _, _, f in rows]).astype(np.float32)
    Y = np.concatenate([((act[ids] > t) & (act[ids] <= t + HORIZON)).astype(np.float32)
                        for t, ids, _ in rows])
    return X, Y


def init_params(seed: int = 0) -> np.ndarray:
    """Random start: normal weights with variance 2 / fan-in, zero biases."""
    ni, nh = 34, 64
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0.0, np.sqrt(2.0 / ni), ni * nh), np.zeros(nh),
             rng.normal(0.0, np.sqrt(2.0 / nh), nh * nh), np.zeros(nh),
             rng.normal(0.0, np.sqrt(1.0 / nh), nh), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def standardise(X):
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    return mean.astype(np.float32), (1.0 / np.maximum(std, 1e-6)).astype(np.float32)


def metrics(prob: np.ndarray, Y: np.ndarray, thr: float = 0.5) -> dict:
    pred = prob > thr
    tp = float(np.sum(pred & (Y > 0.5)))
    return {"samples": int(len(Y)), "positives": int(np.sum(Y > 0.5)),
            "precision": tp / max(float(np.sum(pred)), 1.0),
            "recall": tp / max(float(np.sum(Y > 0.5)), 1.0),
            "accuracy": float(np.mean(pred == (Y > 0.5)))}


def train(L, X, Y, epochs: int = 30, batch: int = 4096, lr: float = 2e-3, seed: int = 0):
    """Adam on the library's kernels; returns params, mean, scale, losses."""
    import torch
    mean, scale = standardise(X)
    mlp = L.MLP(batch)
    mlp.set_params(init_params(seed))
    mlp.set_scaling(mean, scale)
    Xt = torch.tensor(X, device="cuda")
    Yt = torch.tensor(Y, device="cuda")
    rng = np.random.default_rng(seed)
    t = 0
    losses = []
    for _ in range(epochs):
        perm = torch.tensor(rng.permutation(len(Y)), device="cuda")
        tot = 0.0
        for k in range(0, len(Y), batch):
            idx = perm[k:k + batch]
            loss, _ = mlp.loss_grad(Xt[idx], Yt[idx])
            t += 1
            mlp.adam(lr, t)
            tot += loss * len(idx)
        losses.append(tot / len(Y))
    params = mlp.params()
    mlp.close()
    return params, mean, scale, losses


def load_model(L, path: str = WEIGHTS, max_batch: int = 1):
    """An lbm_mlp holding the stored parameters and standardisation."""
    d = np.load(path)
    mlp = L.MLP(max_batch)
    mlp.set_params(d["params"])
    mlp.set_scaling(d["mean"], d["scale"])
    return mlp


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--epochs", type=int, default=30)
    args = ap.parse_args(argv)
    import torch
    from . import build as B
    B.build()
    from . import lbm as L
    t0 = time.time()
    tr = [collect(L, s, args.n, args.steps) for s in TRAIN_SEEDS]
    va = [collect(L, s, args.n, args.steps) for s in VALID_SEEDS]
    X = np.concatenate([a for a, _ in tr]); Y = np.concatenate([b for _, b in tr])
    Xv = np.concatenate([a for a, _ in va]); Yv = np.concatenate([b for _, b in va])
    t1 = time.time()
    params, mean, scale, losses = train(L, X, Y, epochs=args.epochs)
    t2 = time.time()
    mlp = L.MLP(max(len(Yv), 1))
    mlp.set_params(params)
    mlp.set_scaling(mean, scale)
    pv = mlp.forward(torch.tensor(Xv, device="cuda"), bf16=True).cpu().numpy()
    mlp.close()
    info = {"train": metrics(np.zeros(0), np.zeros(0)) if len(Y) == 0 else None,
            "valid_bf16": metrics(pv, Yv), "losses": [round(v, 5) for v in losses],
            "trace_seconds": round(t1 - t0, 1), "train_seconds": round(t2 - t1, 1),
            "grid": args.n, "steps": args.steps, "horizon": HORIZON,
            "train_seeds": list(TRAIN_SEEDS), "valid_seeds": list(VALID_SEEDS),
            "train_samples": int(len(Y)), "train_positives": int(np.sum(Y > 0.5))}
    info.pop("train")
    np.savez(args.out, params=params, mean=mean, scale=scale, info=json.dumps(info))
    print(json.dumps(info))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
