"""Trains the weights of the learned T5 selection -- TEST INFRASTRUCTURE, run by hand:

    python -m oracle.train_t5_mlp            # writes paper_2407_18231_gb300/data/t5_mlp_pu200.json

The paper's LST selections include machine-learning methods (Sec. 1) whose trained weights
are not published; this script trains a network of the same role on the synthetic events
the tests and benchmark use, with the oracle as the only source of candidates and inputs.

Candidates: every pair of T3s sharing an MD (T3 (a, b, c) followed by T3 (c, d, e)) that
the oracle's chain builds on PU200-like events in the flat geometry, restricted to those
passing the full-circle radius and the (a, c, e) r-z conditions -- the two conditions the
network leaves in place.  Label: all ten hits of the five MDs come from one simulated
track.  Inputs: ``oracle.t5_features`` (binary32, the library's definition).

Model and fit: 8-16-16-1 rectified network, logistic loss with the positives weighted 5x,
Adam (learning rate 3e-3, batches of 4096, 60 epochs), float64 numpy from a fixed seed;
weights rounded once to float32.  Working point: the output bias is lowered until
``KEEP`` of the training positives pass under the oracle's binary32 evaluation of the
network.  The file also records, on events not trained on, the fraction of true T5
candidates kept and the non-true candidates accepted, for the network and the cuts.
Re-running reproduces the stored weights up to the rounding of numpy's matrix products.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import lst_synth as S  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(ROOT, "paper_2407_18231_gb300", "data", "t5_mlp_pu200.json")
TRAIN_EVENTS = range(1000, 1016)
HELDOUT_EVENTS = range(2000, 2004)
KEEP = 0.999
NF, NH = oracle.T5_NF, oracle.T5_NH
INPUTS = ["d1/(d1+rhs1)", "d2/(d2+rhs2)", "d1/(d1+|kin|+|kout|+k0)", "d2/(d2+|kbr|+|kfull|+k0)",
          "(tin+tout)/((tin+tout)+|kin|+|kout|+k0)", "|kfull|/kmax", "rz(a,c,e) l/(l+t)", "rz(b,c,d) l/(l+t)"]


def candidates(og, ev):
    """(inputs, true?, passes the cuts?) of the T5 candidates of one event that pass the
    radius and (a, c, e) r-z conditions."""
    r = oracle.run(og, ev)
    md, t3 = r["md"], r["t3"]
    P = np.stack([ev.x, ev.y, ev.z], 1)
    starting = {}
    for k, t in enumerate(t3):
        starting.setdefault(int(t[0]), []).append(k)
    F, Y, CUT = [], [], []
    for t in t3:
        for k2 in starting.get(int(t[2]), []):
            ch = [int(t[0]), int(t[1]), int(t[2]), int(t3[k2][1]), int(t3[k2][2])]
            mods, pts = md[ch, 0], P[md[ch, 1]]
            mask, _, _ = oracle.t5_eval(og, mods, pts)
            if mask & (oracle.T5_RADIUS | oracle.T5_RZ) != oracle.T5_RADIUS | oracle.T5_RZ:
                continue
            hits = np.concatenate([ev.sim[md[ch, 1]], ev.sim[md[ch, 2]]])
            F.append(oracle.t5_features(og, mods, pts))
            Y.append(bool(hits[0] >= 0 and np.all(hits == hits[0])))
            CUT.append(mask == 15)
    return np.array(F, np.float32).reshape(-1, NF), np.array(Y), np.array(CUT)


def collect(og, events):
    parts = [candidates(og, S.make_event("pu200", i)) for i in events]
    return tuple(np.concatenate([p[k] for p in parts]) for k in range(3))


def forward(W, X):
    a1 = X @ W[0].T + W[1]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W[2].T + W[3]
    h2 = np.maximum(a2, 0.0)
    return h2 @ W[4] + W[5][0], (a1, h1, a2, h2)


def gradients(W, X, Y, wt):
    """Gradients of the weighted mean logistic loss (back-propagation by hand)."""
    z, (a1, h1, a2, h2) = forward(W, X)
    g = (1.0 / (1.0 + np.exp(-z)) - Y) * wt / wt.sum()
    gh2 = np.outer(g, W[4]) * (a2 > 0)
    gh1 = gh2 @ W[2] * (a1 > 0)
    return [gh1.T @ X, gh1.sum(0), gh2.T @ h1, gh2.sum(0), h2.T @ g, np.array([g.sum()])]


def train(X, Y, seed=1, epochs=60, batch=4096, lr=3e-3, pos_weight=5.0):
    rng = np.random.default_rng(seed)
    W = [rng.normal(0, np.sqrt(2.0 / NF), (NH, NF)), np.zeros(NH), rng.normal(0, np.sqrt(2.0 / NH), (NH, NH)),
         np.zeros(NH), rng.normal(0, np.sqrt(1.0 / NH), NH), np.zeros(1)]
    m = [np.zeros_like(w) for w in W]
    v = [np.zeros_like(w) for w in W]
    X = X.astype(np.float64)
    Yf = Y.astype(np.float64)
    wt = np.where(Y, pos_weight, 1.0)
    b1, b2, step = 0.9, 0.999, 0
    for _ in range(epochs):
        perm = rng.permutation(len(Y))
        for s in range(0, len(Y), batch):
            idx = perm[s:s + batch]
            G = gradients(W, X[idx], Yf[idx], wt[idx])
            step += 1
            for k in range(6):
                m[k] = b1 * m[k] + (1 - b1) * G[k]
                v[k] = b2 * v[k] + (1 - b2) * G[k] ** 2
                W[k] -= lr * (m[k] / (1 - b1 ** step)) / (np.sqrt(v[k] / (1 - b2 ** step)) + 1e-8)
    return W


def pack(W) -> np.ndarray:
    """float32 weights in the library's order: W1, b1, W2, b2, w3, b3."""
    w = np.concatenate([W[0].ravel(), W[1], W[2].ravel(), W[3], W[4], W[5]]).astype(np.float32)
    assert w.size == oracle.T5_NPARAM
    return w


def logits(w, X):
    """The oracle's binary32 network output for every row of X."""
    return np.array([oracle.t5_logit(w, x) for x in X], np.float32)


def main():
    t0 = time.time()
    og = oracle.Geometry(S.geometry(False).modules)
    X, Y, CUT = collect(og, TRAIN_EVENTS)
    W = train(X, Y)
    w = pack(W)
    # working point: lower b3 so that KEEP of the training positives have z > 0
    zpos = np.sort(logits(w, X[Y]))
    q = float(zpos[int(np.floor((1.0 - KEEP) * len(zpos)))])
    w[-1] = np.float32(float(w[-1]) - q + 1e-6 * max(1.0, abs(q)))
    z = logits(w, X)
    Xh, Yh, CUTh = collect(og, HELDOUT_EVENTS)
    zh = logits(w, Xh)
    rec = {
        "format": "lst-t5-mlp-1",
        "inputs": INPUTS,
        "hidden": NH,
        "order": "W1[16][8], b1[16], W2[16][16], b2[16], w3[16], b3",
        "decision": "z > 0",
        "training": {
            "workload": "pu200 (flat geometry)", "events": [TRAIN_EVENTS.start, TRAIN_EVENTS.stop],
            "candidates": int(len(Y)), "true": int(Y.sum()), "keep": KEEP,
            "true_kept": float(np.mean(z[Y] > 0)), "cut_true_kept": float(np.mean(CUT[Y])),
        },
        "heldout": {
            "events": [HELDOUT_EVENTS.start, HELDOUT_EVENTS.stop], "candidates": int(len(Yh)), "true": int(Yh.sum()),
            "true_kept": float(np.mean(zh[Yh] > 0)), "cut_true_kept": float(np.mean(CUTh[Yh])),
            "other_accepted": int(np.sum((zh > 0) & ~Yh)), "cut_other_accepted": int(np.sum(CUTh & ~Yh)),
        },
        "weights": [float(x) for x in w],
    }
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps({k: rec[k] for k in ("training", "heldout")}), f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
