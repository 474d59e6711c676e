"""Learned decision heuristic (not in the paper): trace, train, evaluate.

1. Solve training programs with the plain heuristic and decision tracing
   (asp_solve_batch, trace_capacity > 0): at every decision about one
   applicable rule in eight is sampled with its 16 features; when the search
   finds an answer set, each sample is labelled by whether the rule's body
   holds in it (programs without an answer set give no labels).
2. Standardise the features, train the 16-64-1 MLP on the device
   (asp_train_mlp: SGD with momentum on binary cross-entropy), then fold the
   standardisation into the first layer so the solver reads raw features.
3. The solver (heuristic = ASP_HEUR_LEARNED) chooses the applicable rule with
   the largest log1p(occurrences of its head) + log P(body holds in an answer
   set): the plain heuristic's impact estimate weighted by the learned
   probability that the choice is right.  With ASP_HEUR_LEARNED_STATIC the
   score is computed once per rule when the program is loaded, with the
   search-state features at their values before the first decision; the
   model for it is trained with those features held at the same values
   (fit(..., static=True)), so it learns a rule order from the program's
   structure alone and costs nothing per decision.

Propagation, learning and the stability check are untouched, so answer sets
and SAT/UNSAT answers do not depend on the weights; only the search order
does.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import aspgpu

N_FEATURES, N_HIDDEN = aspgpu.MLP_FEATURES, 64
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "heuristic_mlp.json")


def init_weights(seed: int = 0) -> np.ndarray:
    """He-style initialisation of W1, zero biases, small w2 (float32)."""
    rng = np.random.default_rng(seed)
    w = np.zeros(aspgpu.MLP_PARAMS, np.float32)
    w[:N_FEATURES * N_HIDDEN] = rng.normal(0, np.sqrt(2.0 / N_FEATURES), N_FEATURES * N_HIDDEN)
    o = N_FEATURES * N_HIDDEN + N_HIDDEN
    w[o:o + N_HIDDEN] = rng.normal(0, np.sqrt(1.0 / N_HIDDEN), N_HIDDEN)
    return w


def split(w):
    W1 = w[:N_FEATURES * N_HIDDEN].reshape(N_HIDDEN, N_FEATURES)
    b1 = w[N_FEATURES * N_HIDDEN:N_FEATURES * N_HIDDEN + N_HIDDEN]
    w2 = w[N_FEATURES * N_HIDDEN + N_HIDDEN:N_FEATURES * N_HIDDEN + 2 * N_HIDDEN]
    b2 = w[-1:]
    return W1, b1, w2, b2


def collect_traces(programs, conflict_budget: int = 200, trace_capacity: int = 4096, chunk: int = 2048, **kw):
    """Solve programs (batched, plain heuristic, `chunk` programs loaded at a
    time) and gather (features, labels)."""
    X, y = [], []
    programs = list(programs)
    for c0 in range(0, len(programs), chunk):
        P = [aspgpu.Program(p, conflict_budget=conflict_budget, trace_capacity=trace_capacity,
                            deps_levels=1024, learned_capacity=1 << 20, **kw) for p in programs[c0:c0 + chunk]]
        aspgpu.solve_batch(P, max_models_each=1, cap_each=1)
        for q in P:
            f, lab = q.trace(trace_capacity)
            keep = lab >= 0
            X.append(f[keep])
            y.append(lab[keep])
            q.close()
    return np.concatenate(X) if X else np.zeros((0, N_FEATURES), np.float32), \
        np.concatenate(y).astype(np.float32) if y else np.zeros(0, np.float32)


def static_features(X: np.ndarray) -> np.ndarray:
    """The features a rule has before the first decision (what the solver
    uses for ASP_HEUR_LEARNED_STATIC): activity 0, every negative body atom
    unassigned (feature 2 = |B-|), none false, level 1, no conflicts, empty
    trail."""
    Z = np.array(X, np.float32, copy=True)
    Z[:, 8] = 0.0
    Z[:, 9] = Z[:, 2]
    Z[:, 10] = 0.0
    Z[:, 11] = 1.0 / 64.0
    Z[:, 12:] = 0.0
    return Z


def fit(X: np.ndarray, y: np.ndarray, epochs: int = 60, learning_rate: float = 0.05, seed: int = 0,
        static: bool = False):
    """Train on standardised features, return weights for raw features and
    the training statistics.  static: train on static_features(X)."""
    if static:
        X = static_features(X)
    mu = X.mean(0)
    sd = X.std(0)
    sd[sd < 1e-6] = 1.0
    Z = ((X - mu) / sd).astype(np.float32)
    w = aspgpu.train_mlp(Z, y, init_weights(seed), epochs=epochs, learning_rate=learning_rate)
    out = fold_standardisation(w, mu, sd)
    p = 1.0 / (1.0 + np.exp(-forward_np(w, Z)))
    stats = dict(samples=int(X.shape[0]), positive=float(y.mean()) if y.size else 0.0,
                 train_logloss=float(-np.mean(y * np.log(p + 1e-7) + (1 - y) * np.log(1 - p + 1e-7))),
                 train_accuracy=float(np.mean((p > 0.5) == (y > 0.5))))
    return out, stats


def fold_standardisation(w: np.ndarray, mu: np.ndarray, sd: np.ndarray) -> np.ndarray:
    """Weights of a network trained on standardised features (x - mu) / sd,
    rewritten for raw features: W1' = W1 / sd, b1' = b1 - W1' mu (the same
    logit for every x)."""
    W1, b1, w2, b2 = split(np.asarray(w, np.float32).copy())
    W1r = W1 / sd[None, :]
    b1r = b1 - W1r @ mu
    return np.concatenate([W1r.reshape(-1), b1r, w2, b2]).astype(np.float32)


def forward_np(w: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Plain fp64 forward pass (the reference for the device kernels)."""
    W1, b1, w2, b2 = (a.astype(np.float64) for a in split(w))
    h = np.maximum(X.astype(np.float64) @ W1.T + b1, 0.0)
    return h @ w2 + b2[0]


def save(weights: np.ndarray, path: str = DEFAULT_WEIGHTS, **meta):
    with open(path, "w") as f:
        json.dump({"weights": [float(x) for x in weights], **meta}, f)


def load(path: str = DEFAULT_WEIGHTS) -> np.ndarray:
    with open(path) as f:
        return np.asarray(json.load(f)["weights"], np.float32)
