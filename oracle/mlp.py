"""Oracle of the learned swap proposal (no counterpart in the paper) -- test infrastructure.

* ``move_features``: the 8 features of a swap move (close open facility j,
  open closed facility k) of one individual, from its swap statistics
  (``oracle.swap_stats``), and the regression target (exact cost change of the
  swap / Z, Z = max(cost / p, 1)).
* A 3-layer perceptron F(16, the 8 features zero-padded) -> 128 -> 128 -> 1
  with ReLU, its mean-squared-error gradients and the Adam update (Kingma &
  Ba, "Adam: A Method for Stochastic Optimization", ICLR 2015: beta1 = 0.9,
  beta2 = 0.999, eps = 1e-8, bias-corrected moments).

Arithmetic is float64.  ``bf16=True`` reproduces where the CUDA path rounds to
bfloat16 (inputs, weight copies, the hidden activations and their gradients
that feed tensor-core products); everything else is exact float64, so the
CUDA path (float32 accumulation) must agree within a tolerance.
"""

from __future__ import annotations

import numpy as np

F_IN = 8      # features per move
F_PAD = 16    # padded input width (one k-step of a 16-bit tensor-core product)
HIDDEN = 128

BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((u >> 16) & 1)
    r = ((u + bias) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _r(x, bf16):
    return bf16_round(x) if bf16 else np.asarray(x, dtype=np.float64)


# --------------------------------------------------------------------------
# Move features
# --------------------------------------------------------------------------

def move_features(gain, cap, loss, assign, cost, n, m, p, j, k):
    """Feature vector (length 8) of closing j and opening k, from one individual's swap statistics."""
    Z = max(float(cost) / p, 1.0)
    per = n / p
    lj, gk = float(loss[j]), float(gain[k])
    return np.array([
        lj / Z,
        gk / Z,
        assign[j] / per,
        cap[k] / per,
        (lj - gk) / Z,
        np.log1p(lj / Z),
        np.log1p(gk / Z),
        p / m,
    ], dtype=np.float64)


def move_target(cost_before, cost_after, p):
    """Regression target: the exact cost change of the swap divided by Z."""
    Z = max(float(cost_before) / p, 1.0)
    return (float(cost_after) - float(cost_before)) / Z


# --------------------------------------------------------------------------
# The perceptron
# --------------------------------------------------------------------------

def init_params(seed=0):
    """He-style initialisation (fixed seed); float64 master weights."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.normal(0, np.sqrt(2.0 / F_IN), size=(F_PAD, HIDDEN)),
        "b1": np.zeros(HIDDEN),
        "W2": rng.normal(0, np.sqrt(2.0 / HIDDEN), size=(HIDDEN, HIDDEN)),
        "b2": np.zeros(HIDDEN),
        "w3": rng.normal(0, np.sqrt(1.0 / HIDDEN), size=(HIDDEN,)),
        "b3": np.zeros(1),
    }


def forward(params, X, bf16=False):
    """y (B,) and the cache for backward.  X is (B, 16)."""
    x = _r(X, bf16)
    W1, W2, w3 = _r(params["W1"], bf16), _r(params["W2"], bf16), _r(params["w3"], bf16)
    z1 = x @ W1 + params["b1"]
    h1 = _r(np.maximum(z1, 0.0), bf16)
    z2 = h1 @ W2 + params["b2"]
    h2 = _r(np.maximum(z2, 0.0), bf16)
    y = h2 @ w3 + params["b3"][0]
    return y, (x, h1, h2, W1, W2, w3)


def loss_and_grads(params, X, t, bf16=False):
    """Mean squared error and its gradients with respect to every parameter."""
    y, (x, h1, h2, W1, W2, w3) = forward(params, X, bf16)
    B = X.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    g = {"b3": np.array([dy.sum()]), "w3": h2.T @ dy}
    dh2 = np.outer(dy, w3) * (h2 > 0)
    dh2 = _r(dh2, bf16)
    g["b2"] = dh2.sum(axis=0)
    g["W2"] = h1.T @ dh2
    dh1 = (dh2 @ W2.T) * (h1 > 0)
    dh1 = _r(dh1, bf16)
    g["b1"] = dh1.sum(axis=0)
    g["W1"] = x.T @ dh1
    return loss, g


def adam_init(params):
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in params.items()},
            "v": {k: np.zeros_like(v) for k, v in params.items()}}


def adam_step(params, grads, state, lr):
    """One Adam update in place (Kingma & Ba 2015, Algorithm 1)."""
    state["t"] += 1
    t = state["t"]
    for k in params:
        g = grads[k]
        state["m"][k] = BETA1 * state["m"][k] + (1 - BETA1) * g
        state["v"][k] = BETA2 * state["v"][k] + (1 - BETA2) * g * g
        mhat = state["m"][k] / (1 - BETA1 ** t)
        vhat = state["v"][k] / (1 - BETA2 ** t)
        params[k] = params[k] - lr * mhat / (np.sqrt(vhat) + EPS)
    return params


# --------------------------------------------------------------------------
# Training: the epoch shuffle and the loop (the library's pm_model_train)
# --------------------------------------------------------------------------

OP_SHUFFLE = 0x300


def fmix32(h: int) -> int:
    """MurmurHash3's 32-bit finaliser (Appleby): xor-shift 16, multiply 0x85ebca6b, xor-shift 13, multiply
    0xc2b2ae35, xor-shift 16, all mod 2^32."""
    h &= 0xFFFFFFFF
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & 0xFFFFFFFF
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & 0xFFFFFFFF
    h ^= h >> 16
    return h


def shuffle_keys(seed: int, epoch: int):
    """The four Feistel round keys of an epoch: the words of Philox4x32-10 at counter (epoch, 0, 0x300 * 2^16, 0)
    with key (seed lo, seed hi)."""
    from oracle import philox4x32_10

    return [int(v) for v in philox4x32_10([epoch, 0, OP_SHUFFLE << 16, 0],
                                          [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])]


def shuffle_order(rows: int, seed: int, epoch: int):
    """Row held by each position of the epoch: a four-round Feistel network on the smallest even number of bits
    b >= 2 with 2^b >= rows (round r: (L, R) -> (R, L ^ (fmix32(R ^ K_r) mod 2^(b/2)))), re-applied while the
    result is >= rows (cycle walking)."""
    keys = shuffle_keys(seed, epoch)
    bits = 2
    while (1 << bits) < rows:
        bits += 2
    half = bits // 2
    mask = (1 << half) - 1

    def once(x):
        L, R = x >> half, x & mask
        for r in range(4):
            L, R = R, L ^ (fmix32(R ^ keys[r]) & mask)
        return (L << half) | R

    out = []
    for i in range(rows):
        x = once(i)
        while x >= rows:
            x = once(x)
        out.append(x)
    return np.array(out, dtype=np.int64)


def train(params, X, t, epochs: int, batch: int, lr: float, seed: int, state=None):
    """Adam over `epochs` passes of (X, t) in mini-batches of `batch` rows taken in the order of shuffle_order;
    returns (params, state, the mean squared error of every batch before its update)."""
    state = adam_init(params) if state is None else state
    rows = X.shape[0]
    losses = []
    for e in range(epochs):
        order = shuffle_order(rows, seed, e)
        for b0 in range(0, rows, batch):
            idx = order[b0:b0 + batch]
            loss, g = loss_and_grads(params, X[idx], np.asarray(t)[idx], bf16=True)
            losses.append(loss)
            adam_step(params, g, state, lr)
    return params, state, losses


def flatten(params):
    """Parameters in the library's flat order: W1 (16x128), b1, W2 (128x128), b2, w3, b3."""
    return np.concatenate([params["W1"].ravel(), params["b1"], params["W2"].ravel(), params["b2"], params["w3"],
                           params["b3"]])


def unflatten(v):
    v = np.asarray(v, dtype=np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (F_PAD, HIDDEN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
                        ("w3", (HIDDEN,)), ("b3", (1,))):
        size = int(np.prod(shape))
        out[name] = v[o:o + size].reshape(shape).copy()
        o += size
    return out


N_PARAMS = F_PAD * HIDDEN + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1


# --------------------------------------------------------------------------
# The learned try when every candidate scores the same (a model whose parameters are all zero)
# --------------------------------------------------------------------------

def first_candidate_try(pi, delta, m: int, p: int):
    """The learned try of one generation (between the crossover and the mutation cycles) for a model that gives
    every candidate move the same score, as an ``extra_try`` for ``oracle.ga_run``.

    The library's learned try ranks the candidates of an individual as rows a * T + b (the a-th open facility in
    ascending order, the b-th closed facility by gain descending, ties by lower id) and takes the lowest score,
    ties to the lowest row; with equal scores that is row 0: close the lowest open facility, open the closed
    facility of largest gain.  The child is evaluated exactly (one evaluation per individual) and replaces the
    individual, marked as improved so the mutation cycle skips it, iff strictly cheaper."""
    from . import eval_scan, swap_stats

    def extra(gen, X, c, enhanced):
        P = X.shape[0]
        gain, _, _, _ = swap_stats(pi, delta, m, X)
        child = X.copy()
        for t in range(P):
            bits = np.unpackbits(X[t].view(np.uint8), bitorder="little")[:m].astype(bool)
            j = int(np.flatnonzero(bits)[0])
            closed = np.flatnonzero(~bits)
            # largest gain, then lowest id: argmax over (gain, -id) among the closed facilities
            g = gain[t, closed]
            k = int(closed[np.flatnonzero(g == g.max())[0]]) if closed.size else 0
            child[t, j >> 5] &= np.uint32(~(1 << (j & 31)) & 0xFFFFFFFF)
            child[t, k >> 5] |= np.uint32(1 << (k & 31))
        cc = eval_scan(pi, delta, child)
        for t in range(P):
            if cc[t] < c[t]:
                X[t] = child[t]
                c[t] = cc[t]
                enhanced[t] = 1
        return P

    return extra
