"""FP64 NumPy oracle of the warm-start message-passing network.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The network predicts the steady-state populations p of the Lindblad
equation from the graph, so that rho0 = diag(p_hat) can start the RK4
iteration near its fixed point. Definition (the CUDA library implements the
same definition independently):

Node features x_i (8 per node):
    [1, omega, log1p(in-strength), log1p(out-strength), log1p(in-degree),
     log1p(out-degree), log(N pi_i), dangles]
where A_ij = w for the link j -> i (Supplementary Note 1), in-strength_i =
sum_j A_ij, out-strength_i = sum_j A_ji, degrees count nonzero entries, pi is
the classical PageRank: the stationary vector of G = alpha S + (1 - alpha) F
(the omega = 1 limit of the method), from 200 steps of power iteration
started at the uniform vector, and dangles = 1 for a node without out-links.

Aggregation P_ij = (A_ij + A_ji) / s_i with s_i = sum_j (A_ij + A_ji) (a zero
row when s_i = 0).

Layers l = 1..4 (width 64): z_l = h_{l-1} Ws_l + (P h_{l-1}) Wn_l + b_l,
h_l = relu(z_l), h_0 = x. Readout s = h_4 wo + bo, p_hat = softmax(s) over
the graph's nodes. Loss L = -sum_i p_i log p_hat_i.

Weights are stored in FP32 and used rounded to BF16 (round to nearest, ties
to even); biases and wo, bo are used as stored.

Flat parameter layout: Ws1 [8][64], Wn1 [8][64], b1 [64], then for l = 2..4:
Ws_l [64][64], Wn_l [64][64], b_l [64]; then wo [64], bo [1].
"""
from __future__ import annotations

import numpy as np

F_IN = 8
WIDTH = 64
LAYERS = 4


def param_shapes():
    shapes = [("Ws1", (F_IN, WIDTH)), ("Wn1", (F_IN, WIDTH)), ("b1", (WIDTH,))]
    for l in range(2, LAYERS + 1):
        shapes += [(f"Ws{l}", (WIDTH, WIDTH)), (f"Wn{l}", (WIDTH, WIDTH)), (f"b{l}", (WIDTH,))]
    shapes += [("wo", (WIDTH,)), ("bo", (1,))]
    return shapes


def param_count() -> int:
    return int(sum(np.prod(s) for _, s in param_shapes()))


def unpack(flat):
    out, o = {}, 0
    for name, shp in param_shapes():
        k = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + k], dtype=np.float64).reshape(shp)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in param_shapes()])


def round_bf16(x):
    """FP32 values rounded to BF16 (nearest, ties to even), returned as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def adjacency(n, src, dst, w=None):
    """Dense A with A[dst, src] += w (self-loops and zero weights dropped)."""
    A = np.zeros((n, n))
    w = np.ones(len(src)) if w is None else np.asarray(w, dtype=np.float64)
    for s, d, x in zip(src, dst, w):
        if s != d and x != 0.0:
            A[d, s] += x
    return A


def google_matrix(A, alpha):
    n = A.shape[0]
    outdeg = A.sum(axis=0)
    F = (np.ones((n, n)) - np.eye(n)) / (n - 1)
    S = np.where(outdeg[None, :] > 0, A / np.where(outdeg > 0, outdeg, 1.0)[None, :], F)
    return alpha * S + (1.0 - alpha) * F


def features(A, omega, alpha):
    n = A.shape[0]
    G = google_matrix(A, alpha)
    pi = np.full(n, 1.0 / n)
    for _ in range(200):
        pi = G @ pi
        pi = pi / pi.sum()
    x = np.zeros((n, F_IN))
    x[:, 0] = 1.0
    x[:, 1] = omega
    x[:, 2] = np.log1p(A.sum(axis=1))
    x[:, 3] = np.log1p(A.sum(axis=0))
    x[:, 4] = np.log1p((A > 0).sum(axis=1))
    x[:, 5] = np.log1p((A > 0).sum(axis=0))
    x[:, 6] = np.log(n * pi)
    x[:, 7] = (A.sum(axis=0) == 0).astype(np.float64)
    return x


def aggregation(A):
    B = A + A.T
    s = B.sum(axis=1)
    return np.where(s[:, None] > 0, B / np.where(s > 0, s, 1.0)[:, None], 0.0)


def forward(params_flat, x, P, bf16=True):
    """Returns (logits, p_hat, cache). bf16=False uses the weights unrounded
    (for finite-difference checks of the backward pass)."""
    prm = unpack(params_flat)
    rnd = round_bf16 if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    h = x
    cache = []
    for l in range(1, LAYERS + 1):
        Ws, Wn = rnd(prm[f"Ws{l}"]), rnd(prm[f"Wn{l}"])
        m = P @ h
        z = h @ Ws + m @ Wn + prm[f"b{l}"]
        cache.append((h, m, z))
        h = np.maximum(z, 0.0)
    s = h @ prm["wo"] + prm["bo"][0]
    e = np.exp(s - s.max())
    p_hat = e / e.sum()
    cache.append(h)
    return s, p_hat, cache


def loss(p_hat, p):
    return float(-np.sum(p * np.log(p_hat)))


def backward(params_flat, P, p_hat, p, cache, bf16=True):
    """Gradient of L with respect to the flat parameters (the BF16-rounded
    weights count as the weights)."""
    prm = unpack(params_flat)
    rnd = round_bf16 if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    g = {}
    h4 = cache[-1]
    # L = -sum_i p_i log p_hat_i with p_hat = softmax(s): dL/ds = p_hat sum(p) - p
    ds = p_hat * p.sum() - p
    g["wo"] = h4.T @ ds
    g["bo"] = np.array([ds.sum()])
    dh = np.outer(ds, prm["wo"])
    for l in range(LAYERS, 0, -1):
        h, m, z = cache[l - 1]
        Ws, Wn = rnd(prm[f"Ws{l}"]), rnd(prm[f"Wn{l}"])
        dz = dh * (z > 0)
        g[f"Ws{l}"] = h.T @ dz
        g[f"Wn{l}"] = m.T @ dz
        g[f"b{l}"] = dz.sum(axis=0)
        dh = dz @ Ws.T + P.T @ (dz @ Wn.T)
    return pack(g)


def loss_and_grad(params_flat, n, src, dst, w, omega, alpha, p):
    A = adjacency(n, src, dst, w)
    x = features(A, omega, alpha)
    P = aggregation(A)
    s, p_hat, cache = forward(params_flat, x, P)
    return loss(p_hat, p), backward(params_flat, P, p_hat, p, cache), p_hat
