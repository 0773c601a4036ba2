"""FP64 reference of the learned point proposer's network (test oracle).

TEST INFRASTRUCTURE ONLY.  The proposer is not in the paper; it scores grid
points so that pivoted Cholesky (Section II.A) can run on a short candidate
list.  Network: 8 inputs -> 64 -> 64 -> 1, ReLU after each hidden layer,
logistic output.  Loss: class-weighted binary cross entropy
    L = -sum_i w_i [y_i log p_i + (1 - y_i) log(1 - p_i)] / sum_i w_i.
Parameters are one flat vector in the order W1 (8x64, row-major), b1 (64),
W2 (64x64), b2 (64), W3 (64), b3 (1) -- the layout the CUDA kernels use.
Gradients are derived by hand (chain rule written out below) and pinned
against central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 8, 64
SIZES = [("W1", (N_IN, N_H)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SIZES])


def init_params(rng):
    """He-style initialisation (fan-in scaled normals), zero biases."""
    p = {
        "W1": rng.standard_normal((N_IN, N_H)) * np.sqrt(2.0 / N_IN),
        "b1": np.zeros(N_H),
        "W2": rng.standard_normal((N_H, N_H)) * np.sqrt(2.0 / N_H),
        "b2": np.zeros(N_H),
        "W3": rng.standard_normal(N_H) * np.sqrt(1.0 / N_H),
        "b3": np.zeros(1),
    }
    return pack(p)


def forward(theta, X):
    P = unpack(theta)
    a1 = X @ P["W1"] + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"] + P["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ P["W3"] + P["b3"][0]
    return z, (X, a1, h1, a2, h2)


def loss_and_grad(theta, X, y, w):
    """Class-weighted BCE and its gradient with respect to theta."""
    z, (X, a1, h1, a2, h2) = forward(theta, X)
    P = unpack(theta)
    W = np.sum(w)
    # log p = -softplus(-z), log(1-p) = -softplus(z), computed stably
    sp_pos = np.logaddexp(0.0, z)
    sp_neg = np.logaddexp(0.0, -z)
    L = np.sum(w * (y * sp_neg + (1.0 - y) * sp_pos)) / W
    p = 1.0 / (1.0 + np.exp(-z))
    dz = w * (p - y) / W                     # dL/dz
    g = {}
    g["W3"] = h2.T @ dz
    g["b3"] = np.array([np.sum(dz)])
    dh2 = np.outer(dz, P["W3"]) * (a2 > 0)  # through ReLU 2
    g["W2"] = h1.T @ dh2
    g["b2"] = np.sum(dh2, axis=0)
    dh1 = (dh2 @ P["W2"].T) * (a1 > 0)      # through ReLU 1
    g["W1"] = X.T @ dh1
    g["b1"] = np.sum(dh1, axis=0)
    return L, pack(g)


def adam_step(theta, m, v, grad, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma & Ba) with bias correction; t counts from 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
