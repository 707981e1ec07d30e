"""FP64 oracle of the step-controller MLP (forward, loss, gradient).

TEST INFRASTRUCTURE ONLY.  The controller is not part of the paper; it follows the
stated design: o = W2 relu(W1 phi + b1) + b2, multiplier 2^(2 tanh o), loss = mean over
samples of (2 tanh(o) - t)^2.  Parameter vector layout: W1[64][5], b1[64], W2[64], b2.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 5, 64
N_PARAMS = N_IN * N_HID + 2 * N_HID + 1


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    W1 = w[:N_IN * N_HID].reshape(N_HID, N_IN)
    b1 = w[N_IN * N_HID:N_IN * N_HID + N_HID]
    W2 = w[N_IN * N_HID + N_HID:N_PARAMS - 1]
    b2 = w[N_PARAMS - 1]
    return W1, b1, W2, b2


def forward(w, phi):
    W1, b1, W2, b2 = unpack(w)
    z = np.asarray(phi, dtype=np.float64) @ W1.T + b1
    h = np.maximum(z, 0.0)
    return h @ W2 + b2, z, h


def multiplier(w, phi):
    o, _, _ = forward(w, phi)
    return 2.0 ** (2.0 * np.tanh(o))


def loss(w, phi, t):
    o, _, _ = forward(w, phi)
    e = 2.0 * np.tanh(o) - np.asarray(t, dtype=np.float64)
    return float(np.mean(e * e))


def gradient(w, phi, t):
    """Backpropagation of `loss` with respect to the parameter vector."""
    phi = np.asarray(phi, dtype=np.float64)
    W1, b1, W2, b2 = unpack(w)
    o, z, h = forward(w, phi)
    th = np.tanh(o)
    n = len(o)
    dlo = 2.0 * (2.0 * th - t) * 2.0 * (1.0 - th * th) / n          # dL/do
    gW2 = h.T @ dlo
    gb2 = dlo.sum()
    dh = np.outer(dlo, W2) * (z > 0.0)
    gW1 = dh.T @ phi
    gb1 = dh.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2, [gb2]])
