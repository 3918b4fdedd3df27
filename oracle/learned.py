"""Learned correction of the preconditioner's branch diagonal (oracle; test
infrastructure only, the GPU library never imports it).

The preconditioner of Eq. (Precond) is P = A diag(Z_b) A^T with the diagonal
D_e of Z_b on each branch.  The learned form replaces D_e by
D'_e = D_e (1 + g(f_e)), g a small network of per-branch features f_e, and
keeps the plain P (g = 0) as the fallback and as the judge of GMRES
iteration counts.

Network: f [F] -> tanh(W1 f + b1) [H] -> tanh(W2 h1 + b2) [H] -> g = s tanh(w3 . h2 + b3),
s = 0.5 (|g| < 1/2 keeps D' away from zero).  Training target: the per-branch
probing scale, the least-squares factor that maps D alpha onto Z_b alpha over
probe currents alpha, t_e = sum Re(conj(D_e a_e) (Z_b a)_e) / sum |D_e a_e|^2 - 1,
clipped to |t| <= 0.45; loss: mean squared error (1/n) sum (g_e - t_e)^2.
Forward and backward are written out plainly (FP64) and pinned by finite
differences in tests/test_oracle_learned.py.
"""
from __future__ import annotations

import numpy as np

SCALE = 0.5
CLIP = 0.45


def init_params(F, H, seed=0):
    """Glorot-uniform weights, zero biases, and a zero output layer (g = 0: the
    plain preconditioner) unless trained."""
    rng = np.random.default_rng(seed)
    a1, a2 = np.sqrt(6.0 / (F + H)), np.sqrt(6.0 / (2 * H))
    return dict(W1=rng.uniform(-a1, a1, (H, F)), b1=np.zeros(H), W2=rng.uniform(-a2, a2, (H, H)),
                b2=np.zeros(H), w3=np.zeros(H), b3=np.zeros(1))


def forward(p, f):
    """g [n] and the activations needed by the backward pass; f [n, F]."""
    h1 = np.tanh(f @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    z = h2 @ p["w3"] + p["b3"][0]
    return SCALE * np.tanh(z), (f, h1, h2, z)


def loss_and_grad(p, f, t):
    """MSE loss (1/n) sum (g - t)^2 and its gradient with respect to every parameter."""
    g, (f, h1, h2, z) = forward(p, f)
    n = f.shape[0]
    r = g - t
    loss = float(np.mean(r * r))
    dg = 2.0 * r / n
    dz = dg * SCALE * (1.0 - np.tanh(z) ** 2)
    gw3 = h2.T @ dz
    gb3 = np.array([dz.sum()])
    dh2 = np.outer(dz, p["w3"]) * (1.0 - h2 * h2)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ p["W2"]) * (1.0 - h1 * h1)
    gW1 = dh1.T @ f
    gb1 = dh1.sum(axis=0)
    return loss, dict(W1=gW1, b1=gb1, W2=gW2, b2=gb2, w3=gw3, b3=gb3)


def adam_step(p, g, state, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of every parameter (t: the step number from 1)."""
    for k in p:
        m, v = state.setdefault(k, (np.zeros_like(p[k]), np.zeros_like(p[k])))
        m = beta1 * m + (1 - beta1) * g[k]
        v = beta2 * v + (1 - beta2) * g[k] * g[k]
        state[k] = (m, v)
        mh, vh = m / (1 - beta1 ** t), v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def probe_target(D, Zb_alpha, alpha):
    """Per-branch probing scale minus one, clipped: D [n] complex, alpha and
    Z_b alpha [k, n] complex (k probes)."""
    Da = D[None, :] * alpha
    num = np.sum(np.real(np.conj(Da) * Zb_alpha), axis=0)
    den = np.sum(np.abs(Da) ** 2, axis=0)
    return np.clip(num / den - 1.0, -CLIP, CLIP)


N_FEATURES = 6
MU0_4PI = 1e-7   # mu0 / (4 pi)


def features(zs_abs, cl, gram_diag, l_diag):
    """Per-branch features at one frequency (F = 6), quarter decades:
    |Z_s| G_ee, c_L Lt_ee, their ratio, G_ee, Lt_ee and omega (= c_L / (mu0 / 4 pi)),
    each as 0.25 log10(max(x, 1e-300)) clipped to [-20, 20]."""
    a = zs_abs * gram_diag
    b = cl * l_diag
    q = lambda x: np.clip(0.25 * np.log10(np.maximum(x, 1e-300)), -20.0, 20.0)
    cols = [q(a), q(b), q(np.maximum(a, 1e-300) / np.maximum(b, 1e-300)), q(gram_diag), q(l_diag),
            q(np.full_like(a, cl / MU0_4PI))]
    return np.stack(cols, axis=1)
