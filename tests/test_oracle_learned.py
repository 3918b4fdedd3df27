"""Pins of the learned-correction oracle (oracle/learned.py): analytic gradients
against central finite differences of the loss for every parameter; the
initial network is the plain preconditioner (g = 0 everywhere); the first Adam
step moves every parameter by lr * sign(gradient) (bias-corrected moments of
one step); the probing target recovers a known per-branch scale exactly and is
clipped."""
import numpy as np

from oracle.learned import init_params, forward, loss_and_grad, adam_step, probe_target, SCALE, CLIP


def random_params(F, H, seed):
    p = init_params(F, H, seed)
    rng = np.random.default_rng(seed + 1)
    p["w3"] = rng.uniform(-1, 1, H)
    p["b1"] = rng.uniform(-0.5, 0.5, H)
    p["b2"] = rng.uniform(-0.5, 0.5, H)
    p["b3"] = rng.uniform(-0.5, 0.5, 1)
    return p


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    F, H, n = 6, 8, 40
    p = random_params(F, H, 3)
    f = rng.standard_normal((n, F))
    t = rng.uniform(-0.4, 0.4, n)
    _, g = loss_and_grad(p, f, t)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            lp, _ = loss_and_grad(p, f, t)
            flat[i] = old - h
            lm, _ = loss_and_grad(p, f, t)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[i]) < 1e-7 * max(1.0, abs(fd)), (k, i)


def test_initial_network_is_the_plain_preconditioner():
    p = init_params(6, 16, 1)
    g, _ = forward(p, np.random.default_rng(1).standard_normal((10, 6)))
    assert np.all(g == 0.0)


def test_first_adam_step():
    rng = np.random.default_rng(2)
    p = random_params(4, 5, 7)
    q = {k: v.copy() for k, v in p.items()}
    f = rng.standard_normal((12, 4))
    t = rng.uniform(-0.3, 0.3, 12)
    _, g = loss_and_grad(p, f, t)
    adam_step(p, g, {}, lr=1e-2, t=1)
    for k in p:
        expect = q[k] - 1e-2 * g[k] / (np.abs(g[k]) + 1e-8)
        assert np.allclose(p[k], expect, atol=1e-12, rtol=0)


def test_probe_target():
    rng = np.random.default_rng(3)
    n, k = 50, 4
    D = rng.uniform(1, 2, n) + 1j * rng.uniform(1, 2, n)
    c = rng.uniform(-0.3, 0.3, n)
    a = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    assert np.allclose(probe_target(D, (1 + c) * D * a, a), c, atol=1e-14)
    big = probe_target(D, 3.0 * D * a, a)
    assert np.all(big == CLIP)
    assert SCALE > CLIP


def test_features_definition():
    from oracle.learned import features, MU0_4PI
    zs = np.array([1e-2, 2e-2])
    G = np.array([1e2, 1e4])
    L = np.array([1e-6, 1e-4])
    w = 2 * np.pi * 1e9
    f = features(zs, w * MU0_4PI, G, L)
    a, b = zs * G, w * MU0_4PI * L
    assert f.shape == (2, 6)
    assert np.allclose(f[:, 0], 0.25 * np.log10(a)) and np.allclose(f[:, 1], 0.25 * np.log10(b))
    assert np.allclose(f[:, 2], f[:, 0] - f[:, 1])
    assert np.allclose(f[:, 5], 0.25 * np.log10(w))
    # DC: c_L = 0 gives the clipped floor for the inductive term and the clipped ceiling for the ratio
    f0 = features(zs, 0.0, G, L)
    assert np.all(f0[:, 1] == -20.0) and np.all(f0[:, 2] == 20.0) and np.all(f0[:, 5] == -20.0)
