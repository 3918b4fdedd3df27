"""GPU parity of the learned preconditioner correction (oracle/learned.py).

* features of every branch against the oracle's definition evaluated on the
  oracle's Gram and direct self terms (FP32 output, 2e-6 absolute);
* the network's forward pass and loss gradient against the FP64 oracle
  (FP32 kernels: 1e-5 on g, 1e-4 relative on the gradient);
* the probing target against the oracle's from the oracle's branch product;
* a new network (zero output layer) leaves the preconditioner bit for bit
  unchanged: the plain form is the fallback;
* one Adam step moves every parameter by lr * sign(gradient); training lowers
  the loss;
* the plain preconditioner judges the learned one: both solves reach the same
  impedance, and the iteration counts of both are reported.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.pfft import PfftSystem, PfftParams
from oracle.mom import branch_zs
from oracle import learned as OL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, PREC_FP64  # noqa: E402

PRM = dict(grid=(16, 8, 4), order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=0.0)


@pytest.fixture(scope="module")
def wires():
    m = synth.tiny_wires()
    O = build_loops(m)
    S = PfftSystem(m, O, PfftParams(grid=PRM["grid"], order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8))
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    return m, O, S, api.Plan(M, L, PRM)


def oracle_diag(m, O, S, w):
    G = S.G.diagonal()
    Ld = S.op.near_matrix(S.op.L_direct).diagonal()
    zs = branch_zs(m, O, w, None)
    zs = np.broadcast_to(zs, G.shape) if np.ndim(zs) == 0 else zs
    return zs, G, Ld


def test_features_match_oracle(wires):
    m, O, S, P = wires
    for f in (1e6, 1e9, 2e10):
        w = 2 * np.pi * f
        zs, G, Ld = oracle_diag(m, O, S, w)
        ref = OL.features(np.abs(zs), w * OL.MU0_4PI, G, Ld)
        got = api.branch_features(P, w).cpu().numpy()
        assert np.abs(got - ref).max() < 2e-6


def random_params(H, seed):
    p = OL.init_params(6, H, seed)
    rng = np.random.default_rng(seed + 1)
    p["w3"] = rng.uniform(-1, 1, H)
    p["b1"] = rng.uniform(-0.5, 0.5, H)
    p["b2"] = rng.uniform(-0.5, 0.5, H)
    p["b3"] = rng.uniform(-0.5, 0.5, 1)
    return p


def flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["w3"], p["b3"]])


@pytest.mark.parametrize("H", [16, 32])
def test_forward_and_gradient_match_oracle(H):
    rng = np.random.default_rng(H)
    n = 1000
    p = random_params(H, 5)
    f = rng.uniform(-3, 3, (n, 6))
    t = rng.uniform(-0.4, 0.4, n)
    net = api.MLP(H, seed=1)
    net.set_params(flat(p).astype(np.float32))
    p32 = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    fd = torch.from_numpy(f.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    g_ref, _ = OL.forward(p32, f.astype(np.float32).astype(np.float64))
    assert np.abs(net.forward(fd).cpu().numpy() - g_ref).max() < 1e-5
    loss_ref, grad_ref = OL.loss_and_grad(p32, f.astype(np.float32).astype(np.float64), t.astype(np.float32))
    loss, grad = net.grad(fd, td)
    assert abs(loss - loss_ref) < 1e-5 * max(1.0, loss_ref)
    gr = flat(grad_ref)
    assert np.abs(grad - gr).max() < 1e-4 * np.abs(gr).max()


def test_width128_fp16_network_matches_oracle():
    # the configured network (6 -> 128 -> 128 -> 1) computes with FP16 roundings of
    # its FP32 master parameters and FP32 accumulation: the oracle's FP64 forward,
    # loss and gradient at those rounded parameters (straight-through gradient)
    H = 128
    rng = np.random.default_rng(H)
    n = 3000   # several CTA partials and a ragged last tile
    p = random_params(H, 7)
    f = rng.uniform(-3, 3, (n, 6))
    t = rng.uniform(-0.4, 0.4, n)
    net = api.MLP(H, seed=1)
    net.set_params(flat(p).astype(np.float32))
    p16 = {k: v.astype(np.float32).astype(np.float16).astype(np.float64) for k, v in p.items()}
    f32 = f.astype(np.float32).astype(np.float64)
    fd = torch.from_numpy(f.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    g_ref, _ = OL.forward(p16, f32)
    assert np.abs(net.forward(fd).cpu().numpy() - g_ref).max() < 2e-5
    loss_ref, grad_ref = OL.loss_and_grad(p16, f32, t.astype(np.float32))
    loss, grad = net.grad(fd, td)
    assert abs(loss - loss_ref) < 1e-5 * max(1.0, loss_ref)
    gr = flat(grad_ref)
    assert np.abs(grad - gr).max() < 2e-4 * np.abs(gr).max()
    # Adam moves the FP32 masters; the network then computes with their new FP16 roundings
    before = net.params()
    net.train(fd, td, 1, lr=1e-3)
    after = net.params()
    assert np.abs(after - before).max() > 0
    keys = ("W1", "b1", "W2", "b2", "w3", "b3")
    parts = np.split(after, np.cumsum([p[k].size for k in keys])[:-1])
    pa = {k: v.reshape(p[k].shape).astype(np.float16).astype(np.float64) for k, v in zip(keys, parts)}
    g_after, _ = OL.forward(pa, f32)
    assert np.abs(net.forward(fd).cpu().numpy() - g_after).max() < 2e-5


def test_width128_new_network_is_the_plain_preconditioner(wires):
    m, O, S, P = wires
    om = 2 * np.pi * np.array([1e8, 1e9, 5e9])
    y = torch.from_numpy(synth.complex_gaussian(O.nl, 3, seed=14)).cuda()
    z0 = api.pfft_precond_apply(P, y, om)
    net = api.MLP(128, seed=3)
    api.set_learned(P, net)
    z1 = api.pfft_precond_apply(P, y, om)
    api.set_learned(P, None)
    assert torch.equal(z0, z1)


def test_probe_target_matches_oracle(wires):
    m, O, S, P = wires
    w = 2 * np.pi * 1e9
    alpha = synth.complex_gaussian(O.nb, 4, seed=12)
    zs, G, Ld = oracle_diag(m, O, S, w)
    D = zs * G + 1j * w * OL.MU0_4PI * Ld
    zb = np.stack([S.branch_product(alpha[k], w) for k in range(4)])
    ref = OL.probe_target(D, zb, alpha)
    got = api.branch_probe_target(P, torch.from_numpy(alpha).cuda(), w).cpu().numpy()
    assert np.abs(got - ref).max() < 2e-5


def test_new_network_is_the_plain_preconditioner(wires):
    m, O, S, P = wires
    om = 2 * np.pi * np.array([1e8, 1e9, 5e9])
    y = torch.from_numpy(synth.complex_gaussian(O.nl, 3, seed=13)).cuda()
    z0 = api.pfft_precond_apply(P, y, om)
    net = api.MLP(32, seed=3)
    api.set_learned(P, net)
    z1 = api.pfft_precond_apply(P, y, om)
    api.set_learned(P, None)
    z2 = api.pfft_precond_apply(P, y, om)
    assert torch.equal(z0, z1) and torch.equal(z0, z2)


def training_data(P, nb, freqs, seed):
    fs, ts = [], []
    for i, f in enumerate(freqs):
        w = 2 * np.pi * f
        alpha = torch.from_numpy(synth.complex_gaussian(nb, 4, seed=seed + i)).cuda()
        fs.append(api.branch_features(P, w))
        ts.append(api.branch_probe_target(P, alpha, w))
    return torch.cat(fs), torch.cat(ts)


def test_adam_step_and_training(wires):
    m, O, S, P = wires
    feats, target = training_data(P, O.nb, [1e7, 1e8, 1e9, 1e10], 20)
    net = api.MLP(32, seed=4)
    p0 = random_params(32, 9)
    net.set_params(flat(p0).astype(np.float32))
    _, g = net.grad(feats, target)
    before = net.params()
    net.train(feats, target, 1, lr=1e-3)
    step = net.params() - before
    nz = np.abs(g) > 1e-6
    assert np.allclose(step[nz], -1e-3 * np.sign(g[nz]), rtol=1e-3, atol=1e-9)
    losses = net.train(feats, target, 300, lr=3e-3)
    assert losses[-1] < 0.9 * losses[0]


def test_plain_preconditioner_judges_the_learned_one(wires):
    m, O, S, P = wires
    feats, target = training_data(P, O.nb, [1e7, 1e8, 1e9, 1e10], 30)
    net = api.MLP(32, seed=6)
    net.train(feats, target, 400, lr=3e-3)
    # held out: a bar, at a frequency not trained on
    mb = synth.tiny_bar()
    Mb = api.Mesh.from_synth(mb)
    Lb = api.Loops(Mb, mb.ports)
    Pb = api.Plan(Mb, Lb, dict(PRM, grid=(16, 8, 8)))
    freqs = [3e9]
    Z0, st0 = api.sie_solve(Pb, freqs, tol=1e-8, restart=100, prec=PREC_FP64)
    api.set_learned(Pb, net)
    Z1, st1 = api.sie_solve(Pb, freqs, tol=1e-8, restart=100, prec=PREC_FP64)
    api.set_learned(Pb, None)
    assert st0["converged"] and st1["converged"]
    assert np.abs(Z1 - Z0).max() < 1e-6 * np.abs(Z0).max()
    print("GMRES iterations, plain / learned:", st0["iterations_max"], st1["iterations_max"])
