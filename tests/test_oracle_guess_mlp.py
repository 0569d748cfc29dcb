"""Pins of the FP64 reference of the learned con2prim guess (oracle/guess_mlp.py).

* backward() against central finite differences of the loss (every parameter block, both outputs), and
  the BF16 rounding of h1, h2 as a straight-through step;
* a network reduced to one unit per layer, evaluated in closed form with math.exp;
* the first Adam step moves every parameter by lr * sign(g) (bias-corrected m/sqrt(v) = g/|g|);
* BF16 rounding of values with known nearest-even results, and against torch's bfloat16 cast;
* features and targets of the state at rest without field, where mu = 1/h and mu_+ = 1 in closed form;
  of cold moving states without field, where mu = mu_+ = 1/W and eps(mu_+) = 0; and targets of random
  states against the oracle's own con2prim root and W.
"""
import math

import numpy as np
import pytest

from oracle import guess_mlp as M
from paper_2410_09146_gb300 import inputs as I


def _net(seed, scale=0.4):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, scale, M.NPARAM)
    norm = np.concatenate([rng.normal(0, 0.5, 8), rng.uniform(0.5, 2, 8), rng.normal(0, 1, 2),
                           rng.uniform(0.5, 3, 2)])
    return theta, norm


def test_gradient_matches_finite_differences():
    theta, norm = _net(1)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (12, 8))
    T = rng.normal(0, 2, (12, 2))
    aux = 0.3
    _, g = M.loss_and_grad(theta, norm, X, T, aux)
    # every bias and output weight, and a random sample of each weight matrix
    idx = []
    for name, (o, shape) in M.OFFSETS.items():
        size = int(np.prod(shape))
        if name.startswith("b") or name == "W4":
            idx.extend(range(o, o + size))
        else:
            idx.extend(o + rng.choice(size, 40, replace=False))
    # finite differences of the unrounded network (BF16 rounding makes the loss piecewise constant)
    _, g = M.loss_and_grad(theta, norm, X, T, aux, round_h=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (M.loss_and_grad(tp, norm, X, T, aux, round_h=False)[0]
              - M.loss_and_grad(tm, norm, X, T, aux, round_h=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_rounded_forward_is_straight_through():
    # rounding h1, h2 changes only the activations: the rounded network's gradient is the unrounded
    # formula evaluated on the rounded activations, i.e. equal to the unrounded gradient of a network whose
    # layer-2 and layer-3 inputs are the rounded values; check the forward values and the W2/W3 blocks
    theta, norm = _net(3, scale=0.3)
    rng = np.random.default_rng(4)
    X = rng.normal(0, 1, (9, 8))
    T = rng.normal(0, 2, (9, 2))
    y, c = M.forward(theta, norm, X, cache=True, round_h=True)
    assert np.array_equal(c["h1"], M.bf16_round(c["h1"])) and np.array_equal(c["h2"], M.bf16_round(c["h2"]))
    P = M.unpack(theta)
    assert np.allclose(c["z2"], c["h1"] @ P["W2"].T + P["b2"], rtol=1e-14, atol=1e-14)
    _, g = M.loss_and_grad(theta, norm, X, T, 0.5, round_h=True)
    G = M.unpack(g)
    e = c["o"] - (T - norm[16:18]) / norm[18:20]
    do = 2.0 * np.array([1.0, 0.5]) * e / len(X)
    d3 = (do @ P["W4"]) * (lambda z: (1 / (1 + np.exp(-z))) * (1 + z * (1 - 1 / (1 + np.exp(-z)))))(c["z3"])
    assert np.allclose(G["W3"], d3.T @ c["h2"], rtol=1e-12, atol=1e-15)


def test_rounded_deltas_bound():
    """round_delta (the tensor-core training form) rounds only the deltas of layers 3 and 2 to BF16: the output
    layer's gradient is unchanged bit for bit, and each other block moves by no more than the rounding bound
    it implies -- |delta_bf16 - delta| <= 2^-8 |delta| element by element, carried linearly into the W3, b3
    and the W2, b2 blocks, and through |W3|, |W2| and |dsilu| into the lower layers."""
    theta, norm = _net(5, scale=0.3)
    rng = np.random.default_rng(9)
    X = rng.normal(0, 1, (40, 8))
    T = rng.normal(0, 2, (40, 2))
    _, g0 = M.loss_and_grad(theta, norm, X, T, 0.3, round_delta=False)
    _, g1 = M.loss_and_grad(theta, norm, X, T, 0.3, round_delta=True)
    G0, G1 = M.unpack(g0), M.unpack(g1)
    assert np.array_equal(G0["W4"], G1["W4"]) and np.array_equal(G0["b4"], G1["b4"])
    P = M.unpack(theta)
    _, c = M.forward(theta, norm, X, cache=True)
    e = c["o"] - (T - norm[16:18]) / norm[18:20]
    do = 2.0 * np.array([1.0, 0.3]) * e / len(X)
    ds = lambda z: (1 / (1 + np.exp(-z))) * (1 + z * (1 - 1 / (1 + np.exp(-z))))
    d3 = np.abs((do @ P["W4"]) * ds(c["z3"]))
    u = 2.0 ** -8
    assert np.all(np.abs(G1["W3"] - G0["W3"]) <= u * d3.T @ np.abs(c["h2"]) + 1e-300)
    assert np.all(np.abs(G1["b3"] - G0["b3"]) <= u * d3.sum(0) + 1e-300)
    # |delta2| with the rounded delta3 (bounded by (1 + u) |delta3| |W3| |dsilu|): the W2 block's change
    d2 = (1 + u) * (d3 @ np.abs(P["W3"])) * np.abs(ds(c["z2"]))
    bound_W2 = (u * (1 + u) * d2 + u * d2).T @ np.abs(c["h1"])
    assert np.all(np.abs(G1["W2"] - G0["W2"]) <= bound_W2 + 1e-300)
    assert np.abs(G1["W2"] - G0["W2"]).max() > 0  # the rounding does act


def test_single_unit_chain_closed_form():
    P = {k: np.zeros(s) for k, (_, s) in M.OFFSETS.items()}
    a1, c1, a2, c2, a3, c3, a40, a41, c40, c41 = 0.7, -0.2, 1.3, 0.1, -0.9, 0.4, 1.1, -0.6, 0.05, 0.3
    P["W1"][0, 2] = a1; P["b1"][0] = c1
    P["W2"][0, 0] = a2; P["b2"][0] = c2
    P["W3"][0, 0] = a3; P["b3"][0] = c3
    P["W4"][0, 0] = a40; P["W4"][1, 0] = a41; P["b4"][:] = (c40, c41)
    theta = M.pack(P)
    norm = np.zeros(M.NNORM)
    norm[0:8] = 0.25; norm[8:16] = 2.0; norm[16:18] = (1.5, -0.5); norm[18:20] = (3.0, 0.5)
    X = np.array([[0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0]])

    def silu(z):
        return z / (1.0 + math.exp(-z))

    x2 = (1.0 - 0.25) * 2.0
    h3 = silu(a3 * silu(a2 * silu(a1 * x2 + c1) + c2) + c3)
    want = [(a40 * h3 + c40) * 3.0 + 1.5, (a41 * h3 + c41) * 0.5 - 0.5]
    got = M.forward(theta, norm, X, round_h=False)[0]
    assert np.allclose(got, want, rtol=1e-14, atol=1e-15)


def test_first_adam_step_is_lr_sign():
    rng = np.random.default_rng(3)
    theta = rng.normal(size=50)
    g = rng.normal(size=50)
    th, m, v = M.adam_step(theta, np.zeros(50), np.zeros(50), g, 1, lr=1e-3)
    assert np.allclose(th, theta - 1e-3 * np.sign(g), rtol=0, atol=1e-3 * 1e-8 / np.min(np.abs(g)) + 1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding():
    vals = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -20, -(1 + 2.0 ** -8), 0.0,
                     3.0e38, 1e-40], np.float32)
    want = np.array([1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -1.0, 0.0], np.float64)
    got = M.bf16_round(vals)
    assert np.array_equal(got[:6], want)
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    r = (rng.normal(size=10000) * 10.0 ** rng.uniform(-5, 5, 10000)).astype(np.float32)
    ref = torch.tensor(r).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(r), ref)
    assert np.array_equal(M.bf16_round(vals), torch.tensor(vals).to(torch.bfloat16).to(torch.float64).numpy())


def test_features_targets_at_rest(orc):
    s = I.linear_wave_setup(8)
    p = orc.params(s)
    eps = np.array([1e-6, 1e-3, 0.1, 1.0, 30.0])
    rho = np.array([1.0, 0.3, 1e-4, 2.0, 0.01])
    P = np.zeros((5, 8))
    P[:, 0] = rho
    P[:, 4] = rho * eps
    x = np.zeros((5, 3))
    U = orc.prim2con_points(p, x, P)["U"]
    q, r2, b2, rb2 = M.invariants_flat(U)
    assert np.allclose(q, eps, rtol=1e-14) and np.all(r2 == 0) and np.all(b2 == 0)
    mu, mup, eps_p, W_p = orc.c2p_mu_points(p, x, U, aux=True)
    h = 1.0 + s.gamma_eos * eps
    assert np.allclose(mup, 1.0, rtol=1e-15) and np.allclose(mu, 1.0 / h, rtol=1e-13)
    # at mu_+ = 1 with r = 0: W = 1 and eps = q
    assert np.allclose(W_p, 1.0, rtol=1e-15) and np.allclose(eps_p, eps, rtol=1e-13)
    X = M.features(q, r2, b2, rb2, eps_p, W_p)
    assert np.allclose(X[:, 0], np.log1p(eps), rtol=1e-14) and np.allclose(X[:, 6], 0.1 * np.log(eps), rtol=1e-12)
    assert np.all(X[:, 1:6] == 0) and np.all(X[:, 7] == 0)
    T = M.targets(mu, mup, np.ones(5))
    assert np.allclose(T[:, 0], np.log(h / (h - 1.0)), rtol=1e-9) and np.all(T[:, 1] == 0)
    # the guess map inverts the first target
    assert np.allclose(M.guess_from_output(T[:, 0], mup), mu, rtol=1e-12)


def test_features_of_cold_moving_states(orc):
    # cold gas, B = 0, moving: q = W - 1, r^2 = W^2 - 1, so mu_+ = 1/W is the root itself, W(mu_+) = W
    # and eps(mu_+) = 0 (to roundoff of the W-sized terms)
    s = I.linear_wave_setup(8)
    p = orc.params(s)
    W = np.array([1.5, 3.0, 10.0, 40.0])
    d = np.array([[1.0, 0, 0], [0, 0.6, 0.8], [0.0, 0, 1.0], [0.48, 0.6, 0.64]])
    P = np.zeros((4, 8))
    P[:, 0] = 0.5
    P[:, 1:4] = np.sqrt(W * W - 1)[:, None] * d
    x = np.zeros((4, 3))
    U = orc.prim2con_points(p, x, P)["U"]
    q, r2, b2, rb2 = M.invariants_flat(U)
    assert np.allclose(q, W - 1, rtol=1e-13) and np.allclose(r2, W * W - 1, rtol=1e-13)
    mu, mup, eps_p, W_p = orc.c2p_mu_points(p, x, U, aux=True)
    assert np.allclose(mup, 1.0 / W, rtol=1e-13) and np.allclose(W_p, W, rtol=1e-12)
    assert np.all(np.abs(eps_p) <= 1e-13 * W * W)
    X = M.features(q, r2, b2, rb2, eps_p, W_p)
    assert np.all(X[:, 6] <= 0.1 * np.log(1e-13 * W * W) + 1e-12) and np.allclose(X[:, 7], np.log(W), rtol=1e-12)


def test_targets_of_random_states(orc):
    s = I.linear_wave_setup(8)
    p = orc.params(s)
    Ps = I.c2p_states(3000, seed=21)
    x = np.zeros((len(Ps), 3))
    U = orc.prim2con_points(p, x, Ps)["U"]
    mu, mup = orc.c2p_mu_points(p, x, U)
    Po, st, _ = orc.c2p_points(p, x, U, floors=False)
    ok = st == 0
    W = np.sqrt(1.0 + np.sum(Po[:, 1:4] ** 2, 1))
    T = M.targets(mu, mup, W)
    assert np.all(mu <= mup) and np.all(mu > 0)
    assert np.all((T[:, 0] >= 0) & (T[:, 0] <= M.Y0_MAX))
    # the root is 1/(h W) of the recovered primitives
    h = 1.0 + s.gamma_eos * Po[:, 4] / Po[:, 0]
    assert np.allclose((mu * h * W)[ok], 1.0, rtol=1e-9)
    # ... and W of the generating primitives on well-conditioned states
    W0 = np.sqrt(1.0 + np.sum(Ps[:, 1:4] ** 2, 1))
    good = ok & (W0 < 10)
    assert np.allclose(T[good, 1], np.log(W0[good]), atol=1e-9)
