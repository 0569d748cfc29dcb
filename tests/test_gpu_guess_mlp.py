"""GPU tests of the learned con2prim guess against the FP64 reference network and the oracle's con2prim.

* forward outputs and the gradient of the loss of the CUDA kernels against oracle/guess_mlp.py evaluated
  in FP64 on the same BF16-rounded weights and the same inputs (1000 samples: 7 full tiles and a ragged
  tail of 104);
* the first Adam step: master weights move by lr * sign(g), the BF16 copy is the nearest-even rounding;
* features and targets recorded by the guided con2prim against the oracle's invariants, root and W;
* the fused kernel's guess (hidden layers on the tensor cores) against the FP64 reference network;
* without a guess the guided batch reproduces the plain batch; with a network trained on oracle-solved
  pairs both network paths (FP32 cores, tensor cores) need fewer iterations for the same roots and
  rarely fall back to the standard start.
"""
import numpy as np
import pytest

from oracle import guess_mlp as M
from paper_2410_09146_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _setup():
    import torch
    from paper_2410_09146_gb300 import grmhd as G
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.lib()
    return torch, G


def _oracle_pairs(orc, n, seed):
    s = I.linear_wave_setup(8)
    p = orc.params(s)
    Ps = I.c2p_states(n, seed=seed)
    x = np.zeros((n, 3))
    U = orc.prim2con_points(p, x, Ps)["U"]
    mu, mup, eps_p, W_p = orc.c2p_mu_points(p, x, U, aux=True)
    Po, st, _ = orc.c2p_points(p, x, U, floors=False)
    W = np.sqrt(1.0 + np.sum(Po[:, 1:4] ** 2, 1))
    X = M.features(*M.invariants_flat(U), eps_p, W_p)
    T = M.targets(mu, mup, W)
    return U, X, T, st, mu, mup


def _random_norm(rng):
    return np.concatenate([rng.normal(0, 0.3, 8), rng.uniform(0.5, 2, 8), rng.normal(10, 1, 1), rng.normal(1, 0.2, 1),
                           rng.uniform(2, 5, 1), rng.uniform(0.5, 1, 1)]).astype(np.float32)


def test_forward_and_gradient_match_fp64_reference(orc):
    torch, G = _setup()
    rng = np.random.default_rng(5)
    net = G.GuessNet(seed=7)
    theta = (G.init_weights(7) + rng.normal(0, 0.05, M.NPARAM)).astype(np.float32)  # nonzero biases too
    norm = _random_norm(rng)
    net.set_weights(theta, norm)
    master, wb = net.weights()
    assert np.array_equal(master, theta)
    assert np.array_equal(wb.astype(np.float64), M.bf16_round(theta))
    U, X, T, _, _, _ = _oracle_pairs(orc, 1000, seed=6)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Td = torch.tensor(T, dtype=torch.float32, device="cuda")
    X32 = Xd.cpu().numpy().astype(np.float64)
    T32 = Td.cpu().numpy().astype(np.float64)
    Yg = net.forward(Xd)
    torch.cuda.synchronize()
    Yr = M.forward(wb, norm.astype(np.float64), X32)
    scale = norm[18:20].astype(np.float64)
    # FP32 sums of 64 terms per layer; h1, h2 are rounded to BF16 on both sides, and a value within an
    # FP32 rounding error of a BF16 rounding boundary can round the other way (a few samples in 1000)
    err = np.abs(Yg.cpu().numpy() - Yr) / (scale + np.abs(Yr))
    assert np.percentile(err, 99) < 1e-4 and err.max() < 2e-2, (np.percentile(err, 99), err.max())
    aux = 0.25
    loss_g, grad_g = net.grad(Xd, Td, aux)
    loss_r, grad_r = M.loss_and_grad(wb, norm.astype(np.float64), X32, T32, aux)
    assert abs(loss_g - loss_r) <= 1e-5 * loss_r
    for name, (o, shape) in M.OFFSETS.items():
        sz = int(np.prod(shape))
        gg, gr = grad_g[o:o + sz].astype(np.float64), grad_r[o:o + sz]
        rel = np.linalg.norm(gg - gr) / np.linalg.norm(gr)
        assert rel < 1e-4, (name, rel)


def test_tensor_core_gradient_matches_fp64_reference(orc):
    """grmhd_mlp_grad_tc (the 64 x 64 products and weight gradients as tcgen05 MMAs) against the FP64 reference
    network with the same BF16 roundings (forward activations h1, h2 and the deltas of layers 3 and 2), on the
    same BF16 weights: 1000 samples, 7 full tiles of 128 and a ragged tail of 104."""
    torch, G = _setup()
    rng = np.random.default_rng(15)
    net = G.GuessNet(seed=17)
    theta = (G.init_weights(17) + rng.normal(0, 0.05, M.NPARAM)).astype(np.float32)
    norm = _random_norm(rng)
    net.set_weights(theta, norm)
    _, wb = net.weights()
    U, X, T, _, _, _ = _oracle_pairs(orc, 1000, seed=16)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Td = torch.tensor(T, dtype=torch.float32, device="cuda")
    X32 = Xd.cpu().numpy().astype(np.float64)
    T32 = Td.cpu().numpy().astype(np.float64)
    aux = 0.25
    loss_t, grad_t = net.grad(Xd, Td, aux, tc=True)
    loss_r, grad_r = M.loss_and_grad(wb, norm.astype(np.float64), X32, T32, aux, round_delta=True)
    loss_f, grad_f = net.grad(Xd, Td, aux)  # the FP32-core gradient (unrounded deltas)
    _, grad_u = M.loss_and_grad(wb, norm.astype(np.float64), X32, T32, aux, round_delta=False)
    assert abs(loss_t - loss_r) <= 1e-5 * loss_r and abs(loss_t - loss_f) <= 1e-5 * loss_r
    worst = {}
    for name, (o, shape) in M.OFFSETS.items():
        sz = int(np.prod(shape))
        gt, gr = grad_t[o:o + sz].astype(np.float64), grad_r[o:o + sz]
        worst[name] = np.linalg.norm(gt - gr) / np.linalg.norm(gr)
        # the rounded deltas move the lower blocks by about the BF16 unit against the unrounded gradient
        drift = np.linalg.norm(gr - grad_u[o:o + sz]) / np.linalg.norm(grad_u[o:o + sz])
        assert drift < 1e-2, (name, drift)
    print("tensor-core gradient vs the reference with BF16 deltas:", worst)
    assert max(worst.values()) < 1e-4, worst


def test_tensor_core_training_reduces_the_loss(orc):
    """A few hundred Adam steps of grmhd_mlp_train_tc on oracle-solved pairs lower the loss as the FP32-core
    training does from the same start."""
    torch, G = _setup()
    U, X, T, st, _, _ = _oracle_pairs(orc, 20000, seed=21)
    keep = (st & (8 | 16)) == 0
    Xd = torch.tensor(X[keep], dtype=torch.float32, device="cuda")
    Td = torch.tensor(T[keep], dtype=torch.float32, device="cuda")
    out = {}
    for tc in (False, True):
        net = G.GuessNet(seed=23)
        net.fit_norm(Xd, Td)
        losses = torch.zeros(300, dtype=torch.float32, device="cuda")
        net.train(Xd, Td, batch=2048, steps=300, lr=3e-3, lr_end=3e-4, losses=losses, tc=tc)
        torch.cuda.synchronize()
        lh = losses.cpu().numpy()
        out[tc] = (float(lh[:10].mean()), float(lh[-20:].mean()))
        assert net.grad(Xd[:128], Td[:128], 0.1, tc=tc)[0] >= 0  # no tensor-core wait timed out
    print("loss first / last (FP32 cores, tensor cores):", out)
    assert out[True][1] < 0.1 * out[True][0]
    assert out[True][1] < 3.0 * out[False][1]


def test_first_adam_step(orc):
    torch, G = _setup()
    rng = np.random.default_rng(8)
    net = G.GuessNet(seed=3)
    theta = G.init_weights(3)
    net.set_weights(theta, _random_norm(rng))
    U, X, T, _, _, _ = _oracle_pairs(orc, 700, seed=9)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Td = torch.tensor(T, dtype=torch.float32, device="cuda")
    _, g = net.grad(Xd, Td, 0.1)  # the gradient stays in the workspace for Adam
    lr = 1e-3
    net.adam(lr)
    master, wb = net.weights()
    want, _, _ = M.adam_step(theta.astype(np.float64), np.zeros(M.NPARAM), np.zeros(M.NPARAM), g.astype(np.float64),
                             1, lr)
    nz = g != 0
    assert np.allclose(master[nz], want[nz], rtol=0, atol=2e-7)
    assert np.array_equal(master[~nz], theta[~nz])
    assert np.array_equal(wb.astype(np.float64), M.bf16_round(master))


def test_tensor_core_network_matches_fp64_reference(orc):
    # the fused kernel's guess (hidden layers as tcgen05 MMAs) against the FP64 reference network on the
    # features the library records for the same states (standard path), over 2.5 tiles of 128 plus a
    # ragged tail
    torch, G = _setup()
    rng = np.random.default_rng(12)
    n = 20000 + 77
    U, X, T, st_o, _, _ = _oracle_pairs(orc, n, seed=13)
    net = G.GuessNet(seed=4)
    theta = (G.init_weights(4) + rng.normal(0, 0.02, M.NPARAM)).astype(np.float32)
    norm = np.concatenate([X.mean(0), 1.0 / X.std(0), [12.0, 1.0], [3.0, 0.7]]).astype(np.float32)
    net.set_weights(theta, norm)
    _, wb = net.weights()
    ctx = G.Context(I.Setup(n=(0, 0, 0)))
    Ud = torch.tensor(U.T.copy(), device="cuda")
    P1, P2 = torch.zeros_like(Ud), torch.zeros_like(Ud)
    st1 = torch.zeros(n, dtype=torch.uint8, device="cuda")
    st2 = torch.zeros_like(st1)
    it2 = torch.zeros(n, dtype=torch.int32, device="cuda")
    Xg = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    guess = torch.full((2, n), -1.0, dtype=torch.float64, device="cuda")
    ctx.c2p_guess(Ud, P1, st1, None, X=Xg)
    ctx.c2p_guess(Ud, P2, st2, it2, net=net, guess=guess)
    stats = ctx.stats()
    torch.cuda.synchronize()
    assert int(stats[6]) == 0  # no tile abandoned
    g = guess.cpu().numpy()
    ok = st1.cpu().numpy() == 0
    assert np.all(g[1, ok] > 0) and np.all(g[0, ok] <= g[1, ok])
    y_tc = -np.log1p(-g[0] / g[1])
    y_ref = M.forward(wb, norm.astype(np.float64), Xg.cpu().numpy().astype(np.float64))[:, 0]
    m = ok & (y_ref > 0.5) & (y_ref < 29.5)
    assert m.mean() > 0.9
    d = np.abs(y_tc[m] - y_ref[m])
    assert np.median(d) < 1e-4 and np.percentile(d, 99) < 2e-3 and d.max() < 0.1, (np.median(d), d.max())
    # same statuses as the standard start, and every state converged
    assert np.array_equal(st1.cpu().numpy(), st2.cpu().numpy())
    assert not np.any(st2.cpu().numpy() & 8)
    assert int(stats[0]) == int(it2.cpu().numpy().sum())


def test_features_targets_and_plain_equivalence(orc):
    torch, G = _setup()
    n = 20000
    U, X, T, st_o, mu, mup = _oracle_pairs(orc, n, seed=10)
    ctx = G.Context(I.Setup(n=(0, 0, 0)))
    Ud = torch.tensor(U.T.copy(), device="cuda")
    P1 = torch.zeros_like(Ud)
    P2 = torch.zeros_like(Ud)
    st1 = torch.zeros(n, dtype=torch.uint8, device="cuda")
    st2 = torch.zeros_like(st1)
    it1 = torch.zeros(n, dtype=torch.int32, device="cuda")
    it2 = torch.zeros_like(it1)
    Xg = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    Tg = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    ctx.c2p(Ud, P1, st1, it1)
    ctx.c2p_guess(Ud, P2, st2, it2, X=Xg, T=Tg)
    stats = ctx.stats()
    torch.cuda.synchronize()
    # no guess: the same solve as the plain batch
    assert np.array_equal(st1.cpu().numpy(), st2.cpu().numpy())
    assert np.mean(it1.cpu().numpy() == it2.cpu().numpy()) > 0.999
    a, b = P1.cpu().numpy(), P2.cpu().numpy()
    sc = np.abs(a).max(axis=0, keepdims=True) + 1e-300
    assert np.max(np.abs(a - b) / sc) < 1e-13
    assert int(stats[0]) == int(it2.cpu().numpy().sum())
    # recorded features against the oracle's (FP32 features of FP64 invariants); ln eps(mu_+) is compared
    # where eps(mu_+) is above the roundoff of the energy terms it is the difference of
    Xn = Xg.cpu().numpy().astype(np.float64)
    cols = [0, 1, 2, 3, 4, 5, 7]
    assert np.max(np.abs(Xn[:, cols] - X[:, cols]) / (1.0 + np.abs(X[:, cols]))) < 2e-6
    q = M.invariants_flat(U)[0]
    resolved = X[:, 6] > 0.1 * np.log(1e-9 * (1.0 + np.abs(q)))
    assert resolved.mean() > 0.5
    assert np.max(np.abs(Xn[resolved, 6] - X[resolved, 6])) < 1e-5
    # recorded targets against the oracle's root: d y0 = (d mu / mu) e^{y0}, so roots that agree to the solve
    # tolerance 1e-10 give |d y0| <= 1e-10 e^{y0} (plus the FP32 rounding of y0)
    Tn = Tg.cpu().numpy().astype(np.float64)
    ok = (st_o == 0) & (st2.cpu().numpy() == 0)
    assert ok.mean() > 0.99
    bound = 1e-10 * np.exp(T[ok, 0]) + 4e-6 * (1.0 + T[ok, 0])
    assert np.all(np.abs(Tn[ok, 0] - T[ok, 0]) <= bound)
    assert np.max(np.abs(Tn[ok, 1] - T[ok, 1])) < 1e-5


def test_trained_guess_reduces_iterations(orc):
    torch, G = _setup()
    # training pairs: oracle-solved states (features and targets from oracle/guess_mlp.py)
    _, X, T, st, _, _ = _oracle_pairs(orc, 300000, seed=31)
    keep = st == 0
    Xd = torch.tensor(X[keep], dtype=torch.float32, device="cuda")
    Td = torch.tensor(T[keep], dtype=torch.float32, device="cuda")
    net = G.GuessNet(seed=1)
    net.fit_norm(Xd, Td)
    losses = torch.zeros(3000, dtype=torch.float32, device="cuda")
    net.train(Xd, Td, batch=152 * 128, steps=3000, lr=3e-3, lr_end=3e-5, aux=0.1, losses=losses)
    torch.cuda.synchronize()
    lh = losses.cpu().numpy()
    assert np.all(np.isfinite(lh)) and lh[-100:].mean() < 0.2 * lh[:10].mean()
    # held-out states
    Ue, Xe, Te, st_e, _, _ = _oracle_pairs(orc, 100000, seed=32)
    n = len(Ue)
    ctx = G.Context(I.Setup(n=(0, 0, 0)))
    Ud = torch.tensor(Ue.T.copy(), device="cuda")
    Ps, Pn = torch.zeros_like(Ud), torch.zeros_like(Ud)
    sts = torch.zeros(n, dtype=torch.uint8, device="cuda")
    stn = torch.zeros_like(sts)
    its = torch.zeros(n, dtype=torch.int32, device="cuda")
    itn = torch.zeros_like(its)
    guess = torch.zeros((2, n), dtype=torch.float64, device="cuda")
    Pt = torch.zeros_like(Ud)
    stt = torch.zeros_like(sts)
    itt = torch.zeros_like(its)
    ctx.c2p_guess(Ud, Ps, sts, its)
    ctx.c2p_guess(Ud, Pn, stn, itn, net=net, guess=guess, fp32=True)
    fallbacks = int(ctx.stats()[7])
    ctx.c2p_guess(Ud, Pt, stt, itt, net=net)
    stats_tc = ctx.stats()
    torch.cuda.synchronize()
    its, itn, itt = its.cpu().numpy(), itn.cpu().numpy(), itt.cpu().numpy()
    sts, stn, stt = sts.cpu().numpy(), stn.cpu().numpy(), stt.cpu().numpy()
    assert np.array_equal(sts, stn) and np.array_equal(sts, stt)
    assert np.mean(stn & 8) == 0 and np.mean(stt & 8) == 0  # every state converged
    assert int(stats_tc[6]) == 0
    # the guess: median error of y0 on the held-out states
    g = guess.cpu().numpy()
    y0 = -np.log1p(-g[0] / g[1])
    good = (st_e == 0) & (Te[:, 0] < 25)
    yerr = np.abs(y0[good] - Te[good, 0])
    assert np.median(yerr) < 0.1, np.median(yerr)
    assert fallbacks <= 0.01 * n and int(stats_tc[7]) <= 0.01 * n
    # fewer iterations on both network paths
    for it in (itn, itt):
        assert it.mean() <= its.mean() - 1.0, (its.mean(), it.mean())
        assert np.percentile(it, 99) <= np.percentile(its, 99)
    # both solutions reproduce U to roundoff (the conditioning-free measure) ...
    s = I.linear_wave_setup(8)
    p = orc.params(s)
    x = np.zeros((n, 3))
    plain = sts == 0
    scale = np.abs(Ue[:, 0]) + np.abs(Ue[:, 4]) + np.linalg.norm(Ue[:, 1:4], axis=1)
    for Pd in (Ps, Pn, Pt):
        Ub = orc.prim2con_points(p, x, Pd.cpu().numpy().T.copy())["U"]
        be = (np.max(np.abs(Ub - Ue), axis=1) / scale)[plain]
        assert be.max() < 1e-11 and np.median(be) < 1e-14
    # ... and agree where the primitives are well-conditioned functions of U (W <= 10, b^2/rho <= 10,
    # p/rho >= 1e-4 of the generating states); elsewhere they differ by condition number x tolerance
    Pg = I.c2p_states(n, seed=32)
    W = np.sqrt(1 + np.sum(Pg[:, 1:4] ** 2, 1))
    sig = np.sum(Pg[:, 5:8] ** 2, 1) / (Pg[:, 0] * W * W)
    good = plain & (W <= 10) & (sig <= 10) & (Pg[:, 4] * (s.gamma_eos - 1.0) / Pg[:, 0] >= 1e-4)
    assert good.mean() > 0.05
    a = Ps.cpu().numpy()[:5, good]
    for Pd in (Pn, Pt):
        b = Pd.cpu().numpy()[:5, good]
        assert np.max(np.abs(a - b) / (np.abs(a) + np.abs(a[0]))) < 1e-10
