"""FP64 reference of the learned con2prim initial guess (test infrastructure only).

Only tests, the smoke check and the benchmark's CPU-baseline leg use this module; the library never
imports it.

The network maps eight features of a conserved state to a guess for the root mu = 1/(h W) of the
Kastaun master function (Sec. 3.1 of the paper; the root lies in the bracket (0, mu_+]). Six features
are functions of the invariants q = tau/D, r^2, b^2, (r.b)^2; the other two, ln(eps)/10 and ln W of the
master-function intermediates at mu_+, carry the thermal content that fixes how close the root is to
mu_+ (features()).

    x  = (features - mean_x) * invstd_x
    h1 = bf16(silu(W1 x + b1)),  h2 = bf16(silu(W2 h1 + b2)),  h3 = silu(W3 h2 + b3)
    o  = W4 h3 + b4,             y = o * std_y + mean_y

with 64 hidden units per layer, SiLU(z) = z / (1 + e^-z) and bf16() the round-to-nearest-even BF16
rounding of the two activations that feed the 64 x 64 layers (tensor-core operands on the GPU). The two outputs are
y0 = -ln(1 - mu/mu_+) (clipped to [0, 30]) and y1 = ln W at the root. The loss is the mean over
samples of (o0 - t0)^2 + aux (o1 - t1)^2 in standardised units t = (y - mean_y)/std_y.

Flat parameter vector (float32 on the device, BF16 copy used by every forward pass):
W1 [64][8], b1 [64], W2 [64][64], b2 [64], W3 [64][64], b3 [64], W4 [2][64], b4 [2] (row-major,
[out][in]). Standardisation vector: mean_x [8], invstd_x [8], mean_y [2], std_y [2].

Pins (tests/test_oracle_guess_mlp.py): central finite differences of the loss against backward();
a one-unit chain evaluated in closed form; the first Adam step moving every parameter by lr*sign(g);
BF16 rounding of values with known nearest-even results; features and targets of hand-computed states.
"""
from __future__ import annotations

import numpy as np

NIN, HID, NOUT = 8, 64, 2
Y0_MAX = 30.0
EPS_P_MIN = 1e-30

_shapes = [("W1", (HID, NIN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID, HID)),
           ("b3", (HID,)), ("W4", (NOUT, HID)), ("b4", (NOUT,))]
OFFSETS = {}
_o = 0
for _name, _shape in _shapes:
    OFFSETS[_name] = (_o, _shape)
    _o += int(np.prod(_shape))
NPARAM = _o  # 9026
NNORM = 2 * NIN + 2 * NOUT


def unpack(theta):
    """Flat parameter vector -> dict of float64 arrays (views where possible)."""
    theta = np.asarray(theta, dtype=np.float64)
    return {k: theta[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in OFFSETS.items()}


def pack(d):
    out = np.zeros(NPARAM)
    for k, (o, s) in OFFSETS.items():
        out[o:o + int(np.prod(s))] = np.asarray(d[k], dtype=np.float64).ravel()
    return out


def bf16_round(a):
    """Round float32 values to the nearest BF16 value, ties to even (returned as float64)."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def invariants_flat(U):
    """Inputs of the master function in flat space (gamma_ij = delta_ij), U [n][8] undensitized.

    q = tau/D, r_i = S_i/D, b^i = B^i/sqrt(D); returns (q, r2, b2, rb2).
    """
    U = np.asarray(U, dtype=np.float64)
    D = U[:, 0]
    q = U[:, 4] / D
    r = U[:, 1:4] / D[:, None]
    b = U[:, 5:8] / np.sqrt(D)[:, None]
    r2 = np.sum(r * r, 1)
    b2 = np.sum(b * b, 1)
    rb = np.sum(r * b, 1)
    return q, r2, b2, rb * rb


def features(q, r2, b2, rb2, eps_p, W_p):
    """The eight raw features [n][8] of the network (before standardisation).

    eps_p and W_p are eps and W of the master-function intermediates at the bracket end mu_+ (Kastaun
    et al. 2021; the oracle's con2prim returns them). eps_p measures the thermal content: it is zero
    exactly when the root sits on mu_+ (the cold limit).
    """
    q = np.maximum(np.asarray(q, dtype=np.float64), 0.0)
    r2 = np.asarray(r2, dtype=np.float64)
    b2 = np.asarray(b2, dtype=np.float64)
    rb2 = np.asarray(rb2, dtype=np.float64)
    r = np.sqrt(r2)
    X = np.empty((len(q), NIN))
    X[:, 0] = np.log1p(q)
    X[:, 1] = 0.5 * np.log1p(r2)
    X[:, 2] = 0.5 * np.log1p(b2)
    X[:, 3] = 0.25 * np.log1p(rb2)
    X[:, 4] = r / (1.0 + q)
    X[:, 5] = b2 / (1.0 + q)
    X[:, 6] = 0.1 * np.log(np.maximum(np.asarray(eps_p, dtype=np.float64), EPS_P_MIN))
    X[:, 7] = np.log(np.asarray(W_p, dtype=np.float64))
    return X


def targets(mu, mup, W):
    """Training targets [n][2]: y0 = -ln(1 - mu/mu_+) clipped to [0, 30], y1 = ln W."""
    ratio = np.asarray(mu, dtype=np.float64) / np.asarray(mup, dtype=np.float64)
    with np.errstate(divide="ignore"):
        y0 = -np.log1p(-np.minimum(ratio, 1.0))
    T = np.empty((len(ratio), NOUT))
    T[:, 0] = np.clip(y0, 0.0, Y0_MAX)
    T[:, 1] = np.log(np.asarray(W, dtype=np.float64))
    return T


def guess_from_output(y0, mup):
    """Newton start mu_0 = mu_+ (1 - e^{-y0}) for the (clipped) first output."""
    return np.asarray(mup) * (1.0 - np.exp(-np.clip(y0, 0.0, Y0_MAX)))


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, norm, X, cache: bool = False, round_h: bool = True):
    """Network outputs y [n][2] (de-standardised) for raw features X [n][8].

    round_h: the hidden activations h1 and h2 (the inputs of the two 64 x 64 layers, the tensor-core
    operands on the GPU) are rounded to BF16, as every forward pass of the library does; the gradient
    passes through the rounding unchanged (straight-through).
    """
    P = unpack(theta)
    norm = np.asarray(norm, dtype=np.float64)
    rnd = bf16_round if round_h else (lambda a: a)
    x = (np.asarray(X, dtype=np.float64) - norm[:NIN]) * norm[NIN:2 * NIN]
    z1 = x @ P["W1"].T + P["b1"]
    h1 = rnd(_silu(z1))
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = rnd(_silu(z2))
    z3 = h2 @ P["W3"].T + P["b3"]
    h3 = _silu(z3)
    o = h3 @ P["W4"].T + P["b4"]
    y = o * norm[2 * NIN + 2:] + norm[2 * NIN:2 * NIN + 2]
    if cache:
        return y, dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3, o=o)
    return y


def loss_and_grad(theta, norm, X, T, aux: float, round_h: bool = True, round_delta: bool = False):
    """Loss (mean over samples) and its gradient [NPARAM] for raw features X and raw targets T.

    round_delta: the deltas back-propagated into layers 3 and 2 (the operands of the tensor-core products of
    the library's tensor-core training kernel: delta3 W3, delta2 W2 and the weight gradients delta^T h) are
    rounded to BF16 where they enter those products; delta1 and the output layer's quantities are not."""
    P = unpack(theta)
    norm = np.asarray(norm, dtype=np.float64)
    _, c = forward(theta, norm, X, cache=True, round_h=round_h)
    n = len(X)
    t = (np.asarray(T, dtype=np.float64) - norm[2 * NIN:2 * NIN + 2]) / norm[2 * NIN + 2:]
    wgt = np.array([1.0, aux])
    e = c["o"] - t
    loss = float(np.sum(wgt * e * e) / n)
    do = 2.0 * wgt * e / n
    g = {}
    g["W4"] = do.T @ c["h3"]
    g["b4"] = do.sum(0)
    rd = bf16_round if round_delta else (lambda a: a)
    d3 = rd((do @ P["W4"]) * _dsilu(c["z3"]))
    g["W3"] = d3.T @ c["h2"]
    g["b3"] = d3.sum(0)
    d2 = rd((d3 @ P["W3"]) * _dsilu(c["z2"]))
    g["W2"] = d2.T @ c["h1"]
    g["b2"] = d2.sum(0)
    d1 = (d2 @ P["W2"]) * _dsilu(c["z1"])
    g["W1"] = d1.T @ c["x"]
    g["b1"] = d1.sum(0)
    return loss, pack(g)


def adam_step(theta, m, v, g, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) of theta; returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
