"""ORACLE -- test infrastructure only.

FP64 reference of the top-m proposal network that the CUDA library trains
and runs: 64 -> 256 -> 256 -> K with GELU (tanh form,
0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))), softmax cross-entropy on
the exact Gaussian-selection label, plain backpropagation.
The input of a patch is its DC-free values scaled by sqrt(beta); log(1/beta)
enters the first layer through a learned per-unit coefficient, so the label
(which depends on beta through Eq. 14) is a function of the input.

Parameter layout (flat FP32/FP64 vector, matrices row-major [out][in]):
W1[256][64], b1[256], wb[256], W2[256][256], b2[256], W3[K][256], b3[K].

The network's definition fixes its precision: the weight matrices are used
rounded to BF16 (round to nearest, ties to even) in every forward pass; the
inference form also rounds the DC-free patch and the hidden activations to
BF16 (``forward_infer``).  ``round_weights`` and ``bf16`` state those roundings.
"""
from __future__ import annotations

import math

import numpy as np

H1 = H2 = 256
D = 64


def sizes(K: int):
    return [("W1", (H1, D)), ("b1", (H1,)), ("wb", (H1,)), ("W2", (H2, H1)), ("b2", (H2,)),
            ("W3", (K, H2)), ("b3", (K,))]


def n_params(K: int) -> int:
    return sum(int(np.prod(s)) for _, s in sizes(K))


def unpack(theta, K: int):
    out, o = {}, 0
    for name, s in sizes(K):
        n = int(np.prod(s))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(s)
        o += n
    return out


def pack(p, K: int):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in sizes(K)])


GA = math.sqrt(2.0 / math.pi)
GB = 0.044715


def gelu(x):
    """GELU in its tanh form (within 5e-4 of x Phi(x) everywhere)."""
    return 0.5 * x * (1.0 + np.tanh(GA * (x + GB * x ** 3)))


def gelu_grad(x):
    t = np.tanh(GA * (x + GB * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GA * (1.0 + 3.0 * GB * x * x)


def inputs(images, H: int, W: int, img_idx, anchors, log_ib):
    """DC-free 8x8 patches (periodic, top-left anchors) scaled by sqrt(beta)."""
    X = np.empty((len(anchors), D))
    for n, (im, a) in enumerate(zip(img_idx, anchors)):
        i, j = divmod(int(a), W)
        z = images[im][np.ix_((np.arange(8) + i) % H, (np.arange(8) + j) % W)].ravel().astype(np.float64)
        X[n] = (z - z.mean()) * math.exp(-0.5 * float(log_ib[n]))
    return X


def forward(p, X, cond):
    a1 = X @ p["W1"].T + p["b1"] + np.outer(cond, p["wb"])
    h1 = gelu(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(a2)
    logits = h2 @ p["W3"].T + p["b3"]
    return logits, (a1, h1, a2, h2)


def loss(p, X, cond, labels):
    logits, _ = forward(p, X, cond)
    m = logits.max(axis=1, keepdims=True)
    lse = m[:, 0] + np.log(np.exp(logits - m).sum(axis=1))
    return float(np.mean(lse - logits[np.arange(len(labels)), labels]))


def loss_and_grad(p, X, cond, labels):
    """Mean softmax cross-entropy and its gradient (dict like p)."""
    B = X.shape[0]
    logits, (a1, h1, a2, h2) = forward(p, X, cond)
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    prob = e / e.sum(axis=1, keepdims=True)
    lse = m[:, 0] + np.log(e.sum(axis=1))
    L = float(np.mean(lse - logits[np.arange(B), labels]))
    d3 = prob.copy()
    d3[np.arange(B), labels] -= 1.0
    d3 /= B
    g = {"W3": d3.T @ h2, "b3": d3.sum(axis=0)}
    d2 = (d3 @ p["W3"]) * gelu_grad(a2)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * gelu_grad(a1)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    g["wb"] = d1.T @ cond
    return L, g


def bf16(x):
    """Round to the nearest BF16 value (ties to even), from the float32 value of x:
    the 16 low bits of the float32 pattern are rounded away."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out.reshape(np.shape(x))


def round_weights(p):
    """The parameters every forward pass uses: W1, W2, W3 rounded to BF16."""
    q = dict(p)
    for name in ("W1", "W2", "W3"):
        q[name] = bf16(p[name])
    return q


def patches(images, H: int, W: int, img_idx, anchors):
    """DC-free 8x8 patches (periodic, top-left anchors), unscaled."""
    Z = np.empty((len(anchors), D))
    for n, (im, a) in enumerate(zip(img_idx, anchors)):
        i, j = divmod(int(a), W)
        z = images[im][np.ix_((np.arange(8) + i) % H, (np.arange(8) + j) % W)].ravel().astype(np.float64)
        Z[n] = z - z.mean()
    return Z


def forward_infer(p, Z, ibeta: float):
    """Logits of the inference form at one beta (1/beta = ibeta): BF16 patch,
    first layer W1 (sqrt(beta) z) = sqrt(beta) (W1 z) with log(1/beta) through wb,
    BF16 hidden activations."""
    q = round_weights(p)
    a1 = (bf16(Z) @ q["W1"].T) / math.sqrt(ibeta) + q["b1"] + math.log(ibeta) * q["wb"]
    h1 = bf16(gelu(a1))
    h2 = bf16(gelu(h1 @ q["W2"].T + q["b2"]))
    return h2 @ q["W3"].T + q["b3"]


def topm(logits, m: int):
    """Indices of the m largest logits per row (lowest index first on ties) and
    their softmax mass."""
    order = np.argsort(-logits, axis=1, kind="stable")[:, :m]
    mx = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - mx)
    mass = np.take_along_axis(e, order, axis=1).sum(axis=1) / e.sum(axis=1)
    return order, mass


# Exponential decay rates and epsilon of the optimiser (Kingma & Ba's defaults).
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8
# Parameter blocks whose weight decays (the matrices; biases and wb do not).
DECAYED = ("W1", "W2", "W3")


def adamw_step(p, g, m, v, step: int, lr: float, wd: float):
    """One AdamW step (Loshchilov & Hutter, "Decoupled weight decay
    regularization", ICLR 2019, Algorithm 2 with the schedule multiplier
    eta_t = lr and alpha = 1): first and second moment estimates
    m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, their bias corrections
    m_hat = m / (1 - b1^t), v_hat = v / (1 - b2^t), and the update
    theta <- theta - lr (m_hat / (sqrt(v_hat) + eps) + wd theta), where the
    decay term appears only for the weight matrices and is not part of the
    gradient that the moments see.  p, g, m, v are dicts of FP64 arrays; returns
    the new (p, m, v); `step` is t >= 1, the index of this step."""
    c1 = 1.0 - ADAM_B1 ** step
    c2 = 1.0 - ADAM_B2 ** step
    p2, m2, v2 = {}, {}, {}
    for name in p:
        mk = ADAM_B1 * m[name] + (1.0 - ADAM_B1) * g[name]
        vk = ADAM_B2 * v[name] + (1.0 - ADAM_B2) * g[name] * g[name]
        upd = (mk / c1) / (np.sqrt(vk / c2) + ADAM_EPS)
        if name in DECAYED:
            upd = upd + wd * p[name]
        p2[name] = p[name] - lr * upd
        m2[name] = mk
        v2[name] = vk
    return p2, m2, v2
