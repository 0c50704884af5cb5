"""Normalising-flow proposal for the acceptance walk, and its maximum-likelihood training.

The paper (Sec. 5) motivates flow-accelerated nested sampling (Nessai; Prathaban et al.) as a
natural fit for a batched GPU sampler but specifies no architecture.  Every choice below is a
reading, kept deliberately plain:

* a RealNVP affine-coupling flow (Dinh, Sohl-Dickstein & Bengio 2017) on the unit cube;
* the fixed pre-map z0 = (logit(u) - mu) / sigma, with mu and sigma the per-dimension mean and
  standard deviation of logit(u) over the training points (so the flow starts at the
  identity on standardised data);
* L coupling layers; layer l conditions on the dimensions d with (d + l) even (mask m_l = 1)
  and transforms the others:
      a   = m_l * z
      h1  = tanh(W1 a + b1),  h2 = tanh(W2 h1 + b2),  o = W3 h2 + b3  (o = [s_raw | t], 2 D)
      s   = (1 - m_l) * S tanh(s_raw / S),  t <- (1 - m_l) * t,  S = 2
      z'  = m_l * z + (1 - m_l) * (z exp(s) + t),   log|det| += sum(s)
* base density N(0, I_D) on x = z_L, so
      log q(u) = log N(x) + sum_l sum(s_l) - sum_d log sigma_d - sum_d log(u_d (1 - u_d));
* inverse (sampling): z_{l-1} = m_l z_l + (1 - m_l)(z_l - t) exp(-s), u = sigmoid(sigma z_0 + mu);
* loss = mean over the training points of -log q(u), minimised by Adam (Kingma & Ba 2015,
  beta = (0.9, 0.999), eps = 1e-8, bias-corrected), full batch; the step counter advances
  every step, and a gradient component that is not finite leaves its parameter and moments
  unchanged;
* initial weights: W1 and W2 uniform on (-1, 1) / sqrt(fan_in) from Philox block
  (l, mat, e // 4, 5), word e % 4 (mat 0 = W1, 1 = W2; e the row-major element index);
  W3 and every bias start at zero, so the initial flow is the identity.

`bf16=True` evaluates the method at the precision the tensor-core path uses: every matrix
product takes its operands rounded to bfloat16 (round to nearest, ties to even; weights, the
masked input a, h1, h2 and, in the backward pass, the output and hidden-layer gradients),
accumulates exactly (FP64 here) and adds the biases unrounded; tanh derivatives use the
rounded activations.  With bf16=False everything is plain FP64.

This module is test infrastructure (see the package header).  Pins: forward o inverse = id,
log q against the log-determinant of a finite-difference Jacobian, gradients against central
finite differences, the 2-D density integrating to 1, Adam's first step, training recovering
a Gaussian's entropy, bf16 rounding against torch's conversion.
"""
import math

import numpy as np

from .philox import philox4x64_vec, open_unit_vec

S_CLAMP = 2.0
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8
LOG_2PI = math.log(2.0 * math.pi)


def round_bf16(x):
    """Round to the nearest bfloat16 value (8 significant bits), ties to even; FP64 in and out."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                     # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def masks(n_dim: int, n_layers: int) -> np.ndarray:
    """m[l, d] = 1 for the dimensions layer l conditions on ((d + l) even), else 0."""
    d = np.arange(n_dim)[None, :]
    l = np.arange(n_layers)[:, None]
    return ((d + l) % 2 == 0).astype(np.float64)


class Flow:
    """Parameters of an L-layer coupling flow in D dimensions with hidden width H."""

    def __init__(self, n_dim: int, n_hidden: int = 128, n_layers: int = 8):
        self.D, self.H, self.L = n_dim, n_hidden, n_layers
        self.mask = masks(n_dim, n_layers)
        D, H = n_dim, n_hidden
        self.W1 = [np.zeros((H, D)) for _ in range(n_layers)]
        self.b1 = [np.zeros(H) for _ in range(n_layers)]
        self.W2 = [np.zeros((H, H)) for _ in range(n_layers)]
        self.b2 = [np.zeros(H) for _ in range(n_layers)]
        self.W3 = [np.zeros((2 * D, H)) for _ in range(n_layers)]
        self.b3 = [np.zeros(2 * D) for _ in range(n_layers)]
        self.mu = np.zeros(D)
        self.sigma = np.ones(D)

    # parameter vector: per layer W1, b1, W2, b2, W3, b3 (row-major), layers in order
    NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")

    def flat(self) -> np.ndarray:
        return np.concatenate([getattr(self, n)[l].ravel() for l in range(self.L) for n in self.NAMES])

    def set_flat(self, v):
        v = np.asarray(v, dtype=np.float64)
        o = 0
        for l in range(self.L):
            for n in self.NAMES:
                a = getattr(self, n)[l]
                a[...] = v[o:o + a.size].reshape(a.shape)
                o += a.size
        assert o == v.size

    def n_params(self) -> int:
        D, H = self.D, self.H
        return self.L * (H * D + H + H * H + H + 2 * D * H + 2 * D)

    def copy(self):
        f = Flow(self.D, self.H, self.L)
        f.set_flat(self.flat())
        f.mu, f.sigma = self.mu.copy(), self.sigma.copy()
        return f


def init_flow(n_dim: int, n_hidden: int, n_layers: int, key) -> Flow:
    """Seeded initial weights (W1, W2 uniform / sqrt(fan_in); W3 and biases zero)."""
    f = Flow(n_dim, n_hidden, n_layers)
    for l in range(n_layers):
        for mat, (W, fan_in) in enumerate(((f.W1[l], n_dim), (f.W2[l], n_hidden))):
            e = np.arange(W.size, dtype=np.uint64)
            blk = philox4x64_vec(np.uint64(l), np.uint64(mat), e // np.uint64(4), np.uint64(5), key)
            words = np.stack(blk, axis=-1)[np.arange(W.size), (np.arange(W.size) % 4)]
            W[...] = ((2.0 * open_unit_vec(words) - 1.0) / math.sqrt(fan_in)).reshape(W.shape)
    return f


def standardise(flow: Flow, u):
    """Set mu, sigma from the training points (population std of logit u)."""
    z = np.log(u) - np.log1p(-u)
    flow.mu = z.mean(axis=0)
    flow.sigma = z.std(axis=0)
    flow.sigma = np.where(flow.sigma > 0.0, flow.sigma, 1.0)


def _q(x, bf16):
    return round_bf16(x) if bf16 else x


def _coupling_net(flow: Flow, l: int, a, bf16: bool):
    """(s, t, cache) of layer l for masked inputs a [n, D]."""
    D = flow.D
    W1, W2, W3 = (_q(W[l], bf16) for W in (flow.W1, flow.W2, flow.W3))
    aq = _q(a, bf16)
    h1 = np.tanh(aq @ W1.T + flow.b1[l])
    h1q = _q(h1, bf16)
    h2 = np.tanh(h1q @ W2.T + flow.b2[l])
    h2q = _q(h2, bf16)
    o = h2q @ W3.T + flow.b3[l]
    keep = 1.0 - flow.mask[l]
    th = np.tanh(o[:, :D] / S_CLAMP)
    s = keep * S_CLAMP * th
    t = keep * o[:, D:]
    return s, t, (aq, h1q, h2q, th, W1, W2, W3)


def pre_map(flow: Flow, u):
    """z0 and the log-Jacobian of u -> z0 summed over dimensions."""
    u = np.asarray(u, dtype=np.float64)
    lg = np.log(u) - np.log1p(-u)
    z0 = (lg - flow.mu) / flow.sigma
    logj = -np.sum(np.log(u) + np.log1p(-u), axis=1) - np.sum(np.log(flow.sigma))
    return z0, logj


def forward(flow: Flow, u, bf16: bool = False):
    """x = F(u) and log q(u) for points u [n, D] strictly inside the unit cube."""
    z, logj = pre_map(flow, u)
    logdet = np.zeros(z.shape[0])
    for l in range(flow.L):
        m = flow.mask[l]
        s, t, _ = _coupling_net(flow, l, m * z, bf16)
        z = m * z + (1.0 - m) * (z * np.exp(s) + t)
        logdet += s.sum(axis=1)
    logn = -0.5 * np.sum(z * z, axis=1) - 0.5 * flow.D * LOG_2PI
    return z, logn + logdet + logj


def inverse(flow: Flow, x, bf16: bool = False):
    """u = F^-1(x) and log q(u) for base points x [n, D]."""
    z = np.array(x, dtype=np.float64, copy=True)
    logn = -0.5 * np.sum(z * z, axis=1) - 0.5 * flow.D * LOG_2PI
    logdet = np.zeros(z.shape[0])
    for l in reversed(range(flow.L)):
        m = flow.mask[l]
        s, t, _ = _coupling_net(flow, l, m * z, bf16)
        z = m * z + (1.0 - m) * (z - t) * np.exp(-s)
        logdet += s.sum(axis=1)
    w = flow.sigma * z + flow.mu
    u = 1.0 / (1.0 + np.exp(-w))
    # -log(u (1 - u)) = softplus(w) + softplus(-w), computed without forming 1 - u
    sp = np.logaddexp(0.0, w) + np.logaddexp(0.0, -w)
    logj = np.sum(sp, axis=1) - np.sum(np.log(flow.sigma))
    return u, logn + logdet + logj


def loss_and_grad(flow: Flow, u, bf16: bool = False):
    """Mean of -log q(u) over the points and its gradient (flat, same order as Flow.flat)."""
    n = u.shape[0]
    z, logj = pre_map(flow, u)
    zs, caches, ss = [], [], []
    logdet = np.zeros(n)
    for l in range(flow.L):
        m = flow.mask[l]
        zs.append(z)
        s, t, cache = _coupling_net(flow, l, m * z, bf16)
        caches.append(cache)
        ss.append(s)
        z = m * z + (1.0 - m) * (z * np.exp(s) + t)
        logdet += s.sum(axis=1)
    logq = -0.5 * np.sum(z * z, axis=1) - 0.5 * flow.D * LOG_2PI + logdet + logj
    loss = -logq.mean()

    grads = {}
    g = z.copy()                                   # d(-log q)/dx per point
    D = flow.D
    for l in reversed(range(flow.L)):
        m = flow.mask[l]
        keep = 1.0 - m
        zin, s = zs[l], ss[l]
        aq, h1q, h2q, th, W1, W2, W3 = caches[l]
        e = np.exp(s)
        g_s = keep * (g * zin * e - 1.0)
        g_t = keep * g
        g_o = np.concatenate([g_s * (1.0 - th * th), g_t], axis=1)
        g_oq = _q(g_o, bf16)
        dW3 = g_oq.T @ h2q
        db3 = g_o.sum(axis=0)
        g_p2 = (g_oq @ W3) * (1.0 - h2q * h2q)
        g_p2q = _q(g_p2, bf16)
        dW2 = g_p2q.T @ h1q
        db2 = g_p2.sum(axis=0)
        g_p1 = (g_p2q @ W2) * (1.0 - h1q * h1q)
        g_p1q = _q(g_p1, bf16)
        dW1 = g_p1q.T @ aq
        db1 = g_p1.sum(axis=0)
        g_a = g_p1q @ W1
        g = m * g + keep * g * e + m * g_a
        grads[l] = (dW1 / n, db1 / n, dW2 / n, db2 / n, dW3 / n, db3 / n)
    flat = np.concatenate([x.ravel() for l in range(flow.L) for x in grads[l]])
    return loss, flat


class Adam:
    """Adam state for a flat parameter vector."""

    def __init__(self, n: int, lr: float = 1e-3):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr = lr

    def step(self, params, grad):
        """Returns the updated parameters; non-finite gradient components are skipped."""
        self.t += 1
        ok = np.isfinite(grad)
        g = np.where(ok, grad, 0.0)
        m = ADAM_B1 * self.m + (1.0 - ADAM_B1) * g
        v = ADAM_B2 * self.v + (1.0 - ADAM_B2) * g * g
        self.m = np.where(ok, m, self.m)
        self.v = np.where(ok, v, self.v)
        mh = self.m / (1.0 - ADAM_B1 ** self.t)
        vh = self.v / (1.0 - ADAM_B2 ** self.t)
        return np.where(ok, params - self.lr * mh / (np.sqrt(vh) + ADAM_EPS), params)


def train(flow: Flow, u, epochs: int, adam: Adam, bf16: bool = False, restandardise: bool = True):
    """Full-batch maximum-likelihood training on points u; returns the loss before each step."""
    if restandardise:
        standardise(flow, u)
    losses = []
    p = flow.flat()
    for _ in range(epochs):
        loss, g = loss_and_grad(flow, u, bf16)
        losses.append(loss)
        p = adam.step(p, g)
        flow.set_flat(p)
    return losses


def base_normals(t: int, walkers, it: int, n_dim: int, key) -> np.ndarray:
    """Standard normal base points x [W, D] of walk step t (Box-Muller on Philox blocks
    (t, w, it, 16 + c), c = 0, 1, ...: words (0, 1) give x[4c], x[4c+1], words (2, 3) give
    x[4c+2], x[4c+3] as r cos(2 pi U2), r sin(2 pi U2), r = sqrt(-2 ln U1))."""
    w = np.asarray(walkers, dtype=np.uint64)
    out = np.empty((w.size, 4 * ((n_dim + 3) // 4)))
    for c in range((n_dim + 3) // 4):
        blk = philox4x64_vec(np.uint64(t), w, np.uint64(it), np.uint64(16 + c), key)
        for p in range(2):
            u1 = open_unit_vec(blk[2 * p])
            u2 = open_unit_vec(blk[2 * p + 1])
            r = np.sqrt(-2.0 * np.log(u1))
            out[:, 4 * c + 2 * p] = r * np.cos(2.0 * math.pi * u2)
            out[:, 4 * c + 2 * p + 1] = r * np.sin(2.0 * math.pi * u2)
    return out[:, :n_dim]


def flow_step_draws(t: int, walkers, it: int, p_flow: float, key):
    """(is a flow step, ln U of its acceptance test) of walk step t: Philox block (t, w, it, 6),
    word 0 -> flow step iff U0 < p_flow, word 1 -> U1."""
    w = np.asarray(walkers, dtype=np.uint64)
    blk = philox4x64_vec(np.uint64(t), w, np.uint64(it), np.uint64(6), key)
    return open_unit_vec(blk[0]) < p_flow, np.log(open_unit_vec(blk[1]))
