"""FP64 oracle of the learned surrogate used for delayed acceptance.

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU baseline,
never by the library.  The paper has no surrogate; this part follows the
problem statement of the delayed-acceptance configuration:

* features: 16 Gaussian radial features of a position r against its neighbours
  j within rc,  G_k = sum_j w_j exp(-eta (r_j - c_k)^2) f_c(r_j),
  centres c_k = 0.8 + 1.7 k / 15 (k = 0..15), eta = 1 / (2 (1.7/15)^2),
  cutoff f_c(r) = (cos(pi r / rc) + 1) / 2, weight w_j = eps between the mobile
  species and the neighbour's species (element-weighted radial functions);
* network: 16 -> 64 -> 64 -> 1, SiLU hidden activations, scalar output e~(r),
  the predicted interaction energy of a particle at r; the sampler's copy
  rounds its weights and every layer's inputs to bfloat16;
* loss: mean squared error against the exact interaction energy e(r),
  targets clipped from above at a fixed value;
* optimiser: Adam.

Parameter vector (5313 values): W1 [16][64], b1 [64], W2 [64][64], b2 [64],
W3 [64], b3 [1], row-major.
"""
from __future__ import annotations

import math

import numpy as np

N_FEAT, N_HID = 16, 64
N_PARAMS = N_FEAT * N_HID + N_HID + N_HID * N_HID + N_HID + N_HID + 1
CENTRES = 0.8 + 1.7 * np.arange(N_FEAT) / 15.0
ETA = 1.0 / (2.0 * (1.7 / 15.0) ** 2)


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    o = 0
    W1 = theta[o:o + N_FEAT * N_HID].reshape(N_FEAT, N_HID); o += N_FEAT * N_HID
    b1 = theta[o:o + N_HID]; o += N_HID
    W2 = theta[o:o + N_HID * N_HID].reshape(N_HID, N_HID); o += N_HID * N_HID
    b2 = theta[o:o + N_HID]; o += N_HID
    W3 = theta[o:o + N_HID]; o += N_HID
    b3 = theta[o:o + 1]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, W3, np.ravel(b3)])


def init_params(seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded initial parameters (fan-in scaled normal weights, zero biases)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(size=(N_FEAT, N_HID)) * scale / math.sqrt(N_FEAT)
    W2 = rng.normal(size=(N_HID, N_HID)) * scale / math.sqrt(N_HID)
    W3 = rng.normal(size=N_HID) * scale / math.sqrt(N_HID)
    return pack(W1, np.zeros(N_HID), W2, np.zeros(N_HID), W3, np.zeros(1))


def to_bf16(theta) -> np.ndarray:
    """Round each value to binary32, then to the nearest bfloat16 value (ties to even)."""
    f = np.asarray(theta, np.float32).view(np.uint32).astype(np.uint64)
    rounded = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def weight_mask() -> np.ndarray:
    """True for the entries of theta that are weights (W1, W2, W3), False for
    the biases."""
    m = np.zeros(N_PARAMS, bool)
    W1, b1, W2, b2, W3, b3 = unpack(np.arange(N_PARAMS, dtype=np.float64))
    for w in (W1, W2, W3):
        m[np.asarray(w, np.int64).ravel()] = True
    return m


def inference_params(theta) -> np.ndarray:
    """The parameters the sampler's network uses: weights rounded to bfloat16,
    biases rounded to binary32."""
    theta = np.asarray(theta, np.float64)
    out = np.asarray(theta, np.float32).astype(np.float64)
    m = weight_mask()
    out[m] = to_bf16(theta[m])
    return out


def cutoff(r, rc):
    return np.where(r < rc, 0.5 * (np.cos(np.pi * r / rc) + 1.0), 0.0)


def features(r, w, rc):
    """Features of one position from its neighbour distances r [n] and
    weights w [n] (neighbours at r >= rc contribute nothing)."""
    r = np.asarray(r, np.float64)
    w = np.asarray(w, np.float64)
    fc = cutoff(r, rc) * w
    g = np.exp(-ETA * (r[:, None] - CENTRES[None, :]) ** 2)
    return (g * fc[:, None]).sum(axis=0)


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def forward(theta, X, bf16_inputs: bool = False):
    """Predicted energies for feature rows X [n, 16]; returns (e [n], cache).

    bf16_inputs: round every layer's inputs (the features, then the hidden
    activations) to bfloat16, as the sampler's network takes them (training
    keeps them in full precision)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.atleast_2d(np.asarray(X, np.float64))
    r = to_bf16 if bf16_inputs else (lambda a: a)
    z1 = r(X) @ W1 + b1
    h1 = r(silu(z1))
    z2 = h1 @ W2 + b2
    h2 = r(silu(z2))
    e = h2 @ W3 + b3[0]
    return e, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, y):
    """Mean squared error and its gradient with respect to theta (analytic
    backward pass through the two SiLU layers)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    e, (X, z1, h1, z2, h2) = forward(theta, X)
    n = X.shape[0]
    r = e - np.asarray(y, np.float64)
    loss = float(np.mean(r * r))
    g = 2.0 * r / n                       # d loss / d e
    dW3 = h2.T @ g
    db3 = np.array([g.sum()])
    dz2 = np.outer(g, W3) * dsilu(z2)
    dW2 = h1.T @ dz2
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * dsilu(z1)
    dW1 = X.T @ dz1
    db1 = dz1.sum(axis=0)
    return loss, pack(dW1, db1, dW2, db2, dW3, db3)


def loss_and_grad_bf16(theta, X, y):
    """The mean squared error and its gradient as mixed-precision training
    defines them: every matrix product takes bfloat16 operands (nearest, ties
    to even) -- bf(X) bf(W1), bf(h1) bf(W2), bf(h1)^T bf(dz2), bf(dz2)
    bf(W2)^T, bf(X)^T bf(dz1) -- and everything else (the output layer, the
    biases, SiLU and its derivative, the products with them, the sums over
    rows) is taken without rounding (FP64 here).  Products of bfloat16 values
    and their sums are exact in FP64 to far below the accumulation error of
    any FP32 implementation."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    bf = to_bf16
    X = np.atleast_2d(np.asarray(X, np.float64))
    n = X.shape[0]
    xb, W1b, W2b = bf(X), bf(W1), bf(W2)
    z1 = xb @ W1b + b1
    h1 = silu(z1)
    h1b = bf(h1)
    z2 = h1b @ W2b + b2
    h2 = silu(z2)
    e = h2 @ W3 + b3[0]
    r = e - np.asarray(y, np.float64)
    loss = float(np.mean(r * r))
    g = 2.0 * r / n
    dW3 = h2.T @ g
    db3 = np.array([g.sum()])
    dz2 = np.outer(g, W3) * dsilu(z2)
    dz2b = bf(dz2)
    dW2 = h1b.T @ dz2b
    db2 = dz2.sum(axis=0)
    dz1 = (dz2b @ W2b.T) * dsilu(z1)
    dW1 = xb.T @ bf(dz1)
    db1 = dz1.sum(axis=0)
    return loss, pack(dW1, db1, dW2, db2, dW3, db3)


def batch_rows(step, batch, count, key):
    """Row indices of Adam step number `step` (from 1) of a mini-batch of
    `batch` rows drawn uniformly from `count` rows: row i is (P0 count) >> 32
    with P = Philox4x32-10((i, step, 0, 6), key)."""
    from . import oracle as O
    out = np.zeros(batch, np.int64)
    for i in range(batch):
        p0 = O.philox4x32_10((i, step, 0, 6), key)[0]
        out[i] = (int(p0) * int(count)) >> 32
    return out


class Adam:
    """Adam (Kingma & Ba) with bias correction."""

    def __init__(self, n, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, theta, grad):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)
