"""FP64 reference of the surrogate sensor network -- TEST INFRASTRUCTURE ONLY.

The paper has no learned component; the surrogate is an extension of its sensor
(eq. gamma): a multilayer perceptron 12 -> 64 -> 64 -> 2 maps the cell-vertex inputs of
``or_features`` (per corner: vertex-candidate mean minus cell mean and the h-scaled
vertex gradient, over ||u^e||_e + eps) to an estimate of gamma_e and a confidence.
Only tests/, the package smoke check and the benchmark's CPU leg may import this file.

Definitions (readings S1-S6, restated where the GPU path implements them):
  S1  parameters, one flat FP32 vector: W1 (64, 12), b1 (64), W2 (64, 64), b2 (64),
      W3 (2, 64), b3 (2)  -- 5,122 values, row-major, in that order;
  S3  GELU in its tanh form 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)));
  S4  outputs o = W3 a2 + b3; gamma_hat = sigmoid(o0), confidence = sigmoid(o1);
  S5  loss per sample (gamma_hat - gamma)^2 + lam * BCE(sigmoid(o1), t) with the target
      t = 1 if |gamma_hat - gamma| < tau (no gradient through t), lam = 0.1,
      tau = 0.05, averaged over the batch;
  S6  BF16 storage: the forward pass reads the inputs and the weights rounded to
      bfloat16 (round to nearest even); gradients are taken with respect to the
      rounded weights and applied to the FP32 master copy; sums in FP32 or better;
  S7  a cell with ||u^e||_e <= 1e-5 (|cell mean| + 1) holds rounding-level variation
      only: it takes gamma_e = 1 without the network and is left out of training.
Everything here is FP64 numpy; bf16 rounding is emulated where S6 places it.
"""
from __future__ import annotations

import numpy as np

NIN, NH, NOUT = 12, 64, 2
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NOUT, NH)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)
LAM, TAU = 0.1, 0.05
_C = np.sqrt(2.0 / np.pi)


NEAR_FLAT = 1e-5


def near_flat(norm, mean):
    """Reading S7: cells whose semi-norm is rounding-level next to their mean."""
    return np.asarray(norm) <= NEAR_FLAT * (np.abs(np.asarray(mean)) + 1.0)


def unpack(theta):
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shp)
        k += n
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], np.float64).reshape(-1) for name, _ in SHAPES])


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64: the float32
    value's low 16 bits are rounded away."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(_C * (x + 0.044715 * x ** 3)))


def gelu_prime(x):
    t = np.tanh(_C * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * _C * (1.0 + 3 * 0.044715 * x * x)


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def forward(theta, X, bf16: bool = True, act_bf16: bool = False):
    """Forward pass on inputs X (n, 12).  bf16: round inputs and weights (S6);
    act_bf16: also round the hidden activations fed to the next layer (the tensor-core
    inference path).  Returns the intermediate arrays."""
    P = unpack(theta)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    ra = bf16_round if act_bf16 else (lambda a: a)
    x = r(X)
    z1 = x @ r(P["W1"]).T + P["b1"]
    a1 = ra(gelu(z1))
    z2 = a1 @ r(P["W2"]).T + P["b2"]
    a2 = ra(gelu(z2))
    o = a2 @ r(P["W3"]).T + P["b3"]
    return dict(x=x, z1=z1, a1=a1, z2=z2, a2=a2, o=o, gamma_hat=sigmoid(o[:, 0]), conf=sigmoid(o[:, 1]))


def loss(theta, X, y, bf16: bool = True, target=None):
    f = forward(theta, X, bf16)
    gh = f["gamma_hat"]
    t = (np.abs(gh - y) < TAU).astype(np.float64) if target is None else target
    o1 = f["o"][:, 1]
    bce = np.logaddexp(0.0, o1) - t * o1  # -[t log s + (1-t) log(1-s)], s = sigmoid(o1)
    return float(np.mean((gh - y) ** 2 + LAM * bce)), t


def loss_and_grad(theta, X, y, bf16: bool = True):
    """Mean loss (S5) and its gradient with respect to the (rounded) parameters,
    by the chain rule written out layer by layer."""
    P = unpack(theta)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    f = forward(theta, X, bf16)
    n = X.shape[0]
    gh, o1 = f["gamma_hat"], f["o"][:, 1]
    t = (np.abs(gh - y) < TAU).astype(np.float64)
    L = float(np.mean((gh - y) ** 2 + LAM * (np.logaddexp(0.0, o1) - t * o1)))
    do = np.zeros((n, NOUT))
    do[:, 0] = 2.0 * (gh - y) * gh * (1.0 - gh) / n
    do[:, 1] = LAM * (sigmoid(o1) - t) / n
    g = {}
    g["W3"] = do.T @ f["a2"]
    g["b3"] = do.sum(0)
    dz2 = (do @ r(P["W3"])) * gelu_prime(f["z2"])
    g["W2"] = dz2.T @ f["a1"]
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ r(P["W2"])) * gelu_prime(f["z1"])
    g["W1"] = dz1.T @ f["x"]
    g["b1"] = dz1.sum(0)
    return L, pack(g)


def adam(theta, m, v, g, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba) with bias correction; step counts from 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
