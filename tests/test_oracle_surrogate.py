"""Pins of the surrogate-sensor oracle (oracle/surrogate.py, or_features): the GELU and
sigmoid identities, bfloat16 rounding, the analytic gradient against central finite
differences, closed forms of the inputs on linear and polynomial data, Adam's first
step, and that the reference training loop fits a small set."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import surrogate as S
from paper_2601_16911_gb300 import inputs as I


def test_gelu_identities_and_derivative():
    x = np.linspace(-6, 6, 241)
    assert S.gelu(np.array([0.0]))[0] == 0.0
    assert np.allclose(S.gelu(x) - S.gelu(-x), x, atol=1e-15)  # x s(x) with s(x) + s(-x) = 1
    assert abs(S.gelu(np.array([30.0]))[0] - 30.0) < 1e-12
    h = 1e-6
    fd = (S.gelu(x + h) - S.gelu(x - h)) / (2 * h)
    assert np.allclose(S.gelu_prime(x), fd, atol=1e-8)
    assert np.allclose(S.sigmoid(x), 1.0 / (1.0 + np.exp(-x)), atol=1e-15)


def test_bf16_rounding():
    exact = np.array([1.0, -2.0, 0.0, 0.5, 3.0, 1.0 + 2.0 ** -7])
    assert np.array_equal(S.bf16_round(exact), exact)
    assert S.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0               # tie -> even
    assert S.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6  # tie -> even (up)
    assert S.bf16_round(np.array([1.0 + 2.0 ** -8 + 2.0 ** -12]))[0] == 1.0 + 2.0 ** -7
    x = np.random.default_rng(0).standard_normal(10000) * 100
    r = S.bf16_round(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) + 1e-300)
    # bfloat16 has 8 significant bits: the result times 2^7 over its binade is an integer
    e = np.floor(np.log2(np.abs(r)))
    assert np.allclose(r / 2.0 ** (e - 7), np.round(r / 2.0 ** (e - 7)))


def random_problem(seed, n=37):
    rng = np.random.default_rng(seed)
    theta = np.array(I.mlp_init(seed)) + 0.05 * rng.standard_normal(S.NPARAM)
    X = rng.uniform(-2, 2, (n, 12))
    y = rng.uniform(0, 1, n)
    return theta, X, y


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    theta, X, y = random_problem(seed)
    L, g = S.loss_and_grad(theta, X, y, bf16=False)
    _, t = S.loss(theta, X, y, bf16=False)
    rng = np.random.default_rng(seed + 5)
    idx = np.concatenate([rng.choice(S.NPARAM, 60, replace=False), [S.NPARAM - 1, S.NPARAM - 2, 0, 767, 768]])
    h = 1e-6
    for k in idx:
        e = np.zeros(S.NPARAM)
        e[k] = h
        fd = (S.loss(theta + e, X, y, bf16=False, target=t)[0] - S.loss(theta - e, X, y, bf16=False, target=t)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 + 1e-5 * abs(fd), (k, fd, g[k])
    assert abs(L - S.loss(theta, X, y, bf16=False)[0]) < 1e-15


def test_zero_network_outputs_its_bias():
    parts = {name: np.zeros(shp) for name, shp in S.SHAPES}
    parts["b3"] = np.array([0.7, -1.2])
    f = S.forward(S.pack(parts), np.random.default_rng(1).standard_normal((5, 12)))
    assert np.allclose(f["gamma_hat"], 1.0 / (1.0 + math.exp(-0.7)))
    assert np.allclose(f["conf"], 1.0 / (1.0 + math.exp(1.2)))


def test_adam_first_step():
    rng = np.random.default_rng(2)
    theta = rng.standard_normal(50)
    g = rng.standard_normal(50)
    new, m, v = S.adam(theta, np.zeros(50), np.zeros(50), g, 1, 1e-3)
    # bias-corrected moments equal g and g^2 at the first step
    assert np.allclose(new, theta - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_reference_training_fits_a_small_set():
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (256, 12))
    y = S.sigmoid(2.0 * X[:, 0] - X[:, 5])  # a smooth target in (0, 1)
    theta = np.array(I.mlp_init(7))
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    L0 = S.loss(theta, X, y)[0]
    for step in range(1, 301):
        L, g = S.loss_and_grad(theta, X, y)
        theta, m, v = S.adam(theta, m, v, g, step, 3e-3)
    f = S.forward(theta, X)
    assert np.mean((f["gamma_hat"] - y) ** 2) < 0.02 * np.mean((y - y.mean()) ** 2) + 1e-4
    assert S.loss(theta, X, y)[0] < 0.5 * L0


def test_features_of_linear_data():
    """u = a x + b y: every candidate equals u, so the mean differences vanish and the
    gradient inputs are h a / (||u||_e + eps) with ||u||_e = sqrt(dx dy (a^2 + b^2))
    (eq. snorm keeps only the first derivatives, weighted by h^0)."""
    a, b = 0.7, -1.3
    d = I.mesh(2, 6, 5, degree=2, system=I.BURGERS, bc=I.TRANSMISSIVE, domain=(0.0, 1.2, -0.5, 0.5))
    P = [0.0] * 25
    P[1], P[5] = a, b
    u = O.project(d, I.IC_POLY, P)
    f, g, nrm = O.features(d, u)
    dx, dy = 1.2 / 6, 1.0 / 5
    h = math.hypot(dx, dy)
    s = math.sqrt(dx * dy * (a * a + b * b))
    assert np.allclose(nrm, s, rtol=1e-12)
    assert np.abs(f[:, 0::3]).max() < 1e-12
    assert np.allclose(f[:, 1::3], h * a / (s + d["eps"]), rtol=1e-10)
    assert np.allclose(f[:, 2::3], h * b / (s + d["eps"]), rtol=1e-10)
    assert np.allclose(g, 1.0)


def test_features_of_polynomial_and_constant_data():
    rng = np.random.default_rng(4)
    d = I.mesh(2, 5, 5, degree=3, system=I.BURGERS, bc=I.TRANSMISSIVE)
    P = [0.0] * 25
    for j in range(4):
        for i in range(4):
            P[i + 5 * j] = rng.uniform(-1, 1)
    u = O.project(d, I.IC_POLY, P)
    f, _, nrm = O.features(d, u)
    assert np.abs(f[:, 0::3]).max() < 1e-11  # every candidate is the polynomial itself
    # gradient inputs: h d_x u at each vertex over the norm
    dx = dy = 0.2
    h = math.hypot(dx, dy)
    for e in (0, 7, 24):
        i, j = e % 5, e // 5
        for c in range(4):
            x, y = (i + (c & 1)) * dx, (j + (c >> 1)) * dy
            ux = sum(P[a + 5 * bb] * a * x ** (a - 1) * y ** bb for a in range(1, 4) for bb in range(4))
            assert abs(f[e, 3 * c + 1] - h * ux / (nrm[e] + 1e-6)) < 1e-9 * (1 + abs(f[e, 3 * c + 1]))
    uc = O.project(d, I.IC_CONST, [2.5])
    fc, gc, nc = O.features(d, uc)
    # rounding-level numerators over s = eps
    # (gamma of rounding-level data is a ratio of rounding errors: not checked)
    assert np.abs(fc).max() < 1e-6 and np.abs(nc).max() < 1e-10
