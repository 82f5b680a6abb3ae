"""Pins of the CPU reference of the indicator network and of the oracle's
indicator features: finite-difference gradients, BF16 rounding, Adam on a
separable problem, and the features' closed forms on uniform and linear
fields."""
import math

import numpy as np

import oracle as O
from oracle import mlp
from paper_2609_07387_gb300 import inputs as I


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    th = mlp.init(3)
    X = rng.normal(size=(40, 32))
    y = (rng.random(40) > 0.4).astype(float)
    g = mlp.grad(th, X, y, 2.0, 0.5)
    for k in rng.choice(mlp.N_PARAMS, 25, replace=False):
        e = np.zeros(mlp.N_PARAMS)
        e[k] = 1e-6
        fd = (mlp.loss(th + e, X, y, 2.0, 0.5) - mlp.loss(th - e, X, y, 2.0, 0.5)) / 2e-6
        assert abs(fd - g[k]) <= 1e-7 + 1e-5 * abs(g[k]), (k, fd, g[k])


def test_bf16_rounding_is_nearest_even():
    v = np.array([1.0, 1 + 2 ** -8, 1 + 1.5 * 2 ** -8, 1 + 3 * 2 ** -8, -2.75, 3.0e-3])
    r = mlp.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0            # tie -> even
    assert r[2] == 1 + 2 ** -7 and r[3] == 1 + 2 ** -6  # above tie -> up; tie at odd -> even (up)
    assert r[4] == -2.75
    assert abs(r[5] - 3.0e-3) <= 3.0e-3 * 2 ** -8


def test_adam_learns_a_separable_rule():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(512, 32))
    y = ((X[:, 0] + 0.5 * X[:, 3]) > 0).astype(float)
    th = mlp.init(0)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    l0 = mlp.loss(th, X, y)
    for t in range(1, 301):
        th, m, v = mlp.adam_step(th, mlp.grad(th, X, y), m, v, t, lr=3e-3)
    z, _ = mlp.forward(th, X)
    assert mlp.loss(th, X, y) < 0.2 * l0
    assert np.mean((z > 0) == (y > 0.5)) > 0.97


def test_features_closed_forms():
    nodes, cells, box = I.hex_lattice(8, jitter=0.1, seed=2)
    c = O.Case(nodes, cells, box, O.Params(order=2, scheme=1, Mach=0.3))
    U = np.zeros((5, len(cells)))
    u = np.array([0.3, -0.2, 0.1])
    U[0] = 1.2
    U[1:4] = (1.2 * u)[:, None]
    p = 2.0
    U[4] = p / 0.4 + 0.5 * 1.2 * u @ u
    F = c.features(U)
    a = math.sqrt(1.4 * p / 1.2)
    assert np.abs(F[:, :29]).max() < 1e-12                 # no jumps, zero smoothness indicators
    assert np.allclose(F[:, 29], np.linalg.norm(u) / a, rtol=1e-13)
    assert np.abs(F[:, 30:]).max() < 1e-12                 # uniform velocity: no divergence, no vorticity
    # a solid-body rotation u = w x r (cell averages by quadrature are exact for linear fields):
    # |curl u| = 2|w|, div u = 0
    vol, cen, hh = c.geometry()
    w = np.array([0.0, 0.0, 0.05])
    i = 4 + 8 * (4 + 8 * 4)  # an interior cell: its stencil does not wrap
    uu = np.cross(w, cen - cen[i])
    U2 = U.copy()
    U2[1:4] = 1.2 * uu.T
    U2[4] = p / 0.4 + 0.5 * 1.2 * np.sum(uu * uu, axis=1)
    F2 = c.features(U2)
    a_i = a  # kinetic energy of the rotation is zero at the centre cell
    assert abs(F2[i, 31] - hh[i] * 2 * 0.05 / a_i) < 1e-10
    assert abs(F2[i, 30]) < 1e-12
