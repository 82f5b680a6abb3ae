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
    # a uniform dilatation u = d (x - x_i): div u = 3 d, no vorticity
    uu = 0.04 * (cen - cen[i])
    U3 = U.copy()
    U3[1:4] = 1.2 * uu.T
    U3[4] = p / 0.4 + 0.5 * 1.2 * np.sum(uu * uu, axis=1)
    F3 = c.features(U3)
    assert abs(F3[i, 30] - hh[i] * 3 * 0.04 / a) < 1e-10
    assert abs(F3[i, 31]) < 1e-12 and abs(F3[i, 29]) < 1e-12


def test_adam_bias_correction_closed_forms():
    """Adam with bias correction (Kingma and Ba): under a constant gradient g
    the corrected moments are g and g^2 exactly, so every step moves each
    parameter by lr g / (|g| + eps); after two gradients g1, g2 they are the
    weighted means (b1 g1 + g2)/(1 + b1) and (b2 g1^2 + g2^2)/(1 + b2)."""
    rng = np.random.default_rng(3)
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    g, th0 = rng.normal(size=50), rng.normal(size=50)
    th, m, v = th0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 8):
        th, m, v = mlp.adam_step(th, g, m, v, t, lr, b1, b2, eps)
        assert np.abs(th - (th0 - t * lr * g / (np.abs(g) + eps))).max() < 1e-14
    g1, g2 = rng.normal(size=50), rng.normal(size=50)
    th, m, v = mlp.adam_step(th0, g1, np.zeros(50), np.zeros(50), 1, lr, b1, b2, eps)
    th, m, v = mlp.adam_step(th, g2, m, v, 2, lr, b1, b2, eps)
    mh, vh = (b1 * g1 + g2) / (1 + b1), (b2 * g1 ** 2 + g2 ** 2) / (1 + b2)
    ref = th0 - lr * g1 / (np.abs(g1) + eps) - lr * mh / (np.sqrt(vh) + eps)
    assert np.abs(th - ref).max() < 1e-14


def test_features_of_linear_density_and_pressure():
    """Features of linear fields at rest on jittered hexahedra (cell averages
    of a linear field are its centroid values): rho = rho0 (1 + s.(x - x_i))
    gives density jumps rho0 s.(x_m - x_i) / rho_i to each central-stencil
    member and SI/(SI + (0.1 rho_i)^2) with SI = V^(2/3) |grad rho|^2 (the
    P2 fit is exact for a linear field); a linear pressure at uniform density
    gives the pressure jumps to the first six members and the energy's
    SI/(SI + (0.1 rho a^2)^2) with SI = V^(2/3) |grad E|^2; every other
    feature is zero."""
    nodes, cells, box = I.hex_lattice(8, jitter=0.1, seed=2)
    c = O.Case(nodes, cells, box, O.Params(order=2, scheme=1, Mach=0.3))
    vol, cen, hh = c.geometry()
    i = 4 + 8 * (4 + 8 * 4)
    mem, sh, _, _ = c.stencil(i)
    assert np.all(sh == 0)  # an interior cell: its stencil does not wrap
    s = np.array([0.04, -0.03, 0.05])
    d = (cen - cen[i]) @ s
    g, rho0, p0 = 1.4, 1.3, 2.0
    # linear density, uniform pressure, at rest
    U = np.zeros((5, c.n_cells))
    U[0], U[4] = rho0 * (1 + d), p0 / (g - 1)
    F = c.features(U)[i]
    assert np.allclose(F[:18], d[mem[:18]], rtol=0, atol=1e-13)  # rho_i = rho0
    si = vol[i] ** (2 / 3) * rho0 ** 2 * (s @ s)
    assert math.isclose(F[24], si / (si + (0.1 * rho0) ** 2), rel_tol=1e-9)
    assert np.abs(F[18:24]).max() < 1e-13 and np.abs(F[25:]).max() < 1e-13
    # linear pressure, uniform density, at rest
    U = np.zeros((5, c.n_cells))
    U[0], U[4] = rho0, p0 * (1 + d) / (g - 1)
    F = c.features(U)[i]
    assert np.allclose(F[18:24], d[mem[:6]], rtol=0, atol=1e-13)
    si = vol[i] ** (2 / 3) * (p0 / (g - 1)) ** 2 * (s @ s)
    q = 0.1 * rho0 * (g * p0 / rho0)
    assert math.isclose(F[28], si / (si + q * q), rel_tol=1e-9)
    assert np.abs(F[:18]).max() < 1e-13 and np.abs(F[24:28]).max() < 1e-13 and np.abs(F[29:]).max() < 1e-13


def test_bf16_rounding_places_worked_example():
    """Where the BF16 form rounds, on a network that routes one value through:
    x = e0, W1 = e0 e0^T, b1 = 2^-10 e0 (biases stay FP64), W2 = e0 e0^T,
    w3 = e0. Then h1 = 1 + 2^-10, which rounds to 1 (half a BF16 ulp at 1 is
    2^-8) before the second layer, so z = 1 exactly against 1 + 2^-10 in
    FP64. With y = 0 the back-propagated dh2 = sigmoid(1) is not BF16: the
    bias gradient of the second layer takes it unrounded, the weight
    gradient W2[0, 0] = bf16(sigmoid(1)) h1r[0] = bf16(sigmoid(1))."""
    p = {k: np.zeros(s) for k, s in mlp.SHAPES.items()}
    p["W1"][0, 0] = p["W2"][0, 0] = p["w3"][0] = 1.0
    p["b1"][0] = 2.0 ** -10
    th = mlp.flatten(p)
    X = np.zeros((1, 32))
    X[0, 0] = 1.0
    y = np.zeros(1)
    assert mlp.forward(th, X, bf16_round=True)[0][0] == 1.0
    assert mlp.forward(th, X)[0][0] == 1.0 + 2.0 ** -10
    g = mlp.unflatten(mlp.grad(th, X, y, bf16_round=True))
    s1 = 1.0 / (1.0 + math.exp(-1.0))
    assert mlp.bf16(s1) != s1
    assert g["b2"][0] == s1 and g["b3"][0] == s1
    assert g["W2"][0, 0] == mlp.bf16(s1) and g["w3"][0] == 1.0 * s1
    assert np.count_nonzero(g["W2"]) == 1 and np.count_nonzero(g["b2"]) == 1


def test_labels_vanish_on_a_uniform_flow_and_flag_a_step():
    """The label is the largest deviation of the CWENOZ weights from the
    linear ones (lambda_1 = lambda_c / (lambda_c + nd), the rest 1 / (lambda_c
    + nd)). On a uniform flow every smoothness indicator is zero, so the
    weights equal the linear ones and every deviation is zero (to rounding); a
    density step flags the cells whose stencils straddle it and only those
    (the step is two lattice planes, the stencils reach at most three
    cells)."""
    n = 16
    nodes, cells, box = I.hex_lattice(n)
    c = O.Case(nodes, cells, box, O.Params(order=2, scheme=1))
    U = np.zeros((5, c.n_cells))
    U[0], U[1], U[4] = 1.0, 0.2, 2.5
    dev, lab = c.labels(U)
    assert dev.max() < 1e-15 and not lab.any()      # zero up to the normalisation's rounding
    _, cen, _ = c.geometry()
    ix = np.floor(cen[:, 0] / (2 * math.pi / n)).astype(int)
    U[0] = np.where(ix < n // 2, 1.0, 0.5)
    U[1] = 0.2 * U[0]
    dev, lab = c.labels(U)
    dist = np.minimum(np.abs(ix - (n // 2 - 0.5)), np.abs((ix + n // 2) % n - (n // 2 - 0.5)))  # to either step plane
    assert lab[dist < 1].all()                        # cells next to a step
    assert (dist > 3).sum() == 4 * n * n and not lab[dist > 3].any()  # beyond every stencil's reach
