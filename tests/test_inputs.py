"""The seeded synthetic input recipe (CPU): lattice numbering and VTK order,
the jitter's amplitude, seed and interior-only rule, the 6-tet split's
orientation and volume, the Taylor-Green closed form (uniform temperature),
the perturbation's rms, and reproducibility of every seeded generator."""
import math

import numpy as np
import pytest

from paper_2609_07387_gb300 import inputs as I


def _tet_volumes(nodes, tets):
    p = nodes[tets]
    return np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0]) / 6.0


def test_lattice_numbering_and_vtk_order():
    nodes, cells, box = I.hex_lattice((3, 4, 5), length=(3.0, 4.0, 5.0))
    assert nodes.shape == (4 * 5 * 6, 3) and cells.shape == (60, 8)
    assert np.allclose(box, [3.0, 4.0, 5.0])
    # node id = i + 4 (j + 5 k) at (i, j, k) (unit spacing here)
    i, j, k = 2, 3, 4
    assert np.allclose(nodes[i + 4 * (j + 5 * k)], [i, j, k])
    # cell (1, 2, 3): VTK corner offsets
    c = cells[1 + 3 * (2 + 4 * 3)]
    off = nodes[c] - nodes[c[0]]
    assert np.allclose(off, [[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])


def test_jitter_amplitude_seed_and_interior_rule():
    n, a = 8, 0.1
    h = 2 * math.pi / n
    base, _, _ = I.hex_lattice(n)
    j1, _, _ = I.hex_lattice(n, jitter=a, seed=1)
    j1b, _, _ = I.hex_lattice(n, jitter=a, seed=1)
    j2, _, _ = I.hex_lattice(n, jitter=a, seed=2)
    assert np.array_equal(j1, j1b) and not np.array_equal(j1, j2)
    d = j1 - base
    assert np.abs(d).max() <= a * h
    assert np.abs(d).max() > 0.9 * a * h  # the uniform draw reaches near the bound
    idx = np.round(base / h).astype(int)
    boundary = np.any((idx == 0) | (idx == n), axis=1)
    assert np.all(d[boundary] == 0.0) and np.all(np.abs(d[~boundary]).max(axis=1) > 0)
    # the documented draw: one uniform(-1, 1) array (n_nodes, 3) in node order, scaled by a h
    ref = np.random.default_rng(1).uniform(-1.0, 1.0, size=base.shape) * (a * h)
    assert np.allclose(d[~boundary], ref[~boundary], rtol=0, atol=1e-15)


def test_tets_positive_and_fill_the_box():
    nodes, cells, _ = I.hex_lattice(4, jitter=0.1, seed=3)
    tets = I.split_tets(cells)
    assert tets.shape == (6 * 64, 4)
    vol = _tet_volumes(nodes, tets)
    assert np.all(vol > 0)
    assert math.isclose(vol.sum(), (2 * math.pi) ** 3, rel_tol=1e-12)


def test_prisms_oriented_and_fill_the_box():
    """Each prism of the split: base triangle counter-clockwise seen from
    the top (its normal points at the top triangle), top node k+3 above base
    node k; the prisms of a lattice hexahedron fill it, all along the same
    diagonal."""
    nodes, cells, _ = I.hex_lattice(4)
    pr = I.split_prisms(cells)
    assert pr.shape == (2 * 64, 6)
    p = nodes[pr]
    nb = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    up = p[:, 3:].mean(axis=1) - p[:, :3].mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", nb, up) > 0)
    assert np.allclose(p[:, 3:, :2], p[:, :3, :2]) and np.all(p[:, 3:, 2] > p[:, :3, 2])
    h = 2 * math.pi / 4
    area = 0.5 * np.linalg.norm(nb, axis=1)
    assert np.allclose(area, 0.5 * h * h) and math.isclose((area * h).sum(), (2 * math.pi) ** 3, rel_tol=1e-12)
    assert np.array_equal(pr[0::2, [0, 2]], pr[1::2, [0, 1]])  # both share the diagonal 0-2


def test_pyramids_oriented_and_fill_the_box():
    """Each hexahedron's six pyramids: one per face, the apex (an appended
    node) at the hexahedron's vertex mean, the base counter-clockwise seen
    from the apex; on the lattice each has volume h^3/6 and they fill it."""
    nodes, cells, _ = I.hex_lattice(3)
    n2, pyr = I.split_pyramids(nodes, cells)
    assert n2.shape == (nodes.shape[0] + 27, 3) and pyr.shape == (6 * 27, 5)
    assert np.array_equal(pyr[:, 4], np.repeat(nodes.shape[0] + np.arange(27), 6))
    assert np.allclose(n2[nodes.shape[0]:], nodes[cells].mean(axis=1))
    p = n2[pyr]
    nb = np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 1])          # base normal
    toward = p[:, 4] - p[:, :4].mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", nb, toward) > 0)
    h = 2 * math.pi / 3
    vol = 0.5 * np.linalg.norm(nb, axis=1) * np.abs(np.einsum("ij,ij->i", nb, toward)) / np.linalg.norm(nb, axis=1) / 3
    assert np.allclose(vol, h ** 3 / 6) and math.isclose(vol.sum(), (2 * math.pi) ** 3, rel_tol=1e-12)


@pytest.mark.parametrize("mach", [0.1, 1.25])
def test_tgv_closed_form_and_uniform_temperature(mach):
    nodes, cells, _ = I.hex_lattice(6)
    x = I.cell_vertex_means(nodes, cells)
    U = I.tgv_state(nodes, cells, mach)
    rho, u, v, w = U[0], U[1] / U[0], U[2] / U[0], U[3] / U[0]
    p = 0.4 * (U[4] - 0.5 * rho * (u * u + v * v + w * w))
    assert np.allclose(u, np.sin(x[:, 0]) * np.cos(x[:, 1]) * np.cos(x[:, 2]), atol=1e-13)
    assert np.allclose(v, -np.cos(x[:, 0]) * np.sin(x[:, 1]) * np.cos(x[:, 2]), atol=1e-13)
    assert np.all(w == 0.0)
    p_ref = 1.0 / (1.4 * mach * mach)
    assert np.allclose(p, p_ref + (np.cos(2 * x[:, 2]) + 2) * (np.cos(2 * x[:, 0]) + np.cos(2 * x[:, 1])) / 16,
                       rtol=1e-12)
    assert np.allclose(p / rho, 1.0 / (1.4 * mach * mach), rtol=1e-13)  # T = p / (rho R) = 1


def test_perturbation_rms_and_seeds():
    nodes, cells, _ = I.hex_lattice(10, jitter=0.1, seed=3)
    x = I.cell_vertex_means(nodes, cells)
    d = I.random_phase_velocity(x, 0.05, seed=4)
    assert math.isclose(math.sqrt(np.mean(np.sum(d * d, axis=1))), 0.05, rel_tol=1e-12)
    assert np.array_equal(d, I.random_phase_velocity(x, 0.05, seed=4))
    assert not np.array_equal(d, I.random_phase_velocity(x, 0.05, seed=5))
    U0 = I.tgv_state(nodes, cells, 1.25)
    U = I.tgv_perturbed_state(nodes, cells, 1.25, 0.05, seed=4)
    assert np.array_equal(U[0], U0[0])  # density and pressure untouched
    assert np.allclose(U[1:4] / U[0] - U0[1:4] / U0[0], d.T, atol=1e-13)


def test_noisy_state_bounds_and_seed():
    nodes, cells, _ = I.hex_lattice(6)
    U0 = I.tgv_state(nodes, cells, 0.1)
    a = I.noisy_state(nodes, cells, 0.1, 0.05, seed=3)
    assert np.array_equal(a, I.noisy_state(nodes, cells, 0.1, 0.05, seed=3))
    r = a[0] / U0[0] - 1.0
    assert np.abs(r).max() <= 0.05 and np.abs(r).max() > 0.04
    assert np.all(a[0] > 0)
