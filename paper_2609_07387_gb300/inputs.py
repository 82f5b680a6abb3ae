"""Seeded synthetic inputs for the Taylor-Green workloads.

This module builds the *inputs* that both the CUDA library and the CPU oracle
consume: mesh node coordinates and cell connectivity (uniform or jittered
hexahedral lattices of the periodic box [0, 2*pi]^3, optionally split into
tetrahedra) and point-sampled flow states.  It holds none of the
finite-volume arithmetic (no geometry, quadrature, reconstruction or flux):
callers pass its arrays to ``ucns_mesh_create`` / the oracle, which do all of
that themselves.

Conventions
-----------
* Nodes of an n^3 lattice: (n+1)^3 points, id = i + (n+1)*(j + (n+1)*k) with
  i the x index (fastest), k the z index (slowest).  Coordinates are
  ``L*i/n``.  Nodes on the box faces are repeated on both sides; periodicity
  is recovered by the consumer from the box lengths.
* Hex cells: id = i + n*(j + n*k), nodes in VTK hexahedron order
  (0:(0,0,0) 1:(1,0,0) 2:(1,1,0) 3:(0,1,0) 4:(0,0,1) 5:(1,0,1) 6:(1,1,1)
  7:(0,1,1) in cell-local lattice offsets).
* Jitter: every node with 0<i,j,k<n moves by independent U(-a*h, a*h) per
  coordinate: ``numpy.random.default_rng(seed).uniform(-1, 1)`` drawn as one
  array of shape (n_nodes, 3) in node-id order (x, y, z per node), scaled by
  a*h per axis; boundary
  nodes do not move, so periodic images stay exact translations.
* Tetrahedra: each hexahedron is split into the 6 Kuhn (Freudenthal) tets
  around its 0-6 diagonal, conforming across the lattice, each listed with
  positive orientation ((p1-p0) x (p2-p0) . (p3-p0) > 0).
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi

# Kuhn split of the unit cube along the 0-6 diagonal, VTK local node ids,
# odd permutations re-ordered so every tet has positive volume.
_KUHN_TETS = np.array(
    [
        [0, 1, 2, 6],
        [0, 5, 1, 6],
        [0, 2, 3, 6],
        [0, 3, 7, 6],
        [0, 4, 5, 6],
        [0, 7, 4, 6],
    ],
    dtype=np.int64,
)

_HEX_OFFSETS = np.array(
    [[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]],
    dtype=np.int64,
)


def hex_lattice(n, length=TWO_PI, jitter: float = 0.0, seed: int | None = None):
    """Return (nodes [(nx+1)(ny+1)(nz+1), 3] f64, cells [nx*ny*nz, 8] i64, box [3] f64).

    ``n`` is an int (cube) or a triple (nx, ny, nz); ``length`` a float or a
    triple (Lx, Ly, Lz).  Spacing h_d = L_d / n_d; the jitter amplitude is
    ``jitter * h_d`` per coordinate.
    """
    nx, ny, nz = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
    Lx, Ly, Lz = (length,) * 3 if np.isscalar(length) else tuple(float(v) for v in length)
    if min(nx, ny, nz) < 1:
        raise ValueError("lattice needs at least one cell per direction")
    mx, my, mz = nx + 1, ny + 1, nz + 1
    kk, jj, ii = np.meshgrid(np.arange(mz), np.arange(my), np.arange(mx), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    nodes = np.stack(
        [Lx * ii.astype(np.float64) / nx, Ly * jj.astype(np.float64) / ny, Lz * kk.astype(np.float64) / nz],
        axis=1,
    )
    if jitter:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-1.0, 1.0, size=(mx * my * mz, 3)) * (jitter * np.array([Lx / nx, Ly / ny, Lz / nz]))
        interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny) & (kk > 0) & (kk < nz)
        nodes[interior] += d[interior]
    ck, cj, ci = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)
    cells = np.empty((nx * ny * nz, 8), dtype=np.int64)
    for a in range(8):
        o = base + _HEX_OFFSETS[a]
        cells[:, a] = o[:, 0] + mx * (o[:, 1] + my * o[:, 2])
    box = np.array([Lx, Ly, Lz], dtype=np.float64)
    return nodes, cells, box


def split_tets(cells: np.ndarray) -> np.ndarray:
    """Split VTK hexahedra [n, 8] into 6 Kuhn tets each -> [6n, 4] (hex-major)."""
    cells = np.asarray(cells, dtype=np.int64)
    return cells[:, _KUHN_TETS].reshape(-1, 4)


# the two triangular prisms of a VTK hexahedron, split through the base and
# top diagonals 0-2 and 4-6: base triangle counter-clockwise seen from the top,
# top node k+3 above base node k
_WEDGES = np.array([[0, 1, 2, 4, 5, 6], [0, 2, 3, 4, 6, 7]], dtype=np.int64)


def split_prisms(cells: np.ndarray) -> np.ndarray:
    """Split VTK hexahedra [n, 8] into 2 triangular prisms each -> [2n, 6]
    (hex-major), every hexahedron along the same diagonal so that the
    triangles of periodic neighbours match."""
    cells = np.asarray(cells, dtype=np.int64)
    return cells[:, _WEDGES].reshape(-1, 6)


# the six faces of a VTK hexahedron, each ordered counter-clockwise seen from
# the hexahedron's inside (the pyramid bases below)
_HEX_FACES_INWARD = np.array([[0, 3, 7, 4], [1, 5, 6, 2], [0, 4, 5, 1], [3, 2, 6, 7], [0, 1, 2, 3],
                              [4, 7, 6, 5]], dtype=np.int64)


def split_pyramids(nodes: np.ndarray, cells: np.ndarray):
    """Split VTK hexahedra [n, 8] into 6 pyramids each, one per face, with
    the apex at the hexahedron's vertex mean (a node appended per
    hexahedron): -> (nodes [n_nodes + n, 3], pyramids [6n, 5], hex-major),
    base counter-clockwise seen from the apex, apex last."""
    nodes = np.asarray(nodes, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    apex = nodes.shape[0] + np.arange(cells.shape[0], dtype=np.int64)
    out = np.concatenate([nodes, nodes[cells].mean(axis=1)])
    base = cells[:, _HEX_FACES_INWARD]                    # [n, 6, 4]
    pyr = np.concatenate([base, np.broadcast_to(apex[:, None, None], (cells.shape[0], 6, 1))], axis=2)
    return out, pyr.reshape(-1, 5)


def cell_vertex_means(nodes: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """Mean of each cell's node coordinates [n_cells, 3] (a sampling point only)."""
    return np.asarray(nodes)[np.asarray(cells)].mean(axis=1)


def tgv_primitive(x: np.ndarray, mach: float, gamma: float = 1.4):
    """Taylor-Green vortex initial field at points x [n, 3] -> (rho, u, v, w, p).

    Velocity and pressure as given for the compressible TGV; uniform
    temperature T0 = 1 with R = 1/(gamma M^2), so rho = gamma M^2 p.
    """
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p = 1.0 / (gamma * mach * mach) + (np.cos(2 * Z) + 2.0) * (np.cos(2 * X) + np.cos(2 * Y)) / 16.0
    rho = gamma * mach * mach * p
    return rho, u, v, w, p


def primitive_to_conserved(rho, u, v, w, p, gamma: float = 1.4) -> np.ndarray:
    """Stack conserved variables as SoA [5, n] (rho, rho u, rho v, rho w, rho E)."""
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E]).astype(np.float64)


def tgv_state(nodes, cells, mach: float, gamma: float = 1.4) -> np.ndarray:
    """TGV conserved state sampled at each cell's vertex mean, SoA [5, n_cells]."""
    x = cell_vertex_means(nodes, cells)
    return primitive_to_conserved(*tgv_primitive(x, mach, gamma), gamma=gamma)


def random_phase_velocity(x: np.ndarray, amplitude: float, seed: int, n_modes: int = 8):
    """Seeded divergence-free-agnostic random-phase velocity perturbation.

    Sum of ``n_modes`` Fourier modes per component, integer wave vectors with
    |k|_inf <= 3, uniform random phases, scaled so the perturbation's rms over
    the sample points equals ``amplitude``.  Returns [n, 3].
    """
    rng = np.random.default_rng(seed)
    out = np.zeros((x.shape[0], 3))
    for c in range(3):
        ks = rng.integers(-3, 4, size=(n_modes, 3))
        ks[np.all(ks == 0, axis=1)] = [1, 0, 0]
        ph = rng.uniform(0.0, TWO_PI, size=n_modes)
        for kv, f in zip(ks, ph):
            out[:, c] += np.sin(x @ kv.astype(np.float64) + f)
    rms = math.sqrt(float(np.mean(np.sum(out * out, axis=1))))
    return out * (amplitude / rms)


def tgv_perturbed_state(nodes, cells, mach: float, amplitude: float, seed: int, gamma: float = 1.4):
    """TGV at Mach ``mach`` plus a seeded random-phase velocity perturbation."""
    x = cell_vertex_means(nodes, cells)
    rho, u, v, w, p = tgv_primitive(x, mach, gamma)
    d = random_phase_velocity(x, amplitude, seed)
    return primitive_to_conserved(rho, u + d[:, 0], v + d[:, 1], w + d[:, 2], p, gamma=gamma)


def noisy_state(nodes, cells, mach: float, noise: float, seed: int, gamma: float = 1.4) -> np.ndarray:
    """TGV state with seeded multiplicative cell noise (rough data that drives
    the nonlinear weights away from the linear ones)."""
    U = tgv_state(nodes, cells, mach, gamma)
    rng = np.random.default_rng(seed)
    rho, m, E = U[0], U[1:4], U[4]
    u = m / rho
    p = (gamma - 1.0) * (E - 0.5 * rho * np.sum(u * u, axis=0))
    rho = rho * (1.0 + noise * rng.uniform(-1, 1, size=rho.shape))
    p = p * (1.0 + noise * rng.uniform(-1, 1, size=p.shape))
    u = u + noise * rng.uniform(-1, 1, size=u.shape)
    return primitive_to_conserved(rho, u[0], u[1], u[2], p, gamma=gamma)
