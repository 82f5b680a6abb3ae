"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: counts
printed in the paper's benchmark matrix, closed forms, exact invariants
(free-stream preservation, discrete conservation, closed-surface sums),
k-exactness of the least-squares reconstruction (Eqs. 3-4), library
least-squares on the same systems, textbook properties of the HLLC and
Newtonian viscous fluxes, the jump-penalised face gradient of Eq. 7 on an
odd-even mode (exact) and a shear wave (convergent), the SSP-RK3 stability
polynomial, the design order of accuracy on exact Euler solutions, the
Taylor-Green initial diagnostics and pressure (pressure Poisson equation),
and the dissipation diagnostics of plane waves.  None of these touch the GPU.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2609_07387_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            rows[k] = [float(x) for x in v]
    return rows


@pytest.fixture(scope="module")
def jhex8_p2():
    nodes, cells, box = I.hex_lattice(8, jitter=0.1, seed=1)
    return nodes, cells, box, O.Case(nodes, cells, box, O.Params(order=2, scheme=1))


@pytest.fixture(scope="module")
def jtet_p2():
    nodes, cells, box = I.hex_lattice(5, jitter=0.1, seed=2)
    tets = I.split_tets(cells)
    return nodes, tets, box, O.Case(nodes, tets, box, O.Params(order=2, scheme=1))


@pytest.fixture(scope="module")
def jpyr_p2():
    nodes, cells, box = I.hex_lattice(4, jitter=0.1, seed=6)
    nodes, pyr = I.split_pyramids(nodes, cells)
    return nodes, pyr, box, O.Case(nodes, pyr, box, O.Params(order=2, scheme=1))


@pytest.fixture(scope="module")
def jprism_p2():
    nodes, cells, box = I.hex_lattice(5, jitter=0.1, seed=5)
    prisms = I.split_prisms(cells)
    return nodes, prisms, box, O.Case(nodes, prisms, box, O.Params(order=2, scheme=1))


# --------------------------------------------------------------- counts ---
def test_counts_match_benchmark_matrix(jhex8_p2):
    """Table 4 (TGV-P2): 3 faces per hex, 54M/2M = 27 reconstructed DoF per
    cell and variable (9 central + 6 linear directional x 3), 24M/6M = 4
    quadrature points per face."""
    g = _golden("benchmark_matrix.txt")["TGV-P2"]
    cells, faces, dof, qps = g
    c = jhex8_p2[3]
    assert c.n_faces == round(faces / cells) * c.n_cells
    assert c.K + c.nd * 3 == round(dof / cells)
    assert c.nq == round(qps / faces)
    # Eq. 3: K(r,d) = (r+1)(r+2)(r+3)/6 = 10 terms incl. the mean -> 9 modes
    assert c.K == math.comb(2 + 3, 3) - 1
    assert c.Mc == 2 * c.K and c.nd == 6 and c.Md == 6


def test_counts_p1_and_tets(jtet_p2):
    nodes, cells, box = I.hex_lattice(4)
    c1 = O.Case(nodes, cells, box, O.Params(order=1, scheme=0))
    assert (c1.K, c1.Mc, c1.nd, c1.nq, c1.n_faces) == (3, 6, 0, 1, 3 * 64)
    ct = jtet_p2[3]
    assert ct.n_cells == 6 * 125 and ct.n_faces == 2 * ct.n_cells
    assert (ct.K, ct.Mc, ct.nd, ct.Md, ct.nq) == (9, 18, 4, 6, 4)


def test_counts_pyramids(jpyr_p2):
    """Six pyramids per hexahedron (apex at its vertex mean, one per face),
    five faces each (the base quad, four triangles), every face shared:
    N = 6n^3, F = 15n^3, of which 3n^3 quads (the hexahedra's faces)."""
    nodes, cells, box, c = jpyr_p2
    assert c.n_cells == 6 * 64 and c.n_faces == 15 * 64
    assert (c.nfc, c.K, c.Mc, c.nd, c.Md, c.nq) == (5, 9, 18, 5, 6, 4)
    n = np.array([c.face_quad(f)[1].sum(axis=0) for f in range(c.n_faces)])
    axis = np.abs(n).max(axis=1) / np.linalg.norm(n, axis=1)
    assert (axis > 0.95).sum() == 3 * 64 and (axis < 0.8).sum() == 12 * 64


def test_degenerate_pyramid_stencils_are_rejected():
    """On the unjittered lattice every member of a pyramid's P2 central
    stencil has the same mean of one quadratic mode as the cell itself (a
    zero column of the least-squares matrix): the rank test, taken against
    the matrix's largest column, rejects it instead of returning a
    polynomial with 1e13 coefficients; P1 and the jittered lattice pass."""
    nodes, cells, box = I.hex_lattice(4)
    nodes, pyr = I.split_pyramids(nodes, cells)
    U = np.zeros((5, pyr.shape[0]))
    U[0], U[4] = 1.0, 2.5
    with pytest.raises(O.OracleError, match="rank-deficient"):
        O.Case(nodes, pyr, box, O.Params(order=2, scheme=0)).residual(U)
    assert np.abs(O.Case(nodes, pyr, box, O.Params(order=1, scheme=0)).residual(U)).max() < 1e-13


def test_counts_prisms(jprism_p2):
    """Two prisms per hexahedron, five faces each (two triangles, three
    quads), every face shared: N = 2n^3, F = 5n^3, of which 2n^3 triangles;
    five directional candidates; 4 points on either face shape at P2."""
    nodes, cells, box, c = jprism_p2
    assert c.n_cells == 2 * 125 and c.n_faces == 5 * 125
    assert (c.nfc, c.K, c.Mc, c.nd, c.Md, c.nq) == (5, 9, 18, 5, 6, 4)
    # the triangles are the base and top faces, whose normals are near z
    n = np.array([c.face_quad(f)[1].sum(axis=0) for f in range(c.n_faces)])
    nz = np.abs(n[:, 2]) / np.linalg.norm(n, axis=1)
    assert (nz > 0.9).sum() == 2 * 125 and (nz < 0.3).sum() == 3 * 125


# ------------------------------------------------------------- geometry ---
@pytest.mark.parametrize("kind", ["hex", "tet", "prism", "pyramid"])
def test_geometry_closed_surfaces_and_volume(kind, jhex8_p2, jtet_p2, jprism_p2, jpyr_p2):
    nodes, cells, box, c = {"hex": jhex8_p2, "tet": jtet_p2, "prism": jprism_p2, "pyramid": jpyr_p2}[kind]
    vol, cen, hh = c.geometry()
    assert abs(vol.sum() - (2 * math.pi) ** 3) <= 1e-12 * (2 * math.pi) ** 3
    assert np.all(vol > 0)
    s = c.surface_sums()
    assert np.abs(s).max() <= 1e-14 * hh.max() ** 2 * 10
    # each face's area vectors sum to the owner-outward area vector; the
    # periodic neighbour image is adjacent to the owner
    fo, fn, sh = c.faces()
    d = cen[fn] + sh * box - cen[fo]
    assert np.linalg.norm(d, axis=1).max() < 2.0 * hh.max()


@pytest.mark.parametrize("kind", ["hex", "tet", "prism", "pyramid"])
def test_face_area_vectors_point_from_owner_to_neighbour(kind, jhex8_p2, jtet_p2, jprism_p2, jpyr_p2):
    """Eq. 2 sums sigma G_f with G_f taken through dS oriented from the owner
    to the neighbour: every face's total area vector has a positive
    component along the owner -> neighbour (periodic image) centroid offset."""
    nodes, cells, box, c = {"hex": jhex8_p2, "tet": jtet_p2, "prism": jprism_p2, "pyramid": jpyr_p2}[kind]
    fo, fn, sh = c.faces()
    _, cen, _ = c.geometry()
    for f in range(0, c.n_faces, 7):
        _, dS = c.face_quad(f)
        d = cen[fn[f]] + sh[f] * box - cen[fo[f]]
        assert dS.sum(axis=0) @ d > 0, f


def test_uniform_lattice_centroids_exact():
    n = 6
    nodes, cells, box = I.hex_lattice(n)
    c = O.Case(nodes, cells, box, O.Params(order=1, scheme=0))
    vol, cen, hh = c.geometry()
    h = 2 * math.pi / n
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ref = np.stack([(i.ravel() + 0.5) * h, (j.ravel() + 0.5) * h, (k.ravel() + 0.5) * h], axis=1)
    assert np.abs(cen - ref).max() < 1e-13
    assert np.abs(vol - h ** 3).max() < 1e-13 * h ** 3
    # face quadrature of an axis-aligned square: 1 point, area vector h^2 e_d
    x, dS = c.face_quad(0)
    assert np.isclose(np.linalg.norm(dS), h * h, rtol=1e-14)


@pytest.mark.parametrize("kind", ["hex", "tet", "tet_p1", "prism", "pyramid"])
def test_face_quadrature_integrates_bilinear_exactly(kind, jhex8_p2, jtet_p2, jprism_p2, jpyr_p2):
    """The face rules against the independent volume quadrature, through the
    divergence theorem on every cell: with y = x - x_c (x_c the centroid),
    oint y_j dS_i = V delta_ij and oint y_j y_k dS_i = 0. The 2x2 Gauss rule
    on a bilinear face and the collapsed rule on a triangle at P2 are exact
    for both integrands; the P1 triangle's centroid rule for the linear one."""
    if kind == "tet_p1":
        nodes, cells, box = I.hex_lattice(6, jitter=0.1, seed=3)
        cells = I.split_tets(cells)
        c = O.Case(nodes, cells, box, O.Params(order=1, scheme=0))
    else:
        nodes, cells, box, c = {"hex": jhex8_p2, "tet": jtet_p2, "prism": jprism_p2, "pyramid": jpyr_p2}[kind]
    vol, cen, hh = c.geometry()
    fo, fn, sh = c.faces()
    acc = np.zeros((c.n_cells, 3, 3))
    quad = np.zeros((c.n_cells, 3, 3, 3))
    for f in range(c.n_faces):
        x, dS = c.face_quad(f)
        yo, yn = x - cen[fo[f]], x - sh[f] * box - cen[fn[f]]
        acc[fo[f]] += np.einsum("qi,qj->ij", dS, yo)
        acc[fn[f]] -= np.einsum("qi,qj->ij", dS, yn)
        quad[fo[f]] += np.einsum("qi,qj,qk->ijk", dS, yo, yo)
        quad[fn[f]] -= np.einsum("qi,qj,qk->ijk", dS, yn, yn)
    ref = vol[:, None, None] * np.eye(3)[None]
    assert np.abs(acc - ref).max() < 1e-12 * vol.max()
    if kind != "tet_p1":
        assert np.abs(quad).max() < 1e-12 * (vol * hh).max()


# ------------------------------------------------------ least squares ---
@pytest.mark.parametrize("which", [-1, 0, 3])
def test_pseudo_inverse_matches_lstsq(jhex8_p2, which):
    """P' = A^+ diag(|V_m|) (Eq. 4): a left inverse of A diag(1/|V_m|), and
    equal to numpy's least-squares solution of the same system."""
    nodes, cells, box, c = jhex8_p2
    vol, _, _ = c.geometry()
    for i in (0, 77, 300, 511):
        mem, sh, A, P = c.stencil(i, which)
        Vm = vol[mem]
        K = A.shape[1]
        assert np.abs(P @ (A / Vm[:, None]) - np.eye(K)).max() < 1e-12
        ref = np.linalg.lstsq(A, np.diag(Vm), rcond=None)[0]
        assert np.abs(P - ref).max() < 1e-12 * np.abs(ref).max()


def test_stencil_membership_hex_lattice():
    """P2 central = 6 face + 12 edge neighbours; directional stencil of face
    f = its neighbour plus that neighbour's 5 other face neighbours."""
    n = 6
    nodes, cells, box = I.hex_lattice(n)
    c = O.Case(nodes, cells, box, O.Params(order=2, scheme=1))
    ijk = lambda q: (q % n, (q // n) % n, q // (n * n))
    i = 0
    mem, sh, A, P = c.stencil(i, -1)
    offs = set()
    for m, s in zip(mem, sh):
        a = np.array(ijk(m)) + s * n
        offs.add(tuple(a))
    ref = {(a, b, d) for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1)
           if 1 <= abs(a) + abs(b) + abs(d) <= 2}
    assert offs == ref
    for s_ in range(6):
        mem, sh, A, P = c.stencil(i, s_)
        offs = [tuple(np.array(ijk(m)) + s * n) for m, s in zip(mem, sh)]
        axis = np.array(offs[0])
        assert np.abs(axis).sum() == 1
        for o in offs[1:]:
            assert np.abs(np.array(o) - axis).sum() == 1 and o != (0, 0, 0)


# --------------------------------------------------------- k-exactness ---
def _random_poly(rng, degree):
    p = rng.normal(size=(5, 10))
    if degree < 2:
        p[:, 4:] = 0.0
    if degree < 1:
        p[:, 1:] = 0.0
    p[0, 0] += 5.0
    return p


def _poly_eval(p, x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    m = np.stack([np.ones_like(X), X, Y, Z, X * X, Y * Y, Z * Z, X * Y, X * Z, Y * Z], axis=1)
    g = np.zeros((x.shape[0], 10, 3))
    g[:, 1, 0] = 1; g[:, 2, 1] = 1; g[:, 3, 2] = 1
    g[:, 4, 0] = 2 * X; g[:, 5, 1] = 2 * Y; g[:, 6, 2] = 2 * Z
    g[:, 7, 0] = Y; g[:, 7, 1] = X; g[:, 8, 0] = Z; g[:, 8, 2] = X; g[:, 9, 1] = Z; g[:, 9, 2] = Y
    return m @ p.T, np.einsum("qkj,vk->qvj", g, p)


@pytest.mark.parametrize(
    "order,scheme,degree,kind",
    [(1, 0, 1, "hex"), (2, 0, 2, "hex"), (2, 1, 1, "hex"), (2, 0, 2, "tet"), (2, 1, 1, "tet"),
     (1, 0, 1, "prism"), (2, 0, 2, "prism"), (2, 1, 1, "prism"),
     (1, 0, 1, "pyramid"), (2, 0, 2, "pyramid"), (2, 1, 1, "pyramid")],
)
def test_k_exact_reconstruction(order, scheme, degree, kind):
    """Cell averages of any polynomial of degree <= r are reproduced exactly
    by the degree-r least-squares reconstruction (Eqs. 3-4), including cells
    whose stencils cross the periodic boundary; CWENOZ (Eqs. 5-6) is exact
    for degree <= 1, where every candidate is."""
    nodes, cells, box = I.hex_lattice(6 if kind == "hex" else 5, jitter=0.1, seed=3)
    if kind == "tet":
        cells = I.split_tets(cells)
    elif kind == "prism":
        cells = I.split_prisms(cells)
    elif kind == "pyramid":
        nodes, cells = I.split_pyramids(nodes, cells)
    c = O.Case(nodes, cells, box, O.Params(order=order, scheme=scheme))
    rng = np.random.default_rng(7)
    vol, cen, hh = c.geometry()
    p = _random_poly(rng, degree) * 0.1
    for i in (0, 5, c.n_cells // 2, c.n_cells - 1):
        x = cen[i] + rng.uniform(-0.3, 0.3, size=(4, 3)) * hh[i]
        val, grad = c.kexact_probe(i, p, x)
        rv, rg = _poly_eval(p, x)
        scale = np.abs(rv).max()
        assert np.abs(val - rv).max() < 1e-11 * scale
        assert np.abs(grad - rg).max() < 1e-10 * max(1.0, np.abs(rg).max())


def test_cwenoz_degree2_not_exact_but_linear_weights_are():
    """With a quadratic field the directional (linear) candidates are not
    exact, so the nonlinear CWENOZ weights differ from the linear ones, yet
    their sum reproduces p_opt only when omega = lambda (Eq. 5)."""
    nodes, cells, box = I.hex_lattice(6)
    c = O.Case(nodes, cells, box, O.Params(order=2, scheme=1))
    cl = O.Case(nodes, cells, box, O.Params(order=2, scheme=0))
    rng = np.random.default_rng(1)
    p = _random_poly(rng, 2)
    vol, cen, hh = c.geometry()
    x = cen[10][None] + 0.2 * hh[10]
    v1, _ = c.kexact_probe(10, p, x)
    v0, _ = cl.kexact_probe(10, p, x)
    rv, _ = _poly_eval(p, x)
    assert np.abs(v0 - rv).max() < 1e-11 * np.abs(rv).max()
    assert np.abs(v1 - rv).max() > 1e-9 * np.abs(rv).max()


# ------------------------------------------------ per-cell scheme mask ---
def _face_neighbours(c):
    fo, fn, _ = c.faces()
    nb = [[] for _ in range(c.n_cells)]
    for o, n in zip(fo, fn):
        nb[o].append(n)
        nb[n].append(o)
    return nb


@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_scheme_mask_routes_each_cell(kind):
    """Sec. 2.2, Eqs. 5-6 with a per-cell choice of the polynomial: a flagged
    cell reconstructs with its CWENOZ weights, an unflagged one takes p_opt,
    which is the polynomial of the linear scheme (a separate case built with
    scheme 0, pinned by quadratic k-exactness); so a cell whose own flag and
    its face neighbours' flags agree has that scheme's residual, bit for bit,
    and all flags set (none set) give the CWENOZ (linear) residual.  The mask
    is a half box plus scattered cells, so both kinds of agreeing cells and
    mixed ones occur."""
    nodes, cells, box = I.hex_lattice(7 if kind == "hex" else 5, jitter=0.1, seed=8)
    if kind == "tet":
        cells = I.split_tets(cells)
    prm = dict(order=2, Re=1600.0, Mach=0.3)
    cw = O.Case(nodes, cells, box, O.Params(scheme=1, **prm))
    cl = O.Case(nodes, cells, box, O.Params(scheme=0, **prm))
    cm = O.Case(nodes, cells, box, O.Params(scheme=1, **prm))
    U = I.noisy_state(nodes, cells, 0.3, 0.05, seed=2)
    assert np.all(np.isfinite(cw.residual(U))) and np.all(np.isfinite(cl.residual(U)))
    _, cen, _ = cw.geometry()
    rng = np.random.default_rng(12)
    mask = (cen[:, 0] < np.pi) | (rng.random(cw.n_cells) < 0.1)
    cm.set_scheme_mask(mask)
    kw, kl, km = cw.reconstruct(U), cl.reconstruct(U), cm.reconstruct(U)
    assert np.array_equal(km[mask], kw[mask]) and np.array_equal(km[~mask], kl[~mask])
    assert not np.array_equal(kw[mask], kl[mask])  # the two schemes differ on the flagged cells
    Rw, Rl, Rm = cw.residual(U), cl.residual(U), cm.residual(U)
    nb = _face_neighbours(cw)
    all_w = np.array([mask[i] and all(mask[j] for j in nb[i]) for i in range(cw.n_cells)])
    all_l = np.array([not mask[i] and not any(mask[j] for j in nb[i]) for i in range(cw.n_cells)])
    assert all_w.sum() > 5 and all_l.sum() > 5
    assert np.array_equal(Rm[:, all_w], Rw[:, all_w]) and np.array_equal(Rm[:, all_l], Rl[:, all_l])
    mixed = ~all_w & ~all_l
    assert np.any(Rm[:, mixed] != Rw[:, mixed]) and np.any(Rm[:, mixed] != Rl[:, mixed])
    cm.set_scheme_mask(np.ones(cw.n_cells))
    assert np.array_equal(cm.residual(U), Rw)
    cm.set_scheme_mask(np.zeros(cw.n_cells))
    assert np.array_equal(cm.residual(U), Rl)
    cm.set_scheme_mask(None)
    assert np.array_equal(cm.residual(U), Rw)


def test_scheme_mask_keeps_free_stream_and_conservation():
    """Any mask: the face fluxes are shared by both sides, so the volume-
    weighted residual still sums to zero, and a uniform state still has a
    zero residual (every candidate reproduces a constant)."""
    nodes, cells, box = I.hex_lattice(6, jitter=0.1, seed=9)
    c = O.Case(nodes, cells, box, O.Params(order=2, scheme=1, Re=1600.0, Mach=0.3))
    c.set_scheme_mask(np.random.default_rng(2).random(c.n_cells) < 0.4)
    U = I.noisy_state(nodes, cells, 0.3, 0.05, seed=4)
    vol, _, _ = c.geometry()
    R = c.residual(U)
    assert np.all(np.abs((R * vol).sum(axis=1)) <= 1e-13 * (np.abs(R) * vol).sum(axis=1))
    U1 = np.zeros((5, c.n_cells))
    U1[0], U1[1], U1[2], U1[3], U1[4] = 1.1, 0.3, -0.2, 0.15, 75.0
    assert np.abs(c.residual(U1)).max() <= 1e-13 * 75.0


# -------------------------------------------------- smoothness indicator ---
def test_smoothness_indicator_closed_forms():
    """SI = sum_{1<=|b|<=r} V^(2|b|/3-1) int (d^b p)^2: on a cube of side h
    with xi = (x-x_c)/h, p = c xi gives c^2 and p = c (xi^2 - mean) gives
    c^2 (1/3 + 4)."""
    nodes, cells, box = I.hex_lattice(5)
    c = O.Case(nodes, cells, box, O.Params(order=2, scheme=1))
    a = np.zeros(9); a[0] = 0.7
    assert math.isclose(c.smoothness(3, a, 1), 0.49, rel_tol=1e-13)
    a = np.zeros(9); a[3] = 0.5
    assert math.isclose(c.smoothness(3, a, 2), 0.25 * (1.0 / 3.0 + 4.0), rel_tol=1e-13)
    a = np.zeros(9); a[6] = 1.0  # xi*eta: |grad|^2 mean = 2/12, d_xy^2 = 1
    assert math.isclose(c.smoothness(3, a, 2), 2.0 / 12.0 + 1.0, rel_tol=1e-13)


# ------------------------------------------------------------------ P3 ---
# Cubic reconstruction on hexahedra (the TGV-P3 row of Table 4): K = 19
# modes, central stencils of 2K = 38 cells, 6 linear directional stencils,
# 3 x 3 Gauss points per face.
def _cubic_monomials(x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return np.stack([np.ones_like(X), X, Y, Z, X * X, Y * Y, Z * Z, X * Y, X * Z, Y * Z,
                     X ** 3, Y ** 3, Z ** 3, X * X * Y, X * X * Z, X * Y * Y, Y * Y * Z, X * Z * Z, Y * Z * Z,
                     X * Y * Z], axis=1)


def _cubic_gradients(x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    o, z = np.ones_like(X), np.zeros_like(X)
    gx = [z, o, z, z, 2 * X, z, z, Y, Z, z, 3 * X * X, z, z, 2 * X * Y, 2 * X * Z, Y * Y, z, Z * Z, z, Y * Z]
    gy = [z, z, o, z, z, 2 * Y, z, X, z, Z, z, 3 * Y * Y, z, X * X, z, 2 * X * Y, 2 * Y * Z, z, Z * Z, X * Z]
    gz = [z, z, z, o, z, z, 2 * Z, z, X, Y, z, z, 3 * Z * Z, z, X * X, z, Y * Y, 2 * X * Z, 2 * Y * Z, X * Y]
    return np.stack([np.stack(gx, 1), np.stack(gy, 1), np.stack(gz, 1)], axis=2)  # [n, 20, 3]


def test_counts_p3_match_benchmark_matrix():
    """Table 4 (TGV-P3): 74M/2M = 37 reconstructed DoF per cell and variable
    (19 cubic central + 6 linear directional x 3), 54M/6M = 9 quadrature
    points per face; Eq. 3's K(3, 3) = 20 terms with the mean -> 19 modes."""
    cells_, faces, dof, qps = _golden("benchmark_matrix.txt")["TGV-P3"]
    nodes, cells, box = I.hex_lattice(8, jitter=0.1, seed=3)
    c = O.Case(nodes, cells, box, O.Params(order=3, scheme=1))
    assert c.K == math.comb(3 + 3, 3) - 1 == 19
    assert c.K + c.nd * 3 == round(dof / cells_)
    assert c.nq == round(qps / faces) == 9
    assert c.Mc == 2 * c.K and c.nd == 6 and c.Md == 6
    assert c.n_faces == 3 * c.n_cells


@pytest.mark.parametrize("scheme,degree", [(0, 3), (1, 1)])
def test_k_exact_p3(scheme, degree):
    """Cell averages of a random polynomial of degree <= 3: the central cubic
    reconstruction reproduces it (value and gradient) at arbitrary points,
    including cells whose stencils cross the periodic wrap; CWENOZ at P3 is
    exact for degree <= 1 (every candidate is)."""
    nodes, cells, box = I.hex_lattice(8, jitter=0.1, seed=5)
    c = O.Case(nodes, cells, box, O.Params(order=3, scheme=scheme))
    rng = np.random.default_rng(degree)
    poly = rng.normal(size=(5, 20)) * 0.2
    if degree == 1:
        poly[:, 4:] = 0.0
    for i in (0, 77, 511):
        x = I.cell_vertex_means(nodes, cells)[i:i + 1] + rng.uniform(-0.3, 0.3, size=(4, 3))
        val, grad = c.kexact_probe(i, poly, x)
        ref = _cubic_monomials(x) @ poly.T
        gref = np.einsum("nkj,vk->nvj", _cubic_gradients(x), poly)
        assert np.abs(val - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), (i, np.abs(val - ref).max())
        assert np.abs(grad - gref).max() <= 1e-9 * max(1.0, np.abs(gref).max()), (i, np.abs(grad - gref).max())


def test_smoothness_indicator_cubic_closed_forms():
    """SI with the |beta| = 3 terms (weight V^1), on a cube of side h with
    xi = (x - x_c)/h: p = xi^3 gives int (3 xi^2)^2 + int (6 xi)^2 + 6^2 =
    9/80 + 3 + 36, p = xi eta zeta gives 3/144 + 3/12 + 1, and p = xi^2 eta
    gives 4/144 + 1/80 + 2/3 + 4."""
    nodes, cells, box = I.hex_lattice(8)
    c = O.Case(nodes, cells, box, O.Params(order=3, scheme=1))
    a = np.zeros(19); a[9] = 1.0
    assert math.isclose(c.smoothness(5, a, 3), 9 / 80 + 3 + 36, rel_tol=1e-13)
    a = np.zeros(19); a[18] = 1.0
    assert math.isclose(c.smoothness(5, a, 3), 3 / 144 + 3 / 12 + 1, rel_tol=1e-13)
    a = np.zeros(19); a[12] = 1.0  # xi^2 eta: 4/144 + 1/80, then (2 eta)^2 + (2 xi)^2 -> 2/3, then 2^2
    assert math.isclose(c.smoothness(5, a, 3), 4 / 144 + 1 / 80 + 2 / 3 + 4, rel_tol=1e-13)
    a = np.zeros(19); a[0] = 0.7  # a linear p: the first-derivative term only, as at P1
    assert math.isclose(c.smoothness(5, a, 3), 0.49, rel_tol=1e-13)


def test_smoothness_indicator_cubic_on_a_stretched_cell():
    """The cubic SI closed form on an a x a x 2a cell, where the cube's
    symmetry no longer hides which coordinate a derivative leaves: with
    h = V^(1/3) and xi = (x - x_c)/h the cell spans half-widths
    (alpha, alpha, 2 alpha), alpha = a/(2h), and the cell means of xi^2 are
    m = (alpha^2/3)(1, 1, 4). For p = xi eta zeta the three derivative orders
    give (with V^(2|beta|/3) h^(-2|beta|) = 1) m_y m_z + m_x m_z + m_x m_y,
    then m_z + m_y + m_x (from zeta, eta, xi), then 1."""
    nodes, cells, box = I.hex_lattice(8)
    nodes = nodes * np.array([1.0, 1.0, 2.0])
    box = box * np.array([1.0, 1.0, 2.0])
    c = O.Case(nodes, cells, box, O.Params(order=3, scheme=1))
    vol, _, hh = c.geometry()
    a_side = 2 * math.pi / 8
    assert math.isclose(vol[5], 2 * a_side ** 3, rel_tol=1e-13)
    alpha = a_side / (2 * hh[5])
    mx, my, mz = alpha ** 2 / 3, alpha ** 2 / 3, 4 * alpha ** 2 / 3
    a = np.zeros(19)
    a[18] = 1.0
    ref = (my * mz + mx * mz + mx * my) + (mx + my + mz) + 1.0
    assert math.isclose(c.smoothness(5, a, 3), ref, rel_tol=1e-13)


@pytest.mark.parametrize("scheme", [0, 1])
def test_free_stream_and_conservation_p3(scheme):
    """Uniform flow gives a zero residual; any state's volume-weighted
    residual sums to zero on the periodic box (P3 on jittered hexahedra)."""
    nodes, cells, box = I.hex_lattice(8, jitter=0.1, seed=4)
    c = O.Case(nodes, cells, box, O.Params(order=3, scheme=scheme))
    n = len(cells)
    U = I.primitive_to_conserved(np.ones(n), 0.3 * np.ones(n), -0.2 * np.ones(n), 0.1 * np.ones(n),
                                 np.ones(n) / (1.4 * 0.01))
    R, S = c.residual_terms(U)
    assert np.abs(R).max() <= 1e-12 * S.max()
    U = I.noisy_state(nodes, cells, 0.1, 0.05, seed=2)
    R, S = c.residual_terms(U)
    vol, _, _ = c.geometry()
    tot = np.abs((R * vol).sum(axis=1))
    assert np.all(tot <= 1e-12 * (S * vol).sum(axis=1)), tot


def test_order_density_wave_p3():
    """Smooth density wave (exact Euler solution), P3 linear reconstruction
    with the fourth-order SSP(5,4): L1 error order -> 4 (n = 8, 16, 32)."""
    e = [_density_wave_error(n, 3, 0, integrator=1) for n in (8, 16, 32)]
    rates = [math.log2(e[k] / e[k + 1]) for k in range(2)]
    assert all(r > 3.6 for r in rates), rates


# ------------------------------------------------------------------ P4 ---
# Quartic reconstruction on hexahedra (the TGV-P4 row of Table 4): K = 34
# modes, central stencils of 68 cells, 6 quadratic directional candidates
# (Sec. 2.2) of 18 cells each, 4 x 4 Gauss points per face.
_QUARTIC_EXP = [(4, 0, 0), (0, 4, 0), (0, 0, 4), (3, 1, 0), (3, 0, 1), (1, 3, 0), (0, 3, 1), (1, 0, 3), (0, 1, 3),
                (2, 2, 0), (2, 0, 2), (0, 2, 2), (2, 1, 1), (1, 2, 1), (1, 1, 2)]


def _quartic_monomials(x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return np.concatenate([_cubic_monomials(x), np.stack([X ** a * Y ** b * Z ** c for a, b, c in _QUARTIC_EXP], 1)],
                          axis=1)


def test_counts_p4_match_benchmark_matrix():
    """Table 4 (TGV-P4): 176M/2M = 88 reconstructed DoF per cell and
    variable (34 quartic central + 6 quadratic directional x 9), 96M/6M = 16
    quadrature points per face; K(4, 3) = 35 terms with the mean -> 34."""
    cells_, faces, dof, qps = _golden("benchmark_matrix.txt")["TGV-P4"]
    nodes, cells, box = I.hex_lattice(10, jitter=0.1, seed=3)
    c = O.Case(nodes, cells, box, O.Params(order=4, scheme=1))
    assert c.K == math.comb(4 + 3, 3) - 1 == 34
    assert c.K + c.nd * (c.Md // 2) == round(dof / cells_)
    assert c.nq == round(qps / faces) == 16
    assert c.Mc == 68 and c.nd == 6 and c.Md == 18


@pytest.mark.parametrize("scheme,degree", [(0, 4), (1, 2)])
def test_k_exact_p4(scheme, degree):
    """Cell averages of a random polynomial: the central quartic
    reconstruction reproduces degree <= 4 (values), and CWENOZ at P4, whose
    directional candidates are quadratic, reproduces degree <= 2."""
    nodes, cells, box = I.hex_lattice(10, jitter=0.1, seed=5)
    c = O.Case(nodes, cells, box, O.Params(order=4, scheme=scheme))
    rng = np.random.default_rng(degree + 10)
    poly = rng.normal(size=(5, 35)) * 0.05
    if degree == 2:
        poly[:, 10:] = 0.0
    for i in (0, 333, 999):
        x = I.cell_vertex_means(nodes, cells)[i:i + 1] + rng.uniform(-0.3, 0.3, size=(4, 3))
        val, _ = c.kexact_probe(i, poly, x)
        ref = _quartic_monomials(x) @ poly.T
        assert np.abs(val - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), (i, np.abs(val - ref).max())


def test_smoothness_indicator_quartic_closed_form():
    """The |beta| = 4 term (weight V^(5/3)): on a cube, p = xi^4 gives
    int (4 xi^3)^2 + int (12 xi^2)^2 + int (24 xi)^2 + 24^2 = 16/448 + 144/80
    + 576/12 + 576; a mixed quartic checks that every derivative multi-index
    of each order is taken once."""
    nodes, cells, box = I.hex_lattice(10)
    c = O.Case(nodes, cells, box, O.Params(order=4, scheme=1))
    a = np.zeros(34); a[19] = 1.0
    assert math.isclose(c.smoothness(5, a, 4), 16 / 448 + 144 / 80 + 576 / 12 + 576, rel_tol=1e-13)
    # a mixed quartic, p = xi eta zeta^2 (cell means of xi^2, xi^4: 1/12, 1/80):
    # |beta| = 1: (eta zeta^2)^2, (xi zeta^2)^2, (2 xi eta zeta)^2 -> 1/960 + 1/960 + 4/1728;
    # |beta| = 2: (zeta^2)^2, (2 eta zeta)^2, (2 xi zeta)^2, (2 xi eta)^2 -> 1/80 + 3 (4/144);
    # |beta| = 3: (2 zeta)^2, (2 eta)^2, (2 xi)^2 -> 3 (4/12); |beta| = 4: d_xyzz p = 2 -> 4
    a = np.zeros(34); a[33] = 1.0
    ref = (2 / 960 + 4 / 1728) + (1 / 80 + 12 / 144) + 1.0 + 4.0
    assert math.isclose(c.smoothness(5, a, 4), ref, rel_tol=1e-13)


@pytest.mark.parametrize("scheme", [0, 1])
def test_free_stream_and_conservation_p4(scheme):
    nodes, cells, box = I.hex_lattice(10, jitter=0.1, seed=4)
    c = O.Case(nodes, cells, box, O.Params(order=4, scheme=scheme))
    n = len(cells)
    U = I.primitive_to_conserved(np.ones(n), 0.3 * np.ones(n), -0.2 * np.ones(n), 0.1 * np.ones(n),
                                 np.ones(n) / (1.4 * 0.01))
    R, S = c.residual_terms(U)
    assert np.abs(R).max() <= 1e-12 * S.max()
    U = I.noisy_state(nodes, cells, 0.1, 0.05, seed=2)
    R, S = c.residual_terms(U)
    vol, _, _ = c.geometry()
    assert np.all(np.abs((R * vol).sum(axis=1)) <= 1e-12 * (S * vol).sum(axis=1))


def test_order_density_wave_p4():
    """P4 linear reconstruction with SSP(5,4) on the density wave: the L1
    error falls at rates near 5 (n = 8, 12, 16; the time error is negligible
    there: a 4x smaller dt changes the error by < 1e-6 relative)."""
    e = [_density_wave_error(n, 4, 0, integrator=1) for n in (8, 12, 16)]
    rates = [math.log(e[0] / e[1]) / math.log(12 / 8), math.log(e[1] / e[2]) / math.log(16 / 12)]
    assert all(r > 4.4 for r in rates), rates


# ------------------------------------------------------- slip walls ---
# Boundary treatment beyond the periodic wrap: a box axis given length 0 is
# not periodic, and the faces on its two planes are slip walls (inviscid):
# the ghost state mirrors the owner's reconstructed state (normal momentum
# reversed), and a wall face has no directional candidate.
def _walled(n=8, order=2, scheme=1, jitter=0.1):
    nodes, cells, box = I.hex_lattice(n, jitter=jitter, seed=3)
    c = O.Case(nodes, cells, np.array([box[0], box[1], 0.0]), O.Params(order=order, scheme=scheme, Re=0.0))
    return nodes, cells, c


def test_wall_flux_of_the_mirror_state():
    """HLLC between a state and its mirror image in a wall of normal n: no
    mass, tangential-momentum or energy flux; the normal momentum flux is the
    star pressure, at least the state's own pressure when it moves into the
    wall and at most that when it moves away."""
    rng = np.random.default_rng(4)
    for _ in range(50):
        n = rng.normal(size=3); n /= np.linalg.norm(n)
        rho, p = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
        u = rng.normal(size=3)
        UL = np.array([rho, *(rho * u), p / 0.4 + 0.5 * rho * u @ u])
        mn = UL[1:4] @ n
        UR = UL.copy(); UR[1:4] = UL[1:4] - 2 * mn * n
        F = O.hllc(UL, UR, n)
        scale = abs(F[1:4] @ n) + p
        assert abs(F[0]) <= 1e-14 * scale * 10 and abs(F[4]) <= 1e-13 * scale * 10
        Ft = F[1:4] - (F[1:4] @ n) * n
        assert np.abs(Ft).max() <= 1e-13 * scale
        if mn > 0:  # moving into the wall: compression, p* >= p
            assert F[1:4] @ n >= p * (1 - 1e-12)
        else:  # moving away: an expansion, p* <= p (it may even be negative for a strong one)
            assert F[1:4] @ n <= p * (1 + 1e-12)


@pytest.mark.parametrize("order,scheme", [(1, 0), (2, 0), (2, 1), (3, 1), (4, 1)])
def test_walls_free_stream_and_conservation(order, scheme):
    """Walls on z = 0 and z = L, periodic in x and y: a uniform flow parallel
    to the walls gives a zero residual; for any state, mass, x- and
    y-momentum and energy are conserved to round-off (the walls exert only a
    normal force), and the face count is the periodic one minus the wrapped
    z faces plus the wall faces."""
    nodes, cells, c = _walled(order=order, scheme=scheme)
    n = len(cells)
    assert c.n_faces == 3 * n - 64 + 2 * 64
    U = I.primitive_to_conserved(np.ones(n), 0.3 * np.ones(n), -0.2 * np.ones(n), np.zeros(n), np.ones(n) / 0.014)
    R, S = c.residual_terms(U)
    assert np.abs(R).max() <= 1e-12 * S.max()
    U = I.noisy_state(nodes, cells, 0.1, 0.05, seed=2)
    R, S = c.residual_terms(U)
    vol, _, _ = c.geometry()
    tot = np.abs((R * vol).sum(axis=1)) / (S * vol).sum(axis=1)
    assert np.all(tot[[0, 1, 2, 4]] <= 1e-12), tot
    assert tot[3] > 1e-8  # the wall pressure changes the normal momentum


@pytest.mark.parametrize("order", [2, 3])
def test_walls_k_exact_and_candidate_weights(order):
    """Cells on the walls have one-sided stencils and still reproduce
    polynomials of their degree; their wall faces carry no directional
    candidate (weight 0), and the remaining CWENOZ weights sum to 1."""
    nodes, cells, c = _walled(order=order, scheme=0)
    rng = np.random.default_rng(order)
    nt = 10 if order == 2 else 20
    poly = rng.normal(size=(5, nt)) * 0.2
    xm = I.cell_vertex_means(nodes, cells)
    bottom, top = 3, len(cells) - 5  # cells touching z = 0 and z = L
    for i in (bottom, top):
        x = xm[i:i + 1] + rng.uniform(-0.3, 0.3, size=(4, 3))
        val, _ = c.kexact_probe(i, poly, x)
        ref = (_cubic_monomials(x)[:, :nt]) @ poly.T
        assert np.abs(val - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), i
    _, _, cw = _walled(order=order, scheme=1)
    U = I.noisy_state(nodes, cells, 0.1, 0.05, seed=1)
    _, w = cw.reconstruct(U, weights=True)
    assert np.allclose(w.sum(axis=2), 1.0, atol=1e-14)
    fo, fn, _ = cw.faces()
    walls = fn < 0
    assert walls.sum() == 128
    # a bottom cell: exactly one of its six candidate slots is a wall face, weight 0
    zeros = (w[bottom] == 0.0).all(axis=0)
    assert zeros[1:].sum() == 1 and not zeros[0]


@pytest.mark.parametrize("order,scheme", [(1, 0), (2, 1), (3, 1)])
def test_supersonic_inflow_outflow(order, scheme):
    """x not periodic, inflow of a Mach-2 uniform state at x = 0 and
    extrapolation outflow at x = L (y, z periodic): that state is steady
    (zero residual); an inflow state different from the interior changes
    only the cells whose stencils reach the inflow faces (one-sided
    neighbourhood of x = 0), not those near the outflow."""
    nodes, cells, box = I.hex_lattice(8, jitter=0.1, seed=6)
    n = len(cells)
    rho, p, u = 1.4, 1.0, 2.0  # sound speed 1
    Uinf = (rho, rho * u, 0.0, 0.0, p / 0.4 + 0.5 * rho * u * u)
    prm = O.Params(order=order, scheme=scheme, Re=0.0, bc=(3, 2, 0, 0, 0, 0), inflow=Uinf)
    c = O.Case(nodes, cells, np.array([0.0, box[1], box[2]]), prm)
    U = np.tile(np.array(Uinf)[:, None], (1, n))
    R, S = c.residual_terms(U)
    assert np.abs(R).max() <= 1e-12 * S.max()
    prm2 = O.Params(order=order, scheme=scheme, Re=0.0, bc=(3, 2, 0, 0, 0, 0),
                    inflow=(1.1 * rho, 1.1 * rho * u, 0.0, 0.0, 1.1 * Uinf[4]))
    c2 = O.Case(nodes, cells, np.array([0.0, box[1], box[2]]), prm2)
    R2, _ = c2.residual_terms(U)
    x = I.cell_vertex_means(nodes, cells)[:, 0]
    h = 2 * math.pi / 8
    assert np.abs(R2[:, x < h]).max() > 1e-3 * S.max()      # the inflow cells feel it
    assert np.abs(R2[:, x > 5 * h]).max() <= 1e-12 * S.max()  # downstream, beyond the stencils: unchanged


def test_walls_need_an_inviscid_flow():
    nodes, cells, box = I.hex_lattice(6)
    with pytest.raises(O.OracleError):
        O.Case(nodes, cells, np.array([box[0], box[1], 0.0]), O.Params(order=1, scheme=0, Re=1600.0))


# ------------------------------------------------------------ invariants ---
@pytest.mark.parametrize("kind", ["hex", "tet", "prism", "pyramid"])
def test_free_stream_preservation(kind, jhex8_p2, jtet_p2, jprism_p2, jpyr_p2):
    nodes, cells, box, c = {"hex": jhex8_p2, "tet": jtet_p2, "prism": jprism_p2, "pyramid": jpyr_p2}[kind]
    U = np.zeros((5, c.n_cells))
    U[0], U[1], U[2], U[3], U[4] = 1.1, 0.3, -0.2, 0.15, 75.0
    R = c.residual(U)
    assert np.abs(R).max() <= 1e-13 * 75.0


@pytest.mark.parametrize("kind", ["hex", "tet", "prism", "pyramid"])
def test_discrete_conservation(kind, jhex8_p2, jtet_p2, jprism_p2, jpyr_p2):
    nodes, cells, box, c = {"hex": jhex8_p2, "tet": jtet_p2, "prism": jprism_p2, "pyramid": jpyr_p2}[kind]
    U = I.noisy_state(nodes, cells, 0.3, 0.05, seed=4)
    R = c.residual(U)
    vol, _, _ = c.geometry()
    tot = (R * vol).sum(axis=1)
    scale = (np.abs(R) * vol).sum(axis=1)
    assert np.all(np.abs(tot) <= 1e-13 * scale)


@pytest.mark.parametrize("kind", ["hex", "tet", "prism", "pyramid"])
def test_residual_of_sampled_cells_equals_the_full_residual(kind, jhex8_p2, jtet_p2, jprism_p2, jpyr_p2):
    """The sampled-cell residual (the path the CPU baseline and the full-size
    parity samples take) equals the full residual's columns bit for bit, and
    so do the summed-term magnitudes S."""
    nodes, cells, box, c = {"hex": jhex8_p2, "tet": jtet_p2, "prism": jprism_p2, "pyramid": jpyr_p2}[kind]
    U = I.noisy_state(nodes, cells, 0.3, 0.05, seed=6)
    R, S = c.residual_terms(U)
    sel = np.random.default_rng(4).choice(c.n_cells, 37, replace=False)
    Rs, Ss = c.residual_subset_terms(U, sel)
    assert np.array_equal(Rs, R[:, sel]) and np.array_equal(Ss, S[:, sel])
    assert np.array_equal(c.residual_subset(U, sel), R[:, sel])


@pytest.mark.parametrize("order,scheme", [(1, 0), (2, 1)])
def test_residual_independent_of_cell_numbering(order, scheme):
    """Renumbering the cells permutes the residual and changes nothing else
    (to round-off): which cell of a face is its owner changes with the
    numbering, so any owner/neighbour asymmetry in the face flux (a one-sided
    gradient or state, a penalty or normal of the wrong orientation) shows.
    Viscous (Re = 10) on jittered hexahedra, where every stencil is a whole
    tie group of its ordering; on tetrahedra the stencils' cut-off falls
    inside groups ordered by cell id, so their membership depends on the
    numbering by construction."""
    nodes, cells, box = I.hex_lattice(6, jitter=0.1, seed=11)
    U = I.noisy_state(nodes, cells, 0.3, 0.05, seed=12)
    prm = O.Params(order=order, scheme=scheme, Re=10.0, Mach=0.3)
    R, S = O.Case(nodes, cells, box, prm).residual_terms(U)
    perm = np.random.default_rng(3).permutation(len(cells))
    c2 = O.Case(nodes, cells[perm], box, prm)
    assert not np.array_equal(c2.faces()[0], perm[O.Case(nodes, cells, box, prm).faces()[0]])  # owners do change
    R2, _ = c2.residual_terms(U[:, perm])
    assert (np.abs(R2 - R[:, perm]) / S[:, perm]).max() < 1e-13


def test_residual_deterministic(jhex8_p2):
    nodes, cells, box, c = jhex8_p2
    U = I.noisy_state(nodes, cells, 0.3, 0.05, seed=5)
    assert np.array_equal(c.residual(U), c.residual(U))


# ------------------------------------------------------------------ HLLC ---
def _phys(U, n, g=1.4):
    r, m, E = U[0], U[1:4], U[4]
    u = m / r
    p = (g - 1) * (E - 0.5 * r * u @ u)
    un = u @ n
    return np.concatenate([[r * un], r * u * un + p * n, [(E + p) * un]])


def _cons(r, u, p, g=1.4):
    u = np.asarray(u, float)
    return np.concatenate([[r], r * u, [p / (g - 1) + 0.5 * r * u @ u]])


def test_hllc_consistency_contact_upwind_symmetry():
    rng = np.random.default_rng(0)
    for _ in range(20):
        n = rng.normal(size=3); n /= np.linalg.norm(n)
        U = _cons(rng.uniform(0.5, 2), rng.normal(size=3), rng.uniform(0.5, 3))
        assert np.allclose(O.hllc(U, U, n), _phys(U, n), rtol=1e-14, atol=1e-14)
        # stationary contact: equal pressure, zero normal velocity, any density/tangential velocity
        t = rng.normal(size=3); t -= (t @ n) * n
        UL = _cons(rng.uniform(0.5, 2), t, 1.3)
        UR = _cons(rng.uniform(0.5, 2), -t, 1.3)
        F = O.hllc(UL, UR, n)
        assert np.allclose(F, np.concatenate([[0], 1.3 * n, [0]]), atol=1e-14)
        # supersonic to the right: upwind flux of the left state
        UL = _cons(1.0, 5.0 * n, 1.0)
        UR = _cons(0.7, 4.0 * n + t, 0.8)
        assert np.allclose(O.hllc(UL, UR, n), _phys(UL, n), rtol=1e-14, atol=1e-13)
        # reflection symmetry F(L,R,n) = -F(R,L,-n)
        UL = _cons(rng.uniform(0.5, 2), rng.normal(size=3), rng.uniform(0.5, 3))
        UR = _cons(rng.uniform(0.5, 2), rng.normal(size=3), rng.uniform(0.5, 3))
        assert np.allclose(O.hllc(UL, UR, n), -O.hllc(UR, UL, -n), rtol=1e-13, atol=1e-13)
        # rotational invariance
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        rot = lambda U: np.concatenate([[U[0]], Q @ U[1:4], [U[4]]])
        F1 = O.hllc(rot(UL), rot(UR), Q @ n)
        assert np.allclose(F1, rot(O.hllc(UL, UR, n)), rtol=1e-12, atol=1e-12)


def test_hllc_resolves_an_isolated_shock_exactly():
    """An isolated shock of speed s between U_L and U_R (Rankine-Hugoniot:
    F(U_R) - F(U_L) = s (U_R - U_L)) is an eigenvector of the Roe matrix, so
    the Roe-averaged speed u~ + a~ (u~ - a~ for a left-running shock) is s
    exactly, Einfeldt's bound selects it, the contact speed is the post-shock
    normal velocity and both star states are the post-shock state: HLLC
    returns the exact interface flux, F(U_L) for s > 0 and F(U_R) for s < 0,
    here to round-off. Normal-shock relations at shock Mach 1.2-3, oblique
    normals, tangential velocity continuous, the post-shock gas moving
    against the shock (star branch on the shock's side), with the shock
    running right and its mirror image running left."""
    rng = np.random.default_rng(7)
    g = 1.4

    def mirror(U, n):
        V = U.copy()
        V[1:4] = U[1:4] - 2 * (U[1:4] @ n) * n
        return V

    for Ms in (1.2, 1.5, 3.0):
        for s in (0.3, -0.4, 2.5):
            n = rng.normal(size=3)
            n /= np.linalg.norm(n)
            t = rng.normal(size=3)
            t = 0.3 * (t - (t @ n) * n)
            w = math.sqrt(g) * Ms                     # s - u_R, pre-shock state rho = p = 1
            rL = (g + 1) * Ms ** 2 / ((g - 1) * Ms ** 2 + 2)
            pL = 1 + 2 * g / (g + 1) * (Ms ** 2 - 1)
            UL = _cons(rL, (s - w / rL) * n + t, pL)
            UR = _cons(1.0, (s - w) * n + t, 1.0)
            rh = _phys(UR, n) - _phys(UL, n) - s * (UR - UL)
            assert np.abs(rh).max() < 1e-13
            F = O.hllc(UL, UR, n)
            ref = _phys(UL, n) if s > 0 else _phys(UR, n)
            assert np.abs(F - ref).max() <= 1e-14 * np.abs(ref).max(), (Ms, s)
            A, B = mirror(UR, n), mirror(UL, n)       # the left-running shock, speed -s
            F = O.hllc(A, B, n)
            ref = _phys(B, n) if s > 0 else _phys(A, n)
            assert np.abs(F - ref).max() <= 1e-14 * np.abs(ref).max(), (Ms, -s)


def test_hllc_sod_interface_flux():
    """Sod's shock tube: the exact solution at the interface is the left star
    state (rho = 0.42632, u = 0.92745, p = 0.30313, Toro's tabulated values).
    HLLC approximates that Godunov flux: mass and energy within 10 %."""
    g = 1.4
    n = np.array([1.0, 0.0, 0.0])
    UL, UR = _cons(1.0, [0, 0, 0], 1.0), _cons(0.125, [0, 0, 0], 0.1)
    F = O.hllc(UL, UR, n)
    r, u, p = 0.42632, 0.92745, 0.30313
    E = p / (g - 1) + 0.5 * r * u * u
    ex = np.array([r * u, r * u * u + p, 0.0, 0.0, (E + p) * u])
    assert abs(F[0] - ex[0]) < 0.1 * ex[0]
    assert abs(F[4] - ex[4]) < 0.1 * ex[4]
    assert F[2] == 0.0 and F[3] == 0.0


# ------------------------------------------------------------- viscous ---
def test_viscous_flux_linear_velocity_uniform_temperature():
    """u = G x with uniform T: the flux is the exact Newtonian stress
    tau = mu (G + G^T - 2/3 tr(G) I) dotted with n, plus u . tau . n."""
    rng = np.random.default_rng(2)
    g, Re, Pr, M = 1.4, 1600.0, 0.71, 0.1
    mu = 1 / Re
    Rg = 1 / (g * M * M)
    for _ in range(10):
        G = rng.normal(size=(3, 3))
        x0 = rng.normal(size=3)
        r = rng.uniform(0.5, 2.0)
        u = G @ x0
        T = 1.3
        p = r * Rg * T
        # conserved gradients of (rho = const, m = rho G x, E = p/(g-1) + rho |u|^2/2)
        gU = np.zeros((5, 3))
        gU[1:4] = r * G
        gU[4] = r * (G.T @ u)
        U = _cons(r, u, p)
        n = rng.normal(size=3); n /= np.linalg.norm(n)
        tau = mu * (G + G.T - 2.0 / 3.0 * np.trace(G) * np.eye(3))
        F = O.viscous_flux(U, gU, n, g, Re, Pr, M)
        assert np.allclose(F[1:4], tau @ n, rtol=1e-12, atol=1e-15)
        assert math.isclose(F[4], u @ tau @ n, rel_tol=1e-11, abs_tol=1e-15)
        assert F[0] == 0.0


def test_viscous_flux_of_a_general_state():
    """The Navier-Stokes viscous flux from primitive gradients by the chain
    rule, at states where density, velocity and pressure all vary: with
    grad rho, G = grad u and grad p given, the conserved gradients are
    grad(rho u_a) = u_a grad rho + rho G_a and grad E = grad p/(g - 1) +
    |u|^2/2 grad rho + rho G^T u; the flux is tau n (tau = mu (G + G^T -
    2/3 tr G I)) and u . tau n + kappa grad T . n with T = p/(rho R)."""
    rng = np.random.default_rng(5)
    g, Re, Pr, M = 1.4, 100.0, 0.71, 0.3
    mu = 1 / Re
    Rg = 1 / (g * M * M)
    kap = mu * g * Rg / (g - 1) / Pr
    for _ in range(20):
        r, p = rng.uniform(0.5, 2.0), rng.uniform(5.0, 20.0)
        u = rng.normal(size=3)
        gr, G, gp = rng.normal(size=3), rng.normal(size=(3, 3)), rng.normal(size=3)
        gU = np.zeros((5, 3))
        gU[0] = gr
        gU[1:4] = u[:, None] * gr[None, :] + r * G
        gU[4] = gp / (g - 1) + 0.5 * (u @ u) * gr + r * (G.T @ u)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        tau = mu * (G + G.T - 2.0 / 3.0 * np.trace(G) * np.eye(3))
        gT = gp / (r * Rg) - p * gr / (r * r * Rg)
        F = O.viscous_flux(_cons(r, u, p), gU, n, g, Re, Pr, M)
        assert F[0] == 0.0
        assert np.allclose(F[1:4], tau @ n, rtol=1e-12, atol=1e-14)
        assert math.isclose(F[4], u @ tau @ n + kap * gT @ n, rel_tol=1e-11, abs_tol=1e-13)


def test_viscous_flux_heat_conduction_and_rest():
    g, Re, Pr, M = 1.4, 1600.0, 0.71, 0.1
    mu = 1 / Re
    Rg = 1 / (g * M * M)
    kap = mu * g * Rg / (g - 1) / Pr
    # fluid at rest, uniform pressure, linear T: rho = p/(R T)
    p, T, dT = 71.4, 1.0, np.array([0.3, -0.1, 0.2])
    r = p / (Rg * T)
    dr = -p / (Rg * T * T) * dT
    gU = np.zeros((5, 3)); gU[0] = dr
    U = _cons(r, [0, 0, 0], p)
    n = np.array([0.0, 0.6, 0.8])
    F = O.viscous_flux(U, gU, n, g, Re, Pr, M)
    assert np.allclose(F[:4], 0.0, atol=1e-15)
    assert math.isclose(F[4], kap * dT @ n, rel_tol=1e-12)
    # uniform flow: no viscous flux
    F = O.viscous_flux(_cons(1.0, [0.3, 0.2, 0.1], 2.0), np.zeros((5, 3)), n, g, Re, Pr, M)
    assert np.all(F == 0.0)


def _viscous_part(nodes, cells, box, U, **kw):
    """The residual with viscosity minus the Euler residual of the same state
    and reconstruction: the viscous flux integral alone, +(1/V) sum sigma F_v A."""
    cv = O.Case(nodes, cells, box, O.Params(**kw))
    ci = O.Case(nodes, cells, box, O.Params(**{**kw, "Re": 0.0}))
    return cv.residual(U) - ci.residual(U)


def _shear_state(n, comp, eps, p, g=1.4):
    """Exact cell averages on the uniform n^3 lattice of rho = 1, uniform p and
    the velocity component comp (1: u, 2: v) = eps sin x; also the cell
    averages of sin x and cos 2x."""
    nodes, cells, box = I.hex_lattice(n)
    h = 2 * math.pi / n
    c = O.Case(nodes, cells, box, O.Params(order=1, scheme=0))
    _, cen, _ = c.geometry()
    a = cen[:, 0] - h / 2
    s = (np.cos(a) - np.cos(a + h)) / h
    c2 = (np.sin(2 * (a + h)) - np.sin(2 * a)) / (2 * h)
    U = np.zeros((5, c.n_cells))
    U[0] = 1.0
    U[comp] = eps * s
    U[4] = p / (g - 1) + 0.5 * eps ** 2 * (0.5 - 0.5 * c2)
    return (nodes, cells, box), U, s, c2


def test_jump_penalty_on_the_odd_even_mode():
    """Eq. 7 on the odd-even shear mode v = eps (-1)^i (i the cell's x index),
    rho and p uniform, on a uniform cube lattice at P1. The mode is even about
    every cell, so each symmetric least-squares gradient of it vanishes and the
    averaged face gradient is zero: only the penalty alpha (U_R - U_L) n / L_int,
    L_int = h, acts. The viscous residual is then alpha mu times the discrete
    Laplacian (v_{i+1} - 2 v_i + v_{i-1}) / h^2 = -4 v_i / h^2 in the y
    momentum and zero in the rest (zero face-average velocity, no jump in rho
    or E), exactly."""
    n, eps, Re, M, g = 8, 0.1, 10.0, 0.5, 1.4
    nodes, cells, box = I.hex_lattice(n)
    h = 2 * math.pi / n
    c = O.Case(nodes, cells, box, O.Params(order=1, scheme=0))
    _, cen, _ = c.geometry()
    v = eps * (-1.0) ** np.floor(cen[:, 0] / h)
    p = 1.0 / (g * M * M)
    U = np.zeros((5, c.n_cells))
    U[0], U[2], U[4] = 1.0, v, p / (g - 1) + 0.5 * v * v
    Rv = _viscous_part(nodes, cells, box, U, order=1, scheme=0, Mach=M, Re=Re)
    ref = np.zeros_like(Rv)
    ref[2] = -4.0 * (4.0 / 3.0) / Re * v / h ** 2
    assert np.abs(Rv - ref).max() <= 1e-12 * np.abs(ref).max()


def test_viscous_residual_of_a_shear_wave():
    """v = eps sin x, rho and p uniform (T uniform), on uniform cube lattices at
    P2: the viscous residual tends at second order to the cell averages of
    div F_v = (0, 0, mu v'', 0, (mu v v')') = (0, 0, -mu eps sin x, 0,
    mu eps^2 cos 2x) (Newtonian stress and its work, Eq. 7 gradients; no
    heat flux). The density, x and z rows stay zero to round-off."""
    eps, Re, M, g = 0.1, 10.0, 0.5, 1.4
    mu = 1.0 / Re
    err = []
    for n in (16, 32):
        mesh, U, s, c2 = _shear_state(n, 2, eps, 1.0 / (g * M * M))
        Rv = _viscous_part(*mesh, U, order=2, scheme=0, Mach=M, Re=Re)
        assert np.abs(Rv[[0, 1, 3]]).max() < 1e-14
        err.append((np.abs(Rv[2] + mu * eps * s).max() / (mu * eps),
                    np.abs(Rv[4] - mu * eps ** 2 * c2).max() / (mu * eps ** 2)))
    (m16, e16), (m32, e32) = err
    assert m32 < 0.35 * m16 and m32 < 0.01, err
    assert e32 < 0.5 * e16 and e32 < 0.05, err


# -------------------------------------------------------------------- RK ---
def test_ssprk3_stability_polynomial():
    for z in (-0.3, -1.0, -2.5, 0.7, 0.05):
        ref = 1 + z + z * z / 2 + z ** 3 / 6
        assert math.isclose(O.ssprk3_linear(z, 1.0, 1.0), ref, rel_tol=1e-15)


def _tableau_from_shu_osher(alpha, beta):
    """u_i = sum_j (alpha_ij u_j + dt beta_ij L(u_j)) rewritten as
    u_i = u_0 + dt sum_k A_ik L(u_k): the Butcher matrix (rows of the stages
    u_0..u_{s-1}) and the weights (the row of u_s)."""
    s = alpha.shape[0] - 1
    A = np.zeros((s + 1, s))
    for i in range(1, s + 1):
        for j in range(i):
            A[i] += alpha[i, j] * A[j]
            A[i, j] += beta[i, j]
    return A[:s], A[s]


def test_ssp54_coefficients_meet_the_order_conditions():
    """The fourth-order SSP scheme of Eq. 8 (Spiteri-Ruuth SSP(5,4)) as stored
    in the oracle, against the mathematics of Runge-Kutta methods: every stage
    is consistent (its alpha row sums to 1), all coefficients are nonnegative,
    the weights satisfy the eight order conditions of the rooted trees with at
    most four nodes, an order-5 condition fails (order exactly 4), and the SSP
    coefficient min alpha/beta is 1.508."""
    alpha, beta = O.ssp54_coefficients()
    for i in range(1, 6):
        assert abs(alpha[i, :i].sum() - 1.0) < 3e-15, i
    assert (alpha >= 0).all() and (beta >= 0).all()
    A, b = _tableau_from_shu_osher(alpha, beta)
    c = A.sum(axis=1)
    conditions = [
        (b.sum(), 1.0), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ (A @ c), 1 / 6),
        (b @ c ** 3, 1 / 4), (b @ (c * (A @ c)), 1 / 8), (b @ (A @ c ** 2), 1 / 12), (b @ (A @ (A @ c)), 1 / 24),
    ]
    for k, (got, want) in enumerate(conditions):
        assert abs(got - want) < 1e-14, (k, got, want)
    assert abs(b @ c ** 4 - 1 / 5) > 1e-4
    ssp = min(alpha[i, j] / beta[i, j] for i in range(6) for j in range(5) if beta[i, j] > 0)
    assert 1.5081 < ssp < 1.5082


def test_ssp54_stability_polynomial():
    """One SSP(5,4) step of du/dt = z u is the degree-5 polynomial whose terms
    up to z^4 are those of e^z and whose z^5 coefficient is b A^3 c of the
    tableau (the stepper combines the stages as the coefficients say)."""
    A, b = _tableau_from_shu_osher(*O.ssp54_coefficients())
    c = A.sum(axis=1)
    g = b @ (A @ (A @ (A @ c)))
    assert 0.004 < g < 0.005
    for z in (-0.3, -1.0, -2.5, 0.7, 0.05):
        ref = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24 + g * z ** 5
        assert math.isclose(O.ssp54_linear(z, 1.0, 1.0), ref, rel_tol=1e-14), z


@pytest.mark.parametrize("integrator", [0, 1])
def test_rk_step_composes_the_residual(integrator):
    """One step of the case's integrator is its Shu-Osher combination of the
    case's own residual L = residual(.): SSP-RK3 u1 = u + dt L(u), u2 = 3/4 u
    + 1/4 (u1 + dt L(u1)), u' = 1/3 u + 2/3 (u2 + dt L(u2)); SSP(5,4) with the
    coefficients pinned above; and dt <= 0 takes the CFL time step."""
    nodes, cells, box = I.hex_lattice(6, jitter=0.1, seed=8)
    c = O.Case(nodes, cells, box, O.Params(order=2, scheme=1, integrator=integrator))
    U = I.noisy_state(nodes, cells, 0.3, 0.05, seed=9)
    dt = 0.5 * c.time_step(U)
    L = c.residual
    if integrator == 0:
        u1 = U + dt * L(U)
        u2 = 0.75 * U + 0.25 * (u1 + dt * L(u1))
        ref = U / 3.0 + 2.0 / 3.0 * (u2 + dt * L(u2))
    else:
        al, be = O.ssp54_coefficients()
        u, Ls = [U], []
        for i in range(1, 6):
            Ls.append(L(u[i - 1]))
            u.append(sum(al[i][j] * u[j] + dt * be[i][j] * Ls[j] for j in range(i)))
        ref = u[5]
    got, used = c.rk_step(U, dt)
    assert used == dt
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(U).max()
    got2, used2 = c.rk_step(U)
    assert used2 == c.time_step(U)


def test_rk_orders_on_a_nonlinear_ode():
    """Logistic equation u' = u (1 - u), u(0) = 0.2, to T = 2 against its
    closed form 1 / (1 + 4 e^-T): halving dt divides the error by 2^4 with
    SSP(5,4) and by 2^3 with SSP-RK3."""
    exact = 1.0 / (1.0 + 4.0 * math.exp(-2.0))
    for integrator, order in ((1, 4), (0, 3)):
        e = [abs(O.logistic(0.2, 2.0, n, integrator) - exact) for n in (16, 32, 64, 128)]
        rates = [math.log2(e[k] / e[k + 1]) for k in range(3)]
        assert all(abs(r - order) < 0.25 for r in rates), (integrator, rates)


# ---------------------------------------------------------- Taylor-Green ---
def test_tgv_initial_diagnostics_converge_to_closed_forms():
    gold = _golden("tgv_initial.txt")
    out = []
    for n in (16, 32):
        nodes, cells, box = I.hex_lattice(n)
        c = O.Case(nodes, cells, box, O.Params(order=2, scheme=0, Mach=0.1))
        U = c.cell_average("tgv", [0.1, 1.4])
        out.append(c.diagnostics(U))
    ke = [abs(o[0] - gold["KE0"][0]) for o in out]
    es = [abs(o[1] - gold["eps_s0_Re1600"][0]) for o in out]
    assert ke[1] < 0.3 * ke[0] and ke[1] < 2e-3      # O(h^2) to 1/8
    assert es[1] < 0.3 * es[0] and es[1] < 0.06 * gold["eps_s0_Re1600"][0]
    assert all(o[2] < 1e-3 * gold["eps_s0_Re1600"][0] for o in out)


def test_tgv_initial_ke_mach_independent():
    nodes, cells, box = I.hex_lattice(12)
    kes = []
    for M in (0.1, 1.25):
        c = O.Case(nodes, cells, box, O.Params(order=1, scheme=0, Mach=M))
        kes.append(c.diagnostics(c.cell_average("tgv", [M, 1.4]))[0])
    assert abs(kes[0] - kes[1]) < 2e-3 * 0.125


def test_tgv_initial_pressure_solves_the_poisson_equation():
    """Sec. 4.2 Taylor-Green initial state: for the given velocity, the
    pressure perturbation is the zero-mean periodic solution of the
    incompressible pressure Poisson equation lap p = -d_i u_j d_j u_i =
    -(1 + cos 2z)(cos 2x + cos 2y)/2 (rho_0 = 1), and the temperature is
    uniform, rho = gamma M^2 p, so the mean density is 1. The 7-point
    Laplacian of the cell pressures converges to that right side at second
    order (Mach 0.01: the density is 1 to 1e-4)."""
    g, M = 1.4, 0.01
    err = []
    for n in (16, 32):
        nodes, cells, box = I.hex_lattice(n)
        h = 2 * math.pi / n
        c = O.Case(nodes, cells, box, O.Params(order=1, scheme=0, Mach=M))
        U = c.cell_average("tgv", [M, g])
        _, cen, _ = c.geometry()
        p = (g - 1) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0])
        assert abs(U[0].mean() - 1.0) < 1e-12
        assert np.abs(g * M * M * p / U[0] - 1.0).max() < 1e-6
        ijk = np.floor(cen / h).astype(int)
        P = np.zeros((n, n, n))
        P[ijk[:, 0], ijk[:, 1], ijk[:, 2]] = p
        lap = (sum(np.roll(P, 1, d) + np.roll(P, -1, d) for d in range(3)) - 6 * P) / h ** 2
        x = (np.arange(n) + 0.5) * h
        X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
        rhs = -(1 + np.cos(2 * Z)) * (np.cos(2 * X) + np.cos(2 * Y)) / 2
        err.append(np.abs(lap - rhs).max() / np.abs(rhs).max())
    assert err[1] < 0.35 * err[0] and err[1] < 0.05, err


def test_dissipation_diagnostics_of_plane_waves():
    """Sec. 4.2 diagnostics at P2 on plane waves, rho and p uniform, Re = 10:
    u = eps sin x is pure dilatation, eps_d -> (4/3) mu <(eps cos x)^2> =
    2 mu eps^2/3 and eps_s = 0; v = eps sin x is pure shear, eps_s -> mu
    <(eps cos x)^2> = mu eps^2/2 and eps_d = 0. KE from the cell averages is
    exactly eps^2/4 (sin(h/2)/(h/2))^2 on the uniform lattice. The two
    dissipations converge at second order."""
    eps, Re, M, g = 0.1, 10.0, 0.5, 1.4
    mu = 1.0 / Re
    err = []
    for n in (8, 16, 32):
        h = 2 * math.pi / n
        ke = eps ** 2 / 4 * (math.sin(h / 2) / (h / 2)) ** 2
        row = []
        for comp, k, ref in ((1, 2, 2 * mu * eps ** 2 / 3), (2, 1, mu * eps ** 2 / 2)):
            mesh, U, _, _ = _shear_state(n, comp, eps, 1.0 / (g * M * M))
            c = O.Case(*mesh, O.Params(order=2, scheme=0, Mach=M, Re=Re))
            d = c.diagnostics(U)
            assert math.isclose(d[0], ke, rel_tol=1e-12)
            assert d[3 - k] < 1e-25  # the other dissipation vanishes
            row.append(abs(d[k] - ref) / ref)
        err.append(row)
    for j in range(2):
        assert err[1][j] < 0.3 * err[0][j] and err[2][j] < 0.3 * err[1][j], err
    assert max(err[2]) < 0.02, err


# ---------------------------------------------------- order of accuracy ---
def _density_wave_error(n, order, scheme, T=0.05, integrator=0, split=None):
    nodes, cells, box = I.hex_lattice(n)
    if split is I.split_pyramids:
        nodes, cells = split(nodes, cells)
    elif split is not None:
        cells = split(cells)
    c = O.Case(nodes, cells, box, O.Params(order=order, scheme=scheme, Re=0.0, integrator=integrator))
    p = [1.0, 0.2, 1.0, 0.5, 0.25, 1.0, 0.0, 1.4]
    U = c.cell_average("density_wave", p)
    nst = int(math.ceil(T / c.time_step(U)))
    for _ in range(nst):
        U, _ = c.rk_step(U, T / nst)
    pe = list(p); pe[6] = T
    Ue = c.cell_average("density_wave", pe)
    vol, _, _ = c.geometry()
    return float((np.abs(U[0] - Ue[0]) * vol).sum() / vol.sum())


def _vortex_error(n, order, scheme, T=0.1):
    nodes, cells, box = I.hex_lattice((n, n, 5), (10.0, 10.0, 50.0 / n))
    c = O.Case(nodes, cells, box, O.Params(order=order, scheme=scheme, Re=0.0))
    p = [5.0, 1.0, 5.0, 5.0, 0.5, 0.5, 0.0, 1.4]
    U = c.cell_average("vortex", p)
    nst = int(math.ceil(T / c.time_step(U)))
    for _ in range(nst):
        U, _ = c.rk_step(U, T / nst)
    pe = list(p); pe[6] = T
    Ue = c.cell_average("vortex", pe)
    vol, _, _ = c.geometry()
    return float((np.abs(U[0] - Ue[0]) * vol).sum() / vol.sum())


@pytest.mark.parametrize("order,scheme,lo", [(1, 0, 1.9), (2, 0, 2.75)])
def test_order_density_wave(order, scheme, lo):
    """Smooth density wave advected by a uniform flow (exact Euler
    solution): L1 error order -> 2 (P1), -> 3 (P2)."""
    e = [_density_wave_error(n, order, scheme) for n in (8, 16, 32)]
    assert math.log2(e[1] / e[2]) > lo


def test_order_density_wave_pyramids_p1():
    """P1 on pyramids (n = 4, 8, 16): rates 0.96 -> 1.17, rising like the
    other diagonal splits' (the unjittered lattice's pyramid stencils are
    rank-deficient at P2, see above)."""
    e = [_density_wave_error(n, 1, 0, split=I.split_pyramids) for n in (4, 8, 16)]
    rates = [math.log2(e[k] / e[k + 1]) for k in range(2)]
    assert rates[1] > rates[0] and rates[1] > 1.1, rates


@pytest.mark.parametrize("order,lo", [(1, 1.4), (2, 2.4)])
def test_order_density_wave_prisms(order, lo):
    """The density wave on prisms (each lattice hexahedron split along one
    diagonal, n = 8, 16, 32): the L1 error falls at rates that rise with
    resolution, P1 1.30 -> 1.43 and P2 2.41 -> 2.46, like the tetrahedral
    split's (P1 1.19 -> 1.43, P2 2.08 -> 2.32) and below the lattice's 2 and
    3 at these sizes: the diagonal splits' one-sided stencils are still
    pre-asymptotic there."""
    e = [_density_wave_error(n, order, 0, split=I.split_prisms) for n in (8, 16, 32)]
    rates = [math.log2(e[k] / e[k + 1]) for k in range(2)]
    assert rates[1] > rates[0] and rates[1] > lo, rates


@pytest.mark.slow
@pytest.mark.parametrize("order,scheme,lo", [(1, 0, 1.9), (2, 0, 2.6), (2, 1, 2.6)])
def test_order_isentropic_vortex(order, scheme, lo):
    """Isentropic vortex advected through a periodic box (exact Euler
    solution; core radius 1, box 10): L1 density error order between
    n = 32 and 64 near 2 (P1) and 3 (P2 linear and CWENOZ)."""
    e = [_vortex_error(n, order, scheme) for n in (32, 64)]
    assert math.log2(e[0] / e[1]) > lo


# ------------------------------------------------------ CWENOZ behaviour ---
def test_cwenoz_weights_worked_example():
    """The CWENOZ weights (Eq. 6 as printed, tau the mean |SI_1 - SI_s|) on a
    closed-form example: U = (x - x_i)^2 on a uniform lattice of spacing h
    (cell averages (x - x_i)^2 + h^2/12), P2.  The central polynomial is exact,
    SI_1 = V^(-1/3) int (2x)^2 + V^(1/3) int 2^2 = h^4 (1/3 + 4).  The linear
    directional candidate of face +x fits the differences a^2 h^2 of its six
    cells (offsets (1,0,0), (2,0,0), (1,+-1,0), (1,0,+-1) in h) with
    gradient 13 h / 9 (normal equations diag(9, 2, 2), right side 13 h^2),
    SI = 169 h^4 / 81; those of the y and z faces (offsets (0,1,0), (+-1,1,0),
    (0,2,0), (0,1,+-1)) have gradient 2 h / 9, SI = 4 h^4 / 81; -x, -y, -z
    mirror them.  The weights follow from these by Eq. 6 with lambda =
    (1000, 1, ..., 1)/1006 and eps = 1e-6."""
    n = 8
    h = 2 * math.pi / n
    nodes, cells, box = I.hex_lattice(n)
    c = O.Case(nodes, cells, box, O.Params(order=2, scheme=1))
    xm = I.cell_vertex_means(nodes, cells)
    i = 4 + n * (4 + n * 4)  # a central cell: its stencils do not reach the periodic seam
    u = (xm[:, 0] - xm[i, 0]) ** 2 + h * h / 12.0
    _, w = c.reconstruct(np.tile(u, (5, 1)), weights=True)
    S0, Sx, Syz = h ** 4 * (1 / 3 + 4), 169 * h ** 4 / 81, 4 * h ** 4 / 81
    S = np.array([S0, Sx, Sx, Syz, Syz, Syz, Syz])  # central, then faces -x, +x, -y, +y, -z, +z
    lam = np.array([1000.0] + [1.0] * 6) / 1006.0
    tau = np.abs(S0 - S[1:]).mean()
    wt = lam * (1.0 + tau / (1e-6 + S))
    wt /= wt.sum()
    for v in range(5):
        assert np.abs(w[i, v] - wt).max() <= 1e-13, (w[i, v], wt)


def test_cwenoz_weights_normalised_and_tend_to_linear():
    """Eq. 5: the nonlinear weights are positive and sum to one; on smooth
    data they approach the linear weights as the mesh is refined (mean
    deviation; the maximum sits at critical points of the field)."""
    dev = []
    for n in (8, 16):
        nodes, cells, box = I.hex_lattice(n)
        c = O.Case(nodes, cells, box, O.Params(order=2, scheme=1))
        U = c.cell_average("tgv", [0.3, 1.4])
        _, w = c.reconstruct(U, weights=True)
        assert np.all(w > 0)
        assert np.abs(w.sum(axis=2) - 1.0).max() < 1e-14
        lam = np.array([1000.0] + [1.0] * 6) / 1006.0
        dev.append(np.abs(w - lam).mean())
    assert dev[1] < 0.4 * dev[0]  # mean deviation falls ~h^2


def test_cwenoz_step_is_non_oscillatory():
    """A density step: the linear P2 reconstruction overshoots the jump at
    the face points next to it; CWENOZ shifts weight to the smooth
    directional candidates and stays close to the range of the data."""
    n = 10
    nodes, cells, box = I.hex_lattice(n)
    over = {}
    for scheme in (0, 1):
        c = O.Case(nodes, cells, box, O.Params(order=2, scheme=scheme))
        vol, cen, hh = c.geometry()
        U = np.zeros((5, c.n_cells))
        U[0] = np.where(cen[:, 0] < math.pi, 1.0, 2.0)
        U[4] = 2.5
        worst = 0.0
        for i in np.where(np.abs(cen[:, 0] - math.pi) < 0.7 * hh[0])[0][:10]:
            x = cen[i] + np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]]) * hh[i]
            val, _ = c.eval(U, int(i), x)
            worst = max(worst, val[:, 0].max() - 2.0, 1.0 - val[:, 0].min())
        over[scheme] = worst
        if scheme == 1:
            _, w = c.reconstruct(U, weights=True)
            i = int(np.where(np.abs(cen[:, 0] - math.pi) < 0.7 * hh[0])[0][0])
            assert w[i, 0, 0] < 0.5  # central candidate loses its weight at the step
    assert over[0] > 0.05
    assert over[1] < 0.2 * over[0]


def test_cfl_time_step_closed_form():
    """Uniform state on a uniform cube lattice: h_i = 2|V|/sum|S_f| = side/3 and
    dt = CFL min(h/(|u|+a), rho h^2 Pr/(2 gamma mu))."""
    n = 8
    nodes, cells, box = I.hex_lattice(n)
    c = O.Case(nodes, cells, box, O.Params(order=1, scheme=0, Re=1600.0, cfl=0.5))
    U = np.zeros((5, c.n_cells))
    r, u, p = 1.3, np.array([0.4, -0.1, 0.2]), 0.9
    U[0] = r
    U[1:4] = (r * u)[:, None]
    U[4] = p / 0.4 + 0.5 * r * u @ u
    h = 2 * math.pi / n / 3
    a = math.sqrt(1.4 * p / r)
    conv, visc = h / (np.linalg.norm(u) + a), r * h * h * 0.71 / (2 * 1.4 / 1600.0)
    assert conv < visc
    assert math.isclose(c.time_step(U), 0.5 * conv, rel_tol=1e-13)
    # Re = 1: the viscous limit binds
    c = O.Case(nodes, cells, box, O.Params(order=1, scheme=0, Re=1.0, cfl=0.5))
    visc = r * h * h * 0.71 / (2 * 1.4 / 1.0)
    assert visc < conv
    assert math.isclose(c.time_step(U), 0.5 * visc, rel_tol=1e-13)
