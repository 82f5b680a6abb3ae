"""CPU tests of libucns: the C ABI loads and exports every declared entry
point, argument and call-order errors come back as status codes, and the
host half of ucns_precompute (stencils + Householder-QR pseudo-inverses,
Eq. 4) agrees with the oracle's independent construction (modified
Gram-Schmidt on quadrature-built matrices).  No GPU is touched."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2609_07387_gb300 import inputs as I
from paper_2609_07387_gb300 import ucns

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "ucns.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ucns_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = ucns.load()
    names = _declared()
    assert "ucns_residual" in names and "ucns_rk_step" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(ucns.EXPORTS)


def test_error_codes_without_gpu():
    lib = ucns.load()
    nodes, cells, box = I.hex_lattice(4)
    with pytest.raises(ucns.UcnsError) as e:
        ucns.Mesh(nodes, cells[:, :3], box)  # no element has 3 nodes
    assert e.value.code == -1
    with pytest.raises(ucns.UcnsError) as e:
        ucns.Mesh(nodes, cells, np.array([box[0], -1.0, box[2]]))
    assert e.value.code == -1
    with pytest.raises(ucns.UcnsError) as e:  # an unknown boundary kind
        ucns.Mesh(nodes, cells, np.array([box[0], box[1], 0.0]), bc=[0, 0, 0, 0, 7, 0])
    assert e.value.code == -1
    with pytest.raises(ucns.UcnsError) as e:  # an inflow side without the inflow state
        ucns.Mesh(nodes, cells, np.array([0.0, box[1], box[2]]), bc=[3, 2, 0, 0, 0, 0])
    assert e.value.code == -1
    with pytest.raises(ucns.UcnsError) as e:  # boundary faces need an inviscid flow
        ucns.Mesh(nodes, cells, np.array([box[0], box[1], 0.0])).precompute_host(ucns.Params(order=1, scheme=0))
    assert e.value.code == -1
    with pytest.raises(ucns.UcnsError) as e:  # prisms are built in the FP64 form
        ucns.Mesh(nodes, I.split_prisms(cells), box).precompute_host(ucns.Params(order=2, precision=1))
    assert e.value.code == -1
    bad = cells.copy()
    bad[3, 2] = nodes.shape[0] + 7
    with pytest.raises(ucns.UcnsError) as e:
        ucns.Mesh(nodes, bad, box)
    assert e.value.code == -2
    # a lattice that is not periodic in z for the given box: unpaired faces
    with pytest.raises(ucns.UcnsError) as e:
        ucns.Mesh(nodes, cells, np.array([box[0], box[1], 2 * box[2]]))
    assert e.value.code == -2
    m = ucns.Mesh(nodes, cells, box)
    with pytest.raises(ucns.UcnsError) as e:
        m.stencil(0)
    assert e.value.code == -7
    # residual before precompute: call order error (checked before any CUDA use)
    rc = lib.ucns_residual(m._h, None, None, None)
    assert rc == -7
    with pytest.raises(ucns.UcnsError) as e:
        m.precompute_host(ucns.Params(order=5))
    assert e.value.code == -1
    with pytest.raises(ucns.UcnsError) as e:  # orders 3 and 4 on hexahedra only
        ucns.Mesh(nodes, I.split_tets(cells), box).precompute_host(ucns.Params(order=3))
    assert e.value.code == -1
    with pytest.raises(ucns.UcnsError) as e:
        m.precompute_host(ucns.Params(order=1, scheme=1))
    assert e.value.code == -1
    with pytest.raises(ucns.UcnsError) as e:
        m.precompute_host(ucns.Params(order=1, scheme=0, integrator=2))
    assert e.value.code == -1
    # 2 cells across a periodic box: each face tuple appears 4 times (non-manifold)
    with pytest.raises(ucns.UcnsError) as e:
        ucns.Mesh(*I.hex_lattice(2))
    assert e.value.code == -2
    lib.ucns_mesh_destroy(None)  # NULL-safe


def test_cell_order_is_a_locality_permutation():
    nodes, cells, box = I.hex_lattice(16, jitter=0.1, seed=1)
    m = ucns.Mesh(nodes, cells, box)
    assert np.array_equal(np.sort(m.perm), np.arange(len(cells)))
    # Morton order: consecutive internal cells are close in space
    x = I.cell_vertex_means(nodes, cells)[m.perm]
    d = np.linalg.norm(np.diff(x, axis=0), axis=1)
    assert np.median(d) < 1.5 * (2 * np.pi / 16)


# basis monomials (exponents of x, y, z) in each side's row order: the
# library's as include/ucns.h states it, the oracle's as its source states it
_LIB_BASIS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1),
              (3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1), (0, 1, 2),
              (0, 0, 3), (4, 0, 0), (3, 1, 0), (3, 0, 1), (2, 2, 0), (2, 1, 1), (2, 0, 2), (1, 3, 0), (1, 2, 1),
              (1, 1, 2), (1, 0, 3), (0, 4, 0), (0, 3, 1), (0, 2, 2), (0, 1, 3), (0, 0, 4)]
_ORC_BASIS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1),
              (3, 0, 0), (0, 3, 0), (0, 0, 3), (2, 1, 0), (2, 0, 1), (1, 2, 0), (0, 2, 1), (1, 0, 2), (0, 1, 2),
              (1, 1, 1), (4, 0, 0), (0, 4, 0), (0, 0, 4), (3, 1, 0), (3, 0, 1), (1, 3, 0), (0, 3, 1), (1, 0, 3),
              (0, 1, 3), (2, 2, 0), (2, 0, 2), (0, 2, 2), (2, 1, 1), (1, 2, 1), (1, 1, 2)]


def _mesh_kind(kind, n, seed):
    """(nodes, cells, box, oracle params extra, library boundary kinds) of a test mesh."""
    nodes, cells, box = I.hex_lattice(n, jitter=0.1, seed=seed)
    if kind == "tet":
        cells = I.split_tets(cells)
    elif kind == "prism":
        cells = I.split_prisms(cells)
    elif kind == "pyramid":
        nodes, cells = I.split_pyramids(nodes, cells)
    if kind == "walls":  # z not periodic: slip walls on z = 0 and z = L
        return nodes, cells, np.array([box[0], box[1], 0.0]), {}, None
    if kind == "inflow":  # x not periodic: supersonic inflow at x = 0, outflow at x = L
        return nodes, cells, np.array([0.0, box[1], box[2]]), {"bc": (3, 2, 0, 0, 0, 0)}, [3, 2, 0, 0, 0, 0]
    return nodes, cells, box, {}, None


@pytest.mark.parametrize("kind,order,scheme", [("prism", 1, 0), ("prism", 2, 1), ("pyramid", 2, 1), ("walls", 2, 1),
                                               ("walls", 1, 0), ("inflow", 2, 1)])
def test_host_precompute_matches_oracle_mixed_elements_and_boundaries(kind, order, scheme):
    """Prisms, pyramids (5 faces, 5 directional candidates) and boxes with
    boundary faces: the library's stencils and pseudo-inverses equal the
    oracle's; a cell on a boundary has one-sided stencils and no directional
    candidate across the boundary."""
    nodes, cells, box, extra, bc = _mesh_kind(kind, 6 if kind != "pyramid" else 5, 12)
    re = 0.0 if kind in ("walls", "inflow") else 1600.0
    params = ucns.Params(order=order, scheme=scheme, Re=re)
    m = ucns.Mesh(nodes, cells, box, bc=bc, inflow=(1.4, 2.8, 0.0, 0.0, 5.3) if bc else None).precompute_host(params)
    oc = O.Case(nodes, cells, box, O.Params(order=order, scheme=scheme, Re=re,
                                            inflow=(1.4, 2.8, 0.0, 0.0, 5.3), **extra))
    assert (m.n_faces, m.K, m.Mc, m.nd, m.Md, m.nq, m.nfc) == (oc.n_faces, oc.K, oc.Mc, oc.nd, oc.Md, oc.nq, oc.nfc)
    rng = np.random.default_rng(1)
    fo, fn, _ = oc.faces()
    bcells = set(fo[fn < 0].tolist())
    sample = list(rng.choice(len(cells), size=10, replace=False)) + sorted(bcells)[:6]
    invalid = 0
    for i in sample:
        for which in [-1] + list(range(m.nd)):
            mem, P = m.stencil(int(i), which)
            try:
                omem, _, _, oP = oc.stencil(int(i), which)
            except O.OracleError:  # no candidate across a boundary face
                invalid += 1
                assert np.all(mem == i) and np.all(P == 0.0), (i, which)
                continue
            assert sorted(mem) == sorted(omem), (i, which)
            pos = {c: k for k, c in enumerate(omem)}
            oPm = oP[:, [pos[c] for c in mem]]
            assert np.abs(P - oPm).max() <= 1e-12 * np.abs(oPm).max(), (i, which)
    assert (invalid > 0) == (kind in ("walls", "inflow") and m.nd > 0)


@pytest.mark.parametrize("kind,order,scheme", [("hex", 1, 0), ("hex", 2, 1), ("tet", 2, 1), ("hex", 3, 1),
                                               ("hex", 4, 1)])
def test_host_precompute_matches_oracle(kind, order, scheme):
    """The library's host precompute (moment-form least-squares rows from each
    cell's central moments, Householder QR) against the oracle's (rows by
    quadrature, Gram-Schmidt QR): the same stencil members and the same
    pseudo-inverse P' = A^+ diag(|V_m|) of Eq. 4, row by row after matching the
    two bases' monomials, for central and directional stencils (P4: 18-member
    quadratic candidates)."""
    nodes, cells, box = I.hex_lattice(6 if kind == "hex" and order <= 2 else (8 if kind == "hex" else 5),
                                      jitter=0.1, seed=11)
    if kind == "tet":
        cells = I.split_tets(cells)
    params = ucns.Params(order=order, scheme=scheme)
    m = ucns.Mesh(nodes, cells, box).precompute_host(params)
    oc = O.Case(nodes, cells, box, O.Params(order=order, scheme=scheme))
    assert (m.n_faces, m.K, m.Mc, m.nd, m.Md, m.nq) == (oc.n_faces, oc.K, oc.Mc, oc.nd, oc.Md, oc.nq)
    rng = np.random.default_rng(0)
    for i in rng.choice(len(cells), size=12, replace=False):
        for which in [-1] + list(range(m.nd)):
            mem, P = m.stencil(int(i), which)
            omem, _, _, oP = oc.stencil(int(i), which)
            assert sorted(mem) == sorted(omem), (i, which)
            pos = {c: k for k, c in enumerate(omem)}
            rows = [_ORC_BASIS.index(e) for e in _LIB_BASIS[:P.shape[0]]]
            oPm = oP[rows][:, [pos[c] for c in mem]]
            assert np.abs(P - oPm).max() <= 1e-12 * np.abs(oPm).max(), (i, which, np.abs(P - oPm).max())


def test_product_path_never_touches_the_oracle():
    """The oracle is test infrastructure: no module of the package imports
    it, no library source names it, importing the package does not load it,
    and libucns.so neither exports nor needs one of its symbols."""
    import ast
    import subprocess
    import sys

    pkg = os.path.join(ROOT, "paper_2609_07387_gb300")
    for f in sorted(os.listdir(pkg)):
        if f.endswith(".py"):
            tree = ast.parse(open(os.path.join(pkg, f)).read())
            for node in ast.walk(tree):
                mods = [a.name for a in node.names] if isinstance(node, ast.Import) else \
                    [node.module or ""] if isinstance(node, ast.ImportFrom) else []
                assert not any(m.split(".")[0] == "oracle" for m in mods), (f, mods)
    csrc = os.path.join(pkg, "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".cpp", ".hpp", ".h", ".c")):
            txt = open(os.path.join(csrc, f)).read()
            assert "ucns_oracle" not in txt and not re.search(r"\borc_\w+\s*\(", txt), f
    code = "import sys, paper_2609_07387_gb300 as p; from paper_2609_07387_gb300 import gate, inputs; " \
           "p.load(); print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "False", r.stdout + r.stderr
    nm = subprocess.run(["nm", "-D", ucns.library_path()], capture_output=True, text=True)
    if nm.returncode == 0:
        assert not re.search(r"\borc_\w+", nm.stdout)


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="checks the behaviour without a CUDA device")
def test_compute_without_a_device_fails_loudly():
    """There is no CPU fallback: without a CUDA device the device half of
    ucns_precompute returns an error (its first device allocation fails, so
    the status is UCNS_ERR_NOMEM naming cudaMalloc, or UCNS_ERR_CUDA), the
    Python layer raises it, and the mesh stays unusable for compute calls."""
    m = ucns.Mesh(*I.hex_lattice(4))
    with pytest.raises(ucns.UcnsError) as e:
        m.precompute(ucns.Params())
    assert e.value.code in (-4, -8)
    assert m._lib.ucns_residual(m._h, None, None, None) != 0
