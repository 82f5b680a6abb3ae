"""Full-size configurations, compared on sampled cells (the oracle computes
the residual of a sample of cells with the same arithmetic as its full
residual): the 6 x 96^3 = 5,308,416-tetrahedron Taylor-Green mesh (FP64 and
mixed) and the 128^3 Mach 1.25 perturbed Taylor-Green mesh (FP64 and mixed),
in the launch configuration the solver uses."""
import numpy as np
import pytest

import oracle as O
from paper_2609_07387_gb300 import inputs as I
from paper_2609_07387_gb300 import ucns

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _sampled(m, oc, U, name, n_sample=3000, seed=0):
    """max |dR| / max S per component over the sample; prints it with the
    norm-wise |dR| / |R| and the sample's S / |R|."""
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(m.n_cells, n_sample, replace=False))
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U))).cuda()
    R = m.residual(Ug)
    torch.cuda.synchronize()
    Rg = R[:, torch.from_numpy(m.iperm[sel]).cuda()].cpu().numpy()
    Rc, S = oc.residual_subset_terms(U, sel)
    d = np.abs(Rg - Rc).max(axis=1)
    err = d / S.max(axis=1)
    print(name, "per component: |dR|/max S", err, " |dR|/|R|", d / np.abs(Rc).max(axis=1),
          " max S/|R|", S.max(axis=1) / np.abs(Rc).max(axis=1))
    return err


def test_c3_tetrahedra_full_size():
    nodes, hexes, box = I.hex_lattice(96, jitter=0.1, seed=2)
    cells = I.split_tets(hexes)
    assert len(cells) == 5308416
    U = I.tgv_state(nodes, cells, 0.1)
    oc = O.Case(nodes, cells, box, O.Params(order=2, scheme=1, Mach=0.1))
    m = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, Mach=0.1, precision=0))
    err = _sampled(m, oc, U, "C3 FP64")
    assert np.all(err <= 1e-12), err
    del m
    mm = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, Mach=0.1, precision=1))
    err = _sampled(mm, oc, U, "C3 mixed")
    assert np.all(err <= 2e-5), err


def test_c4_mach125_full_size():
    nodes, cells, box = I.hex_lattice(128, jitter=0.1, seed=3)
    U = I.tgv_perturbed_state(nodes, cells, 1.25, 0.05, seed=4)
    oc = O.Case(nodes, cells, box, O.Params(order=2, scheme=1, Mach=1.25))
    m = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, Mach=1.25, precision=0))
    err = _sampled(m, oc, U, "C4 FP64")
    assert np.all(err <= 1e-12), err
    del m
    mm = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, Mach=1.25, precision=1))
    err = _sampled(mm, oc, U, "C4 mixed")
    assert np.all(err <= 2e-5), err
