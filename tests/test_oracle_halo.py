"""Periodic wrap versus a two-subdomain split of the box (the host-side check
of what a halo exchange would carry; one GPU runs the whole periodic mesh).
The residual of a cell (Eq. 2) is a sum over its faces of fluxes between
reconstructions (Eqs. 3-6) of the cell and of its face neighbours, each from
its own central and directional stencils.  So the residual of the cells of
one slab depends only on the slab and a halo: the stencil members of the
slab's cells and of their face neighbours.  Setting every cell outside slab
and halo to another state must leave the slab's residual bit for bit
unchanged, and changing a halo cell must change it."""
import numpy as np

import oracle as O
from paper_2609_07387_gb300 import inputs as I


def _dependency_set(oc, cells_a):
    fo, fn, _ = oc.faces()
    nbr = [set() for _ in range(oc.n_cells)]
    for o, n in zip(fo, fn):
        nbr[o].add(int(n))
        nbr[n].add(int(o))
    members = {}

    def stencils(j):
        if j not in members:
            s = set(oc.stencil(j)[0].tolist())
            for w in range(oc.nd):
                s |= set(oc.stencil(j, w)[0].tolist())
            members[j] = s | {j}
        return members[j]

    dep = set(int(i) for i in cells_a)
    for i in cells_a:
        for j in {int(i)} | nbr[i]:
            dep |= stencils(j)
    return dep


def test_slab_residual_depends_only_on_slab_and_halo():
    nz = 24
    nodes, cells, box = I.hex_lattice((6, 6, nz), jitter=0.1, seed=3)
    oc = O.Case(nodes, cells, box, O.Params(order=2, scheme=1))
    _, cen, _ = oc.geometry()
    slab = np.where(cen[:, 2] < np.pi)[0]  # the lower half of the periodic box
    dep = _dependency_set(oc, slab)
    halo = np.array(sorted(dep - set(slab.tolist())))
    outside = np.array(sorted(set(range(oc.n_cells)) - dep))
    assert len(halo) > 0 and len(outside) > 0
    # the halo lies on both sides of the slab (across z = pi and across the periodic wrap),
    # a few cell layers deep
    hz = 2 * np.pi / nz
    zh = cen[halo, 2]
    assert np.any((zh > np.pi) & (zh < 2 * np.pi - 6 * hz)) and np.any(zh > 2 * np.pi - 6 * hz)
    assert np.all((np.abs(zh - np.pi) < 6 * hz) | (2 * np.pi - zh < 6 * hz))
    U = I.noisy_state(nodes, cells, 0.3, 0.05, seed=6)
    R = oc.residual_subset(U, slab)
    other = I.noisy_state(nodes, cells, 0.3, 0.05, seed=7)
    U_out = U.copy()
    U_out[:, outside] = other[:, outside]
    assert np.array_equal(oc.residual_subset(U_out, slab), R)
    U_halo = U.copy()
    U_halo[:, halo] = other[:, halo]
    assert not np.array_equal(oc.residual_subset(U_halo, slab), R)
