"""bench.py's per-launch algorithmic counts on CPU, against the per-unit
figures the roofline states: the P2 mixed face kernel reads 24 bytes per
Gauss point (offset and area vector), 44 per face (centroid offset, penalty,
two ids, five FP32 totals) and 200 per cell (its 50 FP32 coefficients once);
the FP64 form twice the words; the mixed P3/P4 reconstruction's algorithmic
bytes equal its tile records (ids, FP32 pseudo-inverses, smoothness
matrices), and the roofline names the kernel that ran."""
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _mesh(K, Mc, nd, Md, nq, N=1000, F=3000):
    return SimpleNamespace(K=K, Mc=Mc, nd=nd, Md=Md, nq=nq, n_cells=N, n_faces=F)


def test_p2_face_bytes_per_unit():
    m = _mesh(9, 18, 6, 6, 4)
    a = bench.algorithmic(m, "face", mixed=True)
    assert a["alg"] == m.n_faces * (4 * 24 + 44) + m.n_cells * 200
    b = bench.algorithmic(m, "face", mixed=False)
    # FP64: the words double, the ids and the penalty factor do not
    assert b["alg"] == m.n_faces * (4 * 48 + 24 + 12 + 40) + m.n_cells * 400
    assert a["flops"] == b["flops"] == bench.FLOPS_FACE_P2_VISC_PER_QP * 4 * m.n_faces


def test_p2_recon_bytes_gated_and_full():
    m = _mesh(9, 18, 6, 6, 4)
    full = bench.algorithmic(m, "recon", mixed=True, frac_dir=1.0)
    lin = bench.algorithmic(m, "recon", mixed=True, frac_dir=0.0)
    per_cell_lin = 9 * 18 * 4 + 18 * 4 + 7 * 4 + 40 + 200
    assert lin["alg"] == m.n_cells * per_cell_lin
    assert full["alg"] - lin["alg"] == m.n_cells * (6 * 3 * 6 * 4 + 6 * 6 * 4)


def test_ho_mixed_recon_bytes_are_the_tile_records():
    # floats per 64-cell tile with CWENOZ (central chunks, smoothness matrix,
    # directional chunks), as the library lays them out
    tiles = {3: 19 * (2 * 64 + 19 * 2 * 64) + 190 * 64 + 6 * (6 * 64 + 3 * 6 * 64),
             4: 17 * (4 * 64 + 34 * 4 * 64) + 595 * 64 + 18 * (6 * 64 + 9 * 6 * 64)}
    for order, (K, Mc, Md) in {3: (19, 38, 6), 4: (34, 68, 18)}.items():
        m = _mesh(K, Mc, 6, Md, order * order, N=64)
        a = bench.algorithmic(m, "recon", mixed=True)
        rest = (K - 3) * 4 + 4 + 5 * 8 + (K + 1) * 5 * 4  # monomial means, 1/h, state, coefficients
        assert a["alg"] - m.n_cells * rest == tiles[order] * 4


def test_roofline_names_the_kernel_that_ran():
    peaks = {"hbm": 6800.0, "hbm_source": "test", "fp32": 80.0, "fp64": 1.0}
    prof = {"recon": (1.0, 1), "face": (2.0, 1)}
    for K, Mc, Md, nq, name in ((9, 18, 6, 4, "k_face_mx<2,true>"), (19, 38, 6, 9, "k_face_mx<3,true>"),
                                (34, 68, 18, 16, "k_face_mx<4,true>")):
        r = bench.roofline(_mesh(K, Mc, 6, Md, nq), prof, "mixed", peaks, "c5")
        assert r["kernel"] == name
    r = bench.roofline(_mesh(34, 68, 6, 18, 16), {"recon": (3.0, 1), "face": (2.0, 1)}, "fp64", peaks, "c5")
    assert r["kernel"] == "k_recon_ho<4,true>"
