"""Mixed-precision form (FP32 pseudo-inverses, contractions and flux
arithmetic; FP64 stencil differences, RK accumulation and reductions):
its error against the FP64 oracle / FP64 GPU path, stated per quantity.

Bars: residual within 2e-5 of the summed-term scale S (the FP32 unit
roundoff is 6e-8, amplified by the O(1e2) flux-to-residual cancellation at
Mach 0.1); discrete conservation to FP64 round-off (the face totals and the
owner-side sum stay FP64); kinetic-energy and dissipation histories within
1e-4 relative of the FP64 path over 100 SSP-RK3 steps (the target accuracy
of the mixed form).
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_07387_gb300 import inputs as I
from paper_2609_07387_gb300 import ucns

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mesh(nodes, cells, box, prec, **kw):
    return ucns.Mesh(nodes, cells, box, ucns.Params(precision=prec, **kw))


@pytest.mark.parametrize("tets,mach,order,scheme,n", [
    (False, 0.1, 2, 1, 10), (False, 1.25, 2, 1, 10), (True, 0.1, 2, 1, 6),
    # 9^3 = 729 cells: 11 full tiles of 64 cells and a ragged one of 25
    (False, 0.1, 1, 0, 9), (False, 0.1, 2, 0, 9), (False, 1.25, 2, 1, 9),
    # P3 / P4 (thread-per-cell kernels, 3 / 2 faces per warp)
    (False, 0.3, 3, 1, 10), (False, 1.25, 3, 1, 10), (False, 0.3, 4, 0, 10), (False, 0.3, 4, 1, 11)])
def test_mixed_residual_error_vs_oracle(tets, mach, order, scheme, n):
    nodes, cells, box = I.hex_lattice(n, jitter=0.1, seed=5)
    if tets:
        cells = I.split_tets(cells)
    m = _mesh(nodes, cells, box, 1, Mach=mach, order=order, scheme=scheme)
    oc = O.Case(nodes, cells, box, O.Params(Mach=mach, order=order, scheme=scheme))
    U = I.tgv_perturbed_state(nodes, cells, mach, 0.05, seed=4)
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U))).cuda()
    R = m.to_user(m.residual(Ug).cpu().numpy())
    Rc, S = oc.residual_terms(U)
    err = np.abs(R - Rc).max(axis=1) / S.max(axis=1)
    print("mixed residual error / S:", err)
    assert np.all(err <= 2e-5), err
    vol, _, _ = oc.geometry()
    tot = np.abs((R * vol).sum(axis=1))
    assert np.all(tot <= 1e-12 * (S * vol).sum(axis=1)), tot


@pytest.mark.parametrize("order,n", [(2, 4), (2, 5), (2, 8), (1, 8), (1, 9)])
def test_mixed_face_batches(order, n):
    """The face kernel takes faces in batches (128 at P2, 512 at P1, 3 n^3 faces
    on the periodic lattice): one full batch and a part (P2, n = 4), a ragged
    last batch (P2 n = 5: 375 = 2 x 128 + 119; P1 n = 9), an exact multiple
    (n = 8: 1536 faces); each batch's distinct cells are copied once."""
    nodes, cells, box = I.hex_lattice(n, jitter=0.1, seed=7)
    m = _mesh(nodes, cells, box, 1, Mach=0.3, order=order, scheme=1 if order == 2 else 0)
    oc = O.Case(nodes, cells, box, O.Params(Mach=0.3, order=order, scheme=1 if order == 2 else 0))
    U = I.noisy_state(nodes, cells, 0.3, 0.05, seed=8)
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U))).cuda()
    R = m.to_user(m.residual(Ug).cpu().numpy())
    Rc, S = oc.residual_terms(U)
    err = np.abs(R - Rc).max(axis=1) / S.max(axis=1)
    print("faces", 3 * n ** 3, "mixed residual error / S:", err)
    assert np.all(err <= 2e-5), err


@pytest.mark.parametrize("order,steps", [(2, 100), (3, 40), (4, 20)])
def test_mixed_ke_and_dissipation_history_vs_fp64(order, steps):
    """16^3 jittered hexahedra, P2 (P3, P4) CWENOZ, TGV Mach 0.1: SSP-RK3 steps
    of the mixed form against the FP64 form from the same state with the same
    dt sequence."""
    nodes, cells, box = I.hex_lattice(16, jitter=0.1, seed=1)
    m64 = _mesh(nodes, cells, box, 0, order=order)
    m32 = _mesh(nodes, cells, box, 1, order=order)
    U0 = np.ascontiguousarray(m64.to_internal(I.tgv_state(nodes, cells, 0.1)))
    a = torch.from_numpy(U0.copy()).cuda()
    b = torch.from_numpy(U0.copy()).cuda()
    worst = {"ke": 0.0, "eps_s": 0.0, "eps_d": 0.0}
    for step in range(steps):
        dt = m64.time_step(a)
        m64.rk_step(a, dt=dt)
        m32.rk_step(b, dt=dt)
        if step % 10 == 9:
            d64, d32 = m64.diagnostics(a), m32.diagnostics(b)
            for k in worst:
                worst[k] = max(worst[k], abs(d32[k] - d64[k]) / abs(d64[k]))
    print("mixed vs fp64 history, worst relative:", worst)
    assert worst["ke"] <= 1e-4 and worst["eps_s"] <= 1e-4, worst
    assert worst["eps_d"] <= 1e-2, worst  # eps_d ~1e-8 of eps_s at Mach 0.1


def test_mixed_deterministic():
    nodes, cells, box = I.hex_lattice(12, jitter=0.1, seed=2)
    m = _mesh(nodes, cells, box, 1)
    U = np.ascontiguousarray(m.to_internal(I.noisy_state(nodes, cells, 0.1, 0.03, seed=1)))
    a = torch.from_numpy(U.copy()).cuda()
    b = torch.from_numpy(U.copy()).cuda()
    for _ in range(3):
        m.rk_step(a)
        m.rk_step(b)
    assert torch.equal(a, b)


def test_float_pair_equals_its_definition():
    """The float pair the mixed form's kernels form from bit patterns is
    hi = fl32(u), lo = fl32(u - hi) (round to nearest even) bit for bit:
    values over 40 decades of both signs, exact zeros, ties to even, values
    just below powers of two (hi rounds up across the binade), the largest
    finite floats and the rounding to infinity, FP32 denormals, random bit
    patterns over the whole exponent range, and the documented lo = 0 below
    2^-74 and where hi is infinite."""
    rng = np.random.default_rng(12)
    bits = rng.integers(0, 2 ** 63, 100000, dtype=np.int64).view(np.float64)
    bits = bits[~np.isnan(bits)] * rng.choice([-1.0, 1.0], 100000)[: (~np.isnan(bits)).sum()]
    u = np.concatenate([
        rng.normal(size=200000) * 10.0 ** rng.integers(-20, 20, 200000),
        np.array([0.0, -0.0, 1.0, -1.0, 1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, -(1 + 2.0 ** -24), 2 - 2.0 ** -30,
                  np.nextafter(4.0, 0.0), 178.57142857142858, 3.0e38, -3.0e38, 2.0 ** -74, 2.0 ** -73, 1e-30,
                  2.0 ** 127, np.nextafter(2.0 ** 128, 0.0), -np.nextafter(2.0 ** 128, 0.0), 2.0 ** 128, 1e39,
                  float(np.finfo(np.float32).max) * (1 + 2.0 ** -25), -float(np.finfo(np.float32).max),
                  1e-40, -1e-42, 2.0 ** -75, np.inf, -np.inf, 1e300, -1e-300]),
        bits,  # random bit patterns (NaN left out) across the whole exponent range
    ])
    hi, lo = ucns.float_pair(torch.from_numpy(u).cuda())
    hi, lo = hi.cpu().numpy(), lo.cpu().numpy()
    with np.errstate(over="ignore"):
        hi_ref = u.astype(np.float32)
    with np.errstate(invalid="ignore", over="ignore"):
        lo_ref = (u - hi_ref.astype(np.float64)).astype(np.float32)
    lo_ref[(np.abs(u) < 2.0 ** -74) | ~np.isfinite(hi_ref)] = 0.0
    assert np.array_equal(hi.view(np.uint32), hi_ref.view(np.uint32))
    assert np.array_equal(lo.view(np.uint32) & 0x7fffffff, lo_ref.view(np.uint32) & 0x7fffffff)  # +-0 alike
    assert np.array_equal(lo, lo_ref)
