"""GPU parity: libucns (CUDA, through the C ABI) against the CPU oracle on the
same seeded inputs.

Bar (FP64 path), per conserved component c, 1e-12 relative:
    max_i |R_gpu,ic - R_cpu,ic| / max_i S_ic <= 1e-12,
where S_ic = (1/|V_i|) sum_f |G_fc| is the magnitude of the face-flux
integrals whose signed sum is R_ic (Eq. 2).  The residual is a cancelling sum:
at Mach 0.1, R_rho is ~1e-2 of its terms, and perturbing the oracle's own input
by 1e-16 moves ||R_rho||_inf by ~5e-12 relative, so two correct FP64
implementations cannot agree to 1e-12 of ||R||_inf there; the rounding error of
a sum is bounded relative to the sum of |terms|, which is the scale used.
Where the residual is not dominated by cancellation the plain norm-wise
||R_gpu - R_cpu||_inf / ||R_cpu||_inf is checked at 1e-12 as well.  The
kinetic-energy history after 100 SSP-RK3 steps must agree within 1e-10
relative.  Sizes span many thread blocks with ragged tails; the full-size
64^3 jittered P2 CWENOZ residual is compared element by element.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2609_07387_gb300 import inputs as I
from paper_2609_07387_gb300 import ucns

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_R = 1e-12
TOL_KE = 1e-10


def _norm_err(a, b):
    den = np.abs(b).max(axis=1)
    return (np.abs(a - b).max(axis=1) / np.where(den > 0, den, 1.0))


def _term_err(a, b, S):
    """max |a - b| / max S per component (S: summed-term magnitudes)."""
    return np.abs(a - b).max(axis=1) / S.max(axis=1)


def _pair(nodes, cells, box, **kw):
    p = ucns.Params(**kw)
    op = O.Params(order=p.order, scheme=p.scheme, gamma=p.gamma, Pr=p.Pr, Re=p.Re, Mach=p.Mach, cfl=p.cfl,
                  lam_central=p.lam_central, eps=p.eps, alpha=p.alpha, integrator=p.integrator)
    return ucns.Mesh(nodes, cells, box, p), O.Case(nodes, cells, box, op)


def _gpu_residual(m, U_user):
    U = torch.from_numpy(np.ascontiguousarray(m.to_internal(U_user))).cuda()
    R = m.residual(U)
    torch.cuda.synchronize()
    return m.to_user(R.cpu().numpy())


CASES = [
    # name, lattice n, jitter, tets, order, scheme, Re, Mach, state
    ("C1_p1_uniform_16", 16, 0.0, False, 1, 0, 1600.0, 0.1, "tgv"),
    ("p1_jitter_13_inviscid", 13, 0.1, False, 1, 0, 0.0, 0.3, "noisy"),
    ("p2_linear_jitter_11", 11, 0.1, False, 2, 0, 1600.0, 0.1, "noisy"),
    ("p2_cwenoz_jitter_13", 13, 0.1, False, 2, 1, 1600.0, 0.1, "noisy"),
    ("p2_cwenoz_jitter_12_M125", 12, 0.1, False, 2, 1, 1600.0, 1.25, "perturbed"),
    ("p2_cwenoz_tets_6", 6, 0.1, True, 2, 1, 1600.0, 0.1, "noisy"),
    ("p2_cwenoz_tets_7_inviscid", 7, 0.1, True, 2, 1, 0.0, 0.5, "noisy"),
    # P3 / P4 (Sec. 2.2; Table 4 TGV-P3/P4): K = 19 / 34 modes over 38 / 68
    # members, 6 linear / 18-member quadratic directional candidates, 9 / 16
    # Gauss points per face; 10^3, 11^3 and 12^3 cells span many blocks with
    # ragged tails (the face kernel packs 3 / 2 faces per warp)
    ("p3_linear_jitter_10", 10, 0.1, False, 3, 0, 1600.0, 0.3, "noisy"),
    ("p3_cwenoz_jitter_11", 11, 0.1, False, 3, 1, 1600.0, 0.3, "noisy"),
    ("p3_cwenoz_jitter_10_M125", 10, 0.1, False, 3, 1, 1600.0, 1.25, "perturbed"),
    ("p4_linear_jitter_10_inviscid", 10, 0.1, False, 4, 0, 0.0, 0.3, "noisy"),
    ("p4_cwenoz_jitter_12", 12, 0.1, False, 4, 1, 1600.0, 0.3, "noisy"),
]


def _state(kind, nodes, cells, mach):
    if kind == "tgv":
        return I.tgv_state(nodes, cells, mach)
    if kind == "noisy":
        return I.noisy_state(nodes, cells, mach, 0.05, seed=3)
    return I.tgv_perturbed_state(nodes, cells, mach, 0.05, seed=4)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_residual_parity(case):
    name, n, jit, tets, order, scheme, Re, M, st = case
    nodes, cells, box = I.hex_lattice(n, jitter=jit, seed=5)
    if tets:
        cells = I.split_tets(cells)
    m, oc = _pair(nodes, cells, box, order=order, scheme=scheme, Re=Re, Mach=M)
    U = _state(st, nodes, cells, M)
    Rg = _gpu_residual(m, U)
    Rc, S = oc.residual_terms(U)
    err = _term_err(Rg, Rc, S)
    assert np.all(err <= TOL_R), err
    # well-conditioned components (|R| not << its terms) also norm-wise
    cond = S.max(axis=1) / np.abs(Rc).max(axis=1)
    nerr = _norm_err(Rg, Rc)
    for c in range(5):
        if cond[c] < 30:
            assert nerr[c] <= TOL_R, (c, nerr, cond)


def test_residual_parity_full_size_64_cwenoz():
    """The benchmark workload itself: 64^3 jittered hexahedra, P2 CWENOZ,
    every one of the 5 x 262144 residual entries against the oracle."""
    nodes, cells, box = I.hex_lattice(64, jitter=0.1, seed=1)
    m, oc = _pair(nodes, cells, box, order=2, scheme=1, Re=1600.0, Mach=0.1)
    U = I.tgv_state(nodes, cells, 0.1)
    Rg = _gpu_residual(m, U)
    Rc, S = oc.residual_terms(U)
    err = _term_err(Rg, Rc, S)
    print("64^3 P2 CWENOZ FP64, per component: |dR|/max S", err, " |dR|/|R|", _norm_err(Rg, Rc),
          " max S/|R|", S.max(axis=1) / np.abs(Rc).max(axis=1))
    assert np.all(err <= TOL_R), err


def test_rk_steps_and_time_step_parity():
    """C1 configuration: 16^3 hexahedra, P1, 10 SSP-RK3 steps at CFL 0.5."""
    nodes, cells, box = I.hex_lattice(16)
    m, oc = _pair(nodes, cells, box, order=1, scheme=0, Re=1600.0, Mach=0.1, cfl=0.5)
    U0 = I.tgv_state(nodes, cells, 0.1)
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U0))).cuda()
    Uc = U0.copy()
    for _ in range(10):
        dtg = m.rk_step(Ug, return_dt=True)
        Uc, dtc = oc.rk_step(Uc, 0.0)
        assert dtg == dtc or abs(dtg - dtc) <= 1e-14 * dtc
    err = _norm_err(m.to_user(Ug.cpu().numpy()), Uc)
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("order,scheme,n,tets", [(1, 0, 12, False), (2, 1, 10, False), (2, 1, 6, True),
                                                (3, 1, 10, False), (4, 1, 10, False)])
def test_ssp54_steps_parity(order, scheme, n, tets):
    """The paper's fourth-order SSP scheme (integrator 1: SSP(5,4), five
    residual evaluations per step): 5 steps with the CFL time step on both
    sides from a noisy state; dt equal, the state within 1e-12 of the oracle's
    (norm-wise per component)."""
    nodes, cells, box = I.hex_lattice(n, jitter=0.1, seed=2)
    if tets:
        cells = I.split_tets(cells)
    m, oc = _pair(nodes, cells, box, order=order, scheme=scheme, Re=1600.0, Mach=0.1, cfl=0.5, integrator=1)
    U0 = I.noisy_state(nodes, cells, 0.1, 0.03, seed=5)
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U0))).cuda()
    Uc = U0.copy()
    for _ in range(5):
        dtg = m.rk_step(Ug, return_dt=True)
        Uc, dtc = oc.rk_step(Uc, 0.0)
        assert dtg == dtc or abs(dtg - dtc) <= 1e-14 * dtc
    err = _norm_err(m.to_user(Ug.cpu().numpy()), Uc)
    assert np.all(err <= 1e-12), err


def test_ssp54_mixed_history_vs_fp64():
    """SSP(5,4) in the mixed form against the FP64 form, 40 steps from the
    Taylor-Green state with the same dt sequence: kinetic energy and
    solenoidal dissipation within 1e-6 relative."""
    nodes, cells, box = I.hex_lattice(12, jitter=0.1, seed=1)
    m64 = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, precision=0, integrator=1))
    m32 = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, precision=1, integrator=1))
    U0 = np.ascontiguousarray(m64.to_internal(I.tgv_state(nodes, cells, 0.1)))
    a = torch.from_numpy(U0.copy()).cuda()
    b = torch.from_numpy(U0.copy()).cuda()
    worst = 0.0
    for step in range(40):
        dt = m64.time_step(a)
        m64.rk_step(a, dt=dt)
        m32.rk_step(b, dt=dt)
        if step % 10 == 9:
            d64, d32 = m64.diagnostics(a), m32.diagnostics(b)
            worst = max(worst, abs(d32["ke"] - d64["ke"]) / d64["ke"], abs(d32["eps_s"] - d64["eps_s"]) / d64["eps_s"])
    m32.check_state()
    assert worst <= 1e-6, worst


@pytest.mark.parametrize("order,scheme,n,jit", [(1, 0, 16, 0.0), (2, 1, 10, 0.1)])
def test_ke_history_100_steps(order, scheme, n, jit):
    """Kinetic-energy (and dissipation) history over 100 steps with the CFL
    time step on both sides: KE within 1e-10 relative at every step."""
    nodes, cells, box = I.hex_lattice(n, jitter=jit, seed=2)
    m, oc = _pair(nodes, cells, box, order=order, scheme=scheme, Re=1600.0, Mach=0.1, cfl=0.5)
    U0 = I.tgv_state(nodes, cells, 0.1)
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U0))).cuda()
    Uc = U0.copy()
    worst_ke = worst_es = 0.0
    for step in range(100):
        m.rk_step(Ug)
        Uc, _ = oc.rk_step(Uc, 0.0)
        if step % 10 == 9 or step == 99:
            dg = m.diagnostics(Ug)
            dc = oc.diagnostics(Uc)
            worst_ke = max(worst_ke, abs(dg["ke"] - dc[0]) / dc[0])
            worst_es = max(worst_es, abs(dg["eps_s"] - dc[1]) / dc[1])
    m.check_state()
    assert worst_ke <= TOL_KE, worst_ke
    assert worst_es <= 1e-9, worst_es


def test_diagnostics_and_time_step_parity():
    nodes, cells, box = I.hex_lattice(12, jitter=0.1, seed=7)
    m, oc = _pair(nodes, cells, box, order=2, scheme=1)
    U = I.noisy_state(nodes, cells, 0.1, 0.02, seed=1)
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U))).cuda()
    dg = m.diagnostics(Ug)
    dc = oc.diagnostics(U)
    assert abs(dg["ke"] - dc[0]) <= 1e-13 * dc[0]
    assert abs(dg["eps_s"] - dc[1]) <= 1e-11 * dc[1]
    assert abs(dg["eps_d"] - dc[2]) <= 1e-11 * max(dc[2], 1e-30)
    assert abs(dg["volume"] - (2 * math.pi) ** 3) <= 1e-12 * (2 * math.pi) ** 3
    dtg, dtc = m.time_step(Ug), oc.time_step(U)
    assert abs(dtg - dtc) <= 1e-14 * dtc  # per-cell limits round differently; the min is exact


@pytest.mark.parametrize("prec,integrator", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_multi_step_entry_point_equals_single_steps(prec, integrator):
    """ucns_rk_steps (several steps in one call; the mixed form carries its
    float pair of the state between them) gives the state and the simulated
    time of as many ucns_rk_step calls, bit for bit, with either integrator."""
    nodes, cells, box = I.hex_lattice(10, jitter=0.1, seed=9)
    m = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, precision=prec, integrator=integrator))
    U = np.ascontiguousarray(m.to_internal(I.noisy_state(nodes, cells, 0.1, 0.03, seed=4)))
    a = torch.from_numpy(U.copy()).cuda()
    b = torch.from_numpy(U.copy()).cuda()
    t = sum(m.rk_step(a, return_dt=True) for _ in range(4))
    tb = m.rk_steps(b, 4)
    assert torch.equal(a, b)
    assert tb == t or abs(tb - t) <= 1e-15 * t  # the device adds the same dts in the same order


@pytest.mark.parametrize("prec,integrator", [(0, 0), (1, 0), (1, 1)])
def test_resume_from_a_saved_state_is_bitwise(prec, integrator):
    """Checkpoint / resume: 3 steps, the state saved to the host and loaded
    into a freshly built mesh, 3 more steps there, equals 6 uninterrupted
    steps bit for bit (time included)."""
    nodes, cells, box = I.hex_lattice(10, jitter=0.1, seed=11)
    p = ucns.Params(order=2, scheme=1, precision=prec, integrator=integrator)
    m = ucns.Mesh(nodes, cells, box, p)
    U = np.ascontiguousarray(m.to_internal(I.noisy_state(nodes, cells, 0.1, 0.03, seed=6)))
    a = torch.from_numpy(U.copy()).cuda()
    ta = m.rk_steps(a, 6)
    b = torch.from_numpy(U.copy()).cuda()
    tb = m.rk_steps(b, 3)
    saved = b.cpu().numpy()
    m2 = ucns.Mesh(nodes, cells, box, p)
    c = torch.from_numpy(saved).cuda()
    tb += m2.rk_steps(c, 3)
    assert torch.equal(a, c)
    assert abs(ta - tb) <= 1e-15 * ta  # the same dts, summed in two groups


def test_deterministic_and_host_entry_point():
    nodes, cells, box = I.hex_lattice(14, jitter=0.1, seed=9)
    m = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1))
    U = np.ascontiguousarray(m.to_internal(I.noisy_state(nodes, cells, 0.1, 0.03, seed=2)))
    a = torch.from_numpy(U.copy()).cuda()
    b = torch.from_numpy(U.copy()).cuda()
    for _ in range(3):
        m.rk_step(a)
        m.rk_step(b)
    assert torch.equal(a, b)
    Ra, Rb = m.residual(a), m.residual(a)
    assert torch.equal(Ra, Rb)
    # host-buffer entry point = device entry point, bit for bit
    h = U.copy()
    t = m.rk_steps_host(h, 3)
    assert t > 0
    assert np.array_equal(h, a.cpu().numpy())


def test_nonphysical_state_reported():
    nodes, cells, box = I.hex_lattice(8)
    m = ucns.Mesh(nodes, cells, box, ucns.Params(order=1, scheme=0))
    U = np.ascontiguousarray(m.to_internal(I.tgv_state(nodes, cells, 0.1)))
    U[0, 17] = -1.0
    Ug = torch.from_numpy(U).cuda()
    with pytest.raises(ucns.UcnsError) as e:
        m.rk_step(Ug, return_dt=True)
    assert e.value.code == -5
    m.check_state()  # the error word was cleared


def test_physicality_test_near_zero_pressure():
    """The RK stage decides rho > 0, p > 0 in FP32 from the float pair where
    the sign of q = 2 rho E - |m|^2 has a margin of 2^-20 of 2 rho E, and in
    FP64 otherwise.  Cells at p = +-1e-8 of their kinetic energy (far inside
    that margin) after a step of dt = 1e-12: the positive ones are physical,
    a negative one is reported.  (FP64 form: the mixed form shares the test,
    but its FP32 flux cannot resolve such pressures against p_ref.)"""
    nodes, cells, box = I.hex_lattice(8)
    m = ucns.Mesh(nodes, cells, box, ucns.Params(order=1, scheme=0, precision=0))
    U = np.ascontiguousarray(m.to_internal(I.tgv_state(nodes, cells, 0.1)))

    def set_cell(i, delta):
        U[1, i], U[2, i], U[3, i] = 3.0 * U[0, i], -2.0 * U[0, i], 1.0 * U[0, i]
        ke2 = (U[1, i] ** 2 + U[2, i] ** 2 + U[3, i] ** 2) / U[0, i]  # |m|^2 / rho = 2 KE
        U[4, i] = 0.5 * ke2 * (1.0 + delta)

    for i in (3, 100, 400):
        set_cell(i, 1e-8)
    a = torch.from_numpy(U.copy()).cuda()
    m.rk_step(a, dt=1e-12)
    m.check_state()  # nothing reported
    assert torch.isfinite(a).all()
    set_cell(100, -1e-8)
    b = torch.from_numpy(U.copy()).cuda()
    m.rk_step(b, dt=1e-12)
    with pytest.raises(ucns.UcnsError) as e:
        m.check_state()
    assert e.value.code == -5
    m.check_state()  # the error word was cleared


def test_residual_requires_device_tensors():
    nodes, cells, box = I.hex_lattice(6)
    m = ucns.Mesh(nodes, cells, box, ucns.Params(order=1, scheme=0))
    with pytest.raises(ValueError):
        m.residual(torch.zeros(5, m.n_cells, dtype=torch.float64))


@pytest.mark.parametrize("Re", [1600.0, 1.0])
def test_time_step_equal_limits_and_low_pressure(Re):
    """The device reduction evaluates the FP64 limit only where an FP32
    estimate is near the block minimum or cannot be trusted; the result must
    still be the FP64 minimum: every cell on the same limit (uniform state on a
    regular lattice), the minimum in cells whose pressure is 1e-5 of their
    energy, and (Re = 1) viscous and convective limits of similar size."""
    nodes, cells, box = I.hex_lattice(12)
    m, oc = _pair(nodes, cells, box, order=1, scheme=0, Re=Re, Mach=0.1)
    n = len(cells)
    ones = np.ones(n)
    U = I.primitive_to_conserved(ones, 0.3 * ones, 0 * ones, 0 * ones, ones / (1.4 * 0.01))
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U))).cuda()
    assert abs(m.time_step(Ug) - oc.time_step(U)) <= 1e-14 * oc.time_step(U)
    rng = np.random.default_rng(3)
    fast = rng.choice(n, 40, replace=False)
    prim_u = 0.3 * ones
    prim_u[fast] = 50.0 + 1e-9 * np.arange(40)  # near-ties among the fast cells
    p = ones / (1.4 * 0.01)
    p[fast] = 1e-5 * 0.5 * 50.0 ** 2
    U = I.primitive_to_conserved(ones, prim_u, 0 * ones, 0 * ones, p)
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U))).cuda()
    dtg, dtc = m.time_step(Ug), oc.time_step(U)
    assert abs(dtg - dtc) <= 1e-14 * dtc
    # a cell with p < 0 (rho > 0) is reported
    U[4, fast[0]] = 0.5 * U[1, fast[0]] ** 2 / U[0, fast[0]] * (1 - 1e-9)
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U))).cuda()
    with pytest.raises(ucns.UcnsError) as e:
        m.time_step(Ug)
    assert e.value.code == -5
    m.check_state()


def test_bounded_wait_timeout_reaches_the_caller():
    """The give-up path of the bounded mbarrier waits, on a phase that
    nothing completes (no copy, no MMA in flight, a ~1 ms limit): the
    reconstruction's wait sets the mesh's error word, the call returns
    UCNS_ERR_TIMEOUT and clears it, and the mesh keeps working (a following
    check is clean and a residual matches the one before); the network's wait
    likewise through its own error word."""
    nodes, cells, box = I.hex_lattice(8, jitter=0.1, seed=2)
    m = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, precision=1))
    U = torch.from_numpy(np.ascontiguousarray(m.to_internal(I.tgv_state(nodes, cells, 0.1)))).cuda()
    R0 = m.residual(U).clone()
    lib = m._lib
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        assert lib.ucns_probe_bounded_wait(m._h, s) == -6  # UCNS_ERR_TIMEOUT
        assert "bounded wait" in lib.ucns_last_error().decode()
        m.check_state()  # cleared
    assert torch.equal(m.residual(U), R0)
    m.check_state()
    net = ucns.Net(seed=2)
    for _ in range(2):
        assert lib.ucns_mlp_probe_bounded_wait(net._h, s) == -6
        net.check()  # cleared
    X = torch.zeros((256, 32), dtype=torch.bfloat16, device="cuda")
    z = net.forward(X)
    net.check()
    assert torch.isfinite(z).all()


# ---- boundary faces and mixed elements (NEXT-3): prisms and pyramids in the
# periodic box, slip walls on z = 0 and z = L, supersonic inflow at x = 0 with
# outflow at x = L; inviscid wherever a boundary face exists
UINF = (1.4, 2.8, 0.0, 0.0, 5.3)  # Mach 2 (rho 1.4, u 2, p 1)
NEXT3 = [
    # name, element, boundary, lattice n, order, scheme, Re
    ("prism_p1", "prism", None, 7, 1, 0, 1600.0),
    ("prism_p2_cwenoz", "prism", None, 7, 2, 1, 1600.0),
    ("pyramid_p2_cwenoz", "pyramid", None, 5, 2, 1, 1600.0),
    ("walls_p1", "hex", "walls", 9, 1, 0, 0.0),
    ("walls_p2_cwenoz", "hex", "walls", 9, 2, 1, 0.0),
    ("walls_tets_p2_cwenoz", "tet", "walls", 6, 2, 1, 0.0),
    ("walls_prism_p2_cwenoz", "prism", "walls", 7, 2, 1, 0.0),
    ("inflow_outflow_p2_cwenoz", "hex", "inflow", 9, 2, 1, 0.0),
]


def _next3_mesh(element, boundary, n):
    nodes, cells, box = I.hex_lattice(n, jitter=0.1, seed=13)
    if element == "tet":
        cells = I.split_tets(cells)
    elif element == "prism":
        cells = I.split_prisms(cells)
    elif element == "pyramid":
        nodes, cells = I.split_pyramids(nodes, cells)
    if boundary == "walls":
        return nodes, cells, np.array([box[0], box[1], 0.0]), None
    if boundary == "inflow":
        return nodes, cells, np.array([0.0, box[1], box[2]]), (3, 2, 0, 0, 0, 0)
    return nodes, cells, box, None


@pytest.mark.parametrize("case", NEXT3, ids=[c[0] for c in NEXT3])
def test_boundaries_and_mixed_elements_parity(case):
    """The residual (1e-12 of the summed-term scale) and one SSP-RK3 step with
    the CFL time step (dt to 1e-14, the state to 1e-12 norm-wise) against the
    oracle: prisms and pyramids (5 faces and 5 directional candidates, bilinear
    quad and collapsed triangle faces in one mesh), boundary faces with the
    ghost state of their side's kind, one-sided stencils and no directional
    candidate across a boundary."""
    name, element, boundary, n, order, scheme, Re = case
    nodes, cells, box, bc = _next3_mesh(element, boundary, n)
    m = ucns.Mesh(nodes, cells, box, bc=bc, inflow=UINF if bc else None)
    m.precompute(ucns.Params(order=order, scheme=scheme, Re=Re, Mach=0.3))
    oc = O.Case(nodes, cells, box, O.Params(order=order, scheme=scheme, Re=Re, Mach=0.3, inflow=UINF,
                                            **({"bc": bc} if bc else {})))
    U = I.noisy_state(nodes, cells, 0.3, 0.05, seed=3)
    Rg = _gpu_residual(m, U)
    Rc, S = oc.residual_terms(U)
    err = _term_err(Rg, Rc, S)
    print(name, "residual err/S", err)
    assert np.all(err <= TOL_R), err
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U))).cuda()
    dtg = m.rk_step(Ug, return_dt=True)
    Uc, dtc = oc.rk_step(U, 0.0)
    assert abs(dtg - dtc) <= 1e-14 * dtc
    e2 = _norm_err(m.to_user(Ug.cpu().numpy()), Uc)
    assert np.all(e2 <= TOL_R), e2
