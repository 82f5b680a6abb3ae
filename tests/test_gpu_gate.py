"""The learned troubled-cell gate on the GPU: the tcgen05 network's logits
and gradients against the FP64 CPU reference (with the same BF16 rounding
points), training on a separable rule, the indicator features and labels
against the oracle, the gated residual at its two extremes (every cell
CWENOZ / every cell linear) against the ungated schemes, and at partial
masks (random, scattered, a trained network's) against the oracle's
residual under the same per-cell scheme mask."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as omlp
from paper_2609_07387_gb300 import inputs as I
from paper_2609_07387_gb300 import ucns

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bf16_tensor(X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda().to(torch.bfloat16).contiguous()


def _net_with(theta):
    net = ucns.Net(seed=0)
    net.set_params(theta.astype(np.float32))
    return net


def _bf16_up(a):
    """The next BF16 value above |a| (a: BF16 values, as float64)."""
    u = np.abs(np.asarray(a, dtype=np.float32)).view(np.uint32) + np.uint32(0x10000)
    return u.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("n", [128, 1000, 5000])
def test_mlp_forward_matches_reference(n):
    """Logits and the first hidden layer against the FP64 reference with the
    same BF16 rounding points.  The tensor cores accumulate W1 x in FP32, so
    an entry of h1 whose exact value lies next to a BF16 rounding midpoint may
    round to the other neighbour: every entry of the GPU's h1 equals the
    reference's, or is its BF16 neighbour with the exact pre-rounding value
    within FP32 accumulation error of the midpoint between them, and such
    flips are rare.  A row without a flip has the reference logit to 1e-5 of
    its summed-term magnitude; a row with flips to that plus the flipped
    entries' reach through W2 and w3."""
    rng = np.random.default_rng(n)
    theta = omlp.init(11).astype(np.float32).astype(np.float64)
    theta[2048:2112] = rng.normal(0, 0.1, 64)  # nonzero biases
    theta[6208:6272] = rng.normal(0, 0.1, 64)
    theta[6336] = 0.3
    X = omlp.bf16(rng.normal(size=(n, 32)))
    net = _net_with(theta)
    h1g, zg = net.hidden(_bf16_tensor(X))
    h1g = h1g.float().cpu().numpy().astype(np.float64)
    zg = zg.cpu().numpy().astype(np.float64)
    z2 = net.forward(_bf16_tensor(X)).cpu().numpy().astype(np.float64)
    net.check()
    assert np.array_equal(zg, z2)  # the read-back changes nothing
    th = theta.astype(np.float32).astype(np.float64)
    zr, act = omlp.forward(th, X, bf16_round=True)
    p = omlp.unflatten(th)
    W1r, W2r, w3r = omlp.bf16(p["W1"]), omlp.bf16(p["W2"]), omlp.bf16(p["w3"])
    a1, h1r = act["a1"], act["h1r"]
    flip = h1g != h1r
    # every flip is to the adjacent BF16 value, with the exact value within
    # 64 FP32 roundings of the terms' magnitude from the midpoint between them
    mag = np.abs(X) @ np.abs(W1r).T + np.abs(p["b1"])
    tol1 = 64 * 2.0 ** -24 * mag
    # at the ReLU's kink: one side 0, the other no larger than the FP32 error
    kink = flip & ((h1g == 0) | (h1r == 0))
    assert np.all(np.maximum(h1g, h1r)[kink] <= tol1[kink] + 1e-30)
    near = flip & ~kink
    if near.any():
        lo, hi = np.minimum(h1g, h1r)[near], np.maximum(h1g, h1r)[near]
        assert np.array_equal(_bf16_up(lo), hi)
        assert np.all(np.abs(a1[near] - 0.5 * (lo + hi)) <= tol1[near])
    rows = flip.any(axis=1)
    print(f"n={n}: BF16 flips in h1 {int(flip.sum())} of {flip.size} entries, in {int(rows.sum())} rows")
    assert flip.sum() <= max(4, 1e-3 * flip.size)
    # per-row magnitude of the terms summed into z: |w3| . (|W2| h1 + |b2|) + |b3|
    scale = (h1r @ np.abs(W2r).T + np.abs(p["b2"])) @ np.abs(w3r) + abs(p["b3"][0])
    err = np.abs(zg - zr)
    assert np.all(err[~rows] <= 1e-5 * scale[~rows]), (err[~rows] / scale[~rows]).max()
    if rows.any():
        reach = (np.abs(h1g - h1r) @ np.abs(W2r).T) @ np.abs(w3r)
        assert np.all(err[rows] <= 1e-5 * scale[rows] + reach[rows])


def test_mlp_gradient_matches_reference():
    """Every gradient entry against the FP64 reference fed the GPU's own BF16
    h1 (its rare accumulation flips, counted in the forward test, taken as
    they are), within 1e-4 of the magnitude of the per-sample terms summed
    into that entry: FP32 accumulation over the samples and the remaining
    BF16 roundings of dH2 and dH1 stay far below that, while a wrong operand
    tile or descriptor for a subset of rows or columns moves whole terms."""
    rng = np.random.default_rng(5)
    n = 3000
    theta = omlp.init(7).astype(np.float32).astype(np.float64)
    theta[2048:2112] = rng.normal(0, 0.1, 64)
    theta[6208:6272] = rng.normal(0, 0.1, 64)
    X = omlp.bf16(rng.normal(size=(n, 32)))
    y = (rng.random(n) > 0.7).astype(np.float64)
    net = _net_with(theta)
    g = net.grad(_bf16_tensor(X), torch.from_numpy(y).cuda(), 2.0, 0.6).cpu().numpy().astype(np.float64)
    h1g, _ = net.hidden(_bf16_tensor(X))
    net.check()
    h1g = h1g.float().cpu().numpy().astype(np.float64)
    gr = omlp.grad(theta, X, y, 2.0, 0.6, bf16_round=True, h1=h1g)
    T = omlp.grad(theta, X, y, 2.0, 0.6, bf16_round=True, h1=h1g, terms=True)
    for name, (a, b) in {"W1": (0, 2048), "b1": (2048, 2112), "W2": (2112, 6208), "b2": (6208, 6272),
                         "w3": (6272, 6336), "b3": (6336, 6337)}.items():
        live = T[a:b] > 0
        e = (np.abs(g[a:b] - gr[a:b])[live] / T[a:b][live]).max()
        print(f"gradient {name}: max |g - g_ref| / sum|terms| = {e:.2e}")
        assert e <= 1e-4, (name, e)
        assert np.all(g[a:b][~live] == 0.0)
    # the same call twice is bitwise identical (fixed-order reductions)
    g2 = net.grad(_bf16_tensor(X), torch.from_numpy(y).cuda(), 2.0, 0.6).cpu().numpy()
    assert np.array_equal(g.astype(np.float32), g2)


def test_mlp_training_learns_a_separable_rule():
    rng = np.random.default_rng(9)
    n = 16384
    X = omlp.bf16(rng.normal(size=(n, 32)))
    y = ((X[:, 0] + 0.5 * X[:, 5] - 0.25 * X[:, 9]) > 0).astype(np.float64)
    Xt, yt = _bf16_tensor(X), torch.from_numpy(y).cuda()
    net = ucns.Net(seed=3)
    l0 = omlp.loss(net.params().astype(np.float64), X, y)
    for _ in range(20):
        net.train(Xt, yt, batch=1024, lr=3e-3)
    net.check()
    th = net.params().astype(np.float64)
    assert omlp.loss(th, X, y) < 0.25 * l0
    z = net.forward(Xt).cpu().numpy()
    assert np.mean((z > 0) == (y > 0.5)) > 0.95


@pytest.mark.parametrize("prec", [0, 1])
def test_features_and_labels_match_oracle(prec):
    """FP64 form: features from FP64 differences; mixed form: from the float
    pair of the state in FP32 arithmetic (9^3 cells: a ragged last tile of the
    blocked layout).  Labels need the FP64 CWENOZ weights (FP64 form only)."""
    nodes, cells, box = I.hex_lattice(10 if prec == 0 else 9, jitter=0.1, seed=4)
    U = I.tgv_perturbed_state(nodes, cells, 1.25, 0.05, seed=4)
    m = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, Mach=1.25, precision=prec))
    oc = O.Case(nodes, cells, box, O.Params(order=2, scheme=1, Mach=1.25))
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U))).cuda()
    X, Xf = m.gate_features(Ug, want_f32=True)
    F = m.to_user(Xf.cpu().numpy().astype(np.float64).T).T
    Fo = oc.features(U)
    err = np.abs(F - Fo)
    assert err.max() <= 1e-4 * max(1.0, np.abs(Fo).max()), (err.max(axis=0))
    # BF16 rows are the rounded FP32 features
    Xb = m.to_user(X.float().cpu().numpy().astype(np.float64).T).T
    assert np.array_equal(Xb, omlp.bf16(F))
    if prec == 1:
        return
    dev = m.to_user(m.gate_labels(Ug).cpu().numpy().astype(np.float64)[None])[0]
    odev, _ = oc.labels(U)
    assert np.abs(dev - odev).max() <= 1e-6


@pytest.mark.parametrize("tets", [False, True])
def test_gated_residual_extremes_equal_the_plain_schemes(tets):
    """Hexahedra (6 directional stencils) and tetrahedra (4): a gate that flags
    every cell gives the ungated CWENOZ residual bit for bit, one that flags
    none the linear-weight residual, in the FP64 and the mixed form."""
    nodes, cells, box = I.hex_lattice(12 if not tets else 7, jitter=0.1, seed=6)
    if tets:
        cells = I.split_tets(cells)
    U = I.tgv_perturbed_state(nodes, cells, 1.25, 0.05, seed=2)
    for prec in (0, 1):
        mw = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, Mach=1.25, precision=prec))
        ml = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=0, Mach=1.25, precision=prec))
        Ug = torch.from_numpy(np.ascontiguousarray(mw.to_internal(U))).cuda()
        Rw, Rl = mw.residual(Ug).clone(), ml.residual(Ug).clone()
        net = ucns.Net(seed=1)
        mw.gate_attach(net, -1e30)  # every logit above: all cells CWENOZ
        mw.gate_enable(True)
        assert torch.equal(mw.residual(Ug), Rw)
        assert mw.gate_flagged() == mw.n_cells
        mw.gate_attach(net, 1e30)   # none above: all cells linear weights
        assert torch.equal(mw.residual(Ug), Rl)
        assert mw.gate_flagged() == 0
        mw.gate_enable(False)
        assert torch.equal(mw.residual(Ug), Rw)
        net.check()


# ---- the gated residual at partial masks against the oracle's masked scheme
TOL_FP64 = 1e-12  # of the summed-term scale S, as in the FP64 parity tests
TOL_MIXED = 2e-5  # of S, as in the mixed-form tests

MASK_MESHES = [
    # name, lattice n, tets: 9^3 = 729 cells (11 tiles of 64 and a ragged one
    # of 25), 13^3 = 2197 (34 and a ragged 21), 6 * 6^3 = 1296 tets (20 and 16)
    ("hex9", 9, False), ("hex13", 13, False), ("tets6", 6, True),
]


def _masked_case(n, tets):
    nodes, cells, box = I.hex_lattice(n, jitter=0.1, seed=7)
    if tets:
        cells = I.split_tets(cells)
    oc = O.Case(nodes, cells, box, O.Params(order=2, scheme=1, Re=1600.0, Mach=0.3))
    # Taylor-Green at Mach 0.3 with seeded 5 % noise inside a ball at the box
    # centre: 40-70 % of the cells troubled by the label rule
    _, cen, _ = oc.geometry()
    blob = np.linalg.norm(cen - np.pi, axis=1) < 1.6
    U = np.where(blob[None], I.noisy_state(nodes, cells, 0.3, 0.05, seed=8), I.tgv_state(nodes, cells, 0.3))
    return nodes, cells, box, np.ascontiguousarray(U), oc


def _mask(kind, N, rng):
    if kind == "random30":
        return rng.random(N) < 0.3
    m = np.zeros(N, dtype=bool)  # "scattered": a handful of isolated cells, the first and last among them
    m[rng.choice(N, 7, replace=False)] = True
    m[0] = m[N - 1] = True
    return m


def _trained_flags(nodes, cells, box, U, mesh):
    """The flags a network trained on this case's own labels gives U: labels
    and features of 3 snapshots of plain FP64 CWENOZ steps, 30 epochs, the
    threshold for recall 0.99 on the first snapshot."""
    from paper_2609_07387_gb300 import gate

    m64 = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, Re=1600.0, Mach=0.3))
    Uc = torch.from_numpy(np.ascontiguousarray(m64.to_internal(U))).cuda()
    S = gate.collect(m64, Uc, 10, every=5)
    y = (S.dev > gate.LABEL_THRESHOLD).float()
    net = gate.train(S.X, y, epochs=30, lr=2e-3, batch=1024, seed=1)
    N = m64.n_cells
    thr = gate.threshold_for_recall(net, S.X[:N].contiguous(), y[:N].contiguous(), 0.99)
    mesh.gate_attach(net, thr)
    mesh.gate_enable(True)
    return net


@pytest.mark.parametrize("mesh_case", MASK_MESHES, ids=[c[0] for c in MASK_MESHES])
@pytest.mark.parametrize("mask_kind", ["random30", "scattered", "network"])
def test_gated_residual_partial_mask_matches_oracle(mesh_case, mask_kind):
    """Every timed learned step routes a ragged subset of cells through the
    gated kernels (FP64: a per-cell branch; mixed: the tile's linear phase,
    then the flagged cells compacted in shared memory, a warp each).  Here
    the gated residual is compared element by element with the oracle's
    residual under the same per-cell scheme mask (Sec. 2.2, Eqs. 5-6) for a
    seeded random 30 % mask, a few scattered cells, and the mask of a network
    trained on the case (its flags read back from the library); FP64 at
    1e-12 of the summed-term scale, mixed at 2e-5 of it."""
    name, n, tets = mesh_case
    nodes, cells, box, U, oc = _masked_case(n, tets)
    rng = np.random.default_rng(n + (7 if tets else 0))
    for prec, tol in ((0, TOL_FP64), (1, TOL_MIXED)):
        m = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, Re=1600.0, Mach=0.3, precision=prec))
        Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U))).cuda()
        if mask_kind == "network":
            net = _trained_flags(nodes, cells, box, U, m)
            R = m.residual(Ug).clone()  # the network evaluates its flags on U
            flags = m.gate_flags().cpu().numpy().astype(bool)
            net.check()
            mask = flags[m.iperm]  # internal -> caller's order
        else:
            mask = _mask(mask_kind, m.n_cells, rng)
            m.gate_set_flags(torch.from_numpy(mask[m.perm].astype(np.uint8)).cuda())
            R = m.residual(Ug).clone()
            assert np.array_equal(m.gate_flags().cpu().numpy().astype(bool), mask[m.perm])
        assert 0 < mask.sum() < m.n_cells, mask.sum()
        assert m.gate_flagged() == int(mask.sum())
        oc.set_scheme_mask(mask)
        Rc, S = oc.residual_terms(U)
        Rg = m.to_user(R.cpu().numpy())
        err = np.abs(Rg - Rc).max(axis=1) / S.max(axis=1)
        print(name, mask_kind, "precision", prec, "flagged", int(mask.sum()), "of", m.n_cells, "err/S", err)
        assert np.all(err <= tol), (prec, err)
        # the mask matters: the linear and the CWENOZ residuals both differ from it
        oc.set_scheme_mask(None)
        Rw = oc.residual(U)
        oc.set_scheme_mask(np.zeros(m.n_cells))
        Rl = oc.residual(U)
        oc.set_scheme_mask(None)
        assert np.abs(Rw - Rc).max() > 1e3 * TOL_FP64 * S.max() and np.abs(Rl - Rc).max() > 1e3 * TOL_FP64 * S.max()


@pytest.mark.parametrize("tets", [False, True])
def test_gated_rk_step_partial_mask_matches_oracle(tets):
    """One SSP-RK3 step with fixed dt under a seeded random mask (the gate's
    flags serve all three stages): FP64 within 1e-12 of the oracle's masked
    step (norm-wise per component), and the caller's flags leave the plain
    scheme in place once cleared."""
    nodes, cells, box, U, oc = _masked_case(7 if tets else 11, tets)
    m = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1, Re=1600.0, Mach=0.3))
    mask = np.random.default_rng(3).random(m.n_cells) < 0.4
    oc.set_scheme_mask(mask)
    dt = 0.5 * oc.time_step(U)
    Uc, _ = oc.rk_step(U, dt)
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U))).cuda()
    m.gate_set_flags(torch.from_numpy(mask[m.perm].astype(np.uint8)).cuda())
    m.rk_step(Ug, dt=dt)
    m.check_state()
    Ugu = m.to_user(Ug.cpu().numpy())
    err = np.abs(Ugu - Uc).max(axis=1) / np.abs(Uc).max(axis=1)
    assert np.all(err <= 1e-12), err
    m.gate_set_flags(None)
    oc.set_scheme_mask(None)
    Ug = torch.from_numpy(np.ascontiguousarray(m.to_internal(U))).cuda()
    Rg = m.to_user(m.residual(Ug).cpu().numpy())
    Rc, S = oc.residual_terms(U)
    assert np.all(np.abs(Rg - Rc).max(axis=1) / S.max(axis=1) <= TOL_FP64)
