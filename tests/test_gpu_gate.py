"""The learned troubled-cell gate on the GPU: the tcgen05 network's logits
and gradients against the FP64 CPU reference (with the same BF16 rounding
points), training on a separable rule, the indicator features and labels
against the oracle, and the gated residual at its two extremes (every cell
CWENOZ / every cell linear) against the ungated schemes."""
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


@pytest.mark.parametrize("n", [128, 1000, 5000])
def test_mlp_forward_matches_reference(n):
    rng = np.random.default_rng(n)
    theta = omlp.init(11).astype(np.float32).astype(np.float64)
    theta[2048:2112] = rng.normal(0, 0.1, 64)  # nonzero biases
    theta[6208:6272] = rng.normal(0, 0.1, 64)
    theta[6336] = 0.3
    X = omlp.bf16(rng.normal(size=(n, 32)))
    net = _net_with(theta)
    z = net.forward(_bf16_tensor(X)).cpu().numpy().astype(np.float64)
    net.check()
    zr, _ = omlp.forward(theta.astype(np.float32).astype(np.float64), X, bf16_round=True)
    err = np.abs(z - zr)
    assert np.median(err) <= 1e-4 * np.abs(zr).max(), np.median(err)
    assert err.max() <= 2e-2 * np.abs(zr).max(), err.max()


def test_mlp_gradient_matches_reference():
    rng = np.random.default_rng(5)
    n = 3000
    theta = omlp.init(7).astype(np.float32).astype(np.float64)
    theta[2048:2112] = rng.normal(0, 0.1, 64)
    theta[6208:6272] = rng.normal(0, 0.1, 64)
    X = omlp.bf16(rng.normal(size=(n, 32)))
    y = (rng.random(n) > 0.7).astype(np.float64)
    net = _net_with(theta)
    g = net.grad(_bf16_tensor(X), torch.from_numpy(y).cuda(), 2.0, 0.6).cpu().numpy().astype(np.float64)
    net.check()
    gr = omlp.grad(theta, X, y, 2.0, 0.6, bf16_round=True)
    for name, (a, b) in {"W1": (0, 2048), "b1": (2048, 2112), "W2": (2112, 6208), "b2": (6208, 6272),
                         "w3": (6272, 6336), "b3": (6336, 6337)}.items():
        e = np.abs(g[a:b] - gr[a:b]).max() / np.abs(gr[a:b]).max()
        assert e <= 2e-2, (name, e)
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
