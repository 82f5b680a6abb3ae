"""What the learned indicator gains: Mach 1.25 Taylor-Green with a 5 %
random-phase perturbation on 48^3 jittered hexahedra (the 128^3
configuration scaled down).  Labels come from 30 plain FP64 CWENOZ steps;
the network is trained on the GPU (60 epochs); then 60 steps of plain FP64, mixed,
learned + mixed, all-linear + mixed and a hand-set jump rule + mixed run from
the same state with the same dt sequence.  The learned form must stay within
1e-4 of the plain FP64 kinetic-energy and dissipation history and beat plain
FP64 in time; the plain-scheme check must switch the gate off when its
bound is violated."""
import numpy as np
import pytest

from paper_2609_07387_gb300 import gate
from paper_2609_07387_gb300 import inputs as I
from paper_2609_07387_gb300 import ucns

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_SIDE, COLLECT, RUN = 48, 30, 60


@pytest.fixture(scope="module")
def setup():
    nodes, cells, box = I.hex_lattice(N_SIDE, jitter=0.1, seed=3)
    base = dict(order=2, scheme=1, Re=1600.0, Mach=1.25, cfl=0.5)
    m64 = ucns.Mesh(nodes, cells, box, ucns.Params(precision=0, **base))
    U0 = np.ascontiguousarray(m64.to_internal(I.tgv_perturbed_state(nodes, cells, 1.25, 0.05, seed=4)))
    U = torch.from_numpy(U0.copy()).cuda()
    S = gate.collect(m64, U, COLLECT, every=5)
    N = m64.n_cells
    y = (S.dev > gate.LABEL_THRESHOLD).float()
    net = gate.train(S.X[: 5 * N].contiguous(), y[: 5 * N].contiguous(), epochs=60, lr=1e-3, batch=4096, seed=0)
    thr = gate.threshold_for_recall(net, S.X[5 * N: 6 * N].contiguous(), y[5 * N: 6 * N].contiguous(), 0.999)
    held = gate.confusion(net, S.X[6 * N:].contiguous(), y[6 * N:].contiguous(), thr)
    return dict(nodes=nodes, cells=cells, box=box, base=base, m64=m64, U0=U0, net=net, thr=thr, held=held, y=y)


def _run(mesh, U0, dts, gated=False):
    U = torch.from_numpy(U0.copy()).cuda()
    hist = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for k, dt in enumerate(dts):
        e0.record()
        mesh.rk_step(U, dt=dt)
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        if k % 10 == 9:
            mesh.check_state()
            d = mesh.diagnostics(U)
            hist.append((d["ke"], d["eps_s"], d["eps_d"]))
    return np.array(hist), ms


def test_learned_gate_gain(setup):
    s = setup
    m64 = s["m64"]
    U = torch.from_numpy(s["U0"].copy()).cuda()
    dts = []
    for _ in range(RUN):
        dts.append(m64.time_step(U))
        m64.rk_step(U, dt=dts[-1])
    h64, ms64 = _run(m64, s["U0"], dts)
    mk = lambda **kw: ucns.Mesh(s["nodes"], s["cells"], s["box"], ucns.Params(**{**s["base"], **kw}))
    m32 = mk(precision=1)
    hmx, msmx = _run(m32, s["U0"], dts)
    g = gate.GatedRun(mk(precision=1), s["net"], s["thr"], check_every=50, bound=1e-3, eval_every=5)
    hlg, mslg = _run(g.mesh, s["U0"], dts)
    flagged = g.mesh.gate_flagged() / g.mesh.n_cells
    hlin, mslin = _run(mk(precision=1, scheme=0), s["U0"], dts)
    r = gate.GatedRun(mk(precision=1), gate.rule_network(0.05), 1e-6, check_every=50, bound=1e-3, eval_every=5)
    hru, msru = _run(r.mesh, s["U0"], dts)
    rflag = r.mesh.gate_flagged() / r.mesh.n_cells
    err = lambda h: (np.abs(h - h64) / np.abs(h64)).max(axis=0)
    report = {"troubled_fraction": float(s["y"].mean()), "held_out": s["held"], "flagged_learned": flagged,
              "flagged_rule": rflag, "ms": {"fp64": ms64, "mixed": msmx, "learned+mixed": mslg,
                                           "linear+mixed": mslin, "rule+mixed": msru},
              "err [ke, eps_s, eps_d]": {"mixed": err(hmx).tolist(), "learned+mixed": err(hlg).tolist(),
                                         "linear+mixed": err(hlin).tolist(), "rule+mixed": err(hru).tolist()}}
    print("gain:", report)
    assert s["held"]["recall"] >= 0.98
    assert err(hlg)[0] <= 1e-4 and err(hlg)[1] <= 1e-4
    assert mslg < ms64 / 3
    assert g.mesh.gate_flagged() <= g.mesh.n_cells


def test_plain_scheme_check_switches_the_gate_off(setup):
    s = setup
    m = ucns.Mesh(s["nodes"], s["cells"], s["box"], ucns.Params(precision=1, **s["base"]))
    U = torch.from_numpy(s["U0"].copy()).cuda()
    gate.GatedRun(m, gate.rule_network(1e9), 1e-6, check_every=1, bound=0.5)  # flags nothing
    rel, off = m.gate_check(U)
    assert rel > 0.0 and not off  # linear weights everywhere differ a little from CWENOZ
    m.gate_configure(eval_every=1, check_every=1, bound=1e-14)
    m.rk_step(U)  # the step's check finds the rates differ by more than 1e-14 and disables the gate
    with pytest.raises(ucns.UcnsError):
        m.gate_check(U)  # not enabled any more
