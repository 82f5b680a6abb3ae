"""What the learned indicator gains over the method without it: the Mach 1.25
Taylor-Green vortex with a 5 % random-phase perturbation on 96^3 jittered
hexahedra (the 128^3 configuration scaled down).  Labels come from 50 plain
FP64 CWENOZ steps; the network is trained on the GPU (60 epochs); then 400
steps (to t ~ 2.2, through the shocklets' formation) of plain FP64, mixed, learned +
mixed, all-linear + mixed and a hand-set jump rule + mixed run from the same
state with the same dt sequence.

Asserted: the learned form keeps the kinetic-energy, solenoidal and
dilatational dissipation histories within 1e-4 of plain FP64 (its
plain-scheme check switching the gate off where the gate's error would grow
past that); while its gate is on it runs faster than the gate-less mixed form
(the network's gain) and than the hand-set rule; without a gate (all-linear
weights) the dissipation history leaves the bound (why a gate is needed).
The check itself switches the gate off when its bound is violated."""
import numpy as np
import pytest

from paper_2609_07387_gb300 import gate
from paper_2609_07387_gb300 import inputs as I
from paper_2609_07387_gb300 import ucns

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_SIDE, COLLECT, RUN, TIMED = 96, 50, 400, 40
BOUND = 1e-4
RECALL = 0.99


@pytest.fixture(scope="module")
def setup():
    nodes, cells, box = I.hex_lattice(N_SIDE, jitter=0.1, seed=3)
    base = dict(order=2, scheme=1, Re=1600.0, Mach=1.25, cfl=0.5)
    m64 = ucns.Mesh(nodes, cells, box, ucns.Params(precision=0, **base))
    mx = ucns.Mesh(nodes, cells, box, ucns.Params(precision=1, **base))
    U0 = np.ascontiguousarray(m64.to_internal(I.tgv_perturbed_state(nodes, cells, 1.25, 0.05, seed=4)))
    U = torch.from_numpy(U0.copy()).cuda()
    S = gate.collect(m64, U, COLLECT, every=5)
    N = m64.n_cells
    y = (S.dev > gate.LABEL_THRESHOLD).float()
    net = gate.train(S.X[: 9 * N].contiguous(), y[: 9 * N].contiguous(), epochs=60, lr=1e-3, batch=4096, seed=0)
    thr = gate.threshold_for_recall(net, S.X[9 * N: 10 * N].contiguous(), y[9 * N: 10 * N].contiguous(), RECALL)
    held = gate.confusion(net, S.X[10 * N:].contiguous(), y[10 * N:].contiguous(), thr)
    thr999 = gate.threshold_for_recall(net, S.X[9 * N: 10 * N].contiguous(), y[9 * N: 10 * N].contiguous(), 0.999)
    held999 = gate.confusion(net, S.X[10 * N:].contiguous(), y[10 * N:].contiguous(), thr999)
    del S
    dts, h64, _ = gate.reference_history(m64, U0, RUN, every=10)
    return dict(m64=m64, mx=mx, U0=U0, net=net, thr=thr, held=held, held999=held999, troubled=float(y.mean()),
                dts=dts, h64=h64)


def _form(s, kind):
    """Configure the mixed mesh for a form: no gate, the trained network,
    all-linear weights (caller flags all zero) or the hand-set rule."""
    mx = s["mx"]
    mx.gate_set_flags(None)
    mx.gate_enable(False)
    if kind == "learned":
        gate.GatedRun(mx, s["net"], s["thr"], check_every=50, bound=BOUND, eval_every=5)
    elif kind == "linear":
        mx.gate_set_flags(torch.zeros(mx.n_cells, dtype=torch.uint8, device="cuda"))
    elif kind == "rule":
        gate.GatedRun(mx, gate.rule_network(0.05), 1e-6, check_every=50, bound=BOUND, eval_every=5)
    return mx


def _timed_ms(m, U0, steps):
    """ms per step of the multi-step call (device dt), after two warm-up steps."""
    U = torch.from_numpy(U0.copy()).cuda()
    m.rk_steps(U, 2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    m.rk_steps(U, steps)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _total_eps_err(h, h64):
    return float((np.abs((h[:, 1] + h[:, 2]) - (h64[:, 1] + h64[:, 2])) / np.abs(h64[:, 1] + h64[:, 2])).max())


def test_learned_gate_gain(setup):
    s = setup
    report, err, ms, status = {}, {}, {}, {}
    for kind in ("mixed", "learned", "linear", "rule"):
        m = _form(s, kind)
        h, _, _ = gate.replay_history(m, s["U0"], s["dts"], every=10)
        err[kind] = gate.history_error(h, s["h64"]) + [_total_eps_err(h, s["h64"])]
        if kind in ("learned", "rule"):
            status[kind] = {**m.gate_status(), "flagged": m.gate_flagged() / m.n_cells}
        m = _form(s, kind)  # fresh counters for the timed run
        ms[kind] = _timed_ms(m, s["U0"], TIMED)
    ms["fp64"] = _timed_ms(s["m64"], s["U0"], 5)
    report = {"troubled_fraction": s["troubled"], "held_out": s["held"], "held_out_at_recall_0.999": s["held999"],
              "ms_per_step": ms,
              "err [ke, eps_s, eps_d, eps]": err, "gate": status}
    print("gain:", report)
    assert s["held"]["recall"] >= 0.97
    # the learned form: within the bound on every history (the check switches
    # the gate off before its error would pass the bound), gated for a good part of the run
    assert max(err["learned"][:3]) <= BOUND, (err["learned"], status["learned"])
    off = status["learned"]["off_step"]
    assert off == -1 or off >= 100, status["learned"]
    # the network's gain while gated: faster than the same scheme without the
    # gate, and than the hand-set rule (which flags more cells)
    assert ms["learned"] < ms["mixed"], ms
    assert ms["learned"] < ms["rule"], ms
    # without a gate the linear weights leave the dissipation history's bound
    assert err["linear"][2] > BOUND, err["linear"]
    assert ms["learned"] < ms["fp64"] / 10


def test_plain_scheme_check_switches_the_gate_off(setup):
    s = setup
    m = _form(s, "none")
    U = torch.from_numpy(s["U0"].copy()).cuda()
    gate.GatedRun(m, gate.rule_network(1e9), 1e-6, check_every=1, bound=0.5)  # flags nothing
    rel, off = m.gate_check(U)
    assert min(rel) > 0.0 and not off  # linear weights everywhere differ a little from CWENOZ
    assert m.gate_status()["last"] == rel
    m.gate_configure(eval_every=1, check_every=1, bound=1e-14)
    m.rk_step(U)  # the step's check finds the gate's error above 1e-14 and disables the gate
    st = m.gate_status()
    assert not st["enabled"] and st["off_step"] == 0 and st["checks"] == 1
    with pytest.raises(ucns.UcnsError):
        m.gate_check(U)  # not enabled any more
    m.gate_enable(False)
    m.gate_attach(None, 0.0)
