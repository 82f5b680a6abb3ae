"""Workflow of the learned troubled-cell indicator, on top of the C ABI.

1. ``collect``: run the plain FP64 CWENOZ scheme and record, every few steps,
   the 32 features (BF16) and the label deviation max |omega_s - lambda_s| of
   every cell (all on the device).
2. ``train``: class-weighted cross-entropy, Adam, on the GPU (tcgen05
   forward/backward kernels), shuffled mini-batches each epoch.
3. ``threshold_for_recall``: the logit threshold that keeps a given recall of
   the troubled cells on held-out samples.
4. ``GatedRun``: a mesh with the trained network attached, plus the safety
   check of the plain scheme (run by the library): every ``check_every`` steps
   the gated and the full reconstruction of the same state are compared, and
   the gate is switched off for good when the estimated error it puts into the
   kinetic-energy history (the difference of the dKE/dt rates, accumulated over
   the check intervals) or the relative difference of the solenoidal or the
   dilatational dissipation of the two reconstructions (local errors do not
   cancel there) exceeds ``bound`` (see ucns_gate_configure).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import ucns

LABEL_THRESHOLD = 1e-2  # a cell is troubled when its CWENOZ weights depart by more than this


@dataclass
class Samples:
    X: "object"        # torch bfloat16 [n, 32] on the device
    dev: "object"      # torch float32 [n]
    step: np.ndarray   # step index of each sample (for held-out splits)


def collect(mesh64: ucns.Mesh, U, steps: int, every: int = 5, stream=None) -> Samples:
    """Advance U (device, in place) by `steps` plain FP64 CWENOZ steps and
    record features and label deviations of the states at steps 0, every, ..."""
    import torch

    Xs, ds, st = [], [], []
    for k in range(steps + 1):
        if k % every == 0:
            X, _ = mesh64.gate_features(U, stream=stream)
            Xs.append(X)
            ds.append(mesh64.gate_labels(U, stream=stream))
            st.append(np.full(mesh64.n_cells, k, dtype=np.int32))
        if k < steps:
            mesh64.rk_step(U, stream=stream)
    mesh64.check_state(stream)
    return Samples(torch.cat(Xs).contiguous(), torch.cat(ds).contiguous(), np.concatenate(st))


def rule_network(tau: float) -> ucns.Net:
    """A hand-set rule written as the same network: flag a cell when any of
    its central-stencil density or pressure jumps (features 0-23) exceeds tau
    in magnitude (z = sum_k relu(|x_k| - tau) > 0)."""
    th = np.zeros(ucns.MLP_PARAMS, np.float32)
    W1 = th[0:2048].reshape(64, 32)
    b1 = th[2048:2112]
    W2 = th[2112:6208].reshape(64, 64)
    w3 = th[6272:6336]
    for k in range(24):
        W1[2 * k, k], b1[2 * k] = 1.0, -tau
        W1[2 * k + 1, k], b1[2 * k + 1] = -1.0, -tau
    for j in range(48):
        W2[j, j] = 1.0
        w3[j] = 1.0
    net = ucns.Net(seed=0)
    net.set_params(th)
    return net


def class_weights(y) -> tuple[float, float]:
    p = float(y.float().mean().item())
    p = min(max(p, 1e-6), 1 - 1e-6)
    return 0.5 / p, 0.5 / (1.0 - p)


def train(X, y, epochs: int = 4, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
          net: ucns.Net | None = None) -> ucns.Net:
    """Train on (X, y) with shuffled mini-batches; returns the network."""
    import torch

    net = net or ucns.Net(seed=seed)
    w_pos, w_neg = class_weights(y)
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        net.train(X[perm].contiguous(), y[perm].contiguous(), batch=batch, lr=lr, w_pos=w_pos, w_neg=w_neg)
    net.check()
    return net


def threshold_for_recall(net: ucns.Net, X, y, recall: float = 0.999) -> float:
    """Largest FP32 logit threshold whose recall of y = 1 on (X, y) is >= recall
    (a cell is flagged when its logit exceeds the threshold): with the troubled
    samples' logits sorted, at most m = floor((1 - recall) n) of them may lie at
    or below it, so it sits just below the (m+1)-th smallest."""
    z = net.forward(X)
    zp = np.sort(z[y > 0.5].float().cpu().numpy().astype(np.float32))
    if zp.size == 0:
        return float("inf")
    m = int(np.floor((1.0 - recall) * zp.size + 1e-9))
    return float(np.nextafter(zp[min(m, zp.size - 1)], np.float32(-np.inf)))


def confusion(net: ucns.Net, X, y, thr: float) -> dict:
    z = net.forward(X)
    pred = z > thr
    yt = y > 0.5
    tp = int((pred & yt).sum().item())
    fn = int((~pred & yt).sum().item())
    fp = int((pred & ~yt).sum().item())
    tn = int((~pred & ~yt).sum().item())
    return {"tp": tp, "fn": fn, "fp": fp, "tn": tn, "recall": tp / (tp + fn) if tp + fn else 1.0,
            "flagged_fraction": (tp + fp) / max(1, tp + fn + fp + tn)}


@dataclass
class GatedRun:
    """A mixed or FP64 mesh with the trained indicator attached; the library
    runs the plain-scheme check every `check_every` steps and switches the
    gate off when its estimated kinetic-energy history error or a dissipation
    difference exceeds `bound` (or, with `bound_rate` > 0, the total KE-rate
    difference exceeds that)."""

    mesh: ucns.Mesh
    net: ucns.Net
    threshold: float
    check_every: int = 10
    bound: float = 1e-4
    eval_every: int = 1
    bound_rate: float = 0.0

    def __post_init__(self):
        self.mesh.gate_attach(self.net, self.threshold)
        self.mesh.gate_configure(self.eval_every, self.check_every, self.bound, self.bound_rate)
        self.mesh.gate_enable(True)

    def step(self, U, dt=None):
        self.mesh.rk_step(U, dt=dt)

    def detach(self):
        self.mesh.gate_enable(False)
        self.mesh.gate_attach(None, 0.0)


def reference_history(mesh64: ucns.Mesh, U0, steps: int, every: int = 10):
    """Plain FP64 run of `steps` CFL steps from the host state U0 (internal
    order): (the dt sequence, diagnostics [KE, eps_s, eps_d] after every
    `every`-th step, the final device state)."""
    import torch

    U = torch.from_numpy(np.array(U0, copy=True)).cuda()
    dts, hist = [], []
    for k in range(steps):
        dts.append(mesh64.rk_step(U, return_dt=True))
        if k % every == every - 1:
            d = mesh64.diagnostics(U)
            hist.append((d["ke"], d["eps_s"], d["eps_d"]))
    mesh64.check_state()
    return dts, np.array(hist), U


def replay_history(mesh: ucns.Mesh, U0, dts, every: int = 10):
    """The same steps with a given dt sequence on another form of the scheme:
    (diagnostics as in reference_history, milliseconds of the steps alone by
    CUDA events, the final device state)."""
    import torch

    U = torch.from_numpy(np.array(U0, copy=True)).cuda()
    hist, ms = [], 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k, dt in enumerate(dts):
        e0.record()
        mesh.rk_step(U, dt=dt)
        e1.record()
        if k % every == every - 1:
            torch.cuda.synchronize()
            d = mesh.diagnostics(U)
            hist.append((d["ke"], d["eps_s"], d["eps_d"]))
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    mesh.check_state()
    return np.array(hist), ms, U


def history_error(h, h_ref) -> list:
    """max over the history of the relative error of KE, eps_s and eps_d; the
    eps_d error is taken against max(|eps_d|, 1e-3 |eps_s|) (at low Mach
    numbers eps_d lies below the arithmetic's resolution of the dissipation),
    as the library's plain-scheme check measures it."""
    h, h_ref = np.asarray(h), np.asarray(h_ref)
    den = np.abs(h_ref).copy()
    den[:, 2] = np.maximum(den[:, 2], 1e-3 * np.abs(h_ref[:, 1]))
    return (np.abs(h - h_ref) / den).max(axis=0).tolist()

