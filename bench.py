#!/usr/bin/env python
"""Throughput of the explicit residual + SSP Runge-Kutta path in cell-RK-stages/s.

Workload (default): compressible Taylor-Green vortex, Mach 0.1, Re 1600, on
64^3 hexahedra of [0, 2 pi]^3 with interior nodes jittered by a seeded
uniform +-10 % of the spacing, P2 least-squares reconstruction with CWENOZ
weights over central + directional stencils, FP64, SSP-RK3 at CFL 0.5 with
the CFL time step computed on the device every step.  One "step" is one full
SSP-RK3 step (3 residual evaluations + the time step reduction); the metric
counts cells x 3 stages per second.  ``--integrator 1`` times the paper's
SSP(5,4) instead (5 stages per step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ucns|reference] [--integrator 0|1]

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica of the workload on its own GPU (the path is replicated, not sharded:
no collective on the data path); value = total cell-stages of all ranks / the
slowest rank's time.  ``--impl reference`` times the CPU oracle instead (on
a bounded sample of the same workload, rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "cell-RK-stages/s at P2 on 1 GB300, plain FP64 vs chosen form at fixed KE error"
UNIT = "cell-RK-stages/s"
STAGES = 3

# Algorithmic flop counts of the kernels (each +,-,*,/,sqrt = 1, FMA = 2), counted
# from the kernel source.  Face kernel, per Gauss point: 2 sides x 5 variables x 33
# (value 9 FMA, gradient 6 FMA + 3 mul) = 330, penalty and averages 80, HLLC 138,
# viscous flux 120, scaling and the Gauss sum 20.  Reconstruction, per cell: 5 x 814
# (central differences + contraction 342, directional 252, smoothness indicators 95,
# weights and combination 125).
FLOPS_FACE_P2_VISC_PER_QP = 688
FLOPS_RECON_P2_CWENOZ_PER_CELL = 4070


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ucns", choices=["ucns", "reference"])
    ap.add_argument("--n", type=int, default=64, help="lattice cells per direction")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--integrator", type=int, default=0, choices=[0, 1],
                    help="0: SSP-RK3 (the benchmark configuration), 1: the paper's SSP(5,4) (5 stages per step)")
    ap.add_argument("--train-epochs", type=int, default=60,
                    help="indicator training epochs of the learned form (fewer: faster setup, more flagged cells)")
    ap.add_argument("--forms", default="fp64,mixed,learned",
                    help="comma list of forms to time: fp64, mixed, learned (indicator + mixed)")
    return ap.parse_args()


def workload(n: int):
    from paper_2609_07387_gb300 import inputs as I

    nodes, cells, box = I.hex_lattice(n, jitter=0.1, seed=1)
    U = I.tgv_state(nodes, cells, 0.1)
    return nodes, cells, box, U


def rk_name() -> str:
    return "SSP(5,4)" if STAGES == 5 else "SSP-RK3"


def config(n: int, N: int, world: int) -> dict:
    return {
        "workload": f"TGV M0.1 Re1600, {n}^3 jittered (+-10% h, seed 1) hex = {N} cells, P2 CWENOZ, "
                    f"{rk_name()} CFL 0.5, device CFL dt every step; plain FP64 and the mixed form timed",
        "cells": N,
        "stages_per_step": STAGES,
        "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
        "l2": "inputs larger than L2 (pseudo-inverses ~0.57 GB at 64^3)",
    }


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.rows = []
        self.proc = None
        self.bus_id = bus_id

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if self.bus_id:
            cmd[1:1] = ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash() -> str:
    """Hash of every CUDA source of the library (a stored ncu traffic figure
    is used only while it matches)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2609_07387_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, n: int, form: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source for this form (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d.get(f"{kernel}/{form}")
        if e and e.get("source_hash") == kernel_source_hash():
            return e["dram_bytes_per_launch_scaled_to"].get(str(n))
    except (OSError, ValueError, KeyError):
        pass
    return None


def fp64_peak_tflops(torch) -> float | None:
    """Measured FP64 throughput: cuBLAS DGEMM 4096^3, best of 3."""
    try:
        n = 4096
        a = torch.randn(n, n, dtype=torch.float64, device="cuda")
        b = torch.randn(n, n, dtype=torch.float64, device="cuda")
        torch.matmul(a, b)
        torch.cuda.synchronize()
        best = math.inf
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        del a, b
        return 2.0 * n ** 3 / best / 1e12
    except Exception:
        return None


# ------------------------------------------------------------ CPU oracle
def oracle_sample(nodes, cells, box, U, n: int, layers: int):
    """Build the oracle on the workload and pick a sample: `layers` z-layers
    of the lattice (layers * n^2 cells)."""
    import oracle as O

    oc = O.Case(nodes, cells, box, O.Params(order=2, scheme=1, Re=1600.0, Mach=0.1, cfl=0.5,
                                            integrator=1 if STAGES == 5 else 0))
    sel = np.arange(layers * n * n, dtype=np.int64)
    oc.residual_subset(U, sel[:8])  # warm the lazy precompute path
    return oc, sel


def oracle_rk_step_on_sample(oc, U, sel, dt):
    """The stages of one step on the sample cells (residual of the sample +
    Shu-Osher combination), the oracle's arithmetic per stage: SSP-RK3, or
    SSP(5,4) with the oracle's coefficients."""
    if STAGES == 5:
        import oracle as O

        alpha, beta = O.ssp54_coefficients()
        Uw = U.copy()
        u, L = [U[:, sel].copy()], []
        for i in range(1, 6):
            L.append(oc.residual_subset(Uw, sel))
            ui = sum(alpha[i, j] * u[j] + dt * beta[i, j] * L[j] for j in range(i))
            u.append(ui)
            Uw[:, sel] = ui
        return u[5]
    U0 = U[:, sel].copy()
    Uw = U.copy()
    R = oc.residual_subset(Uw, sel)
    U1 = U0 + dt * R
    Uw[:, sel] = U1
    R = oc.residual_subset(Uw, sel)
    U2 = 0.75 * U0 + 0.25 * (U1 + dt * R)
    Uw[:, sel] = U2
    R = oc.residual_subset(Uw, sel)
    return U0 / 3.0 + 2.0 / 3.0 * (U2 + dt * R)


def omp_threads() -> int:
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def cpu_baseline(nodes, cells, box, U, n: int) -> dict:
    oc, sel = oracle_sample(nodes, cells, box, U, n, layers=8)
    dt = 1e-3
    oc.residual_subset(U, sel)  # untimed: lazy precompute of the sample's stencils
    t0 = time.perf_counter()
    oracle_rk_step_on_sample(oc, U, sel, dt)
    t = time.perf_counter() - t0
    return {"value": sel.size * STAGES / t, "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
            "sample": f"one {rk_name()} step ({STAGES} residual evaluations + updates) of {sel.size} of the "
                      f"{len(cells)} cells (8 z-layers of the {n}^3 workload), precompute excluded",
            "seconds": t}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    n = args.n
    nodes, cells, box, U = workload(n)
    oc, sel = oracle_sample(nodes, cells, box, U, n, layers=4)
    dt = 1e-3
    for _ in range(args.warmup):
        oracle_rk_step_on_sample(oc, U, sel, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_rk_step_on_sample(oc, U, sel, dt)
    t = time.perf_counter() - t0
    value = sel.size * STAGES * args.steps / t
    sample = (f"each step: one {rk_name()} step ({STAGES} residual evaluations + updates) of {sel.size} of the "
              f"{len(cells)} cells (4 z-layers of the {n}^3 workload)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": config(n, len(cells), 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": omp_threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU arm
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max SM clock


def algorithmic(m, kind: str, mixed: bool, frac_dir: float = 1.0) -> tuple[float, float]:
    """(flops, bytes) of one launch of the face or reconstruction kernel:
    flops as counted above, bytes = each array element read or written once
    (neighbour gathers served by cache).  frac_dir: fraction of cells that
    take the directional stencils (the gate routes the rest to the linear
    weights: central contraction and constant term only, 5 x 354 flops)."""
    w = 4 if mixed else 8
    N, F = m.n_cells, m.n_faces
    row = (m.K + 1) * 5 * w  # one cell's coefficients
    if kind == "face":
        # per point: offsets, normal, |dS|; per face: penalty, owner/neighbour ids, 5 totals (FP32 in the
        # mixed form); per cell: its coefficient row
        flops = FLOPS_FACE_P2_VISC_PER_QP * m.nq * F
        nbytes = F * (m.nq * 10 * w + w + 2 * 4 + 5 * w) + N * row
    else:
        # per cell: central pseudo-inverse and ids, moments and 1/h (FP32 rows in the mixed form), the
        # state (or its float pair), the coefficient row; per flagged (or CWENOZ) cell: the directional
        # pseudo-inverses and ids
        flops = N * (5 * 354 + frac_dir * (FLOPS_RECON_P2_CWENOZ_PER_CELL - 5 * 354))
        cell = 7 * 4 if mixed else 7 * 8
        nbytes = N * (m.K * m.Mc * w + m.Mc * 4 + cell + 5 * 8 + row
                      + frac_dir * (m.nd * 3 * m.Md * w + m.nd * m.Md * 4))
    return flops, nbytes


def roofline(m, prof: dict, mixed: bool, peak64, hbm_gbs: float, n: int, frac_dir: float = 1.0,
             form: str = "fp64") -> dict:
    kinds = {k: v for k, v in prof.items() if v[1] > 0 and k in ("recon", "face")}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms, dom_n = kinds[dom]
    avg_s = dom_ms / dom_n / 1e3
    kind = "face" if dom == "face" else "recon"
    flops, nbytes = algorithmic(m, kind, mixed, frac_dir)
    name = {("face", False): "k_face<2,true>", ("recon", False): "k_recon<2,true,6>",
            ("face", True): "k_face_mx<2,true>", ("recon", True): "k_recon_mx<2,true,6>"}[(kind, mixed)]
    if kind == "recon" and mixed and frac_dir < 1.0:
        name = "k_recon_mx<2,false,6,gated>"
    if mixed:
        alu_peak, alu_src = FP32_PEAK_TFLOPS, "FP32: 152 SMs x 128 lanes x 2 x 2.07 GHz"
    elif peak64 and 0.3 < peak64 < 5.0:
        alu_peak, alu_src = peak64, "measured cuBLAS DGEMM FP64"
    else:
        alu_peak, alu_src = 1.25, "nominal FP64 1.25 TFLOP/s"
    alu = flops / avg_s / 1e12
    bw = nbytes / avg_s / 1e9
    alu_frac, hbm_frac = alu / alu_peak, bw / hbm_gbs
    if alu_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu_frac,
                "peak_source": alu_src + " (of measured)" if "measured" in alu_src else alu_src}
    else:
        roof = {"bound": "hbm", "achieved": bw, "peak": hbm_gbs, "unit": "GB/s", "frac": hbm_frac,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    roof.update({"kernel": name, "traffic": measured_traffic(name, n, form), "avg_launch_ms": avg_s * 1e3,
                 "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": nbytes,
                 "alu_frac": alu_frac, "hbm_frac": hbm_frac})
    return roof


def max_over_ranks(t: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time (all ranks get it); plain value when world == 1."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist

    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(t_local: float, cells_per_rank: int, steps: int, world: int, device: str = "cuda"):
    """(slowest time, whole-job cell-stages/s): every rank runs a replica of
    `cells_per_rank` cells for `steps` SSP-RK3 steps."""
    t = max_over_ranks(t_local, world, device)
    return t, world * cells_per_rank * STAGES * steps / t


def hbm_peak() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def run_ucns(args, rank: int, world: int, local_rank: int):
    import torch
    import torch.distributed as dist

    from paper_2609_07387_gb300 import ucns

    torch.cuda.set_device(local_rank)
    n = args.n
    nodes, cells, box, U_user = workload(n)
    N = len(cells)
    stream = torch.cuda.current_stream()
    base = dict(order=2, scheme=1, Re=1600.0, Mach=0.1, cfl=0.5, integrator=args.integrator)
    forms = [f for f in args.forms.split(",") if f]
    prec = {"fp64": 0, "mixed": 1, "learned": 1}
    meshes = {f: ucns.Mesh(nodes, cells, box, ucns.Params(precision=prec[f], **base)) for f in forms}
    U0 = np.ascontiguousarray(next(iter(meshes.values())).to_internal(U_user))
    gate_info = None
    if "learned" in meshes:
        # untimed setup: labels from 50 plain FP64 CWENOZ steps, training, threshold
        from paper_2609_07387_gb300 import gate

        m64 = meshes.get("fp64") or ucns.Mesh(nodes, cells, box, ucns.Params(precision=0, **base))
        t0 = time.perf_counter()
        Uc = torch.from_numpy(U0.copy()).cuda()
        S = gate.collect(m64, Uc, 50, every=5)
        y = (S.dev > gate.LABEL_THRESHOLD).float()
        # 60 epochs: at full held-out recall the network then flags ~1 % of the cells (3 epochs: ~8 %)
        net = gate.train(S.X[: 9 * N].contiguous(), y[: 9 * N].contiguous(), epochs=args.train_epochs, lr=1e-3,
                         batch=4096, seed=0)
        thr = gate.threshold_for_recall(net, S.X[9 * N:].contiguous(), y[9 * N:].contiguous(), 0.999)
        held = gate.confusion(net, S.X[10 * N:].contiguous(), y[10 * N:].contiguous(), thr)
        gated = gate.GatedRun(meshes["learned"], net, thr, check_every=50, bound=1e-3, eval_every=5)
        gate_info = {"train_samples": 9 * N, "train_epochs": args.train_epochs,
                     "troubled_fraction": float(y.mean().item()), "threshold": thr,
                     "held_out_last_snapshot": held, "setup_s": time.perf_counter() - t0,
                     "eval_every": 5, "check_every": 50, "check_bound": 1e-3, "_net": net, "_gated": gated}
    bus = None
    try:
        bus = torch.cuda.get_device_properties(local_rank).pci_bus_id
    except Exception:
        bus = None

    def barrier():
        if world > 1:
            dist.barrier()

    prof_steps = min(args.steps, 50)

    def timed(m):
        U = torch.from_numpy(U0.copy()).cuda()
        m.rk_steps(U, args.warmup)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(bus) as clk:
            e0.record(stream)
            m.rk_steps(U, args.steps)  # the library's multi-step call: K steps, dt on the device
            e1.record(stream)
            torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        m.check_state()
        # per-kernel times from a separate run on a copy of the state: the
        # events the library records around each launch when profiling cost
        # ~40 us per step, which the timed run must not include
        Up = U.clone()
        m.profile(True)
        m.rk_steps(Up, prof_steps)
        torch.cuda.synchronize()
        prof = m.profile_read()
        m.profile(False)
        m.check_state()
        t, value = job_throughput(ms / 1e3, N, args.steps, world)
        return {"t": t, "ms": ms, "prof": prof, "U": U, "clocks": clk.summary(), "value": value}

    res = {k: timed(m) for k, m in meshes.items()}
    if gate_info is not None:
        gate_info["flagged_fraction_last_step"] = meshes["learned"].gate_flagged() / N
        # the library switches the gate off for good when a plain-scheme check
        # fails; a gate still on after the timed and the profiled steps was on
        # throughout the timed run
        try:
            rel, _ = meshes["learned"].gate_check(res["learned"]["U"].clone())
            gate_info["gate_on_after_runs"] = True
            gate_info["check_rel_diff_after_runs"] = rel
        except ucns.UcnsError:
            gate_info["gate_on_after_runs"] = False
    # the fixed-error comparison: every form ran warmup + steps from the same state
    errs = {}
    if "fp64" in res:
        d64 = meshes["fp64"].diagnostics(res["fp64"]["U"])
        for f in res:
            if f != "fp64":
                d = meshes[f].diagnostics(res[f]["U"])
                e = {k: abs(d[k] - d64[k]) / abs(d64[k]) for k in ("ke", "eps_s")}
                errs[f] = {"ke_rel_err": e["ke"], "eps_s_rel_err": e["eps_s"], "within": max(e.values()) <= 1e-4}
        ok_forms = ["fp64"] + [f for f in errs if errs[f]["within"]]
        chosen = max(ok_forms, key=lambda f: res[f]["value"])
    else:
        chosen = forms[0]
    mc = meshes[chosen]
    # ---- end to end through the host-buffer entry point (pinned memory)
    Uh = torch.from_numpy(U0.copy()).pin_memory()
    mc.rk_steps_host(Uh, 1)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        mc.rk_steps_host(Uh, 1)
    te, e2e = job_throughput(time.perf_counter() - t0, N, args.e2e_steps, world)
    if rank != 0:
        return
    peak64 = fp64_peak_tflops(torch)
    hbm = hbm_peak()

    def shares(prof):
        # the time step runs on a side stream, overlapped with the first stage's kernels: its event
        # time is wall time on that stream (shared SMs), reported but kept out of the shares
        kinds = {k: v for k, v in prof.items() if v[1] > 0}
        tot = sum(v[0] for k, v in kinds.items() if k != "dt")
        return {k: {"ms_per_launch": v[0] / v[1], "launches": v[1],
                    "share": None if k == "dt" else v[0] / tot,
                    **({"note": "side stream, overlapped with the first stage"} if k == "dt" else {})}
                for k, v in kinds.items()}

    r = res[chosen]
    prof = r["prof"]
    # kernels per step of the profiled run (dt and the check reduction launch two
    # each, a gated reconstruction two, the rest one), scaled to the timed steps
    counted = round((sum(v[1] for k, v in prof.items()) + prof["dt"][1] +
                     (prof["recon"][1] if chosen == "learned" else 0)) * args.steps / prof_steps)
    frac_dir = gate_info["flagged_fraction_last_step"] if (chosen == "learned" and gate_info) else 1.0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(nodes, cells, box, U_user, n)
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if chosen == "fp64" else "f32+f64+bf16" if chosen == "learned" else "f32+f64",
        "data": "synthetic",
        "impl": "ucns", "form": chosen,
        "config": config(n, N, world),
        "clocks": r["clocks"],
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 5 * N * 8, "d2h_bytes_per_step": 5 * N * 8 + 16,
                "steps": args.e2e_steps, "via": "ucns_rk_steps_host, pinned host buffer"},
        "gpu_launches": counted,
        "roofline": roofline(mc, prof, chosen != "fp64", peak64, hbm, n, frac_dir, chosen),
        "kernels": shares(prof),
        "fixed_error": {"compared_after_steps": args.warmup + args.steps, "bound": 1e-4, "vs": "plain FP64",
                        "forms": errs},
        "forms": {f: {"value": res[f]["value"], "ms_per_step": res[f]["ms"] / args.steps,
                      "kernels": shares(res[f]["prof"])} for f in res},
        "learned_gate": None if gate_info is None else {k: v for k, v in gate_info.items() if not k.startswith("_")},
        "plain_fp64": None if "fp64" not in res else {
            "value": res["fp64"]["value"], "ms_per_step": res["fp64"]["ms"] / args.steps,
            "roofline": roofline(meshes["fp64"], res["fp64"]["prof"], False, peak64, hbm, n, 1.0, "fp64"),
            "kernels": shares(res["fp64"]["prof"]), "clocks": res["fp64"]["clocks"]},
        "speedup_vs_plain_fp64": r["value"] / res["fp64"]["value"] if "fp64" in res else None,
        "fp64_dgemm_tflops": peak64,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def main():
    global STAGES
    args = parse()
    STAGES = 5 if args.integrator == 1 else 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ucns(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
