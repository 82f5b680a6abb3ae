#!/usr/bin/env python
"""Throughput of the explicit residual + SSP Runge-Kutta path in cell-RK-stages/s.

Workloads (``--config``, synthetic and seeded; P2 least-squares reconstruction
with CWENOZ weights over central + directional stencils, Re 1600, SSP-RK3 at
CFL 0.5 with the CFL time step computed on the device every step):

  c5 (default)  Mach 1.25 Taylor-Green vortex plus a 5 % random-phase velocity
                perturbation on 128^3 jittered hexahedra (2,097,152 cells):
                plain FP64, mixed precision, and the learned troubled-cell gate
                + mixed precision (network trained on the GPU from labels of 50
                plain FP64 steps); the fixed-error comparison runs 500 steps of
                every form with the plain FP64 run's dt sequence.
  c3            Mach 0.1 Taylor-Green vortex on 6 x 96^3 = 5,308,416
                tetrahedra: plain FP64 and mixed precision (100-step history).
  c2            Mach 0.1 Taylor-Green vortex on 64^3 jittered hexahedra:
                plain FP64, mixed and learned + mixed (200-step history).

One "step" is one full SSP-RK3 step (3 residual evaluations + the time step
reduction); the metric counts cells x 3 stages per second.  ``--integrator 1``
times the paper's SSP(5,4) instead (5 stages per step).  ``value`` is the
fastest form whose kinetic-energy and dissipation histories stay within 1e-4
relative of plain FP64 (the fixed-error comparison).

  python bench.py [--config c5|c3|c2] [--gpus N] [--steps K] [--warmup W] [--impl ucns|reference]

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
import os
import statistics
import subprocess
import sys
import threading
import time
from dataclasses import dataclass

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "cell-RK-stages/s at P2 on 1 GB300, plain FP64 vs chosen form at fixed KE error"
UNIT = "cell-RK-stages/s"
STAGES = 3
ERROR_BOUND = 1e-4  # relative, on the kinetic-energy and dissipation histories

# Algorithmic flop counts of the kernels (each +,-,*,/,sqrt = 1, FMA = 2), counted
# from the kernel source.  Face kernel, per Gauss point: 2 sides x 5 variables x 33
# (value 9 FMA, gradient 6 FMA + 3 mul) = 330, penalty and averages 80, HLLC 138,
# viscous flux 120, scaling and the Gauss sum 20.  Reconstruction, per cell: 5 x 814
# (central differences + contraction 342, directional 252, smoothness indicators 95,
# weights and combination 125); linear weights only: 5 x 354.
FLOPS_FACE_P2_VISC_PER_QP = 688
FLOPS_RECON_P2_CWENOZ_PER_CELL = 4070
FLOPS_RECON_P2_LINEAR_PER_CELL = 5 * 354


@dataclass
class Config:
    key: str
    n: int              # lattice hexahedra per direction
    tets: bool          # split every hexahedron into 6 tetrahedra
    seed: int           # jitter seed
    mach: float
    perturb_seed: int | None  # random-phase velocity perturbation (5 %), None: plain Taylor-Green
    forms: tuple
    history: int        # steps of the fixed-error comparison
    label_steps: int = 50

    def describe(self, n: int, N: int) -> str:
        mesh = (f"6 x {n}^3 = {N} tetrahedra (Kuhn split of a +-10% h jittered lattice, seed {self.seed})"
                if self.tets else f"{n}^3 = {N} hexahedra jittered +-10% h (seed {self.seed})")
        init = (f"Taylor-Green M{self.mach:g} + 5% random-phase velocity (seed {self.perturb_seed})"
                if self.perturb_seed is not None else f"Taylor-Green M{self.mach:g}")
        return f"{init}, Re 1600, {mesh}, P2 CWENOZ, {rk_name()} CFL 0.5, device CFL dt every step"


CONFIGS = {
    "c5": Config("c5", 128, False, 3, 1.25, 4, ("fp64", "mixed", "learned"), 500),
    "c3": Config("c3", 96, True, 2, 0.1, None, ("fp64", "mixed"), 100),
    "c2": Config("c2", 64, False, 1, 0.1, None, ("fp64", "mixed", "learned"), 200),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c5", choices=sorted(CONFIGS))
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ucns", choices=["ucns", "reference"])
    ap.add_argument("--n", type=int, default=0, help="lattice cells per direction (0: the configuration's)")
    ap.add_argument("--history-steps", type=int, default=-1,
                    help="steps of the fixed-error comparison (-1: the configuration's, 0: none)")
    ap.add_argument("--history-every", type=int, default=10)
    ap.add_argument("--history-out", default="", help="write the diagnostics histories to this JSON file")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--integrator", type=int, default=0, choices=[0, 1],
                    help="0: SSP-RK3 (the benchmark configuration), 1: the paper's SSP(5,4) (5 stages per step)")
    ap.add_argument("--train-epochs", type=int, default=60,
                    help="indicator training epochs of the learned form (fewer: faster setup, more flagged cells)")
    ap.add_argument("--check-bound", type=float, default=1e-4,
                    help="plain-scheme check: largest relative difference of the gated and full KE rates")
    ap.add_argument("--forms", default="", help="comma list of forms to time (default: the configuration's)")
    ap.add_argument("--order", type=int, default=2, choices=[2, 3, 4],
                    help="reconstruction degree (3, 4: CWENOZ on the hexahedral configurations; FP64 and mixed forms)")
    return ap.parse_args()


def workload(cfg: Config, n: int):
    from paper_2609_07387_gb300 import inputs as I

    nodes, cells, box = I.hex_lattice(n, jitter=0.1, seed=cfg.seed)
    if cfg.tets:
        cells = I.split_tets(cells)
    if cfg.perturb_seed is not None:
        U = I.tgv_perturbed_state(nodes, cells, cfg.mach, 0.05, seed=cfg.perturb_seed)
    else:
        U = I.tgv_state(nodes, cells, cfg.mach)
    return nodes, cells, box, U


def rk_name() -> str:
    return "SSP(5,4)" if STAGES == 5 else "SSP-RK3"


def config_json(cfg: Config, n: int, N: int, world: int, order: int = 2) -> dict:
    wl = f"{cfg.key.upper()}: " + cfg.describe(n, N)
    if order != 2:
        wl = wl.replace("P2 CWENOZ", f"P{order} CWENOZ")
    return {
        "workload": wl,
        "cells": N,
        "stages_per_step": STAGES,
        "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
        "l2": "inputs larger than L2 (the pseudo-inverses alone exceed 129 MB)",
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


def measured_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source for this workload and form (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d.get(f"{kernel}/{workload}")
        if e and e.get("source_hash") == kernel_source_hash():
            return e["dram_bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        pass
    return None


# ------------------------------------------------------------ CPU oracle
def oracle_sample(nodes, cells, box, U, cfg: Config, n: int, n_cells: int, order: int = 2):
    """Build the oracle on the workload and pick a sample of about n_cells
    cells: whole z-layers of the lattice (for tetrahedra, 6 per hexahedron,
    consecutive in the split's numbering)."""
    import oracle as O

    oc = O.Case(nodes, cells, box, O.Params(order=order, scheme=1, Re=1600.0, Mach=cfg.mach, cfl=0.5,
                                            integrator=1 if STAGES == 5 else 0))
    per_layer = n * n * (6 if cfg.tets else 1)
    layers = n_cells / per_layer if n_cells < per_layer else n_cells // per_layer
    sel = np.arange(min(int(layers * per_layer), len(cells)), dtype=np.int64)
    oc.residual_subset(U, sel)  # untimed: the lazy precompute of the sample's stencils
    return oc, sel, layers


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


def sample_text(cfg: Config, sel, N: int, layers, n: int) -> str:
    what = (f"{layers:g} z-layers of the {n}^3 lattice" if layers >= 1 else
            f"the first {sel.size} cells of one z-layer of the {n}^3 lattice") + \
        (", 6 tetrahedra per hexahedron" if cfg.tets else "")
    return (f"one {rk_name()} step ({STAGES} residual evaluations + updates) of {sel.size} of the {N} cells "
            f"({what}), precompute excluded")


def cpu_baseline(nodes, cells, box, U, cfg: Config, n: int, order: int = 2) -> dict:
    oc, sel, layers = oracle_sample(nodes, cells, box, U, cfg, n, 65536 if order == 2 else 2048, order)
    dt = 1e-4
    t0 = time.perf_counter()
    oracle_rk_step_on_sample(oc, U, sel, dt)
    t = time.perf_counter() - t0
    return {"value": sel.size * STAGES / t, "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
            "sample": sample_text(cfg, sel, len(cells), layers, n), "seconds": t}


def run_reference(args, cfg: Config, n: int, rank: int, world: int):
    if rank != 0:
        return
    nodes, cells, box, U = workload(cfg, n)
    oc, sel, layers = oracle_sample(nodes, cells, box, U, cfg, n, 32768 if args.order == 2 else 1024, args.order)
    dt = 1e-4
    for _ in range(args.warmup):
        oracle_rk_step_on_sample(oc, U, sel, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_rk_step_on_sample(oc, U, sel, dt)
    t = time.perf_counter() - t0
    value = sel.size * STAGES * args.steps / t
    sample = "each step: " + sample_text(cfg, sel, len(cells), layers, n)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": config_json(cfg, n, len(cells), 1, args.order),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": omp_threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU arm
def algorithmic(m, kind: str, mixed: bool, frac_dir: float = 1.0) -> dict:
    """Flops and bytes of one launch of the face or reconstruction kernel.
    flops: as counted above.  bytes: each array element the kernel needs
    crossing HBM once (neighbour gathers served by cache), in two countings:
      "alg": the minimal data -- per Gauss point its position relative to the
        owner's centroid and its area vector (6 words), per face the offset
        between the two centroids (3 words), the penalty factor, two cell ids
        and five face totals; per cell the K+1 coefficients of its 5 variables
        read once (face kernel); the pseudo-inverses, stencil ids, the state,
        the cell geometry the kernel needs (second moments and 1/h) and the
        coefficients written (reconstruction);
      "layout": the arrays as this build stores them (10 words per Gauss point,
        coefficient rows padded to 16 bytes)."""
    w = 4 if mixed else 8
    N, F, nq = m.n_cells, m.n_faces, m.nq
    coef = (m.K + 1) * 5 * w
    if m.K > 9:
        return algorithmic_ho(m, kind, w)
    if kind == "face":
        flops = FLOPS_FACE_P2_VISC_PER_QP * nq * F
        face_common = 4 + 2 * 4 + 5 * w            # penalty (FP32 in both forms' count), ids, totals
        alg = F * (nq * 6 * w + 3 * w + face_common) + N * coef
        row = (((m.K + 1) * 5 + 3) // 4 * 4) * 4 if mixed else coef
        layout = F * (nq * 10 * w + w + 2 * 4 + 5 * w) + N * row
    else:
        lin = FLOPS_RECON_P2_LINEAR_PER_CELL if m.K == 9 else 5 * 2 * m.K * m.Mc
        cw = FLOPS_RECON_P2_CWENOZ_PER_CELL if m.nd else lin
        flops = N * (lin + frac_dir * (cw - lin))
        cell = 7 * w                                 # six second moments and 1/h
        state = 5 * 8                                # the FP64 state, or its float pair
        base = m.K * m.Mc * w + m.Mc * 4 + cell + state
        dirb = m.nd * 3 * m.Md * w + m.nd * m.Md * 4
        alg = N * (base + coef + frac_dir * dirb)
        row = (((m.K + 1) * 5 + 3) // 4 * 4) * 4 if mixed else coef
        layout = N * (base + row + frac_dir * dirb)
    return {"flops": flops, "alg": alg, "layout": layout}


# exponents of the basis monomials beyond P2 (the kernels' order), for the P3/P4 flop counts
_BASIS_HO = [(3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1), (0, 1, 2),
             (0, 0, 3), (4, 0, 0), (3, 1, 0), (3, 0, 1), (2, 2, 0), (2, 1, 1), (2, 0, 2), (1, 3, 0), (1, 2, 1),
             (1, 1, 2), (1, 0, 3), (0, 4, 0), (0, 3, 1), (0, 2, 2), (0, 1, 3), (0, 0, 4)]
_BASIS_P2 = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)]


def algorithmic_ho(m, kind: str, w: int = 8) -> dict:
    """Flops and bytes of one launch of the P3/P4 kernels (w: bytes per word,
    8 in the FP64 form, 4 in the mixed one; ids 4, the state 8), counted
    from their source: face, per Gauss point, 2 sides x 5 variables x 2 flops
    x (K value terms + one gradient term per nonzero exponent), the
    monomials' products (4 per mode and side), HLLC 138, viscous 120,
    penalty/averages 80, scaling and sum 20; reconstruction, per cell, the
    central contraction and differences, the directional contractions twice,
    the smoothness forms (K^2 central, Kd^2 per candidate) and the weights."""
    basis = (_BASIS_P2 + _BASIS_HO)[:m.K]
    N, F, nq, K = m.n_cells, m.n_faces, m.nq, m.K
    kd = m.Md // 2
    if kind == "face":
        g = sum(sum(1 for e in b if e) for b in basis)
        flops = F * nq * (2 * 5 * 2 * (K + g) + 2 * 4 * K + 358)
        alg = F * (nq * 6 * w + 3 * w + 4 + 2 * 4 + 5 * w) + N * (K + 1) * 5 * w
        row = (((K + 1) * 5 + 3) // 4 * 4) * 4 if w == 4 else (K + 1) * 5 * w  # mixed: 16-byte rows
        layout = F * (nq * 10 * w + w + 2 * 4 + 5 * w) + N * row
    else:
        cen = 5 * (2 * K * m.Mc + m.Mc)
        dirf = 5 * 2 * (2 * m.nd * kd * m.Md + m.nd * m.Md) + 5 * 2 * (K * K + m.nd * kd * kd) + 5 * 60
        flops = N * (cen + (dirf if m.nd else 0) + 5 * 2 * K)
        alg = N * (K * m.Mc * w + m.Mc * 4 + m.nd * (kd * m.Md * w + m.Md * 4) + (K * (K + 1) // 2) * w * (m.nd > 0)
                   + (K - 3) * w + w + 5 * 8 + (K + 1) * 5 * w)
        layout = alg
    return {"flops": flops, "alg": alg, "layout": layout}


def roofline(m, prof: dict, form: str, peaks: dict, workload_key: str, frac_dir: float = 1.0) -> dict:
    mixed = form != "fp64"
    kinds = {k: v for k, v in prof.items() if v[1] > 0 and k in ("recon", "face")}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms, dom_n = kinds[dom]
    avg_s = dom_ms / dom_n / 1e3
    a = algorithmic(m, dom, mixed, frac_dir)
    names = {("face", False): "k_face<2,true>", ("recon", False): "k_recon<2,true,nd>",
             ("face", True): "k_face_mx<2,true>", ("recon", True): "k_recon_mx<2,true,nd>"}
    name = names[(dom, mixed)]
    if m.K > 9:
        o = 3 if m.K == 19 else 4
        if dom == "face":  # the mixed face kernel is one kernel for every order
            name = "k_face_mx<%d,true>" % o if mixed else "k_face_ho<%d,true>" % o
        else:
            name = "k_recon_ho%s<%d,true>" % ("_mx" if mixed else "", o)
    if dom == "recon" and mixed and frac_dir < 1.0:
        name = "k_recon_mx<2,false,nd,gated>"
    alu_peak = peaks["fp32"] if mixed else peaks["fp64"]
    alu_src = ("FP32 FMA microbenchmark (ucns_alu_peak), of measured" if mixed
               else "FP64 FMA microbenchmark (ucns_alu_peak), of measured")
    alu = a["flops"] / avg_s / 1e12
    bw = a["alg"] / avg_s / 1e9
    alu_frac, hbm_frac = alu / alu_peak, bw / peaks["hbm"]
    if alu_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu_frac,
                "peak_source": alu_src}
    else:
        roof = {"bound": "hbm", "achieved": bw, "peak": peaks["hbm"], "unit": "GB/s", "frac": hbm_frac,
                "peak_source": peaks["hbm_source"]}
    roof.update({"kernel": name, "traffic": measured_traffic(name, f"{workload_key}/{form}"),
                 "avg_launch_ms": avg_s * 1e3, "algorithmic_flops_per_launch": a["flops"],
                 "algorithmic_bytes_per_launch": a["alg"], "layout_bytes_per_launch": a["layout"],
                 "alu_frac": alu_frac, "hbm_frac": hbm_frac,
                 "hbm_frac_layout_bytes": a["layout"] / avg_s / 1e9 / peaks["hbm"]})
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
    `cells_per_rank` cells for `steps` Runge-Kutta steps."""
    t = max_over_ranks(t_local, world, device)
    return t, world * cells_per_rank * STAGES * steps / t


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs, burst copy (of measured)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "6.8 TB/s, an earlier GB300 measurement (of fallback: MEASURED_PEAKS.json absent)"


def run_ucns(args, cfg: Config, n: int, rank: int, world: int, local_rank: int):
    import torch
    import torch.distributed as dist

    from paper_2609_07387_gb300 import gate, ucns

    torch.cuda.set_device(local_rank)
    t_setup = time.perf_counter()
    nodes, cells, box, U_user = workload(cfg, n)
    N = len(cells)
    stream = torch.cuda.current_stream()
    base = dict(order=args.order, scheme=1, Re=1600.0, Mach=cfg.mach, cfl=0.5, integrator=args.integrator)
    forms = [f for f in (args.forms.split(",") if args.forms else cfg.forms) if f]
    if args.order > 2:
        forms = [f for f in forms if f != "learned"]  # the gate is built for P2
    # one FP64 mesh and one mixed mesh: the learned form is the mixed mesh with the gate attached
    m64 = ucns.Mesh(nodes, cells, box, ucns.Params(precision=0, **base))
    mx = ucns.Mesh(nodes, cells, box, ucns.Params(precision=1, **base)) if set(forms) - {"fp64"} else None
    mesh_of = {"fp64": m64, "mixed": mx, "learned": mx}
    U0 = np.ascontiguousarray(m64.to_internal(U_user))
    gate_info, net, thr = None, None, None
    if "learned" in forms:
        # untimed setup: labels from plain FP64 CWENOZ steps, training, threshold
        t0 = time.perf_counter()
        Uc = torch.from_numpy(U0.copy()).cuda()
        S = gate.collect(m64, Uc, cfg.label_steps, every=5)
        del Uc
        y = (S.dev > gate.LABEL_THRESHOLD).float()
        nsnap = cfg.label_steps // 5 + 1
        ntr = max(1, nsnap - 2) * N
        net = gate.train(S.X[:ntr].contiguous(), y[:ntr].contiguous(), epochs=args.train_epochs, lr=1e-3,
                         batch=4096, seed=0)
        thr = gate.threshold_for_recall(net, S.X[ntr:ntr + N].contiguous(), y[ntr:ntr + N].contiguous(), 0.999)
        held = gate.confusion(net, S.X[ntr + N:].contiguous(), y[ntr + N:].contiguous(), thr)
        gate_info = {"label_steps": cfg.label_steps, "train_samples": ntr, "train_epochs": args.train_epochs,
                     "troubled_fraction": float(y.mean().item()), "threshold": thr,
                     "held_out_last_snapshot": held, "setup_s": time.perf_counter() - t0,
                     "eval_every": 5, "check_every": 50, "check_bound": args.check_bound}
        del S, y

    def attach(kind: str):
        """Configure the mixed mesh for a form: no gate, the trained network,
        all-linear (caller flags all zero) or the hand-set jump rule."""
        mx.gate_set_flags(None)
        mx.gate_enable(False)
        if kind == "learned":
            gate.GatedRun(mx, net, thr, check_every=50, bound=args.check_bound, eval_every=5)
        elif kind == "linear":
            mx.gate_set_flags(torch.zeros(N, dtype=torch.uint8, device="cuda"))
        elif kind == "rule":
            gate.GatedRun(mx, gate.rule_network(0.05), 1e-6, check_every=50, bound=args.check_bound, eval_every=5)

    bus = None
    try:
        bus = torch.cuda.get_device_properties(local_rank).pci_bus_id
    except Exception:
        bus = None

    def barrier():
        if world > 1:
            dist.barrier()

    prof_steps = min(args.steps, 50)
    setup_s = time.perf_counter() - t_setup

    def timed(form):
        m = mesh_of[form]
        if m is mx:
            attach(form)
        U = torch.from_numpy(U0.copy()).cuda()
        m.rk_steps(U, args.warmup)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(bus) as clk:
            torch.cuda.nvtx.range_push(f"timed {form}")  # lets a profiler select the timed kernels
            e0.record(stream)
            m.rk_steps(U, args.steps)  # the library's multi-step call: K steps, dt on the device
            e1.record(stream)
            torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        m.check_state()
        status = m.gate_status() if form == "learned" else None
        flagged = m.gate_flagged() / N if form == "learned" else None
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
        del Up
        t, value = job_throughput(ms / 1e3, N, args.steps, world)
        return {"t": t, "ms": ms, "prof": prof, "clocks": clk.summary(), "value": value, "gate": status,
                "flagged": flagged}

    res = {f: timed(f) for f in forms}
    # ---- the fixed-error comparison: every form from the same state with the plain FP64 run's dt sequence
    hsteps = cfg.history if args.history_steps < 0 else args.history_steps
    every = args.history_every
    hist, errs, hist_ms, hist_gate = {}, {}, {}, {}
    if hsteps > 0 and "fp64" in forms:
        dts, hist["fp64"], _ = gate.reference_history(m64, U0, hsteps, every)
        hforms = [f for f in forms if f != "fp64"]
        if "learned" in forms:
            hforms += ["linear", "rule"]  # what the gate is for: all-linear weights, and a hand-set rule
        for f in hforms:
            attach(f)
            hist[f], hist_ms[f], _ = gate.replay_history(mx, U0, dts, every)
            errs[f] = gate.history_error(hist[f], hist["fp64"])
            if f in ("learned", "rule"):
                hist_gate[f] = {**mx.gate_status(), "flagged_fraction_last_eval": mx.gate_flagged() / N}
        if args.history_out:
            with open(args.history_out, "w") as fh:
                json.dump({"every": every, "dts": dts, "diagnostics [ke, eps_s, eps_d]":
                           {k: v.tolist() for k, v in hist.items()}}, fh)
    fixed = {}
    for f in errs:
        fixed[f] = {"max_rel_err [ke, eps_s, eps_d]": errs[f], "within": max(errs[f]) <= ERROR_BOUND,
                    "ms_per_step_history": hist_ms[f] / hsteps}
        if f in hist_gate:
            fixed[f]["gate"] = hist_gate[f]
    ok_forms = ["fp64"] + [f for f in forms if f != "fp64" and fixed.get(f, {}).get("within")]
    chosen = max([f for f in ok_forms if f in res], key=lambda f: res[f]["value"]) if "fp64" in res else forms[0]
    mc = mesh_of[chosen]
    if mc is mx:
        attach(chosen)
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
    fp32, sms = ucns.alu_peak(0)
    fp32x2, _ = ucns.alu_peak(2)
    fp64, _ = ucns.alu_peak(1)
    hbm, hbm_src = hbm_peak()
    peaks = {"hbm": hbm, "hbm_source": hbm_src, "fp32": max(fp32, fp32x2) / 1e12, "fp64": fp64 / 1e12}

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
    frac_dir = r["flagged"] if (chosen == "learned" and r["flagged"] is not None) else 1.0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(nodes, cells, box, U_user, cfg, n, args.order)
    dtype = {"fp64": "f64", "mixed": "f32+f64", "learned": "f32+f64+bf16"}[chosen]
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "form": chosen,
        "fixed_error": {"bound": ERROR_BOUND, "vs": "plain FP64, same dt sequence", "steps": hsteps,
                        "every": every, "forms": {f: {"err": [float(f"{e:.2e}") for e in fixed[f]["max_rel_err [ke, eps_s, eps_d]"]],
                                                      "within": fixed[f]["within"]} for f in fixed}},
        "speedup_vs_plain_fp64": r["value"] / res["fp64"]["value"] if "fp64" in res else None,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic (seeded mesh jitter and initial state; no dataset)",
        "impl": "ucns",
        "config": config_json(cfg, n, N, world, args.order),
        "clocks": r["clocks"],
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 5 * N * 8, "d2h_bytes_per_step": 5 * N * 8 + 16,
                "steps": args.e2e_steps, "via": "ucns_rk_steps_host, pinned host buffer"},
        "gpu_launches": counted,
        "roofline": roofline(mc, prof, chosen, peaks, cfg.key, frac_dir),
        "cpu_baseline": cpu,
        "forms": {f: {"value": res[f]["value"], "ms_per_step": res[f]["ms"] / args.steps,
                      "clocks": res[f]["clocks"], "kernels": shares(res[f]["prof"]),
                      **({"gate_after_timed_steps": res[f]["gate"], "flagged_fraction": res[f]["flagged"]}
                         if res[f]["gate"] else {})} for f in res},
        "fixed_error_detail": fixed,
        "learned_gate": gate_info,
        "plain_fp64": None if "fp64" not in res else {
            "value": res["fp64"]["value"], "ms_per_step": res["fp64"]["ms"] / args.steps,
            "roofline": roofline(m64, res["fp64"]["prof"], "fp64", peaks, cfg.key, 1.0)},
        "peaks": {"hbm_gbs": peaks["hbm"], "fp32_tflops": peaks["fp32"], "fp32_scalar_tflops": fp32 / 1e12,
                  "fp32_packed_tflops": fp32x2 / 1e12, "fp64_tflops": peaks["fp64"], "sm_count": sms,
                  "source": "HBM: " + hbm_src + "; FP32/FP64: FMA microbenchmarks of this run"},
        "setup_s": setup_s,
        "kernel_source_hash": kernel_source_hash(),
    }
    print(json.dumps(line), flush=True)


def main():
    global STAGES
    args = parse()
    STAGES = 5 if args.integrator == 1 else 3
    cfg = CONFIGS[args.config]
    n = args.n or cfg.n
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, cfg, n, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ucns(args, cfg, n, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
