"""The halo exchange a split of the periodic box would need, on two gloo ranks
(CPU): each rank owns one slab of the box (the lower or the upper half in z)
and holds only its own cells' states; the halo plan is every cell the slab's
residual depends on (the stencil members of the slab's cells and of their face
neighbours, Eqs. 2-6) that the other rank owns; the ranks send each other
those cells' states (point-to-point), then each evaluates the residual of its
own slab.  It must equal the single-mesh residual of those cells bit for bit,
and a cell missing from the plan must show (its state left unset).

This covers the host logic of the exchange only: the GPU path runs the whole
periodic mesh on one GPU (the wrap is in-mesh) and no multi-GPU path is built."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
import torch.distributed as dist
import oracle as O
from paper_2609_07387_gb300 import inputs as I

rank = int(os.environ["RANK"]); world = int(os.environ["WORLD_SIZE"])
drop = os.environ.get("DROP_ONE") == "1"
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:" + os.environ["MASTER_PORT"], rank=rank,
                        world_size=world)
nodes, cells, box = I.hex_lattice((6, 6, 20), jitter=0.1, seed=3)
oc = O.Case(nodes, cells, box, O.Params(order=2, scheme=1, Re=1600.0, Mach=0.3))
_, cen, _ = oc.geometry()
owner = (cen[:, 2] >= np.pi).astype(int)  # rank 0: lower half, rank 1: upper half
fo, fn, _ = oc.faces()
nbr = [set() for _ in range(oc.n_cells)]
for o, n in zip(fo, fn):
    nbr[o].add(int(n)); nbr[n].add(int(o))
memo = {}
def members(j):
    if j not in memo:
        s = set(oc.stencil(j)[0].tolist())
        for w in range(oc.nd):
            s |= set(oc.stencil(j, w)[0].tolist())
        memo[j] = s | {j}
    return memo[j]
def needs(r):
    dep = set()
    for i in np.where(owner == r)[0]:
        for j in {int(i)} | nbr[i]:
            dep |= members(j)
    return sorted(c for c in dep if owner[c] != r)
# the plan: what the other rank needs from me, and what I need from it
peer = 1 - rank
send_ids = np.array(needs(peer), dtype=np.int64)
recv_ids = np.array(needs(rank), dtype=np.int64)
if drop and rank == 0:
    recv_ids = recv_ids[1:]  # a plan missing one halo cell
U_true = I.noisy_state(nodes, cells, 0.3, 0.05, seed=6)
U = np.full_like(U_true, np.nan)
mine = np.where(owner == rank)[0]
U[:, mine] = U_true[:, mine]  # a rank holds only its own cells
# the sizes first, then the states (rank 0 sends first, rank 1 receives first)
n_out = torch.tensor([send_ids.size], dtype=torch.int64)
n_in = torch.zeros(1, dtype=torch.int64)
buf_out = torch.from_numpy(np.ascontiguousarray(U[:, send_ids]))
if rank == 0:
    dist.send(n_out, peer); dist.recv(n_in, peer)
else:
    dist.recv(n_in, peer); dist.send(n_out, peer)
need_full = np.array(needs(rank), dtype=np.int64)
buf_in = torch.zeros((5, int(n_in.item())), dtype=torch.float64)
if rank == 0:
    dist.send(buf_out, peer); dist.recv(buf_in, peer)
else:
    dist.recv(buf_in, peer); dist.send(buf_out, peer)
assert int(n_in.item()) == need_full.size
# received in the peer's order of my needs; a dropped entry leaves its cell unset
keep = np.isin(need_full, recv_ids)
U[:, need_full[keep]] = buf_in.numpy()[:, keep]
R = oc.residual_subset(U, mine)
R_single = oc.residual(U_true)[:, mine]
print(json.dumps({"rank": rank, "cells": int(mine.size), "halo": int(need_full.size),
                  "equal": bool(np.array_equal(R, R_single)), "finite": bool(np.all(np.isfinite(R)))}))
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run(drop: bool):
    port = str(_free_port())
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=port,
                   DROP_ONE="1" if drop else "0", OMP_NUM_THREADS="2")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    out = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e
        out.append(json.loads(o.strip().splitlines()[-1]))
    return out


def test_two_slab_ranks_reproduce_the_single_mesh_residual():
    res = _run(drop=False)
    for r in res:
        assert r["equal"] and r["finite"], r
        assert 0 < r["halo"] < r["cells"]  # a halo of a few layers on each side of the slab
    assert res[0]["cells"] + res[1]["cells"] == 6 * 6 * 20


def test_a_plan_missing_a_halo_cell_shows():
    res = _run(drop=True)
    assert not res[0]["finite"] and not res[0]["equal"]  # the unset state reaches the slab's residual
    assert res[1]["equal"]
