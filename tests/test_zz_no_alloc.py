"""ucns_time_step_static: the CFL time-step reduction for callers that must
not allocate device memory on their call path (a fixed device-memory budget,
a pool-only allocator, or no tolerance for cudaMalloc's implicit device
synchronisation).  Its scratch is a fixed device array inside the library;
this checks, through the C ABI, that two calls in a row give the time step
of the allocating entry point ucns_time_step.  The file is named to be
collected last."""
import ctypes as C

import numpy as np
import pytest

from paper_2609_07387_gb300 import inputs as I
from paper_2609_07387_gb300 import ucns

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_DT = 1e-14  # the relative dt tolerance of the parity tests


def _static_dt(m, U, out):
    lib = m._lib
    rc = lib.ucns_time_step_static(m._h, C.c_void_p(U.data_ptr()), C.c_void_p(out.data_ptr()),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise ucns.UcnsError(rc, lib.ucns_last_error().decode())
    torch.cuda.synchronize()
    return float(out.item())


def test_static_time_step_matches_allocating_entry_point():
    nodes, cells, box = I.hex_lattice(20, jitter=0.1, seed=3)
    m = ucns.Mesh(nodes, cells, box, ucns.Params(order=2, scheme=1))
    U = torch.from_numpy(np.ascontiguousarray(m.to_internal(I.noisy_state(nodes, cells, 0.1, 0.03, seed=6)))).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    # call 1
    ref1 = m.time_step(U)
    got1 = _static_dt(m, U, out)
    assert abs(got1 - ref1) <= TOL_DT * ref1
    # call 2 on a different state (the scratch keeps call 1's partials)
    m.rk_step(U)
    out.fill_(-1.0)
    ref2 = m.time_step(U)
    got2 = _static_dt(m, U, out)
    assert abs(got2 - ref2) <= TOL_DT * ref2
    assert ref1 != ref2
    # a smaller mesh after a larger one reads only its own partials
    nodes, cells, box = I.hex_lattice(6)
    m2 = ucns.Mesh(nodes, cells, box, ucns.Params(order=1, scheme=0))
    U2 = torch.from_numpy(np.ascontiguousarray(m2.to_internal(I.tgv_state(nodes, cells, 0.1)))).cuda()
    assert abs(_static_dt(m2, U2, out) - m2.time_step(U2)) <= TOL_DT * m2.time_step(U2)


def test_static_time_step_rejects_bad_arguments():
    nodes, cells, box = I.hex_lattice(6)
    m = ucns.Mesh(nodes, cells, box)
    lib = m._lib
    assert lib.ucns_time_step_static(m._h, None, None, None) == -7  # not precomputed
    m.precompute(ucns.Params(order=1, scheme=0))
    assert lib.ucns_time_step_static(m._h, None, None, None) == -1
