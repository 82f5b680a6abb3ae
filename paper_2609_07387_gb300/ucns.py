"""Thin ctypes binding of libucns (include/ucns.h).

Argument marshalling only: every step of the residual / Runge-Kutta path
runs in the library's CUDA kernels.  Device states are torch CUDA tensors of
dtype float64 and shape [5, n_cells] (contiguous), in the library's internal
cell order; ``Mesh.to_internal`` / ``Mesh.to_user`` permute numpy or torch
arrays between the caller's order and that order.  There is no CPU fallback:
loading fails loudly when the shared library is missing or cannot be built.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

UCNS_OK = 0
ERRORS = {
    -1: "UCNS_ERR_INVALID_ARG",
    -2: "UCNS_ERR_MESH",
    -3: "UCNS_ERR_STENCIL",
    -4: "UCNS_ERR_CUDA",
    -5: "UCNS_ERR_NONPHYSICAL",
    -6: "UCNS_ERR_TIMEOUT",
    -7: "UCNS_ERR_STATE",
    -8: "UCNS_ERR_NOMEM",
}

# every entry point declared in include/ucns.h
EXPORTS = (
    "ucns_mesh_create", "ucns_mesh_set_boundary", "ucns_precompute", "ucns_precompute_host", "ucns_stencil", "ucns_residual", "ucns_rk_step", "ucns_rk_steps", "ucns_rk_steps_host",
    "ucns_check_state", "ucns_probe_bounded_wait", "ucns_alu_peak", "ucns_diagnostics", "ucns_time_step", "ucns_time_step_static", "ucns_profile",
    "ucns_profile_read",
    "ucns_cell_order", "ucns_mesh_info",
    "ucns_last_error", "ucns_mesh_destroy",
    "ucns_mlp_create", "ucns_mlp_destroy", "ucns_mlp_get_params", "ucns_mlp_set_params", "ucns_mlp_forward",
    "ucns_mlp_grad", "ucns_mlp_train", "ucns_mlp_check", "ucns_mlp_hidden", "ucns_mlp_probe_bounded_wait",
    "ucns_gate_features", "ucns_gate_labels", "ucns_gate_attach", "ucns_gate_enable", "ucns_gate_flagged",
    "ucns_gate_configure", "ucns_gate_check", "ucns_gate_status", "ucns_gate_set_flags", "ucns_gate_flags", "ucns_float_pair",
)
MLP_PARAMS = 6337


class UcnsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Params(C.Structure):
    _fields_ = [
        ("order", C.c_int32), ("scheme", C.c_int32), ("precision", C.c_int32), ("integrator", C.c_int32),
        ("gamma", C.c_double), ("prandtl", C.c_double), ("reynolds", C.c_double), ("mach", C.c_double),
        ("cfl", C.c_double), ("lambda_central", C.c_double), ("epsilon", C.c_double), ("alpha", C.c_double),
    ]


class _Diag(C.Structure):
    _fields_ = [("kinetic_energy", C.c_double), ("eps_solenoidal", C.c_double),
                ("eps_dilatational", C.c_double), ("volume", C.c_double)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libucns.so (building it with nvcc first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise OSError(f"libucns.so not built: {path}")
            _build.build()
        lib = C.CDLL(path)
        P, I64, I32 = C.c_void_p, C.c_int64, C.c_int32
        for name in EXPORTS:
            getattr(lib, name)  # raises AttributeError if an export is missing
        lib.ucns_mesh_create.argtypes = [P, I64, P, I64, I32, P, C.POINTER(P)]
        lib.ucns_mesh_set_boundary.argtypes = [P, P, P]
        lib.ucns_precompute.argtypes = [P, C.POINTER(_Params)]
        lib.ucns_precompute_host.argtypes = [P, C.POINTER(_Params)]
        lib.ucns_stencil.argtypes = [P, I64, I32, P, P]
        lib.ucns_residual.argtypes = [P, P, P, P]
        lib.ucns_rk_step.argtypes = [P, P, C.POINTER(C.c_double), P]
        lib.ucns_rk_steps.argtypes = [P, P, I32, C.POINTER(C.c_double), P]
        lib.ucns_rk_steps_host.argtypes = [P, P, I32, C.POINTER(C.c_double), P]
        lib.ucns_check_state.argtypes = [P, P]
        lib.ucns_probe_bounded_wait.argtypes = [P, P]
        lib.ucns_alu_peak.argtypes = [I32, C.POINTER(C.c_double), C.POINTER(I32), P]
        lib.ucns_mlp_probe_bounded_wait.argtypes = [P, P]
        lib.ucns_diagnostics.argtypes = [P, P, C.POINTER(_Diag), P]
        lib.ucns_time_step.argtypes = [P, P, C.POINTER(C.c_double), P]
        lib.ucns_time_step_static.argtypes = [P, P, P, P]
        lib.ucns_profile.argtypes = [P, I32]
        lib.ucns_profile_read.argtypes = [P, P, P]
        lib.ucns_cell_order.argtypes = [P, P]
        lib.ucns_mesh_info.argtypes = [P, P]
        lib.ucns_last_error.restype = C.c_char_p
        lib.ucns_mesh_destroy.argtypes = [P]
        F32 = C.c_float
        lib.ucns_mlp_create.argtypes = [C.c_uint64, C.POINTER(P)]
        lib.ucns_mlp_destroy.argtypes = [P]
        lib.ucns_mlp_get_params.argtypes = [P, P]
        lib.ucns_mlp_set_params.argtypes = [P, P]
        lib.ucns_mlp_forward.argtypes = [P, P, I64, P, P]
        lib.ucns_mlp_grad.argtypes = [P, P, P, I64, F32, F32, P, P]
        lib.ucns_mlp_hidden.argtypes = [P, P, I64, P, P, P]
        lib.ucns_mlp_train.argtypes = [P, P, P, I64, I64, F32, F32, F32, P]
        lib.ucns_mlp_check.argtypes = [P, P]
        lib.ucns_gate_features.argtypes = [P, P, P, P, P]
        lib.ucns_gate_labels.argtypes = [P, P, P, P]
        lib.ucns_gate_attach.argtypes = [P, P, F32]
        lib.ucns_gate_enable.argtypes = [P, I32]
        lib.ucns_gate_flagged.argtypes = [P, P, P]
        lib.ucns_gate_configure.argtypes = [P, I32, I32, C.c_double, C.c_double]
        lib.ucns_gate_check.argtypes = [P, P, P, C.POINTER(I32), P]
        lib.ucns_gate_status.argtypes = [P, C.POINTER(I32), P, P]
        lib.ucns_gate_set_flags.argtypes = [P, P, P]
        lib.ucns_gate_flags.argtypes = [P, P, P]
        lib.ucns_float_pair.argtypes = [P, P, P, I64, P]
        for name in EXPORTS:
            if name not in ("ucns_last_error", "ucns_mesh_destroy", "ucns_mlp_destroy"):
                getattr(lib, name).restype = C.c_int
        lib.ucns_mesh_destroy.restype = None
        lib.ucns_mlp_destroy.restype = None
        _lib = lib
        return lib


def _check(lib, rc: int):
    if rc != UCNS_OK:
        raise UcnsError(rc, lib.ucns_last_error().decode())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _dev_ptr(t, n_cells: int) -> int:
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
            and tuple(t.shape) == (5, n_cells)):
        raise ValueError(f"expected a contiguous cuda float64 tensor of shape (5, {n_cells})")
    return t.data_ptr()


def alu_peak(which: int, stream=None) -> tuple[float, int]:
    """(measured FLOP/s, SM count) of this GPU: which 0 FP32 FMA, 1 FP64 FMA,
    2 FP32 FMA in packed pairs (ucns_alu_peak)."""
    lib = load()
    f = C.c_double(0.0)
    n = C.c_int32(0)
    _check(lib, lib.ucns_alu_peak(int(which), C.byref(f), C.byref(n), _stream_ptr(stream)))
    return f.value, n.value


def float_pair(u, stream=None):
    """(hi, lo) float32 device tensors of a float64 device tensor u (any shape,
    contiguous): hi = fl32(u), lo = fl32(u - hi), as the mixed form stores its
    states (ucns_float_pair)."""
    import torch

    if not (isinstance(u, torch.Tensor) and u.is_cuda and u.dtype == torch.float64 and u.is_contiguous()):
        raise ValueError("u must be a contiguous float64 CUDA tensor")
    lib = load()
    hi = torch.empty(u.shape, dtype=torch.float32, device=u.device)
    lo = torch.empty_like(hi)
    _check(lib, lib.ucns_float_pair(u.data_ptr(), hi.data_ptr(), lo.data_ptr(), u.numel(), _stream_ptr(stream)))
    return hi, lo


@dataclass
class Params:
    """Scheme parameters (defaults: the Taylor-Green configuration)."""

    order: int = 2
    scheme: int = 1           # 0 linear, 1 CWENOZ
    precision: int = 0        # 0 FP64, 1 mixed
    gamma: float = 1.4
    Pr: float = 0.71
    Re: float = 1600.0        # <= 0: inviscid
    Mach: float = 0.1
    cfl: float = 0.5
    lam_central: float = 1000.0
    eps: float = 1e-6
    alpha: float = 4.0 / 3.0
    integrator: int = 0       # 0 SSP-RK3, 1 SSP(5,4)

    def c_struct(self) -> _Params:
        return _Params(self.order, self.scheme, self.precision, self.integrator, self.gamma, self.Pr, self.Re,
                       self.Mach, self.cfl, self.lam_central, self.eps, self.alpha)


BC_SLIP_WALL, BC_SYMMETRY, BC_SUPERSONIC_OUTFLOW, BC_SUPERSONIC_INFLOW = 0, 1, 2, 3


class Mesh:
    """A mesh of hexahedra, prisms, pyramids or tetrahedra in a box whose axes
    are periodic (length > 0) or bounded (length 0: boundary faces of the
    kinds `bc` gives for the sides x-, x+, y-, y+, z-, z+, with the state
    `inflow` for supersonic inflow sides), with its device-resident precompute."""

    def __init__(self, nodes, cells, box, params: Params | None = None, bc=None, inflow=None):
        lib = load()
        self._lib = lib
        nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        box = np.ascontiguousarray(box, dtype=np.float64)
        h = C.c_void_p()
        _check(lib, lib.ucns_mesh_create(nodes.ctypes.data, nodes.shape[0], cells.ctypes.data, cells.shape[0],
                                         cells.shape[1], box.ctypes.data, C.byref(h)))
        if bc is not None:
            kinds = np.ascontiguousarray(bc, dtype=np.int32)
            inf = None if inflow is None else np.ascontiguousarray(inflow, dtype=np.float64)
            rc = lib.ucns_mesh_set_boundary(h, kinds.ctypes.data, None if inf is None else inf.ctypes.data)
            if rc != UCNS_OK:
                lib.ucns_mesh_destroy(h)
                _check(lib, rc)
        self._h = h
        self.n_cells = int(cells.shape[0])
        perm = np.zeros(self.n_cells, dtype=np.int64)
        _check(lib, lib.ucns_cell_order(h, perm.ctypes.data))
        self.perm = perm
        self.iperm = np.empty_like(perm)
        self.iperm[perm] = np.arange(self.n_cells)
        self.params = None
        self._info()
        if params is not None:
            self.precompute(params)

    def _info(self):
        info = np.zeros(8, dtype=np.int64)
        _check(self._lib, self._lib.ucns_mesh_info(self._h, info.ctypes.data))
        (self.n_cells, self.n_faces, self.K, self.Mc, self.nd, self.Md, self.nq, self.nfc) = (int(v) for v in info)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.ucns_mesh_destroy(h)
        self._h = None

    __del__ = close

    def precompute(self, params: Params):
        p = params.c_struct()
        _check(self._lib, self._lib.ucns_precompute(self._h, C.byref(p)))
        self.params = params
        self._info()
        return self

    def precompute_host(self, params: Params):
        """Host half of the precompute only (no GPU needed); enables stencil()."""
        p = params.c_struct()
        _check(self._lib, self._lib.ucns_precompute_host(self._h, C.byref(p)))
        self.params = params
        self._info()
        return self

    def stencil(self, cell: int, which: int = -1):
        """(members [M] caller ids, P [K, M]) of one stencil (after precompute_host)."""
        M = self.Mc if which < 0 else self.Md
        K = self.K if which < 0 else self.Md // 2
        mem = np.zeros(M, dtype=np.int64)
        P = np.zeros((K, M))
        _check(self._lib, self._lib.ucns_stencil(self._h, int(cell), int(which), mem.ctypes.data, P.ctypes.data))
        return mem, P

    # ---- ordering helpers -------------------------------------------------
    def to_internal(self, U_user):
        """[5, N] caller order -> internal order (numpy or torch)."""
        return U_user[:, self.perm]

    def to_user(self, U_int):
        return U_int[:, self.iperm]

    # ---- device calls -----------------------------------------------------
    def residual(self, U, R=None, stream=None):
        import torch

        if R is None:
            R = torch.empty_like(U)
        _check(self._lib, self._lib.ucns_residual(self._h, _dev_ptr(U, self.n_cells), _dev_ptr(R, self.n_cells),
                                                  _stream_ptr(stream)))
        return R

    def rk_step(self, U, dt: float | None = None, stream=None, return_dt: bool = False):
        """One step of the mesh's integrator (SSP-RK3 or SSP(5,4), Params.integrator)
        in place.  dt=None: CFL dt on the device (no sync unless return_dt); dt>0: fixed."""
        ptr = _dev_ptr(U, self.n_cells)
        if dt is not None and dt > 0:
            d = C.c_double(dt)
            _check(self._lib, self._lib.ucns_rk_step(self._h, ptr, C.byref(d), _stream_ptr(stream)))
            return dt
        if return_dt:
            d = C.c_double(0.0)
            _check(self._lib, self._lib.ucns_rk_step(self._h, ptr, C.byref(d), _stream_ptr(stream)))
            return d.value
        _check(self._lib, self._lib.ucns_rk_step(self._h, ptr, None, _stream_ptr(stream)))
        return None

    def rk_steps(self, U, n_steps: int, stream=None) -> float:
        """n_steps CFL steps of a device state U (in place) in one call; returns
        the simulated time.  Synchronises."""
        t = C.c_double(0.0)
        _check(self._lib, self._lib.ucns_rk_steps(self._h, _dev_ptr(U, self.n_cells), int(n_steps), C.byref(t),
                                                  _stream_ptr(stream)))
        return t.value

    def rk_steps_host(self, U_host, n_steps: int, stream=None) -> float:
        """n_steps on a host [5, N] float64 array/tensor (copied in and out)."""
        if isinstance(U_host, np.ndarray):
            if not (U_host.dtype == np.float64 and U_host.flags.c_contiguous and U_host.shape == (5, self.n_cells)):
                raise ValueError("U_host must be a C-contiguous float64 array of shape (5, n_cells)")
            ptr = U_host.ctypes.data
        else:
            if U_host.is_cuda or U_host.dtype.itemsize != 8 or not U_host.is_contiguous():
                raise ValueError("U_host must be a contiguous float64 host tensor")
            ptr = U_host.data_ptr()
        t = C.c_double(0.0)
        _check(self._lib, self._lib.ucns_rk_steps_host(self._h, ptr, int(n_steps), C.byref(t), _stream_ptr(stream)))
        return t.value

    def check_state(self, stream=None):
        _check(self._lib, self._lib.ucns_check_state(self._h, _stream_ptr(stream)))

    def time_step(self, U, stream=None) -> float:
        d = C.c_double(0.0)
        _check(self._lib, self._lib.ucns_time_step(self._h, _dev_ptr(U, self.n_cells), C.byref(d),
                                                   _stream_ptr(stream)))
        return d.value

    KINDS = ("recon", "face", "rk", "dt", "diag", "other", "features", "mlp")

    def profile(self, enable: bool = True):
        """Open (or close) a per-kernel CUDA-event timing window."""
        _check(self._lib, self._lib.ucns_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        ms = np.zeros(8)
        n = np.zeros(8, dtype=np.int64)
        _check(self._lib, self._lib.ucns_profile_read(self._h, ms.ctypes.data, n.ctypes.data))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.KINDS)}

    # ---- learned troubled-cell gate ---------------------------------------
    def gate_features(self, U, want_f32: bool = False, stream=None):
        """(X bf16 [N, 32], Xf float32 [N, 32] or None) features of U."""
        import torch

        X = torch.empty((self.n_cells, 32), dtype=torch.bfloat16, device=U.device)
        Xf = torch.empty((self.n_cells, 32), dtype=torch.float32, device=U.device) if want_f32 else None
        _check(self._lib, self._lib.ucns_gate_features(self._h, _dev_ptr(U, self.n_cells), X.data_ptr(),
                                                       None if Xf is None else Xf.data_ptr(), _stream_ptr(stream)))
        return X, Xf

    def gate_labels(self, U, stream=None):
        """max_{v,s} |omega_s - lambda_s| per cell (float32 [N]) of the FP64 CWENOZ scheme."""
        import torch

        dev = torch.empty(self.n_cells, dtype=torch.float32, device=U.device)
        _check(self._lib, self._lib.ucns_gate_labels(self._h, _dev_ptr(U, self.n_cells), dev.data_ptr(),
                                                     _stream_ptr(stream)))
        return dev

    def gate_attach(self, net, threshold: float):
        self._gate_net = net  # keep the network alive while attached
        _check(self._lib, self._lib.ucns_gate_attach(self._h, None if net is None else net._h, float(threshold)))

    def gate_enable(self, on: bool = True):
        _check(self._lib, self._lib.ucns_gate_enable(self._h, 1 if on else 0))

    def gate_configure(self, eval_every: int = 1, check_every: int = 10, bound: float = 1e-4,
                       bound_rate: float = 0.0):
        """Gate evaluated every `eval_every` steps; plain-scheme check every
        `check_every` steps, gate off when the estimated kinetic-energy history
        error or the dissipation difference exceeds `bound`, or the total
        KE-rate difference exceeds `bound_rate` (0: not used)."""
        _check(self._lib, self._lib.ucns_gate_configure(self._h, int(eval_every), int(check_every), float(bound),
                                                        float(bound_rate)))

    def gate_check(self, U, stream=None) -> tuple[list, bool]:
        """One plain-scheme check on U: ([total KE-rate difference, local
        KE-rate difference, estimated KE history error, solenoidal and
        dilatational dissipation differences], gate now off)."""
        rel = np.zeros(5)
        dis = C.c_int32(0)
        _check(self._lib, self._lib.ucns_gate_check(self._h, _dev_ptr(U, self.n_cells), rel.ctypes.data,
                                                    C.byref(dis), _stream_ptr(stream)))
        return rel.tolist(), bool(dis.value)

    def gate_status(self) -> dict:
        """{"enabled", "steps", "checks", "off_step" (-1: never), "last": the five measures}."""
        en = C.c_int32(0)
        cnt = np.zeros(3, dtype=np.int64)
        last = np.zeros(5)
        _check(self._lib, self._lib.ucns_gate_status(self._h, C.byref(en), cnt.ctypes.data, last.ctypes.data))
        return {"enabled": bool(en.value), "steps": int(cnt[0]), "checks": int(cnt[1]), "off_step": int(cnt[2]),
                "last": last.tolist()}

    def gate_set_flags(self, flags, stream=None):
        """Use caller flags (cuda uint8/bool tensor [N], internal order; nonzero:
        CWENOZ, 0: linear weights) in place of the network; None returns to it."""
        import torch

        if flags is None:
            _check(self._lib, self._lib.ucns_gate_set_flags(self._h, None, _stream_ptr(stream)))
            self._fixed_flags = None
            return
        f = flags.to(torch.uint8).contiguous()
        if not (f.is_cuda and tuple(f.shape) == (self.n_cells,)):
            raise ValueError(f"flags must be a cuda tensor of shape ({self.n_cells},)")
        self._fixed_flags = f  # kept alive until the stream has copied it
        _check(self._lib, self._lib.ucns_gate_set_flags(self._h, f.data_ptr(), _stream_ptr(stream)))

    def gate_flags(self, stream=None):
        """The flags of the last gate evaluation (cuda uint8 [N], internal order)."""
        import torch

        f = torch.empty(self.n_cells, dtype=torch.uint8, device="cuda")
        _check(self._lib, self._lib.ucns_gate_flags(self._h, f.data_ptr(), _stream_ptr(stream)))
        return f

    def gate_flagged(self, stream=None) -> int:
        n = C.c_int64(0)
        _check(self._lib, self._lib.ucns_gate_flagged(self._h, C.byref(n), _stream_ptr(stream)))
        return n.value

    def diagnostics(self, U, stream=None) -> dict:
        d = _Diag()
        _check(self._lib, self._lib.ucns_diagnostics(self._h, _dev_ptr(U, self.n_cells), C.byref(d),
                                                     _stream_ptr(stream)))
        return {"ke": d.kinetic_energy, "eps_s": d.eps_solenoidal, "eps_d": d.eps_dilatational,
                "volume": d.volume}


class Net:
    """The troubled-cell indicator network (32 -> 64 -> 64 -> 1) on the GPU."""

    def __init__(self, seed: int = 0):
        self._lib = load()
        h = C.c_void_p()
        _check(self._lib, self._lib.ucns_mlp_create(C.c_uint64(seed), C.byref(h)))
        self._h = h

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.ucns_mlp_destroy(h)
        self._h = None

    __del__ = close

    def params(self) -> np.ndarray:
        th = np.zeros(MLP_PARAMS, dtype=np.float32)
        _check(self._lib, self._lib.ucns_mlp_get_params(self._h, th.ctypes.data))
        return th

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        if th.size != MLP_PARAMS:
            raise ValueError(f"expected {MLP_PARAMS} parameters")
        _check(self._lib, self._lib.ucns_mlp_set_params(self._h, th.ctypes.data))

    @staticmethod
    def _x(X):
        import torch

        if not (X.is_cuda and X.dtype == torch.bfloat16 and X.is_contiguous() and X.dim() == 2 and X.shape[1] == 32):
            raise ValueError("X must be a contiguous cuda bfloat16 tensor [n, 32]")
        return X.data_ptr()

    def forward(self, X, stream=None):
        import torch

        z = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _check(self._lib, self._lib.ucns_mlp_forward(self._h, self._x(X), X.shape[0], z.data_ptr(), _stream_ptr(stream)))
        return z

    def hidden(self, X, stream=None):
        """(h1 bf16 [n, 64], z float32 [n]): the first hidden layer as fed to
        the second layer's product, and the logits."""
        import torch

        h1 = torch.empty((X.shape[0], 64), dtype=torch.bfloat16, device=X.device)
        z = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _check(self._lib, self._lib.ucns_mlp_hidden(self._h, self._x(X), X.shape[0], h1.data_ptr(), z.data_ptr(),
                                                    _stream_ptr(stream)))
        return h1, z

    def grad(self, X, y, w_pos: float = 1.0, w_neg: float = 1.0, stream=None):
        import torch

        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=X.device)
        y = y.to(torch.float32).contiguous()
        _check(self._lib, self._lib.ucns_mlp_grad(self._h, self._x(X), y.data_ptr(), X.shape[0], float(w_pos),
                                                  float(w_neg), g.data_ptr(), _stream_ptr(stream)))
        return g

    def train(self, X, y, batch: int = 4096, lr: float = 1e-3, w_pos: float = 1.0, w_neg: float = 1.0, stream=None):
        """One pass over (X, y) in consecutive batches, one Adam step each."""
        import torch

        y = y.to(torch.float32).contiguous()
        _check(self._lib, self._lib.ucns_mlp_train(self._h, self._x(X), y.data_ptr(), X.shape[0], int(batch),
                                                   float(lr), float(w_pos), float(w_neg), _stream_ptr(stream)))

    def check(self, stream=None):
        _check(self._lib, self._lib.ucns_mlp_check(self._h, _stream_ptr(stream)))
