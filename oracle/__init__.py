"""CPU oracle for the explicit finite-volume residual and SSP Runge-Kutta update
(SSP-RK3 and SSP(5,4)).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it; the product path never does.

The arithmetic lives in ``ucns_oracle.c`` (plain FP64 C, compiled with
``-ffp-contract=off``); this module only compiles it with gcc and marshals
numpy arrays through ctypes.  All states are SoA ``[5, n_cells]`` float64 in
the caller's (user) cell order.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ucns_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libucns_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP over cells)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # UCNS_ORACLE_LIB: a library compiled from a modified copy of the
            # source (the mutation tests check that the pins reject it)
            lib = C.CDLL(os.environ.get("UCNS_ORACLE_LIB") or build())
            P, I64, D = C.c_void_p, C.c_int64, C.c_double
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [P, I64, P, I64, C.c_int, P, P]
            lib.orc_destroy.argtypes = [P]
            lib.orc_last_error.restype = C.c_char_p
            lib.orc_counts.argtypes = [P, P]
            lib.orc_geometry.argtypes = [P, P, P, P]
            lib.orc_faces.argtypes = [P, P, P, P]
            lib.orc_face_quad.argtypes = [P, I64, P, P]
            lib.orc_surface_sums.argtypes = [P, P]
            lib.orc_stencil.argtypes = [P, I64, C.c_int, P, P, P, P]
            lib.orc_residual.argtypes = [P, P, P]
            lib.orc_set_scheme_mask.argtypes = [P, P]
            lib.orc_residual_subset.argtypes = [P, P, I64, P, P]
            lib.orc_residual_subset_terms.argtypes = [P, P, I64, P, P, P]
            lib.orc_residual_terms.argtypes = [P, P, P, P]
            lib.orc_rk_step.restype = D
            lib.orc_rk_step.argtypes = [P, P, D]
            lib.orc_time_step.restype = D
            lib.orc_time_step.argtypes = [P, P]
            lib.orc_reconstruct.argtypes = [P, P, P, P]
            lib.orc_eval.argtypes = [P, P, I64, C.c_int, P, P, P]
            lib.orc_smoothness.restype = D
            lib.orc_smoothness.argtypes = [P, I64, P, C.c_int]
            lib.orc_kexact_probe.argtypes = [P, I64, P, C.c_int, P, P, P]
            lib.orc_kexact_probeN.argtypes = [P, I64, P, C.c_int, C.c_int, P, P, P]
            lib.orc_cell_average.argtypes = [P, C.c_int, P, C.c_int, P]
            lib.orc_diagnostics.argtypes = [P, P, P]
            lib.orc_features.argtypes = [P, P, P]
            lib.orc_hllc.argtypes = [P, P, P, D, P]
            lib.orc_viscous_flux.argtypes = [P, P, P, D, D, D, D, P]
            lib.orc_ssprk3_linear.restype = D
            lib.orc_ssprk3_linear.argtypes = [D, D, D]
            lib.orc_ssp54_linear.restype = D
            lib.orc_ssp54_linear.argtypes = [D, D, D]
            lib.orc_ssp54_coeffs.argtypes = [P]
            lib.orc_ssp54_logistic.restype = D
            lib.orc_ssp54_logistic.argtypes = [D, D, C.c_int]
            lib.orc_ssprk3_logistic.restype = D
            lib.orc_ssprk3_logistic.argtypes = [D, D, C.c_int]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Params:
    """Scheme parameters (defaults: the Taylor-Green configuration)."""

    order: int = 2
    scheme: int = 1          # 0 linear (p_opt), 1 CWENOZ
    gamma: float = 1.4
    Pr: float = 0.71
    Re: float = 1600.0       # <= 0 -> inviscid (Euler)
    Mach: float = 0.1
    cfl: float = 0.5
    lam_central: float = 1000.0
    eps: float = 1e-6
    alpha: float = 4.0 / 3.0
    integrator: int = 0      # 0 SSP-RK3, 1 SSP(5,4)
    # boundary kind of each box side x-, x+, y-, y+, z-, z+ of a non-periodic
    # axis (box length 0): 0 or 1 slip wall, 2 supersonic outflow, 3 supersonic
    # inflow of the conserved state `inflow`
    bc: tuple = (0, 0, 0, 0, 0, 0)
    inflow: tuple = (0.0, 0.0, 0.0, 0.0, 0.0)

    def array(self) -> np.ndarray:
        return np.array([self.order, self.scheme, self.gamma, self.Pr, self.Re, self.Mach, self.cfl,
                         self.lam_central, self.eps, self.alpha, self.integrator, *self.bc, *self.inflow],
                        dtype=np.float64)


class OracleError(RuntimeError):
    pass


class Case:
    """One mesh + scheme on the CPU oracle."""

    def __init__(self, nodes, cells, box, params: Params):
        lib = _load()
        self._lib = lib
        self.params = params
        nodes = _f64(nodes)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        box_a = None if box is None else _f64(box)
        self._keep = (nodes, cells, box_a)
        h = lib.orc_create(_p(nodes), nodes.shape[0], _p(cells), cells.shape[0], cells.shape[1],
                           None if box_a is None else _p(box_a), _p(params.array()))
        if not h:
            raise OracleError(lib.orc_last_error().decode())
        self._h = h
        cnt = np.zeros(8, dtype=np.int64)
        lib.orc_counts(h, _p(cnt))
        (self.n_cells, self.n_faces, self.K, self.Mc, self.nd, self.Md, self.nq, self.nfc) = (int(v) for v in cnt)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    def _check(self, rc):
        if rc:
            raise OracleError(self._lib.orc_last_error().decode())

    def geometry(self):
        n = self.n_cells
        vol, cen, hh = np.zeros(n), np.zeros((n, 3)), np.zeros(n)
        self._lib.orc_geometry(self._h, _p(vol), _p(cen), _p(hh))
        return vol, cen, hh

    def faces(self):
        F = self.n_faces
        fo, fn, sh = np.zeros(F, np.int64), np.zeros(F, np.int64), np.zeros((F, 3), np.int32)
        self._lib.orc_faces(self._h, _p(fo), _p(fn), _p(sh))
        return fo, fn, sh

    def face_quad(self, f: int):
        x, dS = np.zeros((self.nq, 3)), np.zeros((self.nq, 3))
        self._lib.orc_face_quad(self._h, f, _p(x), _p(dS))
        return x, dS

    def surface_sums(self):
        out = np.zeros((self.n_cells, 3))
        self._lib.orc_surface_sums(self._h, _p(out))
        return out

    def stencil(self, i: int, which: int = -1):
        M = self.Mc if which < 0 else self.Md
        K = self.K if which < 0 else self.Md // 2
        mem, sh = np.zeros(M, np.int64), np.zeros((M, 3), np.int32)
        A, P = np.zeros((M, K)), np.zeros((K, M))
        self._check(self._lib.orc_stencil(self._h, i, which, _p(mem), _p(sh), _p(A), _p(P)))
        return mem, sh, A, P

    def set_scheme_mask(self, mask):
        """Per-cell scheme of a CWENOZ case (Sec. 2.2, Eqs. 5-6): cells with a
        nonzero mask entry keep CWENOZ, the others take the optimal central
        polynomial p_opt (linear weights).  mask: [n_cells] in the caller's
        cell order, or None for CWENOZ everywhere.  Every later residual,
        reconstruction and step of the case follows it."""
        if mask is None:
            self._check(self._lib.orc_set_scheme_mask(self._h, None))
            self._mask = None
            return
        m = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
        if m.shape != (self.n_cells,):
            raise ValueError(f"mask must have shape ({self.n_cells},)")
        self._check(self._lib.orc_set_scheme_mask(self._h, _p(m)))
        self._mask = m

    def residual(self, U):
        U = _f64(U)
        R = np.zeros_like(U)
        self._check(self._lib.orc_residual(self._h, _p(U), _p(R)))
        return R

    def residual_terms(self, U):
        """(R, S): the residual and S_i = (1/|V_i|) sum_f |G_f| per component,
        the magnitude of the face-flux terms whose signed sum is R."""
        U = _f64(U)
        R, S = np.zeros_like(U), np.zeros_like(U)
        self._check(self._lib.orc_residual_terms(self._h, _p(U), _p(R), _p(S)))
        return R, S

    def residual_subset(self, U, cells):
        """Residual [5, len(cells)] of the given cells only (same arithmetic)."""
        U = _f64(U)
        sel = np.ascontiguousarray(cells, dtype=np.int64)
        R = np.zeros((5, sel.size))
        self._check(self._lib.orc_residual_subset(self._h, _p(U), sel.size, _p(sel), _p(R)))
        return R

    def residual_subset_terms(self, U, cells):
        """(R, S) [5, len(cells)] of the given cells only (same arithmetic)."""
        U = _f64(U)
        sel = np.ascontiguousarray(cells, dtype=np.int64)
        R, S = np.zeros((5, sel.size)), np.zeros((5, sel.size))
        self._check(self._lib.orc_residual_subset_terms(self._h, _p(U), sel.size, _p(sel), _p(R), _p(S)))
        return R, S

    def time_step(self, U) -> float:
        U = _f64(U)
        return float(self._lib.orc_time_step(self._h, _p(U)))

    def rk_step(self, U, dt: float = 0.0):
        """Return (U_new, dt_used); dt <= 0 uses the CFL time step."""
        U = np.array(U, dtype=np.float64, copy=True, order="C")
        dt = self._lib.orc_rk_step(self._h, _p(U), float(dt))
        if dt < 0:
            raise OracleError(self._lib.orc_last_error().decode())
        return U, float(dt)

    def reconstruct(self, U, weights: bool = False):
        U = _f64(U)
        coef = np.zeros((self.n_cells, 5, self.K))
        w = np.zeros((self.n_cells, 5, self.nd + 1)) if weights else None
        self._check(self._lib.orc_reconstruct(self._h, _p(U), _p(coef), None if w is None else _p(w)))
        return (coef, w) if weights else coef

    def eval(self, U, i: int, x):
        U, x = _f64(U), _f64(np.atleast_2d(x))
        val, grad = np.zeros((x.shape[0], 5)), np.zeros((x.shape[0], 5, 3))
        self._check(self._lib.orc_eval(self._h, _p(U), i, x.shape[0], _p(x), _p(val), _p(grad)))
        return val, grad

    def smoothness(self, i: int, a, deg: int) -> float:
        a = _f64(a)
        return float(self._lib.orc_smoothness(self._h, i, _p(a), deg))

    def kexact_probe(self, i: int, poly, x):
        """Reconstruct cell i from the cell averages of a polynomial in the
        physical coordinates (poly [5][10]: up to quadratic, [5][20]: up to
        cubic, [5][35]: up to quartic; terms as in the C source) and evaluate
        it at the points x."""
        poly, x = _f64(poly), _f64(np.atleast_2d(x))
        val, grad = np.zeros((x.shape[0], 5)), np.zeros((x.shape[0], 5, 3))
        if poly.shape[-1] == 10:
            self._check(self._lib.orc_kexact_probe(self._h, i, _p(poly), x.shape[0], _p(x), _p(val), _p(grad)))
        else:
            self._check(self._lib.orc_kexact_probeN(self._h, i, _p(poly), poly.shape[-1], x.shape[0], _p(x),
                                                    _p(val), _p(grad)))
        return val, grad

    def cell_average(self, kind: str, p, nq1d: int = 5):
        kinds = {"tgv": 0, "density_wave": 1, "vortex": 2}
        p = _f64(p)
        U = np.zeros((5, self.n_cells))
        self._lib.orc_cell_average(self._h, kinds[kind], _p(p), nq1d, _p(U))
        return U

    def features(self, U):
        """Troubled-cell indicator features [n_cells, 32] (FP64)."""
        U = _f64(U)
        F = np.zeros((self.n_cells, 32))
        self._check(self._lib.orc_features(self._h, _p(U), _p(F)))
        return F

    def labels(self, U, threshold: float = 1e-2):
        """max over variables and stencils of |omega_s - lambda_s| under the
        CWENOZ weights, and the label (deviation > threshold)."""
        _, w = self.reconstruct(U, weights=True)
        lam = np.array([self.params.lam_central] + [1.0] * self.nd) / (self.params.lam_central + self.nd)
        dev = np.abs(w - lam[None, None, :]).max(axis=(1, 2))
        return dev, dev > threshold

    def diagnostics(self, U):
        U = _f64(U)
        out = np.zeros(3)
        self._check(self._lib.orc_diagnostics(self._h, _p(U), _p(out)))
        return out


def hllc(UL, UR, n, gamma: float = 1.4):
    lib = _load()
    UL, UR, n = _f64(UL), _f64(UR), _f64(n)
    F = np.zeros(5)
    lib.orc_hllc(_p(UL), _p(UR), _p(n), gamma, _p(F))
    return F


def viscous_flux(Uf, gradU, n, gamma=1.4, Re=1600.0, Pr=0.71, Mach=0.1):
    lib = _load()
    Uf, g, n = _f64(Uf), _f64(gradU).reshape(15), _f64(n)
    F = np.zeros(5)
    lib.orc_viscous_flux(_p(Uf), _p(g), _p(n), gamma, Re, Pr, Mach, _p(F))
    return F


def ssprk3_linear(lam: float, dt: float, u0: float = 1.0) -> float:
    return float(_load().orc_ssprk3_linear(lam, dt, u0))


def ssp54_linear(lam: float, dt: float, u0: float = 1.0) -> float:
    """One SSP(5,4) step of du/dt = lam u from u0."""
    return float(_load().orc_ssp54_linear(lam, dt, u0))


def ssp54_coefficients():
    """The oracle's SSP(5,4) Shu-Osher coefficients (alpha, beta), each [6][5]:
    row i gives u_i in terms of u_j, L(u_j), j < i."""
    out = np.zeros(60)
    _load().orc_ssp54_coeffs(_p(out))
    return out[:30].reshape(6, 5), out[30:].reshape(6, 5)


def logistic(u0: float, T: float, n: int, integrator: int) -> float:
    """n steps of u' = u (1 - u) to time T (integrator 0: SSP-RK3, 1: SSP(5,4))."""
    f = _load().orc_ssp54_logistic if integrator == 1 else _load().orc_ssprk3_logistic
    return float(f(u0, T, n))
