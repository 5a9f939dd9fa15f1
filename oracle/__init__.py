"""Oracle for the Parareal/PINN Black-Scholes hot path: TEST INFRASTRUCTURE ONLY.

A plain, serial FP64 CPU implementation (``bs_oracle.c``, compiled with gcc)
plus this thin ctypes wrapper.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library and never imports it.

Paper: Ibrahim, Goetschel, Ruprecht, "Parareal with a physics-informed neural
network as coarse propagator" (arXiv:2303.03848).  Section/equation citations
are on each function in ``bs_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

COARSE_IE = 0
COARSE_PINN = 1
COARSE_PINN_INCR = 2
COARSE_PINN_IE = 3


class Params(ctypes.Structure):
    """Problem parameters of one Black-Scholes instance (tau = time to maturity)."""

    _fields_ = [
        ("K", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("r", ctypes.c_double),
        ("T", ctypes.c_double),
        ("Smax", ctypes.c_double),
        ("Nx", ctypes.c_int32),
        ("P", ctypes.c_int32),
        ("fine_steps", ctypes.c_int32),
        ("coarse_steps", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile ``bs_oracle.c`` into ``liboracle.so`` (plain -O2, ISO C, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(Params)
        i32p = ctypes.POINTER(ctypes.c_int32)
        L.orc_payoff.argtypes = [pp, dp]
        L.orc_right_bc.argtypes = [pp, ctypes.c_double]
        L.orc_right_bc.restype = ctypes.c_double
        L.orc_coefficients.argtypes = [pp, dp, dp, dp]
        L.orc_thomas.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
        L.orc_cn_step.argtypes = [pp, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_ie_step.argtypes = [pp, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_fine.argtypes = [pp, ctypes.c_int, dp, dp]
        L.orc_coarse_ie.argtypes = [pp, ctypes.c_int, dp, dp]
        L.orc_serial_fine.argtypes = [pp, dp]
        L.orc_parareal.argtypes = [pp, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int, dp, dp, i32p]
        L.orc_rel_error.argtypes = [pp, dp, dp]
        L.orc_rel_error.restype = ctypes.c_double
        L.orc_speedup_bound.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.orc_speedup_bound.restype = ctypes.c_double
        L.orc_bs_call.argtypes = [ctypes.c_double] * 5
        L.orc_bs_call.restype = ctypes.c_double
        L.orc_mlp_n_params.argtypes = [ctypes.c_int, i32p]
        L.orc_mlp_n_params.restype = ctypes.c_int64
        L.orc_mlp_eval.argtypes = [ctypes.c_int, i32p, dp, dp, dp, dp, ctypes.c_int64, dp, dp]
        L.orc_pinn_table.argtypes = [pp, ctypes.c_int, i32p, dp, dp, dp, dp]
        L.orc_pinn_loss_grad.argtypes = [
            ctypes.c_int, i32p, dp, dp, dp, dp, ctypes.POINTER(ctypes.c_int8), ctypes.c_int64,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp,
        ]
        L.orc_pinn_loss_grad_y.argtypes = [
            ctypes.c_int, i32p, dp, dp, dp, dp, ctypes.POINTER(ctypes.c_int8), dp, ctypes.c_int64,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp,
        ]
        L.orc_adam.argtypes = [ctypes.c_int64, dp, dp, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=256, P=8, fine_steps=128, coarse_steps=1) -> Params:
    return Params(K, sigma, r, T, Smax, Nx, P, fine_steps, coarse_steps)


def payoff(p: Params) -> np.ndarray:
    V = np.empty(p.Nx)
    lib().orc_payoff(ctypes.byref(p), _dp(V))
    return V


def right_bc(p: Params, tau: float) -> float:
    return lib().orc_right_bc(ctypes.byref(p), tau)


def coefficients(p: Params):
    a, b, c = np.empty(p.Nx), np.empty(p.Nx), np.empty(p.Nx)
    lib().orc_coefficients(ctypes.byref(p), _dp(a), _dp(b), _dp(c))
    return a, b, c


def thomas(lo, di, up, rhs) -> np.ndarray:
    lo, di, up, rhs = (np.ascontiguousarray(v, dtype=np.float64) for v in (lo, di, up, rhs))
    x = np.empty_like(rhs)
    rc = lib().orc_thomas(len(rhs), _dp(lo), _dp(di), _dp(up), _dp(rhs), _dp(x))
    if rc:
        raise ArithmeticError("zero pivot")
    return x


def cn_step(p: Params, dt: float, tau_new: float, V: np.ndarray) -> np.ndarray:
    a, b, c = coefficients(p)
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.empty_like(V)
    if lib().orc_cn_step(ctypes.byref(p), _dp(a), _dp(b), _dp(c), dt, tau_new, _dp(V), _dp(out)):
        raise ArithmeticError("cn step failed")
    return out


def ie_step(p: Params, dt: float, tau_new: float, V: np.ndarray) -> np.ndarray:
    a, b, c = coefficients(p)
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.empty_like(V)
    if lib().orc_ie_step(ctypes.byref(p), _dp(a), _dp(b), _dp(c), dt, tau_new, _dp(V), _dp(out)):
        raise ArithmeticError("ie step failed")
    return out


def fine(p: Params, n: int, V: np.ndarray) -> np.ndarray:
    """F over slice n (Eq. 6): fine_steps Crank-Nicolson steps."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.empty_like(V)
    if lib().orc_fine(ctypes.byref(p), n, _dp(V), _dp(out)):
        raise ArithmeticError("fine failed")
    return out


def coarse_ie(p: Params, n: int, V: np.ndarray) -> np.ndarray:
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.empty_like(V)
    if lib().orc_coarse_ie(ctypes.byref(p), n, _dp(V), _dp(out)):
        raise ArithmeticError("coarse failed")
    return out


def serial_fine(p: Params) -> np.ndarray:
    U = np.empty((p.P + 1, p.Nx))
    if lib().orc_serial_fine(ctypes.byref(p), _dp(U)):
        raise ArithmeticError("serial fine failed")
    return U


def parareal(p: Params, kind: int = COARSE_IE, g: np.ndarray | None = None, tol: float = 1e-10,
             max_iter: int | None = None):
    """Parareal, Eq. 7.  Returns (U [(P+1), Nx], norms [iters], status)."""
    if max_iter is None:
        max_iter = p.P
    U = np.empty((p.P + 1, p.Nx))
    norms = np.zeros(max(max_iter, 1))
    iters = ctypes.c_int32(0)
    if g is None:
        g = np.zeros((p.P + 1, p.Nx))
    g = np.ascontiguousarray(g, dtype=np.float64)
    st = lib().orc_parareal(ctypes.byref(p), kind, _dp(g), tol, max_iter, _dp(U), _dp(norms), ctypes.byref(iters))
    if st < 0:
        raise ArithmeticError("parareal failed")
    return U, norms[: iters.value].copy(), st


def rel_error(p: Params, U: np.ndarray, Uref: np.ndarray) -> float:
    U = np.ascontiguousarray(U, dtype=np.float64)
    Uref = np.ascontiguousarray(Uref, dtype=np.float64)
    return lib().orc_rel_error(ctypes.byref(p), _dp(U), _dp(Uref))


def speedup_bound(P: int, K: int, cc_over_cf: float) -> float:
    return lib().orc_speedup_bound(P, K, cc_over_cf)


def bs_call(S: float, K: float, r: float, sigma: float, tau: float) -> float:
    return lib().orc_bs_call(S, K, r, sigma, tau)


class MLP:
    """Network description for the oracle: widths [d_in, w1, ..., 1], flat FP64 params, input box lo/hi."""

    def __init__(self, widths, params, lo, hi):
        self.widths = np.ascontiguousarray(widths, dtype=np.int32)
        self.params = np.ascontiguousarray(params, dtype=np.float64)
        self.lo = np.ascontiguousarray(lo, dtype=np.float64)
        self.hi = np.ascontiguousarray(hi, dtype=np.float64)
        self.n_lin = len(self.widths) - 1
        assert self.params.size == n_params(self.widths)

    def _w(self):
        return self.widths.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def n_params(widths) -> int:
    w = np.ascontiguousarray(widths, dtype=np.int32)
    return int(lib().orc_mlp_n_params(len(w) - 1, w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))


def mlp_eval(m: MLP, X: np.ndarray, with_derivs: bool = True):
    """u[N] and (u_S, u_SS, u_tau)[N, 3] at points X[N, d_in]."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    N = X.shape[0]
    u = np.empty(N)
    d = np.empty((N, 3)) if with_derivs else None
    lib().orc_mlp_eval(m.n_lin, m._w(), _dp(m.params), _dp(m.lo), _dp(m.hi), _dp(X), N, _dp(u),
                       _dp(d) if d is not None else None)
    return (u, d) if with_derivs else u


def pinn_table(p: Params, m: MLP) -> np.ndarray:
    """Network values on (S_j, tau_n), n = 0..P, Dirichlet nodes exact."""
    g = np.empty((p.P + 1, p.Nx))
    if lib().orc_pinn_table(ctypes.byref(p), m.n_lin, m._w(), _dp(m.params), _dp(m.lo), _dp(m.hi), _dp(g)):
        raise MemoryError("oracle table allocation failed")
    return g


def pinn_loss_grad(m: MLP, X: np.ndarray, kind: np.ndarray, K: float, sigma: float, r: float, Smax: float,
                   smax_over_K: float = 0.0, with_grad: bool = True, y: np.ndarray | None = None):
    """Loss terms (MSE_f, MSE_b, MSE_exp) of Eqs. 12-14 and, optionally, the gradient of Eq. 11.

    y: values of the kind-4 data points (their squared misfit joins term 0)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    kind = np.ascontiguousarray(kind, dtype=np.int8)
    yv = None if y is None else np.ascontiguousarray(y, dtype=np.float64)
    terms = np.empty(3)
    g = np.empty(m.params.size) if with_grad else None
    rc = lib().orc_pinn_loss_grad_y(m.n_lin, m._w(), _dp(m.params), _dp(m.lo), _dp(m.hi), _dp(X),
                                    kind.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                    _dp(yv) if yv is not None else None, X.shape[0], K, sigma, r, Smax,
                                    smax_over_K, _dp(terms), _dp(g) if g is not None else None)
    if rc == -2:
        raise ValueError("kind outside 0..3, or kind 4 without values y")
    if rc:
        raise MemoryError("oracle loss allocation failed")
    return (terms, g) if with_grad else terms


def adam(theta, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step t (1-based) on FP64 arrays."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib().orc_adam(theta.size, _dp(theta), _dp(m), _dp(v), _dp(g), t, lr, b1, b2, eps)
