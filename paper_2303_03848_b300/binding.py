"""ctypes binding of libbsparareal.so (C ABI in include/bsparareal.h).

Argument marshalling only: torch tensors provide device memory and the current
stream; every numerical step runs in the library's kernels.  If the library or
a CUDA device is missing, the calls raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbsparareal.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "bsparareal.h")

BS_OK, BS_EINVAL, BS_ECUDA, BS_ENOMEM, BS_NOT_CONVERGED, BS_DIVERGED, BS_TIMEOUT, BS_EUNSUPPORTED = range(8)
COARSE_IE, COARSE_PINN, COARSE_PINN_INCR, COARSE_PINN_IE = 0, 1, 2, 3
FP64, FP32, TF32, BF16 = 0, 1, 2, 3
PREC = {"fp64": FP64, "fp32": FP32, "tf32": TF32, "bf16": BF16}

_lock = threading.Lock()
_lib = None


class BsError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


class BsParams(ctypes.Structure):
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


class InstanceStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("status", ctypes.c_int32), ("final_norm", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("Nx", ctypes.c_int32), ("M", ctypes.c_int32), ("NW", ctypes.c_int32), ("C", ctypes.c_int32),
                ("S2", ctypes.c_int32), ("ms", ctypes.c_float), ("chosen", ctypes.c_int32)]


def lib() -> ctypes.CDLL:
    """Load the library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2303_03848_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        P = ctypes.POINTER
        L.bs_status_string.argtypes = [ctypes.c_int]
        L.bs_status_string.restype = ctypes.c_char_p
        L.bs_version.argtypes = []
        L.bs_version.restype = ctypes.c_char_p
        L.bs_problem_init.argtypes = [P(BsParams), i32, P(vp)]
        L.bs_problem_init_tuned.argtypes = [P(BsParams), i32, P(vp), P(Tuning), i32, P(i32)]
        L.bs_problem_init_partitioned.argtypes = [P(BsParams), i32, P(Tuning), i32, P(vp)]
        L.bs_problem_destroy.argtypes = [vp]
        L.bs_problem_destroy.restype = None
        L.bs_problem_info.argtypes = [vp, P(i32), P(i64), P(i64)]
        L.bs_problem_partition.argtypes = [vp, i32, P(i32), P(i32), P(i32)]
        L.bs_problem_slices_per_cta.argtypes = [vp, i32, P(i32)]
        L.bs_problem_device_status.argtypes = [vp, P(ctypes.c_int)]
        for f in (L.fine_propagate, L.coarse_propagate):
            f.argtypes = [vp, vp, vp, vp, vp]
        L.serial_fine.argtypes = [vp, vp, vp]
        L.pinn_create.argtypes = [P(i32), i32, P(dbl), P(dbl), ctypes.c_uint64, P(vp)]
        L.pinn_destroy.argtypes = [vp]
        L.pinn_destroy.restype = None
        L.pinn_num_params.argtypes = [vp, P(i64)]
        L.pinn_set_weights.argtypes = [vp, P(dbl)]
        L.pinn_get_weights.argtypes = [vp, P(dbl)]
        L.pinn_get_state.argtypes = [vp, P(dbl), P(dbl), P(dbl), P(i64)]
        L.pinn_set_state.argtypes = [vp, P(dbl), P(dbl), P(dbl), i64]
        L.bs_wait_probe.argtypes = [i32, i64, P(i32)]
        L.pinn_eval.argtypes = [vp, ctypes.c_int, vp, i64, vp, vp, vp]
        L.pinn_device_status.argtypes = [vp, P(ctypes.c_int)]
        L.pinn_loss_grad.argtypes = [vp, vp, vp, i64, P(BsParams), dbl, ctypes.c_int, vp, vp, vp]
        L.pinn_train_step.argtypes = [vp, vp, vp, i64, P(BsParams), dbl, ctypes.c_int, dbl, P(dbl), vp, vp]
        L.pinn_loss_grad_data.argtypes = [vp, vp, vp, vp, i64, P(BsParams), dbl, ctypes.c_int, vp, vp, vp]
        L.pinn_train_step_data.argtypes = [vp, vp, vp, vp, i64, P(BsParams), dbl, ctypes.c_int, dbl, P(dbl), vp, vp]
        L.parareal_solve.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, dbl, i32, vp, P(dbl), P(InstanceStats), vp]
        _lib = L
        return L


def status_string(code: int) -> str:
    return lib().bs_status_string(code).decode()


def version() -> str:
    return lib().bs_version().decode()


def wait_probe(arrive: bool, limit_cycles: int) -> int:
    """bs_wait_probe: run one bounded device wait on a barrier that is completed
    (arrive) or never completed; returns BS_OK or BS_TIMEOUT."""
    s = ctypes.c_int32(-1)
    _check(lib().bs_wait_probe(1 if arrive else 0, int(limit_cycles), ctypes.byref(s)), "bs_wait_probe")
    return s.value


# Checkpoint file of a network's training state: magic, then little-endian
# int32 layer count L and widths[L + 1], float64 lo[d_in] and hi[d_in], int64
# Adam step and n_params, then float64 theta, first and second moments.
CKPT_MAGIC = b"BSPINN01"


def write_checkpoint(path, widths, lo, hi, step, theta, mom1, mom2):
    import struct

    widths = [int(w) for w in widths]
    n = len(theta)
    if len(mom1) != n or len(mom2) != n or len(lo) != widths[0] or len(hi) != widths[0]:
        raise ValueError("inconsistent checkpoint arrays")
    with open(path, "wb") as f:
        f.write(CKPT_MAGIC)
        f.write(struct.pack("<i", len(widths) - 1))
        f.write(struct.pack(f"<{len(widths)}i", *widths))
        f.write(struct.pack(f"<{len(lo)}d", *[float(v) for v in lo]))
        f.write(struct.pack(f"<{len(hi)}d", *[float(v) for v in hi]))
        f.write(struct.pack("<qq", int(step), n))
        for a in (theta, mom1, mom2):
            f.write(np.ascontiguousarray(a, dtype="<f8").tobytes())


def read_checkpoint(path) -> dict:
    import struct

    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != CKPT_MAGIC:
        raise ValueError("not a network checkpoint")
    o = 8
    (nl,) = struct.unpack_from("<i", data, o)
    o += 4
    if not 1 <= nl <= 15:
        raise ValueError("bad layer count")
    widths = list(struct.unpack_from(f"<{nl + 1}i", data, o))
    o += 4 * (nl + 1)
    d = widths[0]
    lo = list(struct.unpack_from(f"<{d}d", data, o))
    o += 8 * d
    hi = list(struct.unpack_from(f"<{d}d", data, o))
    o += 8 * d
    step, n = struct.unpack_from("<qq", data, o)
    o += 16
    if len(data) != o + 3 * 8 * n:
        raise ValueError("truncated or oversized checkpoint")
    arr = np.frombuffer(data, dtype="<f8", count=3 * n, offset=o).astype(np.float64)
    return dict(widths=widths, lo=lo, hi=hi, step=step, theta=arr[:n].copy(), mom1=arr[n:2 * n].copy(),
                mom2=arr[2 * n:].copy())


def header_functions() -> list[str]:
    """Names of the functions the public header declares."""
    import re

    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|void|char\s*\*|const char\s*\*)\s*\*?\s*(\w+)\s*\(",
                                 src, flags=re.M)))


def _check(rc: int, what: str):
    if rc != BS_OK:
        raise BsError(rc, what)


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype, what):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{what}: expected a contiguous CUDA tensor of {dtype}")
    return ctypes.c_void_p(t.data_ptr())


_kinds_checked = {}


def check_loss_inputs(X, kind, y=None):
    """Lengths and kinds of a training batch, checked before any launch: X is
    [N][d_in], kind and y (when given) hold N entries, every kind is 0..3 or,
    with values y, 4.  The range check reads the kinds once per tensor version
    (a cache keyed by the tensor's storage, version and length), so a training
    loop over one batch pays it once."""
    n = X.shape[0] if X.dim() == 2 else -1
    if n < 0:
        raise ValueError("X must be a [N][d_in] tensor")
    if kind.dim() != 1 or kind.numel() != n:
        raise ValueError(f"kind must hold N = {n} entries (has {kind.numel()})")
    if y is not None and (y.dim() != 1 or y.numel() != n):
        raise ValueError(f"y must hold N = {n} entries (has {y.numel()})")
    top = 4 if y is not None else 3
    key = (kind.device.type, kind.data_ptr(), kind._version, n, top)
    if key not in _kinds_checked:
        if n and bool(((kind < 0) | (kind > top)).any()):
            raise ValueError(f"kind values must lie in 0..{top}" + ("" if y is not None else
                                                                     " (kind 4 needs values y)"))
        if len(_kinds_checked) > 64:
            _kinds_checked.clear()
        _kinds_checked[key] = True


def params(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=256, P=8, fine_steps=128, coarse_steps=1) -> dict:
    return dict(K=K, sigma=sigma, r=r, T=T, Smax=Smax, Nx=Nx, P=P, fine_steps=fine_steps, coarse_steps=coarse_steps)


def _to_struct(d) -> BsParams:
    return BsParams(d["K"], d["sigma"], d["r"], d["T"], d["Smax"], d["Nx"], d["P"], d["fine_steps"],
                    d["coarse_steps"])


def _cache_keys(instances) -> dict:
    """Tuning-cache key per grid size: device name, Nx and the class's slice count
    (capped at the tuner's 4096 and rounded up to a power of two)."""
    import torch

    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    slices = {}
    for p in instances:
        slices[p["Nx"]] = slices.get(p["Nx"], 0) + int(p["P"])
    out = {}
    for nx, s in slices.items():
        b = 1
        while b < min(s, 4096):
            b *= 2
        out[nx] = f"{dev}|Nx={nx}|slices={b}"
    return out


def _cache_lookup(path, instances):
    import json
    import os

    if not os.path.exists(path):
        return None
    with open(path) as f:
        cache = json.load(f)
    got = []
    for nx, key in _cache_keys(instances).items():
        e = cache.get(key)
        if e is None:
            return None
        got.append(dict(Nx=nx, M=int(e["M"]), NW=int(e["NW"]), C=int(e["C"]), S2=int(e["S2"])))
    return got


def _cache_store(path, instances, chosen):
    import json
    import os

    cache = {}
    if os.path.exists(path):
        with open(path) as f:
            cache = json.load(f)
    keys = _cache_keys(instances)
    for r in chosen:
        cache[keys[r["Nx"]]] = dict(M=r["M"], NW=r["NW"], C=r["C"], S2=r["S2"])
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class Problem:
    """Handle of bs_problem_init: one or more pricing instances on the current device."""

    def __init__(self, instances, tuned: bool = False, tuning_cache=None, partitions=None):
        """tuned: pick each grid size's partition by timing (bs_problem_init_tuned); the
        timed candidates are kept in self.tuning.  tuning_cache: path of a JSON file of
        earlier tuned choices, keyed by device, grid size and slice count; when it holds
        every grid size of the instances the problem is set up from it without timing
        (bs_problem_init_partitioned), else the tuner runs and its choices are added.
        partitions: explicit choices instead, a list of dicts with keys Nx, M, NW, C, S2
        covering every grid size (bs_problem_init_partitioned).
        self.tuning_source says which ("timed", "cache", "given" or None)."""
        if isinstance(instances, dict):
            instances = [instances]
        self.instances = [dict(p) for p in instances]
        arr = (BsParams * len(self.instances))(*[_to_struct(p) for p in self.instances])
        h = ctypes.c_void_p()
        self.tuning, self.tuning_source = [], None
        cached = _cache_lookup(tuning_cache, self.instances) if (tuned and tuning_cache) else None
        if partitions is not None:
            parts = (Tuning * len(partitions))(*[Tuning(e["Nx"], e["M"], e["NW"], e["C"], e.get("S2", 1), 0.0, 1)
                                                for e in partitions])
            _check(lib().bs_problem_init_partitioned(arr, len(self.instances), parts, len(partitions),
                                                     ctypes.byref(h)), "bs_problem_init_partitioned")
            self.tuning = [dict(e, ms=None, chosen=True) for e in partitions]
            self.tuning_source = "given"
        elif cached is not None:
            parts = (Tuning * len(cached))(*[Tuning(e["Nx"], e["M"], e["NW"], e["C"], e["S2"], 0.0, 1)
                                            for e in cached])
            _check(lib().bs_problem_init_partitioned(arr, len(self.instances), parts, len(cached), ctypes.byref(h)),
                   "bs_problem_init_partitioned")
            self.tuning = [dict(e, ms=None, chosen=True) for e in cached]
            self.tuning_source = "cache"
        elif tuned:
            cap = 256
            rep = (Tuning * cap)()
            nrep = ctypes.c_int32()
            _check(lib().bs_problem_init_tuned(arr, len(self.instances), ctypes.byref(h), rep, cap, ctypes.byref(nrep)),
                   "bs_problem_init_tuned")
            self.tuning = [dict(Nx=r.Nx, M=r.M, NW=r.NW, C=r.C, S2=r.S2, ms=r.ms, chosen=bool(r.chosen))
                           for r in rep[:min(nrep.value, cap)]]
            self.tuning_source = "timed"
            if tuning_cache:
                _cache_store(tuning_cache, self.instances, [r for r in self.tuning if r["chosen"]])
        else:
            _check(lib().bs_problem_init(arr, len(self.instances), ctypes.byref(h)), "bs_problem_init")
        self._h = h
        n, ts, tl = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().bs_problem_info(h, ctypes.byref(n), ctypes.byref(ts), ctypes.byref(tl)), "bs_problem_info")
        self.n_instances, self.total_state, self.total_slice = n.value, ts.value, tl.value
        self.state_off, self.slice_off = [], []
        so = sl = 0
        for p in self.instances:
            self.state_off.append(so)
            self.slice_off.append(sl)
            so += (p["P"] + 1) * p["Nx"]
            sl += p["P"] * p["Nx"]

    def close(self):
        if getattr(self, "_h", None):
            lib().bs_problem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def partition(self, i: int = 0) -> dict:
        """Rows per thread M, warps per CTA NW and CTAs per grid C chosen for instance i."""
        M, NW, C = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().bs_problem_partition(self._h, i, ctypes.byref(M), ctypes.byref(NW), ctypes.byref(C)),
               "bs_problem_partition")
        return dict(M=M.value, NW=NW.value, C=C.value)

    def slices_per_cta(self, i: int = 0) -> int:
        """1, or 2 when instance i's fine propagation runs two slices per CTA."""
        s = ctypes.c_int32()
        _check(lib().bs_problem_slices_per_cta(self._h, i, ctypes.byref(s)), "bs_problem_slices_per_cta")
        return s.value

    def device_status(self) -> int:
        """Synchronises and returns the problem's device status word (BS_OK or BS_TIMEOUT)."""
        s = ctypes.c_int()
        _check(lib().bs_problem_device_status(self._h, ctypes.byref(s)), "bs_problem_device_status")
        return s.value

    # views -------------------------------------------------------------
    def state_view(self, U, i: int):
        p = self.instances[i]
        o = self.state_off[i]
        return U[o:o + (p["P"] + 1) * p["Nx"]].view(p["P"] + 1, p["Nx"])

    def slice_view(self, U, i: int):
        p = self.instances[i]
        o = self.slice_off[i]
        return U[o:o + p["P"] * p["Nx"]].view(p["P"], p["Nx"])

    # calls -------------------------------------------------------------
    def _prop(self, fn, U_in, U_out, active):
        import torch

        if U_out is None:
            U_out = torch.empty(self.total_slice, dtype=torch.float64, device=U_in.device)
        if U_in.numel() != self.total_slice or U_out.numel() != self.total_slice:
            raise ValueError("slice arrays must hold sum_i P_i * Nx_i doubles")
        act = _dev(active, torch.uint8, "active") if active is not None else None
        _check(fn(self._h, _dev(U_in, torch.float64, "U_in"), _dev(U_out, torch.float64, "U_out"), act, _stream()),
               fn.__name__)
        return U_out

    def fine_propagate(self, U_in, U_out=None, active=None):
        return self._prop(lib().fine_propagate, U_in, U_out, active)

    def coarse_propagate(self, U_in, U_out=None, active=None):
        return self._prop(lib().coarse_propagate, U_in, U_out, active)

    def serial_fine(self, U_out=None):
        import torch

        if U_out is None:
            U_out = torch.empty(self.total_state, dtype=torch.float64, device="cuda")
        _check(lib().serial_fine(self._h, _dev(U_out, torch.float64, "U_out"), _stream()), "serial_fine")
        return U_out

    def parareal_solve(self, coarse_kind=COARSE_IE, model=None, prec=FP64, tol=1e-10, max_iter=None, U_out=None,
                       want_stats=True):
        """Returns (U, norms [n_inst, max_iter] or None, stats list or None, status)."""
        import torch

        if max_iter is None:
            max_iter = max(p["P"] for p in self.instances)
        if U_out is None:
            U_out = torch.empty(self.total_state, dtype=torch.float64, device="cuda")
        norms = stats = None
        np_norms = None
        if want_stats:
            np_norms = np.empty(self.n_instances * max_iter)
            stats = (InstanceStats * self.n_instances)()
        rc = lib().parareal_solve(self._h, coarse_kind, model._h if model is not None else None, prec, tol, max_iter,
                                  _dev(U_out, torch.float64, "U_out"),
                                  np_norms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_stats else None,
                                  stats, _stream())
        if rc not in (BS_OK, BS_NOT_CONVERGED, BS_DIVERGED):
            raise BsError(rc, "parareal_solve")
        if want_stats:
            norms = np_norms.reshape(self.n_instances, max_iter)
            stats = [dict(iterations=s.iterations, status=s.status, final_norm=s.final_norm) for s in stats]
        return U_out, norms, stats, rc


class SolveGraph:
    """One Parareal solve captured in a CUDA graph: replay() re-runs the whole
    solve (network table, initial iterate, every iteration's propagation,
    correction and stop test) as one graph launch on the current stream.

    The device-side stop rule makes the captured iterations past convergence
    return at once.  A first solve outside the capture allocates the
    workspace; the captured call reads nothing back, so statistics come from a
    separate parareal_solve call."""

    def __init__(self, prob, coarse_kind=COARSE_IE, model=None, prec=FP64, tol=1e-10, max_iter=None):
        import torch

        self.prob = prob
        self.U = torch.empty(prob.total_state, dtype=torch.float64, device="cuda")
        args = dict(coarse_kind=coarse_kind, model=model, prec=prec, tol=tol, max_iter=max_iter, U_out=self.U,
                    want_stats=False)
        prob.parareal_solve(**args)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="thread_local"):
            prob.parareal_solve(**args)
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()
        return self.U


def _autograd_function():
    import torch

    class PinnLossFunction(torch.autograd.Function):
        """The total training loss of Eq. 11 (residual + boundary + expiry terms)
        as a differentiable function of the network's flat FP64 parameter
        vector theta.  forward loads theta into the model and runs
        pinn_loss_grad (the forward derivative streams and the adjoint on the
        device), keeping the gradient; backward returns it times the incoming
        gradient.  apply(theta, model, X, kind, prob, smax_over_K, prec, y);
        y: values of the kind-4 data points, or None."""

        @staticmethod
        def forward(ctx, theta, model, X, kind, prob, smax_over_K, prec, y):
            model.set_weights(theta.detach().to("cpu", torch.float64).numpy())
            loss3, grad = model.loss_grad(X, kind, prob, smax_over_K, prec, y=y)
            ctx.save_for_backward(grad.to(theta.device))
            return loss3.sum().to(theta.device)

        @staticmethod
        def backward(ctx, g):
            (grad,) = ctx.saved_tensors
            return grad * g, None, None, None, None, None, None, None

    return PinnLossFunction


def pinn_loss(theta, model, X, kind, prob: dict, smax_over_K=0.0, prec=FP32, y=None):
    """Total loss (Eq. 11) of `model` with parameters `theta` (FP64 tensor of
    model.n_params) on collocation points X / kind (y: values of the kind-4
    data points); differentiable in theta (the gradient is the device adjoint
    of pinn_loss_grad / pinn_loss_grad_data)."""
    return _autograd_function().apply(theta, model, X, kind, prob, smax_over_K, prec, y)


class PinnModel:
    """Handle of pinn_create: tanh MLP in (S, tau) [, sigma, r, K]."""

    def __init__(self, widths, lo, hi, seed=0):
        self.widths = [int(w) for w in widths]
        w = (ctypes.c_int32 * len(self.widths))(*self.widths)
        lo_a = (ctypes.c_double * len(lo))(*[float(v) for v in lo])
        hi_a = (ctypes.c_double * len(hi))(*[float(v) for v in hi])
        h = ctypes.c_void_p()
        _check(lib().pinn_create(w, len(self.widths) - 1, lo_a, hi_a, seed, ctypes.byref(h)), "pinn_create")
        self._h = h
        n = ctypes.c_int64()
        _check(lib().pinn_num_params(h, ctypes.byref(n)), "pinn_num_params")
        self.n_params = n.value
        self.lo, self.hi = list(lo), list(hi)

    def close(self):
        if getattr(self, "_h", None):
            lib().pinn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float64)
        if flat.size != self.n_params:
            raise ValueError("wrong parameter count")
        _check(lib().pinn_set_weights(self._h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "pinn_set_weights")

    def get_weights(self) -> np.ndarray:
        out = np.empty(self.n_params)
        _check(lib().pinn_get_weights(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "pinn_get_weights")
        return out

    def get_state(self):
        """(theta, Adam first moment, second moment, Adam step) from pinn_get_state."""
        arrs = [np.empty(self.n_params) for _ in range(3)]
        step = ctypes.c_int64()
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib().pinn_get_state(self._h, dp(arrs[0]), dp(arrs[1]), dp(arrs[2]), ctypes.byref(step)),
               "pinn_get_state")
        return arrs[0], arrs[1], arrs[2], step.value

    def set_state(self, theta, mom1, mom2, step: int):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (theta, mom1, mom2)]
        if any(a.size != self.n_params for a in arrs):
            raise ValueError("wrong parameter count")
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib().pinn_set_state(self._h, dp(arrs[0]), dp(arrs[1]), dp(arrs[2]), int(step)), "pinn_set_state")

    def save(self, path):
        """Checkpoint the training state (write_checkpoint format)."""
        theta, m1, m2, step = self.get_state()
        write_checkpoint(path, self.widths, self.lo, self.hi, step, theta, m1, m2)

    def load(self, path):
        """Resume from a checkpoint of a network of the same shape and input box."""
        c = read_checkpoint(path)
        if c["widths"] != self.widths or c["lo"] != [float(v) for v in self.lo] or \
                c["hi"] != [float(v) for v in self.hi]:
            raise ValueError("checkpoint of a different network")
        self.set_state(c["theta"], c["mom1"], c["mom2"], c["step"])

    def device_status(self) -> int:
        """Synchronise and read the device status word (BS_OK, BS_TIMEOUT or BS_EINVAL)."""
        s = ctypes.c_int(0)
        _check(lib().pinn_device_status(self._h, ctypes.byref(s)), "pinn_device_status")
        return s.value

    def eval(self, X, prec=FP64, derivs=False, out=None):
        """u_theta at the rows of X (device [N][d_in] FP64) into out (or a new tensor)."""
        import torch

        N = X.shape[0]
        u = out if out is not None else torch.empty(N, dtype=torch.float64, device=X.device)
        if u.shape != (N,):
            raise ValueError("out must have shape (N,)")
        d = torch.empty(N, 3, dtype=torch.float64, device=X.device) if derivs else None
        _check(lib().pinn_eval(self._h, prec, _dev(X, torch.float64, "X"), N, _dev(u, torch.float64, "u"),
                               _dev(d, torch.float64, "derivs") if d is not None else None, _stream()), "pinn_eval")
        return (u, d) if derivs else u

    def loss_grad(self, X, kind, prob: dict, smax_over_K=0.0, prec=FP32, y=None):
        """Loss terms and gradient; y (device doubles): values of the kind-4 data points."""
        import torch

        check_loss_inputs(X, kind, y)
        loss3 = torch.empty(3, dtype=torch.float64, device=X.device)
        grad = torch.empty(self.n_params, dtype=torch.float64, device=X.device)
        pp = _to_struct(prob)
        if y is None:
            _check(lib().pinn_loss_grad(self._h, _dev(X, torch.float64, "X"), _dev(kind, torch.int8, "kind"),
                                        X.shape[0], ctypes.byref(pp), smax_over_K, prec,
                                        _dev(loss3, torch.float64, "loss3"), _dev(grad, torch.float64, "grad"),
                                        _stream()), "pinn_loss_grad")
        else:
            _check(lib().pinn_loss_grad_data(self._h, _dev(X, torch.float64, "X"), _dev(kind, torch.int8, "kind"),
                                             _dev(y, torch.float64, "y"), X.shape[0], ctypes.byref(pp), smax_over_K,
                                             prec, _dev(loss3, torch.float64, "loss3"),
                                             _dev(grad, torch.float64, "grad"), _stream()), "pinn_loss_grad_data")
        return loss3, grad

    def train_step(self, X, kind, prob: dict, lr=1e-3, smax_over_K=0.0, prec=FP32, want_loss=False, grad_out=None,
                   y=None):
        """One Adam step on the loss; y (device doubles): values of the kind-4 data points."""
        import torch

        check_loss_inputs(X, kind, y)
        pp = _to_struct(prob)
        loss = (ctypes.c_double * 3)() if want_loss else None
        g = _dev(grad_out, torch.float64, "grad_out") if grad_out is not None else None
        if y is None:
            _check(lib().pinn_train_step(self._h, _dev(X, torch.float64, "X"), _dev(kind, torch.int8, "kind"),
                                         X.shape[0], ctypes.byref(pp), smax_over_K, prec, lr, loss, g, _stream()),
                   "pinn_train_step")
        else:
            _check(lib().pinn_train_step_data(self._h, _dev(X, torch.float64, "X"), _dev(kind, torch.int8, "kind"),
                                              _dev(y, torch.float64, "y"), X.shape[0], ctypes.byref(pp), smax_over_K,
                                              prec, lr, loss, g, _stream()), "pinn_train_step_data")
        return list(loss) if want_loss else None
