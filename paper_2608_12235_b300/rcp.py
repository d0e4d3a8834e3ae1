"""Thin ctypes binding of the C ABI in include/rcp.h (librcp.so, sm_103a).

The functions below carry the C names and only marshal arguments; every step
of the protocol runs in the CUDA library.  There is no CPU fallback: if the
library or a CUDA device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librcp.so")

RCP_FP64, RCP_MIXED = 0, 1
STATUS = {0: "RCP_OK", 1: "RCP_ERR_ARG", 2: "RCP_ERR_IMAGE", 3: "RCP_ERR_OOM", 4: "RCP_ERR_NAN",
          5: "RCP_ERR_CAPACITY", 6: "RCP_ERR_TIMEOUT", 7: "RCP_ERR_MAXITER", 8: "RCP_ERR_CUDA",
          9: "RCP_ERR_UNSUPPORTED"}

# every symbol include/rcp.h declares
EXPORTS = ["rcp_config_default", "rcp_create", "rcp_destroy", "rcp_set_stream", "rcp_set_positions",
           "rcp_build_neighbors", "rcp_energy_grad", "rcp_energy_grad_at", "rcp_adam_step", "rcp_run", "rcp_profile", "rcp_shrink", "rcp_state",
           "rcp_load_state", "rcp_neighbors", "rcp_cell_keys", "rcp_size", "rcp_dim", "rcp_status_str", "rcp_last_error",
           "rcp_energy_grad_noalloc", "rcp_batch_create", "rcp_batch_run", "rcp_batch_tuning", "rcp_batch_destroy",
           "rcp_batch_last_error", "rcp_create_seated", "rcp_frozen", "rcp_cascade"]


class rcp_config(C.Structure):
    _fields_ = [("precision", C.c_int), ("phi0", C.c_double), ("eps", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("adam_eps", C.c_double), ("skin_s", C.c_double),
                ("skin_theta", C.c_double), ("skin_abs", C.c_double), ("lr_x", C.c_double),
                ("lr_kappa", C.c_double), ("delta_star0", C.c_double), ("tol", C.c_double), ("Y", C.c_int),
                ("X", C.c_int), ("n_min", C.c_longlong), ("n_down", C.c_int), ("n_cycles", C.c_int),
                ("max_iters", C.c_longlong), ("chunk", C.c_int), ("cell_occupancy", C.c_double),
                ("placement", C.c_int), ("place_rounds", C.c_int), ("walls", C.c_int),
                ("container", C.c_int)]


class rcp_stop(C.Structure):
    _fields_ = [("max_iters", C.c_longlong), ("max_seconds", C.c_double), ("shrink", C.c_int)]


class rcp_result(C.Structure):
    _fields_ = [("iters", C.c_longlong), ("rebuilds", C.c_longlong), ("pairs", C.c_longlong),
                ("stopped", C.c_int), ("kappa", C.c_double), ("max_delta", C.c_double),
                ("energy", C.c_double), ("kappa_c", C.c_double), ("phi", C.c_double), ("seconds", C.c_double),
                ("launches", C.c_longlong)]


class rcp_scalars(C.Structure):
    _fields_ = [("t", C.c_longlong), ("kappa", C.c_double), ("m_kappa", C.c_double), ("v_kappa", C.c_double),
                ("b1", C.c_double), ("b2", C.c_double), ("rung", C.c_int), ("rung_start", C.c_longlong),
                ("kappa_rung", C.c_double), ("stopped", C.c_int)]


_lib = None


class RcpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str | None = None) -> C.CDLL:
    """Load librcp.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with `python -m paper_2608_12235_b300.build`")
    L = C.CDLL(p)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    L.rcp_config_default.argtypes = [C.POINTER(rcp_config)]
    L.rcp_create.argtypes = [vp, C.c_longlong, ip, vp, C.c_ulonglong, C.POINTER(rcp_config), C.POINTER(vp)]
    L.rcp_destroy.argtypes = [vp]
    L.rcp_set_stream.argtypes = [vp, vp]
    L.rcp_set_positions.argtypes = [vp, vp, C.c_double, ip]
    L.rcp_build_neighbors.argtypes = [vp]
    L.rcp_energy_grad.argtypes = [vp, C.c_double, vp, vp, vp, vp, ip]
    L.rcp_adam_step.argtypes = [vp, vp, C.c_double, C.c_double, C.c_double, ip]
    L.rcp_energy_grad_at.argtypes = [vp, vp, vp, C.c_double, vp, vp, vp, vp]
    L.rcp_run.argtypes = [vp, C.POINTER(rcp_stop), C.POINTER(rcp_result)]
    L.rcp_profile.argtypes = [vp, C.c_longlong, dp, dp, C.POINTER(C.c_longlong)]
    L.rcp_shrink.argtypes = [vp, dp, dp]
    L.rcp_state.argtypes = [vp, vp, vp, vp, C.POINTER(rcp_scalars)]
    L.rcp_load_state.argtypes = [vp, vp, vp, vp, C.POINTER(rcp_scalars)]
    L.rcp_neighbors.argtypes = [vp, vp, vp, C.c_longlong, C.POINTER(C.c_longlong)]
    L.rcp_cell_keys.argtypes = [vp, vp]
    L.rcp_energy_grad_noalloc.argtypes = [vp, vp, C.c_longlong, vp, C.c_double, C.c_double, C.c_double,
                                          vp, vp, vp, vp, vp, vp, vp]
    L.rcp_batch_create.argtypes = [vp, ip, ip, C.POINTER(vp)]
    L.rcp_batch_run.argtypes = [vp, C.POINTER(rcp_stop), vp]
    L.rcp_batch_tuning.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.rcp_batch_destroy.argtypes = [vp]
    L.rcp_batch_last_error.argtypes = [vp]
    L.rcp_batch_last_error.restype = C.c_char_p
    L.rcp_size.argtypes = [vp]
    L.rcp_size.restype = C.c_longlong
    L.rcp_dim.argtypes = [vp]
    L.rcp_dim.restype = C.c_int
    L.rcp_create_seated.argtypes = [vp, vp, C.c_longlong, vp, C.c_longlong, ip, vp, C.c_ulonglong,
                                    C.POINTER(rcp_config), C.POINTER(vp)]
    L.rcp_frozen.argtypes = [vp]
    L.rcp_frozen.restype = C.c_longlong
    L.rcp_cascade.argtypes = [vp, vp, C.c_longlong, ip, vp, C.c_ulonglong, C.POINTER(rcp_config), vp, vp, vp, vp]
    L.rcp_status_str.argtypes = [ip]
    L.rcp_status_str.restype = C.c_char_p
    L.rcp_last_error.argtypes = [vp]
    L.rcp_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("rcp_size", "rcp_dim", "rcp_frozen", "rcp_status_str", "rcp_last_error",
                        "rcp_batch_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(st: int, h=None):
    if st != 0:
        msg = load().rcp_last_error(h).decode() if h else ""
        raise RcpError(st, msg or load().rcp_status_str(st).decode())


def _ptr(a) -> int:
    """Address of a contiguous numpy array or torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def rcp_config_default(**overrides) -> rcp_config:
    cfg = rcp_config()
    _check(load().rcp_config_default(C.byref(cfg)))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def rcp_create(diameters, box=1.0, seed: int = 0, cfg: rcp_config | None = None, d: int = 3):
    D0 = np.ascontiguousarray(diameters, dtype=np.float64)
    b = np.full(d, float(box)) if np.isscalar(box) else np.ascontiguousarray(box, dtype=np.float64)
    h = C.c_void_p()
    _check(load().rcp_create(D0.ctypes.data, D0.size, d, b.ctypes.data, seed,
                             C.byref(cfg) if cfg is not None else None, C.byref(h)))
    return h


def rcp_create_seated(fixed_d, fixed_x, diameters, box=1.0, seed: int = 0, cfg: rcp_config | None = None,
                      d: int = 3):
    """Frozen spheres (contact diameters fixed_d, positions fixed_x [Nf, d])
    first, then the mobile ones (relative diameters)."""
    F = np.ascontiguousarray(fixed_d, dtype=np.float64).ravel()
    X = np.ascontiguousarray(fixed_x, dtype=np.float64).reshape(F.size, d)
    D0 = np.ascontiguousarray(diameters, dtype=np.float64).ravel()
    b = np.full(d, float(box)) if np.isscalar(box) else np.ascontiguousarray(box, dtype=np.float64)
    if cfg is None:
        cfg = rcp_config_default()
    h = C.c_void_p()
    _check(load().rcp_create_seated(F.ctypes.data, X.ctypes.data, F.size, D0.ctypes.data, D0.size, d,
                                    b.ctypes.data, seed, C.byref(cfg), C.byref(h)))
    return h


def rcp_frozen(h) -> int:
    return int(load().rcp_frozen(h))


def rcp_cascade(diameters, cls, box=1.0, seed: int = 0, cfg: rcp_config | None = None, d: int = 3):
    """The sequential cascade.  Returns (positions [N, d], contact diameters
    [N], phi of each stage [2C-1], Adam steps of each stage [2C-1])."""
    D0 = np.ascontiguousarray(diameters, dtype=np.float64).ravel()
    k = np.ascontiguousarray(cls, dtype=np.int32).ravel()
    if k.size != D0.size or k.size == 0:
        raise ValueError("one class per sphere")
    nst = 2 * (int(k.max()) + 1) - 1
    b = np.full(d, float(box)) if np.isscalar(box) else np.ascontiguousarray(box, dtype=np.float64)
    if cfg is None:
        cfg = rcp_config_default()
    x = np.zeros((D0.size, d))
    dm = np.zeros(D0.size)
    ph = np.zeros(max(nst, 1))
    it = np.zeros(max(nst, 1), dtype=np.int64)
    _check(load().rcp_cascade(D0.ctypes.data, k.ctypes.data, D0.size, d, b.ctypes.data, seed, C.byref(cfg),
                              x.ctypes.data, dm.ctypes.data, ph.ctypes.data, it.ctypes.data))
    return x, dm, ph, it


def rcp_destroy(h):
    _check(load().rcp_destroy(h))


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy


def rcp_set_stream(h, stream: int | None):
    """stream: a cudaStream_t address, None for the handle's own stream, or
    CUDA_STREAM_LEGACY for the legacy default stream (torch's default)."""
    _check(load().rcp_set_stream(h, stream), h)


def torch_stream(device=None) -> int:
    """The cudaStream_t of torch's current stream, mapping torch's default
    stream (handle 0) to cudaStreamLegacy so that work stays ordered with it."""
    import torch
    s = torch.cuda.current_stream(device).cuda_stream
    return s if s else CUDA_STREAM_LEGACY


def rcp_set_positions(h, x, kappa: float = 0.0, on_device: bool = False):
    if not on_device:
        x = np.ascontiguousarray(x, dtype=np.float64)
    _check(load().rcp_set_positions(h, _ptr(x), kappa, int(on_device)), h)


def rcp_build_neighbors(h):
    _check(load().rcp_build_neighbors(h), h)


def rcp_energy_grad(h, mu: float, E=None, grad_x=None, dE_dkappa=None, max_delta=None, on_device=False):
    """Fill the given output buffers (numpy float64 on the host, or torch
    float64 CUDA tensors with on_device=True)."""
    _check(load().rcp_energy_grad(h, mu, _ptr(E), _ptr(grad_x), _ptr(dE_dkappa), _ptr(max_delta),
                                  int(on_device)), h)


def rcp_energy_grad_at(h, x_dev, kappa_dev, mu: float, E=None, grad_x=None, dE_dkappa=None, max_delta=None):
    """Device-pointer evaluation (torch CUDA float64 tensors) on the handle's stream."""
    _check(load().rcp_energy_grad_at(h, _ptr(x_dev), _ptr(kappa_dev), mu, _ptr(E), _ptr(grad_x), _ptr(dE_dkappa),
                                     _ptr(max_delta)), h)


def rcp_adam_step(h, grad_x, dE_dkappa: float, lr_x: float, lr_kappa: float, on_device=False):
    if not on_device:
        grad_x = np.ascontiguousarray(grad_x, dtype=np.float64)
    _check(load().rcp_adam_step(h, _ptr(grad_x), dE_dkappa, lr_x, lr_kappa, int(on_device)), h)


def rcp_run(h, max_iters: int = 0, max_seconds: float = 0.0, shrink: bool = True) -> rcp_result:
    st = rcp_stop(max_iters, max_seconds, int(shrink))
    res = rcp_result()
    code = load().rcp_run(h, C.byref(st), C.byref(res))
    if code not in (0,):
        _check(code, h)
    return res


def rcp_profile(h, iters: int):
    """Run `iters` real iterations launched one by one with CUDA events around
    the pair kernel; returns (ms in the pair kernel, ms in whole iterations,
    pair-kernel launches)."""
    a, b, n = C.c_double(), C.c_double(), C.c_longlong()
    _check(load().rcp_profile(h, iters, C.byref(a), C.byref(b), C.byref(n)), h)
    return a.value, b.value, n.value


def rcp_shrink(h):
    kc, phi = C.c_double(), C.c_double()
    _check(load().rcp_shrink(h, C.byref(kc), C.byref(phi)), h)
    return kc.value, phi.value


def rcp_state(h):
    n, d = load().rcp_size(h), load().rcp_dim(h)
    x, m, v = np.zeros((n, d)), np.zeros((n, d)), np.zeros((n, d))
    s = rcp_scalars()
    _check(load().rcp_state(h, x.ctypes.data, m.ctypes.data, v.ctypes.data, C.byref(s)), h)
    return x, m, v, s


def rcp_positions(h, out=None):
    """Current positions only ([N, d] binary64), written into `out` when given
    (e.g. a page-locked array, for a direct device-to-host copy)."""
    n, d = load().rcp_size(h), load().rcp_dim(h)
    x = np.zeros((n, d)) if out is None else out
    if x.shape != (n, d) or x.dtype != np.float64 or not x.flags.c_contiguous:
        raise ValueError("out must be a C-contiguous float64 array of shape (N, d)")
    _check(load().rcp_state(h, x.ctypes.data, None, None, None), h)
    return x


def rcp_load_state(h, x, m, v, s: rcp_scalars):
    x, m, v = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, m, v))
    _check(load().rcp_load_state(h, x.ctypes.data, m.ctypes.data, v.ctypes.data, C.byref(s)), h)


def rcp_neighbors(h):
    n = load().rcp_size(h)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    P = C.c_longlong()
    _check(load().rcp_neighbors(h, rowptr.ctypes.data, None, 0, C.byref(P)), h)
    col = np.zeros(max(P.value, 1), dtype=np.int32)
    _check(load().rcp_neighbors(h, rowptr.ctypes.data, col.ctypes.data, col.size, C.byref(P)), h)
    return rowptr, col[: P.value]


def rcp_cell_keys(h):
    n = load().rcp_size(h)
    k = np.zeros(n, dtype=np.uint64)
    _check(load().rcp_cell_keys(h, k.ctypes.data), h)
    return k


def rcp_energy_grad_noalloc(x, D0, box, kappa: float, mu: float, rowptr, col, E, grad_x, dE_dkappa,
                            max_delta, eps: float = 1.0, stream: int | None = None):
    """Evaluation on caller-owned device buffers with no allocation (torch CUDA
    tensors: x float64 [N,3], D0 float64 [N], rowptr/col int32, outputs
    float64).  Asynchronous on `stream` (a cudaStream_t address)."""
    b = np.full(3, float(box)) if np.isscalar(box) else np.ascontiguousarray(box, dtype=np.float64)
    _check(load().rcp_energy_grad_noalloc(_ptr(x), _ptr(D0), int(D0.shape[0]), b.ctypes.data, kappa, mu, eps,
                                          _ptr(rowptr), _ptr(col), _ptr(E), _ptr(grad_x), _ptr(dE_dkappa),
                                          _ptr(max_delta), stream))


def rcp_size(h) -> int:
    return int(load().rcp_size(h))


def rcp_dim(h) -> int:
    return int(load().rcp_dim(h))


# ----------------------------------------------------------------- convenience
@dataclass
class RunSummary:
    iters: int
    rebuilds: int
    pairs: int
    stopped: bool
    kappa: float
    max_delta: float
    energy: float
    kappa_c: float
    phi: float
    seconds: float
    launches: int


class Packing:
    """One packing on the GPU (owns an rcp handle)."""

    def __init__(self, diameters, box=1.0, seed: int = 0, precision: int = RCP_FP64, d: int = 3,
                 fixed_d=None, fixed_x=None, **cfg):
        """fixed_d / fixed_x (optional): frozen spheres placed before the
        mobile ones (rcp_create_seated)."""
        self.cfg = rcp_config_default(precision=precision, **cfg)
        self.d = int(d)
        if fixed_d is None:
            self.n = int(np.size(diameters))
            self.h = rcp_create(diameters, box, seed, self.cfg, d=self.d)
        else:
            self.n = int(np.size(fixed_d)) + int(np.size(diameters))
            self.h = rcp_create_seated(fixed_d, fixed_x, diameters, box, seed, self.cfg, d=self.d)

    def close(self):
        if self.h:
            rcp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def energy_grad(self, mu: float):
        E, dk, md = np.zeros(1), np.zeros(1), np.zeros(1)
        g = np.zeros((self.n, self.d))
        rcp_energy_grad(self.h, mu, E, g, dk, md)
        return float(E[0]), g, float(dk[0]), float(md[0])

    def run(self, max_iters=0, max_seconds=0.0, shrink=True) -> RunSummary:
        r = rcp_run(self.h, max_iters, max_seconds, shrink)
        return RunSummary(r.iters, r.rebuilds, r.pairs, bool(r.stopped), r.kappa, r.max_delta, r.energy,
                          r.kappa_c, r.phi, r.seconds, r.launches)

    def state(self):
        return rcp_state(self.h)

    def positions(self, out=None):
        return rcp_positions(self.h, out)

    def neighbors(self):
        return rcp_neighbors(self.h)

    def cell_keys(self):
        return rcp_cell_keys(self.h)

    def set_positions(self, x, kappa=0.0):
        rcp_set_positions(self.h, x, kappa)

    def shrink(self):
        return rcp_shrink(self.h)

    def adam_step(self, g, dEdk, lr_x, lr_kappa):
        rcp_adam_step(self.h, g, dEdk, lr_x, lr_kappa)


# ----------------------------------------------------------------- batches
class Batch:
    """Independent packings advanced together by one graph of batched kernels
    (rcp_batch_*).  The packings keep ownership of their state."""

    def __init__(self, packings, autotune: bool = False):
        self.packings = list(packings)
        arr = (C.c_void_p * len(self.packings))(*[p.h.value for p in self.packings])
        b = C.c_void_p()
        st = load().rcp_batch_create(arr, len(self.packings), int(autotune), C.byref(b))
        if st != 0:
            raise RcpError(st, load().rcp_last_error(self.packings[0].h).decode())
        self.b = b

    def run(self, max_iters=0, max_seconds=0.0, shrink=True):
        n = len(self.packings)
        outs = (rcp_result * n)()
        st = rcp_stop(max_iters, max_seconds, int(shrink))
        code = load().rcp_batch_run(self.b, C.byref(st), outs)
        if code != 0:
            raise RcpError(code, load().rcp_batch_last_error(self.b).decode())
        return [RunSummary(r.iters, r.rebuilds, r.pairs, bool(r.stopped), r.kappa, r.max_delta, r.energy,
                           r.kappa_c, r.phi, r.seconds, r.launches) for r in outs]

    def tuning(self):
        a, c = C.c_int(), C.c_int()
        _check(load().rcp_batch_tuning(self.b, C.byref(a), C.byref(c)))
        return a.value, c.value

    def close(self):
        if self.b:
            load().rcp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
