"""Plain FP64 CPU oracle of the Adam-based inflation protocol (arxiv 2608.12235).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its binding) never imports, links or calls it, and it
shares no code with that path.

The arithmetic lives in ``rcp_oracle.c`` (plain C, binary64, no FMA
contraction); this module builds it with gcc on first use and exposes it
through ctypes with numpy arrays.  Each C function cites the passage of the
paper it follows.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rcp_oracle.c")
_LIB = os.path.join(_HERE, "librcp_oracle.so")
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle into ``librcp_oracle.so`` beside its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


class Params(C.Structure):
    _fields_ = [("d", C.c_int), ("L", C.c_double * 3), ("phi0", C.c_double),
                ("eps", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("adam_eps", C.c_double), ("skin_s", C.c_double), ("skin_theta", C.c_double),
                ("skin_abs", C.c_double), ("lr_x", C.c_double), ("lr_kappa", C.c_double),
                ("delta_star0", C.c_double), ("tol", C.c_double), ("Y", C.c_int), ("X", C.c_int),
                ("n_min", C.c_long), ("n_down", C.c_int), ("n_cycles", C.c_int),
                ("max_iters", C.c_long), ("kappa_init", C.c_double), ("walls", C.c_int),
                ("container", C.c_int)]


class Result(C.Structure):
    _fields_ = [("iters", C.c_long), ("rebuilds", C.c_long), ("stopped", C.c_int),
                ("kappa", C.c_double), ("max_delta", C.c_double), ("energy", C.c_double),
                ("kappa_c", C.c_double), ("phi", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        L.orc_set_walls.argtypes = [C.c_int]
        L.orc_get_walls.restype = C.c_int
        L.orc_set_container.argtypes = [C.c_int]
        L.orc_get_container.restype = C.c_int
        L.orc_splitmix64_at.restype = C.c_uint64
        L.orc_splitmix64_at.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_init_positions.argtypes = [C.c_uint64, C.c_long, C.c_int, _dp, _dp]
        L.orc_place.argtypes = [C.c_uint64, C.c_long, C.c_int, _dp, _dp, C.c_double, C.c_int, _dp,
                                np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")]
        L.orc_place.restype = C.c_int
        L.orc_tree_sum.restype = C.c_double
        L.orc_tree_sum.argtypes = [_dp, C.c_long]
        L.orc_cbrt.restype = C.c_double
        L.orc_cbrt.argtypes = [C.c_double]
        L.orc_moments.argtypes = [_dp, C.c_long, _dp]
        L.orc_kappa0.restype = C.c_double
        L.orc_kappa0.argtypes = [_dp, C.c_long, C.c_int, _dp, C.c_double]
        L.orc_n_trig.restype = C.c_double
        L.orc_n_trig.argtypes = [C.c_long, C.c_int, C.c_int, C.c_int]
        L.orc_rho.restype = C.c_double
        L.orc_rho.argtypes = [C.c_double] * 4
        L.orc_levels.restype = C.c_int
        L.orc_levels.argtypes = [_dp, C.c_long, C.c_double, C.c_double, C.c_double,
                                 np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS"), _dp]
        L.orc_grid_n.restype = C.c_long
        L.orc_grid_n.argtypes = [C.c_double, C.c_long, C.c_double, C.c_double]
        L.orc_cell_keys.argtypes = [_dp, _dp, C.c_long, C.c_int, _dp, C.c_double, C.c_double,
                                    C.c_double, C.c_double, _up]
        for nm in ("orc_list_brute", "orc_list_grid"):
            f = getattr(L, nm)
            f.restype = C.c_long
            f.argtypes = [_dp, _dp, C.c_long, C.c_int, _dp, C.c_double, C.c_double, C.c_double,
                          _lp, _ip, C.c_long]
        L.orc_row_brute.restype = C.c_long
        L.orc_row_brute.argtypes = [_dp, _dp, C.c_long, C.c_int, _dp, C.c_double, C.c_double,
                                    C.c_double, C.c_long, _ip, C.c_long]
        L.orc_energy_grad_brute.argtypes = [_dp, _dp, C.c_long, C.c_int, _dp, C.c_double,
                                            C.c_double, C.c_double, _dp, _dp, _dp, _dp]
        L.orc_energy_grad_list.argtypes = [_dp, _dp, C.c_long, C.c_int, _dp, C.c_double,
                                           C.c_double, C.c_double, _lp, _ip, _dp, _dp, _dp, _dp]
        L.orc_row_grad.argtypes = [_dp, _dp, C.c_long, C.c_int, _dp, C.c_double, C.c_double,
                                   C.c_long, _dp, _dp, _dp, _dp]
        L.orc_adam_update.argtypes = [_dp, _dp, _dp, _dp, C.c_long, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_wrap.restype = C.c_double
        L.orc_wrap.argtypes = [C.c_double, C.c_double]
        L.orc_shrink_kappa.restype = C.c_double
        L.orc_shrink_kappa.argtypes = [_dp, _dp, C.c_long, C.c_int, _dp, C.c_double, _lp, _ip]
        L.orc_phi.restype = C.c_double
        L.orc_phi.argtypes = [_dp, C.c_long, C.c_int, _dp, C.c_double]
        L.orc_params_default.argtypes = [C.POINTER(Params)]
        L.orc_sample_iterations.restype = C.c_long
        L.orc_sample_iterations.argtypes = [C.POINTER(Params), _dp, C.c_long, _dp, C.c_double, C.c_double,
                                            C.c_double, C.c_double, C.c_double, C.c_long]
        L.orc_run.restype = C.c_int
        L.orc_run.argtypes = [C.POINTER(Params), _dp, C.c_long, C.c_uint64, _dp, C.c_int,
                              C.POINTER(Result), C.c_void_p, C.c_long]
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    """Threads of the oracle's row loop and Adam step (1 by default); results
    do not depend on it."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


@contextlib.contextmanager
def threads(n: int):
    old = get_threads()
    set_threads(n)
    try:
        yield
    finally:
        set_threads(old)


def _box(L, d=3):
    b = np.zeros(3)
    if np.isscalar(L):
        b[:d] = float(L)
    else:
        b[: len(L)] = np.asarray(L, dtype=np.float64)
    return b


def f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@contextlib.contextmanager
def walls(mask: int, container: int | None = None):
    """Flat hard walls (bit a: walls at 0 and L_a bound axis a) and, when
    given, the curved container (0 none, 1 ball / disk, 2 cylinder about z) for
    the calls inside the block; the previous settings are restored.  A bare
    mask may also be a (mask, container) pair."""
    if isinstance(mask, tuple):
        mask, container = mask
    L = lib()
    before = (L.orc_get_walls(), L.orc_get_container())
    L.orc_set_walls(int(mask))
    if container is not None:
        L.orc_set_container(int(container))
    try:
        yield
    finally:
        L.orc_set_walls(before[0])
        L.orc_set_container(before[1])


# ---------------------------------------------------------------- primitives
def splitmix64_at(seed: int, k: int) -> int:
    return int(lib().orc_splitmix64_at(seed, k))


def init_positions(seed: int, n: int, L=1.0, d: int = 3) -> np.ndarray:
    x = np.zeros(n * d)
    lib().orc_init_positions(seed, n, d, _box(L, d), x)
    return x.reshape(n, d)


def place(seed: int, D0, kappa: float, L=1.0, d: int = 3, max_rounds: int = 10000, x_frozen=None, wall_mask=0):
    """Non-overlapping placement by rounds of random sequential addition
    (orc_place).  Frozen spheres (D0 < 0) stay where x_frozen [n, d] has them.
    Returns (positions [n, d], round of each sphere, rounds or -1)."""
    D0 = f64(D0)
    n = D0.size
    x = np.zeros(n * d) if x_frozen is None else f64(x_frozen).ravel().copy()
    rounds = np.zeros(n, dtype=np.int32)
    with walls(wall_mask):
        r = lib().orc_place(seed, n, d, _box(L, d), D0, kappa, max_rounds, x, rounds)
    return x.reshape(n, d), rounds, int(r)


def tree_sum(a) -> float:
    a = f64(a).ravel()
    return float(lib().orc_tree_sum(a, a.size))


def cbrt(a: float) -> float:
    return float(lib().orc_cbrt(a))


def moments(D0):
    out = np.zeros(3)
    D0 = f64(D0)
    lib().orc_moments(D0, D0.size, out)
    return out


def kappa0(D0, L=1.0, phi0=0.05, d=3) -> float:
    D0 = f64(D0)
    return float(lib().orc_kappa0(D0, D0.size, d, _box(L, d), phi0))


def n_trig(n: int, d: int = 3, Y: int = 2, X: int = 9) -> float:
    return float(lib().orc_n_trig(n, d, Y, X))


def rho(D0: float, kappa_b: float, s: float, sigma0: float) -> float:
    return float(lib().orc_rho(D0, kappa_b, s, sigma0))


def levels(D0, kappa_b, s, sigma0):
    D0 = f64(D0)
    lvl = np.zeros(D0.size, dtype=np.int32)
    rml = np.zeros(32)
    nlev = lib().orc_levels(D0, D0.size, kappa_b, s, sigma0, lvl, rml)
    return lvl, rml[:nlev]


def grid_n(L: float, count: int, V: float, occ: float = 1.0) -> int:
    return int(lib().orc_grid_n(L, count, V, occ))


def cell_keys(x, D0, L, kappa_b, s, sigma0, d=3, occ=1.0):
    x = f64(x).ravel()
    D0 = f64(D0)
    key = np.zeros(D0.size, dtype=np.uint64)
    lib().orc_cell_keys(x, D0, D0.size, d, _box(L, d), kappa_b, s, sigma0, occ, key)
    return key


def _list(fn, x, D0, L, kappa_b, s, sigma0, d, wall_mask=0):
    x = f64(x).ravel()
    D0 = f64(D0)
    n = D0.size
    rowptr = np.zeros(n + 1, dtype=np.int64)
    cap = 32 * n + 64
    while True:
        col = np.zeros(cap, dtype=np.int32)
        with walls(wall_mask):
            P = fn(x, D0, n, d, _box(L, d), kappa_b, s, sigma0, rowptr, col, cap)
        if P <= cap:
            return rowptr, col[:P].copy()
        cap = P


def list_brute(x, D0, L, kappa_b, s, sigma0, d=3, wall_mask=0):
    """The listed set by definition (O(N^2)); CSR with ascending columns."""
    return _list(lib().orc_list_brute, x, D0, L, kappa_b, s, sigma0, d, wall_mask)


def list_grid(x, D0, L, kappa_b, s, sigma0, d=3, wall_mask=0):
    """The same set found through the size-class cell search."""
    return _list(lib().orc_list_grid, x, D0, L, kappa_b, s, sigma0, d, wall_mask)


def row_brute(x, D0, L, kappa_b, s, sigma0, i, d=3):
    x = f64(x).ravel()
    D0 = f64(D0)
    cap = D0.size
    col = np.zeros(cap, dtype=np.int32)
    P = lib().orc_row_brute(x, D0, D0.size, d, _box(L, d), kappa_b, s, sigma0, i, col, cap)
    return col[:P].copy()


def energy_grad(x, D0, L, kappa, mu, eps=1.0, d=3, rowptr=None, col=None, wall_mask=0):
    """Eq. energy, its gradient w.r.t. every coordinate and kappa, and the largest
    fractional overlap.  Brute force over all pairs unless a CSR list is given."""
    x = f64(x).ravel()
    D0 = f64(D0)
    n = D0.size
    E, dk, md = np.zeros(1), np.zeros(1), np.zeros(1)
    g = np.zeros(n * d)
    with walls(wall_mask):
        if rowptr is None:
            lib().orc_energy_grad_brute(x, D0, n, d, _box(L, d), kappa, mu, eps, E, g, dk, md)
        else:
            lib().orc_energy_grad_list(x, D0, n, d, _box(L, d), kappa, mu, eps,
                                       np.ascontiguousarray(rowptr, dtype=np.int64),
                                       np.ascontiguousarray(col, dtype=np.int32), E, g, dk, md)
    return float(E[0]), g.reshape(n, d), float(dk[0]), float(md[0])


def row_grad(x, D0, L, kappa, i, eps=1.0, d=3):
    x = f64(x).ravel()
    D0 = f64(D0)
    g, e, k, md = np.zeros(d), np.zeros(1), np.zeros(1), np.zeros(1)
    lib().orc_row_grad(x, D0, D0.size, d, _box(L, d), kappa, eps, i, g, e, k, md)
    return g, float(e[0]), float(k[0]), float(md[0])


def adam_update(p, m, v, g, eta, b1, b2, beta1=0.9, beta2=0.999, adam_eps=1e-8):
    """In-place Adam step on float64 arrays; b1, b2 are beta^t for this step."""
    lib().orc_adam_update(p, m, v, f64(g).ravel(), p.size, eta, beta1, beta2, adam_eps, b1, b2)


def wrap(x: float, L: float) -> float:
    return float(lib().orc_wrap(x, L))


def shrink_kappa(x, D0, L, kappa, rowptr, col, d=3, wall_mask=0) -> float:
    x = f64(x).ravel()
    D0 = f64(D0)
    with walls(wall_mask):
        return float(lib().orc_shrink_kappa(x, D0, D0.size, d, _box(L, d), kappa,
                                            np.ascontiguousarray(rowptr, dtype=np.int64),
                                            np.ascontiguousarray(col, dtype=np.int32)))


def phi(D0, L, kappa, d=3) -> float:
    D0 = f64(D0)
    return float(lib().orc_phi(D0, D0.size, d, _box(L, d), kappa))


# ---------------------------------------------------------------- the protocol
@dataclass
class RunResult:
    iters: int
    rebuilds: int
    stopped: bool
    kappa: float
    max_delta: float
    energy: float
    kappa_c: float
    phi: float
    x: np.ndarray = field(repr=False)
    trace: np.ndarray | None = field(default=None, repr=False)


def default_params(**kw) -> Params:
    p = Params()
    lib().orc_params_default(C.byref(p))
    for k, v in kw.items():
        if k == "L":
            p.L = (C.c_double * 3)(*_box(v, kw.get("d", 3)))
        else:
            setattr(p, k, v)
    return p


def run(D0, seed=0, x0=None, trace_len=0, **params) -> RunResult:
    """Run the protocol to the stopping criterion and shrink to contact."""
    p = default_params(**params)
    D0 = f64(D0)
    n = D0.size
    x = np.zeros(n * p.d) if x0 is None else f64(x0).ravel().copy()
    res = Result()
    tr = np.zeros(4 * trace_len) if trace_len else None
    st = lib().orc_run(C.byref(p), D0, n, seed, x, 0 if x0 is None else 1, C.byref(res),
                       tr.ctypes.data_as(C.c_void_p) if tr is not None else None, trace_len)
    if st != 0:
        raise RuntimeError(f"oracle run failed with status {st}")
    return RunResult(res.iters, res.rebuilds, bool(res.stopped), res.kappa, res.max_delta,
                     res.energy, res.kappa_c, res.phi, x.reshape(n, p.d),
                     tr.reshape(-1, 4)[: min(trace_len, res.iters + 1)] if tr is not None else None)


# ---------------------------------------------------------------- the cascade
def _boundary(wall_mask):
    """(flat-wall mask, container) from a mask or a (mask, container) pair."""
    return tuple(wall_mask) if isinstance(wall_mask, tuple) else (int(wall_mask), 0)


def _bounded_axes(bd, d):
    """Axes without minimum image or wrap: the flat walls' and the container's."""
    mask, container = bd
    return mask | ((1 << d) - 1 if container == 1 else (3 if container == 2 else 0))


def seated_state(fixed_d, fixed_x, D0, seed=0, L=1.0, d=3, placement=0, place_rounds=10000, phi0=0.05,
                 wall_mask=0):
    """Initial state of a seated packing (Sec. IV: a finer class seated into
    the voids of coarser spheres held fixed).  Spheres 0..nf-1 are frozen, with
    contact diameters fixed_d and positions fixed_x (wrapped into the box);
    spheres nf.. are mobile with relative diameters D0 and positions from the
    uniform draw of the whole index range, or from placement among the frozen
    ones at kappa_0 (placement = 1).  Returns (encoded D0 [n], x [n, d])."""
    fixed_d = f64(fixed_d).ravel()
    nf = fixed_d.size
    Dall = np.concatenate([-fixed_d, f64(D0).ravel()])
    n = Dall.size
    box = _box(L, d)
    x = init_positions(seed, n, L, d)
    fx = f64(fixed_x).reshape(nf, d)
    bd = _boundary(wall_mask)
    bounded = _bounded_axes(bd, d)
    for i in range(nf):
        for a in range(d):
            x[i, a] = fx[i, a] if (bounded >> a) & 1 else wrap(fx[i, a], box[a])
    if placement:
        with walls(*bd):
            k0 = kappa0(Dall, L, phi0, d)
        x, _, r = place(seed, Dall, k0, L, d, place_rounds, x_frozen=x, wall_mask=bd)
        if r < 0:
            raise RuntimeError("placement did not finish")
    return Dall, x


def cascade(D0, cls, seed=0, L=1.0, d=3, placement=0, place_rounds=10000, **params):
    """Sequential multimodal cascade (Sec. IV), one class at a time, class 0
    first.  Stage 0 packs class 0 alone.  Stage s >= 1 seats class s among the
    packed spheres, frozen at their contact diameters (seed + s, mobile
    spheres in ascending caller index after the frozen ones, also in
    ascending caller index), runs the protocol to the stop and shrinks to
    contact; then releases every sphere: a packing of all of them at their
    contact diameters, kappa starting at 1 (phi0 = the seated phi, so that
    kappa_0 and its skin are of that scale), run to the stop and shrunk.  After
    each stage the diameters are the contact diameters (kappa_c D).
    Returns (x [n, d] in caller order, contact diameters [n], list of
    (stage, phase, phi, iters))."""
    D0 = f64(D0).ravel()
    cls = np.asarray(cls).ravel()
    n = D0.size
    nclass = int(cls.max()) + 1
    phi0 = params.pop("phi0", 0.05)
    wall_mask = (params.get("walls", 0), params.get("container", 0))
    order = []          # caller indices of the packed spheres, in stage order
    diam = None         # their contact diameters
    xs = None           # their positions
    log = []
    for s_ in range(nclass):
        new = np.flatnonzero(cls == s_)
        if s_ == 0:
            if placement:
                with walls(*wall_mask):
                    k0 = kappa0(D0[new], L, phi0, d)
                x0, _, r = place(seed, D0[new], k0, L, d, place_rounds, wall_mask=wall_mask)
                if r < 0:
                    raise RuntimeError("placement did not finish")
            else:
                x0 = None
            res = run(D0[new], seed=seed, x0=x0, d=d, L=L, phi0=phi0, **params)
            order = list(new)
            diam = res.kappa_c * D0[new]
            xs = res.x
            log.append((0, "pack", res.phi, res.iters))
            continue
        Dall, x0 = seated_state(diam, xs, D0[new], seed + s_, L, d, placement, place_rounds, phi0, wall_mask)
        res = run(Dall, seed=seed + s_, x0=x0, d=d, L=L, phi0=phi0, **params)
        log.append((s_, "seat", res.phi, res.iters))
        nf = diam.size
        diam = np.concatenate([diam, res.kappa_c * D0[new]])
        order = order + list(new)
        res = run(diam, seed=seed + s_, x0=res.x, d=d, L=L, phi0=res.phi, kappa_init=1.0, **params)
        log.append((s_, "release", res.phi, res.iters))
        diam = res.kappa_c * diam
        xs = res.x
        assert nf + new.size == diam.size
    x_out = np.zeros((n, d))
    d_out = np.zeros(n)
    x_out[order] = xs
    d_out[order] = diam
    return x_out, d_out, log


def sample_iterations(D0, x, kappa, mu, eta_x, eta_k, sigma0, iters, **params) -> int:
    """`iters` protocol iterations from (x, kappa) at fixed rung values, for
    timing the CPU baseline.  x (N x 3) is advanced in place.  Returns the
    number of list builds."""
    p = default_params(**params)
    D0 = f64(D0)
    b = lib().orc_sample_iterations(C.byref(p), D0, D0.size, x.reshape(-1), kappa, mu, eta_x, eta_k, sigma0,
                                    iters)
    if b < 0:
        raise RuntimeError("periodic-image rule violated")
    return int(b)
