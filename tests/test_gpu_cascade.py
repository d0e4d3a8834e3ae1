"""Frozen spheres and the sequential cascade (Sec. IV): the binary64 CUDA path
against the oracle, bit for bit, on the same seeded inputs; the mixed path
within its tolerances (element-wise gradient, E and dE/dkappa against the
magnitudes of their sums) and its runs to the stop beside binary64.

Sizes: a few hundred spheres across several size classes and cell levels,
frozen spheres in the coarsest class (the cascade's case) and in a finer
class than the mobile ones (placement must still see them), d = 3 and d = 2.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rcp():
    import torch
    assert torch.cuda.is_available(), "the CUDA path needs a GPU"
    from paper_2608_12235_b300 import build, rcp as R
    build.build()
    R.load()
    return R


def _lattice(m, L, F, d=3):
    g = (np.arange(m) + 0.25) * (L / m)
    if d == 3:
        X = np.array([[a, b, c] for a in g for b in g for c in g])
    else:
        X = np.array([[a, b] for a in g for b in g])
    return np.full(len(X), F), X


@pytest.mark.parametrize("placement", [0, 1])
def test_seated_initial_state_bitexact(rcp, orc, placement):
    F, X = _lattice(2, 8.0, 2.4)
    D = np.linspace(0.6, 1.0, 300)
    p = rcp.Packing(D, box=8.0, seed=5, fixed_d=F, fixed_x=X, placement=placement)
    assert rcp.rcp_frozen(p.h) == F.size and rcp.rcp_size(p.h) == F.size + D.size
    Dall, x = orc.seated_state(F, X, D, seed=5, L=8.0, placement=placement)
    assert np.array_equal(p.positions(), x)
    p.close()


def test_seated_placement_sees_frozen_spheres_of_a_finer_class(rcp, orc):
    """Frozen spheres much smaller than the mobile ones sit in a finer size
    class; the mobile candidates must still give way to them."""
    F, X = _lattice(4, 8.0, 0.3)
    D = np.full(40, 1.0)
    p = rcp.Packing(D, box=8.0, seed=2, fixed_d=F, fixed_x=X, placement=1, phi0=0.1)
    _, x = orc.seated_state(F, X, D, seed=2, L=8.0, placement=1, phi0=0.1)
    assert np.array_equal(p.positions(), x)
    p.close()


def test_seated_energy_grad_bitexact(rcp, orc):
    F, X = _lattice(2, 8.0, 2.4)
    D = np.linspace(0.6, 1.0, 300)
    Dall, x = orc.seated_state(F, X, D, seed=8, L=8.0, placement=0)
    p = rcp.Packing(D, box=8.0, seed=8, fixed_d=F, fixed_x=X)
    for k in (0.7, 1.3):
        p.set_positions(x, k)
        for mu in (0.0, 0.02):
            E, g, dk, md = p.energy_grad(mu)
            oE, og, odk, omd = orc.energy_grad(x, Dall, 8.0, k, mu)
            assert omd > 0.0
            assert E == oE and dk == odk and md == omd
            assert np.array_equal(g, og)
            assert not g[:F.size].any()
    p.close()


@pytest.mark.parametrize("d", [3, 2])
def test_seated_run_bitexact(rcp, orc, d):
    """A whole seated stage: the protocol to the stop and the shrink, the
    frozen spheres unmoved."""
    if d == 3:
        F, X = _lattice(2, 8.0, 2.4)
        D = np.linspace(0.7, 1.0, 240)
        L = 8.0
    else:
        F, X = _lattice(3, 12.0, 2.4, d=2)
        D = np.linspace(0.7, 1.0, 150)
        L = 12.0
    Dall, x0 = orc.seated_state(F, X, D, seed=9, L=L, d=d, placement=1)
    ref = orc.run(Dall, seed=9, x0=x0, L=L, d=d)
    p = rcp.Packing(D, box=L, seed=9, d=d, fixed_d=F, fixed_x=X, placement=1)
    r = p.run()
    assert r.stopped and ref.stopped and r.iters == ref.iters
    assert r.kappa_c == ref.kappa_c and r.phi == ref.phi
    got = p.positions()
    assert np.array_equal(got, ref.x)
    assert np.array_equal(got[:F.size], X)
    p.close()


def test_cascade_bitexact(rcp, orc):
    """Two classes at diameter ratio 4, placement on: every stage (pack, seat,
    release) takes the oracle's Adam steps to the same phi, and the final
    positions and contact diameters are the oracle's."""
    nc, nf = 32, 256
    D0 = np.concatenate([np.full(nc, 4.0), np.full(nf, 1.0)])
    cls = np.concatenate([np.zeros(nc, int), np.ones(nf, int)])
    # interleave the classes in the caller's order
    perm = np.random.default_rng(1).permutation(D0.size)
    D0, cls = D0[perm], cls[perm]
    xo, do, log = orc.cascade(D0, cls, seed=7, L=12.0, placement=1)
    cfg = rcp.rcp_config_default(placement=1)
    x, dm, phi, iters = rcp.rcp_cascade(D0, cls, box=12.0, seed=7, cfg=cfg)
    assert list(phi) == [f for _, _, f, _ in log]
    assert list(iters) == [t for _, _, _, t in log]
    assert np.array_equal(dm, do)
    assert np.array_equal(x, xo)


def test_cascade_three_classes_bitexact(rcp, orc):
    """Three classes (ratios 3:1.5:1, uniform starts): five stages."""
    D0 = np.concatenate([np.full(40, 3.0), np.full(120, 1.5), np.full(200, 1.0)])
    cls = np.concatenate([np.zeros(40, int), np.ones(120, int), np.full(200, 2)])
    xo, do, log = orc.cascade(D0, cls, seed=3, L=10.0)
    x, dm, phi, iters = rcp.rcp_cascade(D0, cls, box=10.0, seed=3)
    assert len(phi) == 5
    assert list(phi) == [f for _, _, f, _ in log]
    assert list(iters) == [t for _, _, _, t in log]
    assert np.array_equal(dm, do) and np.array_equal(x, xo)


def test_cascade_in_a_ball_bitexact(rcp, orc):
    """A two-class cascade inside a ball container (every axis bounded, so
    no periodic-image limit on the coarse class), placement on."""
    D0 = np.concatenate([np.full(24, 4.0), np.full(120, 1.0)])
    cls = np.concatenate([np.zeros(24, int), np.ones(120, int)])
    xo, do, log = orc.cascade(D0, cls, seed=5, L=14.0, placement=1, container=1)
    cfg = rcp.rcp_config_default(placement=1, container=1)
    x, dm, phi, iters = rcp.rcp_cascade(D0, cls, box=14.0, seed=5, cfg=cfg)
    assert list(phi) == [f for _, _, f, _ in log]
    assert list(iters) == [t for _, _, _, t in log]
    assert np.array_equal(dm, do) and np.array_equal(x, xo)


# ------------------------------------------------------------------ mixed precision
def test_seated_energy_grad_mixed(rcp, orc, term_scale, grad_check, sums_check):
    """Pairs with a frozen sphere take d = (F + kappa D^0)/2 (or (F_i + F_j)/2)
    and half the mobile D^0 in dE/dkappa; frozen rows have no gradient."""
    F, X = _lattice(2, 8.0, 2.4)
    D = np.linspace(0.6, 1.0, 300)
    Dall, x = orc.seated_state(F, X, D, seed=8, L=8.0, placement=0)
    p = rcp.Packing(D, box=8.0, seed=8, fixed_d=F, fixed_x=X, precision=rcp.RCP_MIXED)
    for k in (0.7, 1.3):
        p.set_positions(x, k)
        for mu in (0.0, 0.02):
            E, g, dk, md = p.energy_grad(mu)
            oE, og, odk, omd = orc.energy_grad(x, Dall, 8.0, k, mu)
            assert omd > 0.0
            # the mu terms take the mobile spheres only
            sums_check(E, oE, dk, odk, mu, k, np.where(Dall > 0.0, Dall, 0.0), what="seated mixed")
            assert abs(md - omd) <= 1e-5 * omd
            assert not g[:F.size].any()
            w = grad_check(g, og, term_scale(x, Dall, 8.0, k), what="seated mixed")
            print(f"kappa {k} mu {mu}: worst gradient error / bound {w:.3g}")
    p.close()


def test_seated_run_mixed(rcp, orc):
    """A seated stage in mixed precision to the stop and the shrink: the frozen
    spheres keep their positions bit for bit, and phi lands beside the
    binary64 run's (a whole run is chaotic in the rounding: a few 1e-3 at
    this size)."""
    F, X = _lattice(2, 8.0, 2.4)
    D = np.linspace(0.7, 1.0, 240)
    out = {}
    for prec in (rcp.RCP_FP64, rcp.RCP_MIXED):
        p = rcp.Packing(D, box=8.0, seed=9, fixed_d=F, fixed_x=X, placement=1, precision=prec)
        r = p.run()
        got = p.positions()
        p.close()
        assert r.stopped and r.max_delta < 5e-4
        assert np.array_equal(got[:F.size], X)
        out[prec] = r.phi
    print(f"seated phi: binary64 {out[rcp.RCP_FP64]:.6f}, mixed {out[rcp.RCP_MIXED]:.6f}")
    assert abs(out[rcp.RCP_MIXED] - out[rcp.RCP_FP64]) < 1e-2


def test_cascade_mixed(rcp, orc):
    """The two-class cascade in mixed precision: every stage reaches the stop
    and lands beside the binary64 cascade's phi."""
    nc, nf = 32, 256
    D0 = np.concatenate([np.full(nc, 4.0), np.full(nf, 1.0)])
    cls = np.concatenate([np.zeros(nc, int), np.ones(nf, int)])
    perm = np.random.default_rng(1).permutation(D0.size)
    D0, cls = D0[perm], cls[perm]
    x64, d64, phi64, it64 = rcp.rcp_cascade(D0, cls, box=12.0, seed=7, cfg=rcp.rcp_config_default(placement=1))
    cfg = rcp.rcp_config_default(placement=1, precision=rcp.RCP_MIXED)
    x, dm, phi, iters = rcp.rcp_cascade(D0, cls, box=12.0, seed=7, cfg=cfg)
    print(f"cascade phi: binary64 {list(phi64)}, mixed {list(phi)}")
    assert len(phi) == len(phi64) == 3
    assert all(abs(a - b) < 2e-2 for a, b in zip(phi, phi64))
    assert np.all(np.isfinite(x)) and np.all(dm > 0.0)
