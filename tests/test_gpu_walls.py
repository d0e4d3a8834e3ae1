"""Flat hard walls and the curved container (Sec. II): the binary64 CUDA
path against the oracle, bit for bit, on the same seeded inputs -- lists with
spheres on and beyond the walls, energy and gradient, placement, whole runs
in d = 3 and d = 2, and a seated stage inside walls; the mixed path against
the oracle within its tolerances (lists exact), whole mixed runs beside the
binary64 ones, and batches of bounded packings in both precisions.
"""
import numpy as np
import pytest

from paper_2608_12235_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rcp():
    import torch
    assert torch.cuda.is_available(), "the CUDA path needs a GPU"
    from paper_2608_12235_b300 import build, rcp as R
    build.build()
    R.load()
    return R


def _sigma0(orc, D0, kappa0, cfg):
    m = orc.moments(D0)
    return cfg.skin_abs * ((cfg.lr_x * kappa0) * (m[2] / m[1]))


def _state(orc, n, mask, d, seed):
    rng = np.random.default_rng(seed)
    D0 = inputs.lognormal(n, 0.5, 10.0)
    x = rng.uniform(0.0, 1.0, (n, d))
    for a in range(d):
        if (mask >> a) & 1:
            x[:, a] = rng.uniform(-0.01, 1.01, n)   # some spheres beyond the walls
    return D0, x


@pytest.mark.parametrize("mask,d", [(0b001, 3), (0b101, 3), (0b111, 3), (0b01, 2), (0b11, 2)])
def test_walled_list_and_energy_bitexact(rcp, orc, mask, d):
    n = 3000 if d == 3 else 1500
    D0, x = _state(orc, n, mask, d, seed=mask + 10 * d)
    p = rcp.Packing(D0, box=1.0, seed=1, d=d, walls=mask)
    k = orc.kappa0(D0, 1.0, 0.4, d=d)
    p.set_positions(x, k)
    rp, col = p.neighbors()
    s0 = _sigma0(orc, D0, orc.kappa0(D0, 1.0, 0.05, d=d), p.cfg)
    orp, ocol = orc.list_brute(x, D0, 1.0, k, p.cfg.skin_s, s0, d=d, wall_mask=mask)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    for mu in (0.0, 0.01):
        E, g, dk, md = p.energy_grad(mu)
        oE, og, odk, omd = orc.energy_grad(x, D0, 1.0, k, mu, d=d, wall_mask=mask)
        assert omd > 0.0
        assert E == oE and dk == odk and md == omd
        assert np.array_equal(g, og)
    # positions on walled axes are kept as given, not wrapped
    assert np.array_equal(p.positions(), x)
    p.close()


def test_walled_placement_bitexact(rcp, orc):
    D0 = inputs.lognormal(2000, 0.5, 10.0)
    p = rcp.Packing(D0, box=1.0, seed=6, placement=1, phi0=0.2, walls=0b111)
    k = orc.kappa0(D0, 1.0, 0.2)
    x, _, R = orc.place(6, D0, k, wall_mask=0b111)
    assert R >= 1
    assert np.array_equal(p.positions(), x)
    p.close()


@pytest.mark.parametrize("mask,d", [(0b111, 3), (0b001, 3), (0b11, 2)])
def test_walled_run_bitexact(rcp, orc, mask, d):
    D0 = inputs.lognormal(600, 0.5, 10.0)
    ref = orc.run(D0, seed=2, d=d, walls=mask)
    p = rcp.Packing(D0, box=1.0, seed=2, d=d, walls=mask)
    r = p.run()
    assert r.stopped and ref.stopped and r.iters == ref.iters
    assert r.kappa_c == ref.kappa_c and r.phi == ref.phi
    assert np.array_equal(p.positions(), ref.x)
    p.close()


def test_seated_stage_inside_walls_bitexact(rcp, orc):
    g = (np.arange(2) + 0.25) * 4.0
    X = np.array([[a, b, c] for a in g for b in g for c in g])
    F = np.full(len(X), 1.6)
    D = np.linspace(0.6, 1.0, 200)
    Dall, x0 = orc.seated_state(F, X, D, seed=4, L=8.0, placement=1, wall_mask=0b011)
    ref = orc.run(Dall, seed=4, x0=x0, L=8.0, walls=0b011)
    p = rcp.Packing(D, box=8.0, seed=4, fixed_d=F, fixed_x=X, placement=1, walls=0b011)
    r = p.run()
    assert r.stopped and ref.stopped and r.iters == ref.iters
    assert r.kappa_c == ref.kappa_c and r.phi == ref.phi
    assert np.array_equal(p.positions(), ref.x)
    p.close()


# ------------------------------------------------------------------ curved walls
@pytest.mark.parametrize("container,d", [(1, 3), (2, 3), (1, 2)])
def test_container_list_and_energy_bitexact(rcp, orc, container, d):
    n = 3000 if d == 3 else 1500
    rng = np.random.default_rng(container + 7 * d)
    D0 = inputs.lognormal(n, 0.5, 10.0)
    x = rng.uniform(0.0, 1.0, (n, d))
    cax = list(range(d)) if container == 1 else [0, 1]
    x[:, cax] = rng.uniform(-0.01, 1.01, (n, len(cax)))
    p = rcp.Packing(D0, box=1.0, seed=1, d=d, container=container)
    with orc.walls(0, container):
        k = orc.kappa0(D0, 1.0, 0.3, d=d)
        k0 = orc.kappa0(D0, 1.0, 0.05, d=d)
    p.set_positions(x, k)
    rp, col = p.neighbors()
    s0 = _sigma0(orc, D0, k0, p.cfg)
    orp, ocol = orc.list_brute(x, D0, 1.0, k, p.cfg.skin_s, s0, d=d, wall_mask=(0, container))
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    E, g, dk, md = p.energy_grad(0.01)
    oE, og, odk, omd = orc.energy_grad(x, D0, 1.0, k, 0.01, d=d, wall_mask=(0, container))
    assert omd > 0.0
    assert E == oE and dk == odk and md == omd
    assert np.array_equal(g, og)
    p.close()


@pytest.mark.parametrize("container,d", [(1, 3), (2, 3), (1, 2)])
def test_container_run_from_placement_bitexact(rcp, orc, container, d):
    """The container from App. A's dilute start: placement inside it, then the
    whole protocol and the shrink, against the oracle."""
    D0 = inputs.lognormal(500, 0.5, 10.0)
    with orc.walls(0, container):
        k0 = orc.kappa0(D0, 1.0, 0.05, d=d)
    x0, _, _ = orc.place(5, D0, k0, 1.0, d, wall_mask=(0, container))
    ref = orc.run(D0, seed=5, x0=x0, d=d, container=container)
    p = rcp.Packing(D0, box=1.0, seed=5, d=d, container=container, placement=1)
    assert np.array_equal(p.positions(), x0)
    r = p.run()
    assert r.stopped and ref.stopped and r.iters == ref.iters
    assert r.kappa_c == ref.kappa_c and r.phi == ref.phi
    assert np.array_equal(p.positions(), ref.x)
    p.close()


def test_batch_of_bounded_and_seated_packings_runs_as_solo(rcp):
    """Walled, contained and seated packings advanced by the batched kernels
    stop at the same iteration, kappa_c and phi as when each runs alone."""
    g = (np.arange(2) + 0.25) * 4.0
    X = np.array([[a, b, c] for a in g for b in g for c in g])
    F = np.full(len(X), 1.6)

    def make():
        return [rcp.Packing(inputs.lognormal(400, 0.5, 10.0), box=1.0, seed=1, walls=0b111),
                rcp.Packing(inputs.lognormal(400, 0.5, 10.0), box=1.0, seed=2, container=1, placement=1),
                rcp.Packing(np.linspace(0.6, 1.0, 200), box=8.0, seed=4, fixed_d=F, fixed_x=X, placement=1)]
    solo = make()
    ref = [p.run() for p in solo]
    packs = make()
    b = rcp.Batch(packs)
    res = b.run()
    for r, q, p, s in zip(res, ref, packs, solo):
        assert r.stopped and r.iters == q.iters and r.phi == q.phi and r.kappa_c == q.kappa_c
        assert np.array_equal(p.positions(), s.positions())
    b.close()
    for p in solo + packs:
        p.close()


# ------------------------------------------------------------------ mixed precision
def _bounded_axes(mask, container, d):
    cax = list(range(d)) if container == 1 else ([0, 1] if container == 2 else [])
    return sorted(set([a for a in range(d) if (mask >> a) & 1] + cax))


@pytest.mark.parametrize("mask,container,d", [(0b001, 0, 3), (0b111, 0, 3), (0b11, 0, 2),
                                              (0, 1, 3), (0, 2, 3), (0, 1, 2), (0b100, 2, 3)])
def test_bounded_list_and_energy_mixed(rcp, orc, term_scale, grad_check, sums_check, kappa_mag, mask, container,
                                       d):
    """Walls and the container in mixed precision (each wall a sphere meets is
    one more term of its row, taken in two-term binary32 from the fixed-point
    record): the list is the oracle's, E and dE/dkappa within the mixed sums'
    bound, the gradient element by element within the row-term bound, and
    the largest overlap within 1e-5 of itself; spheres on and beyond the
    walls."""
    n = 3000 if d == 3 else 1500
    rng = np.random.default_rng(100 + mask + 7 * container + 10 * d)
    D0 = inputs.lognormal(n, 0.5, 10.0)
    x = rng.uniform(0.0, 1.0, (n, d))
    for a in _bounded_axes(mask, container, d):
        x[:, a] = rng.uniform(-0.01, 1.01, n)
    wm = (mask, container)
    p = rcp.Packing(D0, box=1.0, seed=1, d=d, walls=mask, container=container, precision=rcp.RCP_MIXED)
    with orc.walls(wm):
        k = orc.kappa0(D0, 1.0, 0.3, d=d)
        k0 = orc.kappa0(D0, 1.0, 0.05, d=d)
    p.set_positions(x, k)
    rp, col = p.neighbors()
    s0 = _sigma0(orc, D0, k0, p.cfg)
    orp, ocol = orc.list_brute(x, D0, 1.0, k, p.cfg.skin_s, s0, d=d, wall_mask=wm)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    for mu in (0.0, 0.01):
        E, g, dk, md = p.energy_grad(mu)
        oE, og, odk, omd = orc.energy_grad(x, D0, 1.0, k, mu, d=d, wall_mask=wm)
        assert omd > 0.0
        # spheres past a wall give negative kappa terms: the bound takes the
        # terms' magnitudes
        sums_check(E, oE, dk, odk, mu, k, D0, what=f"mixed walls {mask} container {container}",
                   k_mag=kappa_mag(x, D0, 1.0, k, d=d, wall_mask=wm))
        assert abs(md - omd) <= 1e-5 * omd
        w = grad_check(g, og, term_scale(x, D0, 1.0, k, d=d, wall_mask=wm),
                       what=f"mixed walls {mask} container {container}")
        print(f"walls {mask} container {container} d={d} mu {mu}: worst gradient error / bound {w:.3g}")
    # positions on bounded axes come back as given, not wrapped (to the
    # records' resolution)
    assert np.allclose(p.positions(), x, rtol=0.0, atol=1e-15)
    p.close()


def test_wall_terms_mixed_near_contact(rcp, orc, term_scale, grad_check, sums_check, kappa_mag):
    """Small overlaps with the walls and between spheres (a relaxed walled
    packing inflated by 0.2 %): the wall clearance rad - h taken in two-term
    arithmetic, where a binary32 difference would cancel."""
    D0 = inputs.lognormal(500, 0.5, 10.0)
    ref = orc.run(D0, seed=3, walls=0b111)
    k = ref.kappa_c * 1.002
    x = ref.x
    p = rcp.Packing(D0, box=1.0, seed=3, walls=0b111, precision=rcp.RCP_MIXED)
    p.set_positions(x, k)
    for mu in (0.0, 0.01):
        E, g, dk, md = p.energy_grad(mu)
        oE, og, odk, omd = orc.energy_grad(x, D0, 1.0, k, mu, wall_mask=0b111)
        assert 5e-4 < omd < 5e-3
        sums_check(E, oE, dk, odk, mu, k, D0, what="mixed walls near contact",
                   k_mag=kappa_mag(x, D0, 1.0, k, wall_mask=(0b111, 0)))
        assert abs(md - omd) <= 1e-5 * omd
        w = grad_check(g, og, term_scale(x, D0, 1.0, k, wall_mask=(0b111, 0)), what="mixed walls near contact")
        print(f"mu {mu}: worst gradient error / bound {w:.3g}")
    p.close()


@pytest.mark.parametrize("mask,container,d", [(0b111, 0, 3), (0b11, 0, 2), (0, 1, 3), (0, 2, 3)])
def test_bounded_run_mixed(rcp, orc, mask, container, d):
    """A bounded packing in mixed precision to the stop and the shrink: no
    binary64 overlap with a sphere or a wall at kappa_c, and phi beside the
    binary64 run's (a whole run is chaotic in the rounding)."""
    D0 = inputs.lognormal(600, 0.5, 10.0)
    out = {}
    for prec in (rcp.RCP_FP64, rcp.RCP_MIXED):
        p = rcp.Packing(D0, box=1.0, seed=2, d=d, walls=mask, container=container, placement=1, precision=prec)
        r = p.run()
        x = p.positions()
        p.close()
        assert r.stopped and r.max_delta < 5e-4
        assert orc.energy_grad(x, D0, 1.0, r.kappa_c, 0.0, d=d, wall_mask=(mask, container))[3] == 0.0
        out[prec] = r.phi
    print(f"walls {mask} container {container} d={d}: phi binary64 {out[rcp.RCP_FP64]:.6f}, "
          f"mixed {out[rcp.RCP_MIXED]:.6f}")
    assert abs(out[rcp.RCP_MIXED] - out[rcp.RCP_FP64]) < 2e-2


def test_batch_of_bounded_and_seated_packings_runs_as_solo_mixed(rcp):
    """The batched mixed kernel with the wall terms: walled, contained and
    seated packings stop at the same iteration, kappa_c and phi, at the same
    positions, as when each runs alone."""
    g = (np.arange(2) + 0.25) * 4.0
    X = np.array([[a, b, c] for a in g for b in g for c in g])
    F = np.full(len(X), 1.6)
    M = rcp.RCP_MIXED

    def make():
        return [rcp.Packing(inputs.lognormal(400, 0.5, 10.0), box=1.0, seed=1, walls=0b111, precision=M),
                rcp.Packing(inputs.lognormal(400, 0.5, 10.0), box=1.0, seed=2, container=1, placement=1,
                            precision=M),
                rcp.Packing(np.linspace(0.6, 1.0, 200), box=8.0, seed=4, fixed_d=F, fixed_x=X, placement=1,
                            precision=M),
                rcp.Packing(inputs.lognormal(400, 0.5, 10.0), box=1.0, seed=3, precision=M)]
    solo = make()
    ref = [p.run() for p in solo]
    packs = make()
    b = rcp.Batch(packs)
    res = b.run()
    for r, q, p, s in zip(res, ref, packs, solo):
        assert r.stopped and r.iters == q.iters and r.phi == q.phi and r.kappa_c == q.kappa_c
        assert np.array_equal(p.positions(), s.positions())
    b.close()
    for p in solo + packs:
        p.close()


def test_seated_stage_inside_walls_mixed(rcp, orc):
    """Frozen spheres inside walls in mixed precision (the kernel with the wall
    terms, instantiated for frozen spheres too): the frozen spheres keep their
    positions bit for bit, nothing overlaps in binary64 at kappa_c, and phi
    lands beside the binary64 stage's."""
    g = (np.arange(2) + 0.25) * 4.0
    X = np.array([[a, b, c] for a in g for b in g for c in g])
    F = np.full(len(X), 1.6)
    D = np.linspace(0.6, 1.0, 200)
    out = {}
    for prec in (rcp.RCP_FP64, rcp.RCP_MIXED):
        p = rcp.Packing(D, box=8.0, seed=4, fixed_d=F, fixed_x=X, placement=1, walls=0b011, precision=prec)
        r = p.run()
        x = p.positions()
        p.close()
        assert r.stopped and r.max_delta < 5e-4
        assert np.array_equal(x[:F.size], X)
        Dall = np.concatenate([-F, D])
        assert orc.energy_grad(x, Dall, 8.0, r.kappa_c, 0.0, wall_mask=0b011)[3] == 0.0
        out[prec] = r.phi
    print(f"seated inside walls: phi binary64 {out[rcp.RCP_FP64]:.6f}, mixed {out[rcp.RCP_MIXED]:.6f}")
    assert abs(out[rcp.RCP_MIXED] - out[rcp.RCP_FP64]) < 2e-2


def test_seated_stage_in_a_ball_mixed(rcp, orc):
    """A seated stage inside a ball in mixed precision, from the same frozen
    configuration as the binary64 stage (class 0 packed in binary64): frozen
    spheres kept to the records' resolution, no binary64 overlap with a
    sphere or the wall at kappa_c, and phi beside the binary64 stage's (on
    eight seeds: within 3e-6 on seven, 3.7e-3 on the eighth, where the two
    trajectories part)."""
    p = rcp.Packing(np.full(24, 4.0), box=14.0, seed=5, placement=1, container=1)
    r0 = p.run()
    X = p.positions()
    p.close()
    F = np.full(24, 4.0 * r0.kappa_c)
    D1 = np.full(120, 1.0)
    Dall = np.concatenate([-F, D1])
    out = {}
    for prec in (rcp.RCP_FP64, rcp.RCP_MIXED):
        q = rcp.Packing(D1, box=14.0, seed=6, fixed_d=F, fixed_x=X, placement=1, container=1, precision=prec)
        r = q.run()
        x = q.positions()
        q.close()
        assert r.stopped and r.max_delta < 5e-4
        assert np.allclose(x[:F.size], X, rtol=0.0, atol=1e-13)
        assert orc.energy_grad(x, Dall, 14.0, r.kappa_c, 0.0, wall_mask=(0, 1))[3] == 0.0
        out[prec] = r.phi
    print(f"seated in a ball: phi binary64 {out[rcp.RCP_FP64]:.7f}, mixed {out[rcp.RCP_MIXED]:.7f}")
    assert abs(out[rcp.RCP_MIXED] - out[rcp.RCP_FP64]) < 1e-2


def test_cascade_in_a_ball_mixed(rcp, orc):
    """The two-class cascade inside a ball in mixed precision: three stages,
    the seated stage denser than the coarse class alone, and the final
    packing inside the ball without overlap.  Its phi is not compared seed by
    seed with the binary64 cascade's: with 24 coarse spheres the stage-0
    configuration decides the seated phi (binary64 over ten seeds: stage 1
    0.569-0.583), and a mixed stage 0 ends in another configuration of the
    same ensemble."""
    D0 = np.concatenate([np.full(24, 4.0), np.full(120, 1.0)])
    cls = np.concatenate([np.zeros(24, int), np.ones(120, int)])
    cfg = rcp.rcp_config_default(placement=1, container=1, precision=rcp.RCP_MIXED)
    x, dm, phi, iters = rcp.rcp_cascade(D0, cls, box=14.0, seed=5, cfg=cfg)
    print(f"cascade in a ball, mixed: phi {list(phi)}, iterations {list(iters)}")
    assert len(phi) == 3 and np.all(iters > 0)
    assert phi[1] > phi[0] + 0.05 and phi[2] >= phi[1] - 1e-3
    rc = np.sqrt(np.sum((x - 7.0) ** 2, axis=1))
    assert np.all(rc + 0.5 * dm <= 7.0 * (1.0 + 1e-9))
    assert orc.energy_grad(x, dm, 14.0, 1.0, 0.0, wall_mask=(0, 1))[3] < 1e-12
