"""Pins of the oracle's frozen spheres and sequential cascade (Sec. IV).

A stage of the cascade holds the coarser classes fixed while a finer class is
inflated among them.  None of these re-types the oracle's arithmetic: the
checks are hand-derived values for one pair, finite differences of the
energy, the closed-form contact scale of one pair, a reduction to the
all-mobile energy, invariants of a run and the growth of phi the paper
reports stage by stage.
"""
import math

import numpy as np
import pytest


def _min_gap(x, diam, L):
    """min over pairs of r_ij / ((d_i + d_j)/2) - 1 (brute force, minimum image)."""
    n = len(diam)
    best = np.inf
    for i in range(n):
        dx = x[i] - x[i + 1:]
        dx -= L * np.round(dx / L)
        r = np.sqrt((dx * dx).sum(axis=1))
        if r.size:
            best = min(best, float((r / (0.5 * (diam[i] + diam[i + 1:])) - 1.0).min()))
    return best


def test_frozen_pair_by_hand(orc):
    """Frozen sphere F = 2 at (1,1,1), mobile D^0 = 1 at (2.2,1,1), kappa 0.8:
    d = (2 + 0.8)/2 = 1.4, r = 1.2, delta = 1/7."""
    x = np.array([[1.0, 1.0, 1.0], [2.2, 1.0, 1.0]])
    D0 = np.array([-2.0, 1.0])
    mu, kappa = 0.3, 0.8
    E, g, dk, md = orc.energy_grad(x, D0, 5.0, kappa, mu)
    delta = 1.0 - 1.2 / 1.4
    assert md == pytest.approx(delta, rel=1e-14)
    # E = 1/2 delta^2 - mu kappa (mobile D^0 only)
    assert E == pytest.approx(0.5 * delta ** 2 - mu * kappa * 1.0, rel=1e-14)
    # dE/dkappa = delta (r / d^2)(D^0 / 2) - mu D^0: only the mobile half of d grows
    assert dk == pytest.approx(delta * (1.2 / 1.4 ** 2) * 0.5 - mu, rel=1e-13)
    # the mobile sphere is pushed along +x with |dE/dx| = delta / d; the frozen one has none
    assert g[1] == pytest.approx([-delta / 1.4, 0.0, 0.0], rel=1e-14, abs=0)
    assert np.array_equal(g[0], np.zeros(3))


def _seated_random(seed=3, nf=5, nm=14, L=4.0):
    rng = np.random.default_rng(seed)
    F = rng.uniform(1.2, 1.8, nf)
    D = rng.uniform(0.5, 1.0, nm)
    x = rng.uniform(0, L, (nf + nm, 3))
    return np.concatenate([-F, D]), x, L


def test_frozen_derivatives_by_finite_differences(orc):
    D0, x, L = _seated_random()
    kappa, mu = 1.1, 0.2
    E, g, dk, md = orc.energy_grad(x, D0, L, kappa, mu)
    assert np.count_nonzero(g[:5]) == 0             # frozen rows: no gradient
    assert md > 0.0 and np.count_nonzero(g[5:]) > 0  # some overlaps exist
    h = 1e-6
    Ep = orc.energy_grad(x, D0, L, kappa + h, mu)[0]
    Em = orc.energy_grad(x, D0, L, kappa - h, mu)[0]
    assert dk == pytest.approx((Ep - Em) / (2 * h), rel=1e-6, abs=1e-9)
    for i in range(5, 19):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = (orc.energy_grad(xp, D0, L, kappa, mu)[0] - orc.energy_grad(xm, D0, L, kappa, mu)[0]) / (2 * h)
            assert g[i, a] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_frozen_at_kappa_diameters_reduce_to_all_mobile(orc):
    """Frozen spheres with F_i = kappa D_i^0 meet every mobile sphere at the
    same contact distance as in the all-mobile packing at kappa: the pair
    energy and the mobile rows' gradient agree to rounding."""
    rng = np.random.default_rng(11)
    n, L, kappa = 24, 3.0, 1.3
    D = rng.uniform(0.6, 1.0, n)
    x = rng.uniform(0, L, (n, 3))
    frozen = np.arange(n) < 8
    Ds = np.where(frozen, -kappa * D, D)
    Ea, ga, _, mda = orc.energy_grad(x, D, L, kappa, 0.0)
    Es, gs, _, mds = orc.energy_grad(x, Ds, L, kappa, 0.0)
    assert Ea > 0
    assert Es == pytest.approx(Ea, rel=1e-13)
    assert mds == pytest.approx(mda, rel=1e-13)
    np.testing.assert_allclose(gs[~frozen], ga[~frozen], rtol=1e-12, atol=1e-14)


def test_frozen_pair_contact_scale(orc):
    """One mobile sphere at distance r from a frozen one touches it at
    kappa* = (2r - F)/D^0; shrink to contact lands just below that."""
    L, F, D, r = 6.0, 2.0, 1.0, 1.7
    x = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
    D0 = np.array([-F, D])
    kappa = 2.0   # overlapping: d = (2 + 2)/2 = 2 > 1.7
    rowptr, col = orc.list_brute(x, D0, L, kappa, 0.0, 0.0)
    kc = orc.shrink_kappa(x, D0, L, kappa, rowptr, col)
    exact = (2 * r - F) / D
    assert exact * (1 - 1e-11) < kc < exact
    assert orc.energy_grad(x, D0, L, kc, 0.0)[3] == 0.0   # no overlap left
    # two frozen spheres set no bound, however much they overlap
    kc2 = orc.shrink_kappa(x, np.array([-F, -3.0]), L, kappa, *orc.list_brute(x, np.array([-F, -3.0]), L,
                                                                                kappa, 0.0, 0.0))
    assert kc2 == kappa * (1 - 2.0 ** -50)


def _lattice_frozen(m=2, L=8.0, F=2.4):
    g = (np.arange(m) + 0.25) * (L / m)
    X = np.array([[a, b, c] for a in g for b in g for c in g])
    return np.full(len(X), F), X


def test_seated_placement_avoids_the_frozen_spheres(orc):
    F, X = _lattice_frozen()
    D = np.full(60, 1.0)
    Dall, x = orc.seated_state(F, X, D, seed=5, L=8.0, placement=1)
    nf = F.size
    assert np.array_equal(x[:nf], X)
    k0 = orc.kappa0(Dall, 8.0, 0.05)
    # kappa_0 puts the mobile spheres alone at phi0
    assert (math.pi / 6) * k0 ** 3 * D.size / 8.0 ** 3 == pytest.approx(0.05, rel=1e-12)
    diam = np.where(Dall < 0, -Dall, k0 * Dall)
    assert _min_gap(x, diam, 8.0) >= 0.0
    # the uniform variant only replaces the frozen rows of the uniform draw
    Dall_u, xu = orc.seated_state(F, X, D, seed=5, L=8.0, placement=0)
    draw = orc.init_positions(5, nf + D.size, 8.0)
    assert np.array_equal(xu[nf:], draw[nf:]) and np.array_equal(xu[:nf], X)


def test_seated_run_holds_the_frozen_spheres(orc):
    F, X = _lattice_frozen()
    D = np.full(120, 1.0)
    Dall, x0 = orc.seated_state(F, X, D, seed=9, L=8.0, placement=1)
    res = orc.run(Dall, seed=9, x0=x0, L=8.0)
    nf = F.size
    assert res.stopped
    assert np.array_equal(res.x[:nf], X)          # not moved, bit for bit
    diam = np.where(Dall < 0, -Dall, res.kappa_c * Dall)
    gap = _min_gap(res.x, diam, 8.0)
    assert 0.0 <= gap < 1e-9                       # shrunk to the last contact
    V = 8.0 ** 3
    assert res.phi == pytest.approx((math.pi / 6) * (diam ** 3).sum() / V, rel=1e-13)


def test_cascade_climbs_stage_by_stage(orc):
    """Two classes at diameter ratio 4 (coarse volume twice the fine): the
    seated stage packs denser than the coarse class alone (Sec. IV, Table:
    phi rises with every class added), the release keeps it, the classes keep
    one contact diameter each and nothing overlaps at the end."""
    nc, nf = 32, 256
    D0 = np.concatenate([np.full(nc, 4.0), np.full(nf, 1.0)])
    cls = np.concatenate([np.zeros(nc, int), np.ones(nf, int)])
    x, diam, log = orc.cascade(D0, cls, seed=7, L=12.0, placement=1)
    phases = [(s, p) for s, p, _, _ in log]
    assert phases == [(0, "pack"), (1, "seat"), (1, "release")]
    phi = [f for _, _, f, _ in log]
    assert 0.55 < phi[0] < 0.66
    assert phi[1] > phi[0] + 0.03
    assert phi[2] > phi[1] - 2e-3
    assert np.ptp(diam[:nc]) == 0.0 and np.ptp(diam[nc:]) == 0.0
    assert _min_gap(x, diam, 12.0) >= 0.0
    assert phi[2] == pytest.approx((math.pi / 6) * (diam ** 3).sum() / 12.0 ** 3, rel=1e-12)


def test_seated_run_inside_walls_and_a_container(orc):
    """Frozen spheres inside a walled box and inside a ball: the mobile ones
    end inside the boundary, the frozen ones unmoved, nothing overlaps."""
    F = np.full(8, 1.6)
    g = (np.arange(2) + 0.25) * 4.0
    X = np.array([[a, b, c] for a in g for b in g for c in g])
    D = np.linspace(0.6, 1.0, 150)
    for walls, container, Xf in ((0b011, 0, X), (0, 1, 4.0 + 0.45 * (X - 4.0))):
        Dall, x0 = orc.seated_state(F, Xf, D, seed=4, L=8.0, placement=1, wall_mask=(walls, container))
        res = orc.run(Dall, seed=4, x0=x0, L=8.0, walls=walls, container=container)
        assert res.stopped and np.array_equal(res.x[:8], Xf)
        E, g_, dk, md = orc.energy_grad(res.x, Dall, 8.0, res.kappa_c, 0.0, wall_mask=(walls, container))
        assert md == 0.0
        rad = 0.5 * res.kappa_c * D
        xm = res.x[8:]
        if walls:
            for a in (0, 1):
                assert (xm[:, a] >= rad).all() and (8.0 - xm[:, a] >= rad).all()
        else:
            assert (np.sqrt(((xm - 4.0) ** 2).sum(axis=1)) + rad <= 4.0).all()


def test_placement_sees_frozen_spheres_of_a_finer_class(orc):
    """Frozen spheres far smaller than the mobile ones (a finer size class)
    still keep every placed candidate off them."""
    g = (np.arange(4) + 0.25) * 2.0
    X = np.array([[a, b, c] for a in g for b in g for c in g])
    F = np.full(len(X), 0.3)
    D = np.full(40, 1.0)
    Dall, x = orc.seated_state(F, X, D, seed=2, L=8.0, placement=1, phi0=0.1)
    k0 = orc.kappa0(Dall, 8.0, 0.1)
    lvl, _ = orc.levels(Dall, k0, 0.0, 0.0)
    assert lvl[:len(X)].min() > lvl[len(X):].max()      # the frozen ones are in a finer class
    diam = np.where(Dall < 0, -Dall, k0 * Dall)
    assert _min_gap(x, diam, 8.0) >= 0.0


def test_two_dimensional_cascade_climbs(orc):
    """Disks: two classes at diameter ratio 4; the seated stage packs denser
    than the coarse class alone and nothing overlaps at the end."""
    D0 = np.concatenate([np.full(40, 4.0), np.full(300, 1.0)])
    cls = np.concatenate([np.zeros(40, int), np.ones(300, int)])
    x, diam, log = orc.cascade(D0, cls, seed=3, L=30.0, d=2, placement=1)
    phi = [f for _, _, f, _ in log]
    assert phi[1] > phi[0] + 0.02 and phi[2] > phi[1] - 2e-3
    n = len(diam)
    dx = x[:, None, :] - x[None, :, :]
    dx -= 30.0 * np.round(dx / 30.0)
    r = np.sqrt((dx ** 2).sum(-1)) + np.eye(n) * 100
    assert (r / (0.5 * (diam[:, None] + diam[None, :])) - 1).min() >= 0.0


def test_release_starts_at_the_given_kappa(orc):
    """kappa_init (the cascade's release) replaces kappa_0 as the first
    iterate while the skin keeps kappa_0's scale."""
    D0 = np.linspace(0.7, 1.0, 60)
    x0 = orc.init_positions(2, 60)
    r = orc.run(D0, seed=2, x0=x0, kappa_init=0.123, max_iters=3, trace_len=3)
    assert r.trace[0, 2] == 0.123
    r0 = orc.run(D0, seed=2, x0=x0, max_iters=3, trace_len=3)
    assert r0.trace[0, 2] == orc.kappa0(D0, 1.0, 0.05)
