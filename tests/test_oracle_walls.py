"""Pins of the oracle's flat hard walls (Sec. II: an axis may be bounded by a
wall instead of being periodic).

The checks are hand values for one sphere, the mirror-image identity (a
sphere against a wall is a pair against its reflection), finite differences,
the cell search against the brute-force definition with spheres on and
beyond the walls, the one-sphere contact scale and the invariants of a run.
"""
import numpy as np
import pytest


def test_one_sphere_against_either_wall_by_hand(orc):
    D0 = np.array([1.0])
    mu = 0.1
    # wall at 0 on x: h = 0.3, rad = 0.5, delta = 1 - 0.3/0.5 = 0.4
    x = np.array([[0.3, 2.0, 2.0]])
    E, g, dk, md = orc.energy_grad(x, D0, 4.0, 1.0, mu, wall_mask=1)
    assert md == pytest.approx(0.4, rel=1e-14)
    assert E == pytest.approx(0.5 * 0.4 ** 2 - mu, rel=1e-14)
    assert dk == pytest.approx(0.4 * 0.6 - mu, rel=1e-14)   # d delta / d kappa = 0.6 at kappa = 1
    assert g[0] == pytest.approx([-0.4 / 0.5, 0.0, 0.0], abs=1e-15)   # pushed towards +x
    # the wall at L on x: h = 0.2, delta = 0.6, pushed towards -x
    x = np.array([[3.8, 2.0, 2.0]])
    E, g, dk, md = orc.energy_grad(x, D0, 4.0, 1.0, mu, wall_mask=1)
    assert md == pytest.approx(0.6, rel=1e-14)
    assert g[0] == pytest.approx([0.6 / 0.5, 0.0, 0.0], rel=1e-14)
    # periodic axis: no wall, no term
    E, g, dk, md = orc.energy_grad(x, D0, 4.0, 1.0, mu, wall_mask=0)
    assert md == 0.0 and E == -mu and not g.any()


def test_wall_term_is_the_pair_with_the_mirror_image(orc):
    """Against a wall at distance h a sphere overlaps as it would overlap its
    reflection at distance 2h (contact distance D): the same overlap and the
    same energy."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        h = rng.uniform(0.05, 0.5)
        D = rng.uniform(0.6, 1.0)
        k = rng.uniform(0.8, 1.2)
        x = np.array([[h, 3.0, 3.0]])
        Ew, _, _, mdw = orc.energy_grad(x, np.array([D]), 6.0, k, 0.0, wall_mask=1)
        pair = np.array([[3.0 + h, 3.0, 3.0], [3.0 - h, 3.0, 3.0]])
        Ep, _, _, mdp = orc.energy_grad(pair, np.array([D, D]), 6.0, k, 0.0)
        assert mdw == pytest.approx(mdp, rel=1e-13, abs=1e-15)
        assert Ew == pytest.approx(Ep, rel=1e-12, abs=1e-300)


def test_walls_derivatives_by_finite_differences(orc):
    rng = np.random.default_rng(8)
    n, L = 30, 3.0
    D0 = rng.uniform(0.5, 1.0, n)
    D0[:4] = -D0[:4]           # a few frozen spheres too
    x = rng.uniform(0.0, L, (n, 3))
    x[:, [0, 2]] = rng.uniform(-0.1, L + 0.1, (n, 2))   # beyond the walls on the walled axes
    mask, kappa, mu = 0b101, 1.1, 0.05
    E, g, dk, md = orc.energy_grad(x, D0, L, kappa, mu, wall_mask=mask)
    assert md > 0.0 and not g[:4].any()
    h = 1e-6
    fd = (orc.energy_grad(x, D0, L, kappa + h, mu, wall_mask=mask)[0] -
          orc.energy_grad(x, D0, L, kappa - h, mu, wall_mask=mask)[0]) / (2 * h)
    assert dk == pytest.approx(fd, rel=1e-6, abs=1e-9)
    for i in range(4, n):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            f = (orc.energy_grad(xp, D0, L, kappa, mu, wall_mask=mask)[0] -
                 orc.energy_grad(xm, D0, L, kappa, mu, wall_mask=mask)[0]) / (2 * h)
            assert g[i, a] == pytest.approx(f, rel=1e-5, abs=1e-8)


@pytest.mark.parametrize("mask", [0b001, 0b011, 0b111])
def test_walled_grid_list_equals_the_definition(orc, mask):
    """Spheres on both sides of the walls, some beyond them: the cell search
    (clamped windows, no wrap on walled axes) finds exactly the brute-force
    set of pairs closer than rho_i + rho_j without minimum image on those axes."""
    rng = np.random.default_rng(mask)
    n, L = 600, 1.0
    D0 = np.exp(rng.normal(0, 0.6, n))
    x = rng.uniform(0.0, 1.0, (n, 3))   # periodic axes hold wrapped positions
    for a in range(3):
        if (mask >> a) & 1:
            x[:, a] = rng.uniform(-0.02, 1.02, n)
    k = 0.03
    rb, cb = orc.list_brute(x, D0, L, k, 0.1, 1e-3, wall_mask=mask)
    rg, cg = orc.list_grid(x, D0, L, k, 0.1, 1e-3, wall_mask=mask)
    assert np.array_equal(rb, rg) and np.array_equal(cb, cg)
    # no pair across a walled axis' boundary: every listed pair is close without wrap
    i = np.repeat(np.arange(n), np.diff(rb))
    dx = x[i] - x[cb]
    for a in range(3):
        if (mask >> a) & 1:
            assert np.abs(dx[:, a]).max() < 0.5
    # and with periodic axes the set differs (pairs across the boundary exist)
    rp, cp = orc.list_brute(x, D0, L, k, 0.1, 1e-3, wall_mask=0)
    assert cp.size > cb.size


def test_one_sphere_wall_contact_scale(orc):
    x = np.array([[0.35, 1.0, 1.0]])
    D0 = np.array([1.0])
    rowptr, col = orc.list_brute(x, D0, 2.0, 1.0, 0.0, 0.0, wall_mask=1)
    kc = orc.shrink_kappa(x, D0, 2.0, 1.0, rowptr, col, wall_mask=1)
    assert 0.7 * (1 - 1e-14) < kc < 0.7
    assert orc.energy_grad(x, D0, 2.0, kc, 0.0, wall_mask=1)[3] == 0.0


@pytest.mark.parametrize("mask,d", [(0b111, 3), (0b001, 3), (0b11, 2)])
def test_walled_run_ends_inside_the_walls(orc, mask, d):
    n, L = 400, 1.0
    D0 = np.linspace(0.7, 1.0, n)
    res = orc.run(D0, seed=5, L=L, d=d, walls=mask)
    assert res.stopped
    x = res.x
    rad = 0.5 * res.kappa_c * D0
    for a in range(d):
        if (mask >> a) & 1:
            assert (x[:, a] >= rad).all() and (L - x[:, a] >= rad).all()
        else:
            assert (x[:, a] >= 0).all() and (x[:, a] < L).all()
    # no overlap left, and the last contact (pair or wall) is reached
    E, g, dk, md = orc.energy_grad(x, D0, L, res.kappa_c, 0.0, d=d, wall_mask=mask)
    assert md == 0.0
    gap_wall = min(((np.minimum(x[:, a], L - x[:, a]) / rad) - 1).min() for a in range(d) if (mask >> a) & 1)
    dx = x[:, None, :] - x[None, :, :]
    for a in range(d):
        if not (mask >> a) & 1:
            dx[..., a] -= L * np.round(dx[..., a] / L)
    r = np.sqrt((dx ** 2).sum(-1)) + np.eye(n) * 10
    gap_pair = (r / (0.5 * res.kappa_c * (D0[:, None] + D0[None, :])) - 1).min()
    assert 0.0 <= min(gap_wall, gap_pair) < 1e-9
    # walls lower the density of a small packing against the periodic box
    per = orc.run(D0, seed=5, L=L, d=d)
    assert res.phi < per.phi


def test_walled_placement_keeps_candidates_off_the_walls(orc):
    D0 = np.linspace(0.5, 1.0, 500)
    k = orc.kappa0(D0, 1.0, 0.2)
    x, rnd, R = orc.place(3, D0, k, wall_mask=0b111)
    assert R >= 1
    rad = 0.5 * k * D0
    assert (x >= rad[:, None]).all() and (1.0 - x >= rad[:, None]).all()


# ------------------------------------------------------------------ curved walls
def test_one_sphere_in_a_ball_and_a_cylinder_by_hand(orc):
    """Container radius R = 2 about the centre of a box of edge 4; a sphere
    D^0 = 1 at kappa = 1 whose centre is 1.7 from the centre (or the axis):
    h = 0.3, delta = 0.4, pushed towards the centre with |dE/dx| = 0.4/0.5."""
    D0 = np.array([1.0])
    mu = 0.1
    x = np.array([[3.7, 2.0, 2.0]])
    E, g, dk, md = orc.energy_grad(x, D0, 4.0, 1.0, mu, wall_mask=(0, 1))
    assert md == pytest.approx(0.4, rel=1e-14)
    assert E == pytest.approx(0.5 * 0.4 ** 2 - mu, rel=1e-14)
    assert dk == pytest.approx(0.4 * 0.6 - mu, rel=1e-14)
    assert g[0] == pytest.approx([0.8, 0.0, 0.0], rel=1e-14, abs=1e-15)
    # diagonal offset: the push points along the offset
    x = np.array([[2.0 + 1.7 / np.sqrt(2), 2.0 - 1.7 / np.sqrt(2), 2.0]])
    E, g, dk, md = orc.energy_grad(x, D0, 4.0, 1.0, mu, wall_mask=(0, 1))
    assert md == pytest.approx(0.4, rel=1e-13)
    assert g[0] == pytest.approx([0.8 / np.sqrt(2), -0.8 / np.sqrt(2), 0.0], rel=1e-12, abs=1e-15)
    # cylinder about z: only the distance in x, y counts; z stays periodic
    x = np.array([[2.0, 3.7, 0.1]])
    E, g, dk, md = orc.energy_grad(x, D0, 4.0, 1.0, mu, wall_mask=(0, 2))
    assert md == pytest.approx(0.4, rel=1e-14)
    assert g[0] == pytest.approx([0.0, 0.8, 0.0], rel=1e-14, abs=1e-15)
    # at the centre: no contact, no term
    E, g, dk, md = orc.energy_grad(np.array([[2.0, 2.0, 2.0]]), D0, 4.0, 1.0, mu, wall_mask=(0, 1))
    assert md == 0.0 and E == -mu and not g.any()


def test_container_derivatives_by_finite_differences(orc):
    rng = np.random.default_rng(21)
    n, L = 30, 3.0
    D0 = rng.uniform(0.5, 1.0, n)
    D0[:3] = -D0[:3]
    x = rng.uniform(-0.1, L + 0.1, (n, 3))
    for container in (1, 2):
        if container == 2:
            x[:, 2] = rng.uniform(0.0, L, n)   # the cylinder's axis stays periodic
        bd = (0, container)
        kappa, mu = 1.05, 0.05
        E, g, dk, md = orc.energy_grad(x, D0, L, kappa, mu, wall_mask=bd)
        assert md > 0.0 and not g[:3].any()
        h = 1e-6
        fd = (orc.energy_grad(x, D0, L, kappa + h, mu, wall_mask=bd)[0] -
              orc.energy_grad(x, D0, L, kappa - h, mu, wall_mask=bd)[0]) / (2 * h)
        assert dk == pytest.approx(fd, rel=1e-6, abs=1e-9)
        for i in range(3, n):
            for a in range(3):
                xp, xm = x.copy(), x.copy()
                xp[i, a] += h
                xm[i, a] -= h
                f = (orc.energy_grad(xp, D0, L, kappa, mu, wall_mask=bd)[0] -
                     orc.energy_grad(xm, D0, L, kappa, mu, wall_mask=bd)[0]) / (2 * h)
                assert g[i, a] == pytest.approx(f, rel=1e-5, abs=1e-8)


@pytest.mark.parametrize("container", [1, 2])
def test_container_grid_list_equals_the_definition(orc, container):
    rng = np.random.default_rng(container + 40)
    n, L = 600, 1.0
    D0 = np.exp(rng.normal(0, 0.6, n))
    x = rng.uniform(0.0, 1.0, (n, 3))
    x[:, :2] = rng.uniform(-0.02, 1.02, (n, 2))
    if container == 1:
        x[:, 2] = rng.uniform(-0.02, 1.02, n)
    rb, cb = orc.list_brute(x, D0, L, 0.03, 0.1, 1e-3, wall_mask=(0, container))
    rg, cg = orc.list_grid(x, D0, L, 0.03, 0.1, 1e-3, wall_mask=(0, container))
    assert np.array_equal(rb, rg) and np.array_equal(cb, cg)


@pytest.mark.parametrize("container,d", [(1, 3), (2, 3), (1, 2)])
def test_run_in_a_container_ends_inside_it(orc, container, d):
    # from the dilute placement inside the container (App. A's start): a
    # uniform draw over the box would leave about half the spheres outside
    n, L = 400, 1.0
    D0 = np.linspace(0.7, 1.0, n)
    with orc.walls(0, container):
        k0 = orc.kappa0(D0, L, 0.05, d=d)
    x0, _, _ = orc.place(3, D0, k0, L, d, wall_mask=(0, container))
    res = orc.run(D0, seed=3, x0=x0, L=L, d=d, container=container)
    assert res.stopped
    x = res.x
    rad = 0.5 * res.kappa_c * D0
    ax = list(range(d)) if container == 1 else [0, 1]
    rc = np.sqrt(((x[:, ax] - 0.5) ** 2).sum(axis=1))
    assert (rc + rad <= 0.5).all()                      # inside the wall
    E, g, dk, md = orc.energy_grad(x, D0, L, res.kappa_c, 0.0, d=d, wall_mask=(0, container))
    assert md == 0.0
    assert ((0.5 - rc) / rad - 1).min() < 1e-3           # it touches the wall somewhere
    # phi over the container's volume
    if d == 3:
        Vc = (4 / 3) * np.pi * 0.125 if container == 1 else np.pi * 0.25
        assert res.phi == pytest.approx((np.pi / 6) * ((res.kappa_c * D0) ** 3).sum() / Vc, rel=1e-12)
    else:
        assert res.phi == pytest.approx((np.pi / 4) * ((res.kappa_c * D0) ** 2).sum() / (np.pi * 0.25), rel=1e-12)
    assert 0.5 < res.phi < 0.9


def test_kappa0_fills_the_container(orc):
    D0 = np.linspace(0.5, 1.0, 300)
    with orc.walls(0, 1):
        k = orc.kappa0(D0, 2.0, 0.1)
    assert (np.pi / 6) * k ** 3 * (D0 ** 3).sum() / ((4 / 3) * np.pi) == pytest.approx(0.1, rel=1e-13)


def test_container_placement_keeps_candidates_inside(orc):
    D0 = np.linspace(0.5, 1.0, 400)
    with orc.walls(0, 1):
        k = orc.kappa0(D0, 1.0, 0.15)
    x, rnd, R = orc.place(8, D0, k, wall_mask=(0, 1))
    assert R >= 1
    rc = np.sqrt(((x - 0.5) ** 2).sum(axis=1))
    assert (rc + 0.5 * k * D0 <= 0.5).all()


def test_run_restores_the_boundary_setting(orc):
    """orc_run takes its boundary from its parameters and leaves the module
    setting as it found it."""
    D0 = np.linspace(0.7, 1.0, 50)
    with orc.walls(5, 2):
        orc.run(D0, seed=1, max_iters=50, walls=0, container=0)
        L = orc.lib()
        assert L.orc_get_walls() == 5 and L.orc_get_container() == 2
    assert orc.lib().orc_get_walls() == 0 and orc.lib().orc_get_container() == 0
