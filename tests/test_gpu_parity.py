"""CUDA path against the CPU oracle, element by element, on the same seeded inputs.

Bar: integer work (cell keys, neighbour lists) bit-exact; the binary64 path
bit-exact as well (same operations in the same order, IEEE-correct on both
sides); the mixed path within 1e-5 relative on energy, dE/dkappa and the
largest overlap, and element by element on the gradient within 1e-5 relative
plus an absolute floor of 1e-6 of the row's summed term magnitudes (see
row_term_scale in conftest.py for why that floor).
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
    Dref = m[2] / m[1]
    return cfg.skin_abs * ((cfg.lr_x * kappa0) * Dref)


def _mk(rcp, D0, seed=0, box=1.0, **cfg):
    return rcp.Packing(D0, box=box, seed=seed, **cfg)


# ------------------------------------------------------------------ initial state
@pytest.mark.parametrize("n", [1, 2, 257, 1000])
def test_initial_positions_and_kappa0_bitexact(rcp, orc, n):
    D0 = inputs.lognormal(n, 0.5, 10.0)
    p = _mk(rcp, D0, seed=42)
    x, m, v, s = p.state()
    assert np.array_equal(x, orc.init_positions(42, n))
    assert s.kappa == orc.kappa0(D0, 1.0, 0.05)
    assert s.t == 0 and not m.any() and not v.any()
    p.close()


# ------------------------------------------------------------------ integer work
@pytest.mark.parametrize("n,sig,S,phi", [(1000, 0.5, 10.0, 0.05), (4097, 1.0, 100.0, 0.4),
                                         (3000, 2.0, 5e4, 0.2), (777, 0.2, 3.0, 0.6)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cell_keys_and_list_bitexact(rcp, orc, n, sig, S, phi, precision):
    # the list does not depend on the precision of the pair arithmetic
    D0 = inputs.lognormal(n, sig, S)
    prec = rcp.RCP_FP64 if precision == "fp64" else rcp.RCP_MIXED
    p = _mk(rcp, D0, seed=n, precision=prec)
    x = orc.init_positions(n, n)
    k = orc.kappa0(D0, 1.0, phi)
    p.set_positions(x, k)
    rcp.rcp_build_neighbors(p.h)
    s0 = _sigma0(orc, D0, orc.kappa0(D0, 1.0, 0.05), p.cfg)
    keys = p.cell_keys()
    assert np.array_equal(keys, orc.cell_keys(x, D0, 1.0, k, p.cfg.skin_s, s0, occ=p.cfg.cell_occupancy))
    rp, col = p.neighbors()
    orp, ocol = orc.list_brute(x, D0, 1.0, k, p.cfg.skin_s, s0)
    assert np.array_equal(rp, orp)
    assert np.array_equal(col, ocol)
    p.close()


def test_empty_and_single_rows(rcp, orc):
    # two far-apart spheres and one lone sphere: empty rows everywhere
    D0 = np.array([1.0, 1.0, 0.5])
    x = np.array([[1.0, 1.0, 1.0], [5.0, 5.0, 5.0], [8.0, 2.0, 6.0]])
    p = _mk(rcp, D0, box=10.0)
    p.set_positions(x, 1.0)
    rp, col = p.neighbors()
    assert rp.tolist() == [0, 0, 0, 0] and col.size == 0
    E, g, dk, md = p.energy_grad(0.1)
    assert E == -0.1 * 2.5 and dk == -0.1 * 2.5 and md == 0.0 and not g.any()
    p.close()


# ------------------------------------------------------------------ binary64 evaluation
def _states(orc):
    out = []
    for n, sig, S, phi, seed in [(1000, 0.5, 10.0, 0.3, 1), (1000, 0.5, 10.0, 0.64, 2), (2049, 1.0, 100.0, 0.5, 3),
                                 (600, 0.3, 4.0, 0.7, 4)]:
        D0 = inputs.lognormal(n, sig, S)
        out.append((D0, orc.init_positions(seed, n), orc.kappa0(D0, 1.0, phi)))
    return out


def test_two_spheres_closed_form_on_gpu(rcp):
    D0 = np.ones(2)
    p = _mk(rcp, D0, box=10.0)
    p.set_positions(np.array([[5.0, 5, 5], [5.9, 5, 5]]), 1.0)
    E, g, dk, md = p.energy_grad(0.01)
    assert E == pytest.approx(0.005 - 0.02, rel=1e-14)
    np.testing.assert_allclose(g, [[0.1, 0, 0], [-0.1, 0, 0]], atol=1e-15)
    assert dk == pytest.approx(0.09 - 0.02, rel=1e-14) and md == pytest.approx(0.1, rel=1e-14)
    p.close()


def test_energy_grad_fp64_bitexact(rcp, orc):
    for D0, x, k in _states(orc):
        p = _mk(rcp, D0)
        p.set_positions(x, k)
        for mu in (0.0, 0.013):
            E, g, dk, md = p.energy_grad(mu)
            oE, og, odk, omd = orc.energy_grad(x, D0, 1.0, k, mu)
            assert E == oE and dk == odk and md == omd
            assert np.array_equal(g, og)
        p.close()


def test_adam_step_fp64_bitexact(rcp, orc):
    D0, x, k = _states(orc)[0]
    p = _mk(rcp, D0)
    p.set_positions(x, k)
    rng = np.random.default_rng(0)
    xo, mo, vo = x.ravel().copy(), np.zeros(x.size), np.zeros(x.size)
    ko, mk, vk = np.array([k]), np.zeros(1), np.zeros(1)
    b1 = b2 = 1.0
    for t in range(5):
        g = rng.standard_normal(x.shape) * 10.0 ** rng.uniform(-4, 2)
        dk = float(rng.standard_normal())
        p.adam_step(g, dk, 1e-3, 1e-4)
        b1 *= 0.9
        b2 *= 0.999
        orc.adam_update(xo, mo, vo, g, 1e-3, b1, b2)
        xo = np.array([orc.wrap(a, 1.0) for a in xo])
        orc.adam_update(ko, mk, vk, np.array([dk]), 1e-4, b1, b2)
    xs, ms, vs, s = p.state()
    assert np.array_equal(xs.ravel(), xo) and np.array_equal(ms.ravel(), mo) and np.array_equal(vs.ravel(), vo)
    assert s.kappa == ko[0] and s.b1 == b1 and s.b2 == b2 and s.t == 5
    p.close()


@pytest.mark.parametrize("d,mask", [(2, 0), (3, 0b101), (2, 0b01)])
def test_adam_step_fp64_bitexact_disks_and_walls(rcp, orc, d, mask):
    """The standalone Adam step with the caller's [N][d] gradient: disks (the
    internal layout has three columns) and walled axes (no wrap there)."""
    n = 700
    D0 = inputs.lognormal(n, 0.5, 10.0)
    x = orc.init_positions(8, n, 1.0, d=d)
    k = orc.kappa0(D0, 1.0, 0.4, d=d)
    p = _mk(rcp, D0, seed=8, d=d, walls=mask)
    p.set_positions(x, k)
    rng = np.random.default_rng(d + 10 * mask)
    xo, mo, vo = x.ravel().copy(), np.zeros(x.size), np.zeros(x.size)
    periodic = np.array([not ((mask >> (a % d)) & 1) for a in range(x.size)])
    b1 = b2 = 1.0
    for t in range(4):
        g = rng.standard_normal(x.shape) * 10.0 ** rng.uniform(-4, 2)
        p.adam_step(g, 0.0, 1e-3, 0.0)
        b1 *= 0.9
        b2 *= 0.999
        orc.adam_update(xo, mo, vo, g, 1e-3, b1, b2)
        xo = np.array([orc.wrap(a, 1.0) if per else a for a, per in zip(xo, periodic)])
    xs, ms, vs, s = p.state()
    assert xs.shape == (n, d)
    assert np.array_equal(xs.ravel(), xo) and np.array_equal(ms.ravel(), mo) and np.array_equal(vs.ravel(), vo)
    assert s.t == 4
    p.close()


def test_shrink_fp64_bitexact(rcp, orc):
    D0, x, k = _states(orc)[1]
    p = _mk(rcp, D0)
    p.set_positions(x, k)
    kc, phi = p.shrink()
    rp, col = orc.list_grid(x, D0, 1.0, k, 0.1, 0.0)
    okc = orc.shrink_kappa(x, D0, 1.0, k, rp, col)
    assert kc == okc and phi == orc.phi(D0, 1.0, okc)
    p.close()


# ------------------------------------------------------------------ the protocol, binary64
def test_full_run_fp64_bitexact_lognormal_n1000(rcp, orc):
    """Lognormal sigma_ln = 0.5, S = 10, N = 1000, seed 0, phi0 = 0.05, run to the
    stopping criterion: same iteration count, same final positions, same phi."""
    D0 = inputs.lognormal(1000, 0.5, 10.0)
    ref = orc.run(D0, seed=0)
    p = _mk(rcp, D0, seed=0)
    r = p.run()
    assert r.stopped and ref.stopped
    assert r.iters == ref.iters
    assert r.kappa_c == ref.kappa_c and r.phi == ref.phi
    assert np.array_equal(p.positions(), ref.x)
    p.close()


@pytest.mark.parametrize("n,sig,S,phi0", [(2000, 0.5, 10.0, 0.05), (3000, 1.5, 200.0, 0.3)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_placement_matches_the_oracle(rcp, orc, n, sig, S, phi0, precision):
    """Non-overlapping placement by rounds: the same positions as the oracle's
    sequential rounds (binary64 positions bit for bit; the mixed handle holds
    them in fixed point)."""
    D0 = inputs.lognormal(n, sig, S)
    prec = rcp.RCP_FP64 if precision == "fp64" else rcp.RCP_MIXED
    p = _mk(rcp, D0, seed=11, precision=prec, placement=1, phi0=phi0)
    k = orc.kappa0(D0, 1.0, phi0)
    x, rnd, R = orc.place(11, D0, k)
    assert R >= 1
    got = p.positions()
    if precision == "fp64":
        assert np.array_equal(got, x)
    else:
        assert np.allclose(got, x, rtol=0.0, atol=1e-15)
    p.close()


def test_full_run_from_placement_fp64_bitexact(rcp, orc):
    """The protocol from the non-overlapping start: same trajectory as the
    oracle's run from the oracle's placement."""
    D0 = inputs.lognormal(800, 0.5, 10.0)
    k = orc.kappa0(D0, 1.0, 0.05)
    x0, _, _ = orc.place(4, D0, k)
    ref = orc.run(D0, seed=4, x0=x0)
    p = _mk(rcp, D0, seed=4, placement=1)
    r = p.run()
    assert r.stopped and ref.stopped and r.iters == ref.iters
    assert r.kappa_c == ref.kappa_c and r.phi == ref.phi
    assert np.array_equal(p.positions(), ref.x)
    p.close()


def test_resume_is_bitexact(rcp):
    D0 = inputs.lognormal(500, 0.5, 10.0)
    a = _mk(rcp, D0, seed=3)
    a.run(max_iters=3000, shrink=False)
    xa, ma, va, sa = a.state()
    b = _mk(rcp, D0, seed=3)
    b.run(max_iters=1500, shrink=False)
    x, m, v, s = b.state()
    c = _mk(rcp, D0, seed=99)
    rcp.rcp_load_state(c.h, x, m, v, s)
    c.run(max_iters=1500, shrink=False)
    xc, mc, vc, sc = c.state()
    assert sc.t == sa.t == 3000
    assert np.array_equal(xc, xa) and np.array_equal(mc, ma) and np.array_equal(vc, va) and sc.kappa == sa.kappa
    for p in (a, b, c):
        p.close()


def test_chunk_size_does_not_change_the_trajectory(rcp):
    D0 = inputs.lognormal(300, 0.5, 10.0)
    xs = []
    for chunk in (1, 7, 64):
        p = _mk(rcp, D0, seed=5, chunk=chunk)
        p.run(max_iters=700, shrink=False)
        xs.append(p.positions())
        p.close()
    assert np.array_equal(xs[0], xs[1]) and np.array_equal(xs[0], xs[2])


# ------------------------------------------------------------------ mixed precision
def test_energy_grad_mixed_within_tolerance(rcp, orc, term_scale, grad_check, sums_check):
    for D0, x, k in _states(orc):
        p = _mk(rcp, D0, precision=rcp.RCP_MIXED)
        p.set_positions(x, k)
        mu = 0.013
        E, g, dk, md = p.energy_grad(mu)
        oE, og, odk, omd = orc.energy_grad(x, D0, 1.0, k, mu)
        sums_check(E, oE, dk, odk, mu, k, D0, what="mixed")
        assert abs(md - omd) <= 1e-5 * omd
        w = grad_check(g, og, term_scale(x, D0, 1.0, k), what="mixed")
        print(f"N={D0.size} worst gradient error / bound {w:.3g}")
        p.close()


def test_mixed_state_follows_the_caller_order(rcp, orc):
    """The mixed path keeps its spheres in cell-key order inside the library
    (rebuilt at every neighbour build): positions, moments and a caller's
    gradient must still come and go in the caller's sphere order."""
    D0, x, k = _states(orc)[0]
    p = _mk(rcp, D0, precision=rcp.RCP_MIXED)
    p.set_positions(x, k)
    rcp.rcp_build_neighbors(p.h)  # reorders the internal state
    assert np.allclose(p.positions(), x, rtol=0.0, atol=1e-15)
    rng = np.random.default_rng(0)
    xo, mo, vo = x.ravel().copy(), np.zeros(x.size), np.zeros(x.size)
    b1 = b2 = 1.0
    for _ in range(3):
        g = rng.standard_normal(x.shape)
        p.adam_step(g, 0.0, 1e-3, 0.0)
        b1 *= 0.9
        b2 *= 0.999
        orc.adam_update(xo, mo, vo, g, 1e-3, b1, b2)
        xo = np.array([orc.wrap(a, 1.0) for a in xo])
        rcp.rcp_build_neighbors(p.h)  # and again, from the moved state
    xs, ms, vs, s = p.state()
    d = np.abs(xs.ravel() - xo)
    d = np.minimum(d, 1.0 - d)  # a coordinate may sit across the periodic wrap
    assert d.max() <= 1e-9
    # binary32 moments: absolute error a few ulp of the moment's scale
    assert np.allclose(ms.ravel(), mo, rtol=1e-5, atol=1e-7)
    assert np.allclose(vs.ravel(), vo, rtol=1e-5, atol=1e-10)
    rcp.rcp_load_state(p.h, xs, ms, vs, s)
    x2, m2, v2, _ = p.state()
    assert np.array_equal(m2, ms) and np.array_equal(v2, vs)
    assert np.allclose(x2, xs, rtol=0.0, atol=1e-15)
    p.close()


def test_energy_grad_mixed_near_contact(rcp, orc, term_scale, grad_check, sums_check):
    """Small overlaps (delta ~ 1e-3, a relaxed packing inflated by 0.2 %): the
    regime where a plain binary32 d - r would cancel."""
    D0 = inputs.lognormal(400, 0.5, 10.0)
    ref = orc.run(D0, seed=2)
    k = ref.kappa_c * 1.002
    x = ref.x
    p = _mk(rcp, D0, precision=rcp.RCP_MIXED)
    p.set_positions(x, k)
    for mu in (0.0, 0.01):
        E, g, dk, md = p.energy_grad(mu)
        oE, og, odk, omd = orc.energy_grad(x, D0, 1.0, k, mu)
        assert 5e-4 < omd < 5e-3
        print(f"mu={mu} relE={abs(E - oE) / abs(oE):.2e} reldk={abs(dk - odk) / abs(odk):.2e} "
              f"relg={np.linalg.norm(g - og) / np.linalg.norm(og):.2e} relmd={abs(md - omd) / omd:.2e}")
        sums_check(E, oE, dk, odk, mu, k, D0, what="mixed near contact")
        assert abs(md - omd) <= 1e-5 * omd
        w = grad_check(g, og, term_scale(x, D0, 1.0, k), what="mixed near contact")
        print(f"worst gradient error / bound {w:.3g}")
    p.close()


def test_mixed_run_reaches_the_criterion(rcp, orc):
    """Mixed precision runs the whole protocol to the stopping criterion; the
    final state has no binary64 overlap at kappa_c.  Rounding differences
    grow chaotically along a trajectory, so phi is compared with the binary64
    oracle statistically: over three seeds the mean difference must sit
    inside the seed-to-seed scatter of this small system."""
    D0 = inputs.lognormal(1000, 0.5, 10.0)
    diffs = []
    for seed in (0, 1, 2):
        p = _mk(rcp, D0, seed=seed, precision=rcp.RCP_MIXED)
        r = p.run()
        assert r.stopped and r.max_delta < 5e-4
        x = p.positions()
        assert orc.energy_grad(x, D0, 1.0, r.kappa_c, 0.0)[3] == 0.0
        p.close()
        ref = orc.run(D0, seed=seed)
        diffs.append(r.phi - ref.phi)
    print("phi(mixed) - phi(binary64) per seed:", diffs)
    assert all(abs(d) < 0.015 for d in diffs)
    assert abs(float(np.mean(diffs))) < 6e-3


# ------------------------------------------------------------------ extreme size ratio, sampled
def test_extreme_ratio_sampled_rows_bitexact(rcp, orc):
    """N = 1e6 truncated lognormal sigma_ln = 2, S = 5e5: sampled rows of the list
    and of the binary64 gradient against brute force over all spheres."""
    D0 = inputs.lognormal(1_000_000, 2.0, 5e5)
    p = _mk(rcp, D0, seed=0)
    k = orc.kappa0(D0, 1.0, 0.3)
    x = orc.init_positions(0, D0.size)
    p.set_positions(x, k)
    rp, col = p.neighbors()
    s0 = _sigma0(orc, D0, orc.kappa0(D0, 1.0, 0.05), p.cfg)
    E, g, dk, md = p.energy_grad(0.0)
    rng = np.random.default_rng(1)
    rows = np.concatenate([rng.integers(0, D0.size, 12), [0, D0.size - 1, D0.size // 2]])
    for i in rows:
        assert np.array_equal(col[rp[i]:rp[i + 1]], orc.row_brute(x, D0, 1.0, k, p.cfg.skin_s, s0, int(i)))
        og, oe, ok, omd = orc.row_grad(x, D0, 1.0, k, int(i))
        assert np.array_equal(g[i], og)
    p.close()


def test_periodic_image_rule_is_enforced(rcp):
    D0 = np.ones(8)
    p = _mk(rcp, D0, box=1.0)
    with pytest.raises(rcp.RcpError) as e:
        p.set_positions(np.random.default_rng(0).random((8, 3)), 0.5)
        rcp.rcp_build_neighbors(p.h)
    assert e.value.status == 2
    p.close()


# ------------------------------------------------------------------ two dimensions
# d = 2 handles hold disks in the plane z = L_z / 2 of the three-axis layout;
# everything the caller sees has two columns and must match the oracle's d = 2
# definitions bit for bit in binary64.
def test_two_dimensional_initial_state_and_kappa0_bitexact(rcp, orc):
    D0 = inputs.lognormal(700, 0.5, 10.0)
    p = _mk(rcp, D0, seed=9, d=2)
    assert rcp.rcp_dim(p.h) == 2
    assert np.array_equal(p.positions(), orc.init_positions(9, 700, 1.0, d=2))
    assert p.state()[3].kappa == orc.kappa0(D0, 1.0, 0.05, d=2)
    p.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_dimensional_list_and_energy(rcp, orc, precision, term_scale, grad_check, sums_check):
    n = 1200
    D0 = inputs.lognormal(n, 1.0, 30.0)
    prec = rcp.RCP_FP64 if precision == "fp64" else rcp.RCP_MIXED
    p = _mk(rcp, D0, seed=3, d=2, precision=prec)
    x = orc.init_positions(3, n, 1.0, d=2)
    k = orc.kappa0(D0, 1.0, 0.45, d=2)
    p.set_positions(x, k)
    rp, col = p.neighbors()
    s0 = _sigma0(orc, D0, orc.kappa0(D0, 1.0, 0.05, d=2), p.cfg)
    orp, ocol = orc.list_brute(x, D0, 1.0, k, p.cfg.skin_s, s0, d=2)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    E, g, dk, md = p.energy_grad(0.01)
    oE, og, odk, omd = orc.energy_grad(x, D0, 1.0, k, 0.01, d=2)
    assert g.shape == (n, 2)
    if precision == "fp64":
        assert E == oE and dk == odk and md == omd and np.array_equal(g, og)
    else:
        sums_check(E, oE, dk, odk, 0.01, k, D0, what="mixed d = 2")
        assert abs(md - omd) <= 1e-5 * omd
        grad_check(g, og, term_scale(x, D0, 1.0, k, d=2), what="mixed d = 2")
    p.close()


def test_two_dimensional_full_run_fp64_bitexact(rcp, orc):
    """Disks, lognormal sigma_ln = 0.5, S = 10, N = 400, run to the stop: the
    oracle's d = 2 trajectory, iteration count and area fraction."""
    D0 = inputs.lognormal(400, 0.5, 10.0)
    ref = orc.run(D0, seed=1, d=2)
    p = _mk(rcp, D0, seed=1, d=2)
    r = p.run()
    assert r.stopped and ref.stopped and r.iters == ref.iters
    assert r.kappa_c == ref.kappa_c and r.phi == ref.phi
    assert np.array_equal(p.positions(), ref.x)
    p.close()


def test_two_dimensional_placement_matches_the_oracle(rcp, orc):
    D0 = inputs.lognormal(1500, 1.0, 30.0)
    p = _mk(rcp, D0, seed=6, d=2, placement=1, phi0=0.2)
    x, _, R = orc.place(6, D0, orc.kappa0(D0, 1.0, 0.2, d=2), d=2)
    assert R >= 1 and np.array_equal(p.positions(), x)
    p.close()
