"""The benchmark's workload at full size: N = 1e6 truncated lognormal
(sigma_ln = 2, S = 5e5), in the launch configuration the benchmark uses
(mixed precision, skin_abs 100, skin fraction 0.02), against the oracle on
every row.

States are inputs the oracle can produce itself (it shares nothing with the
CUDA path and takes nothing from it): uniform positions at phi = 0.3 and at
phi = 0.6 (deep overlaps; the rows of the largest spheres exceed 1024
entries, which the mixed kernel walks in several warp windows), and the
phi = 0.3 state with near-contact pairs planted on chosen rows (overlaps of
1e-3 down to 1e-6: the largest sphere against the smallest, the smallest
against their own size class, random pairs), the regime where 1 - r/d
cancels and where binary32 meets the resolution of the smallest spheres.

Bars: the neighbour list bit-exact (full CSR); binary64 energy, dE/dkappa,
max overlap and every gradient component bit-exact; mixed within 1e-5
relative on the scalars and element by element on the gradient (1e-5
relative plus the floor of conftest.row_term_scale).
"""
import numpy as np
import pytest

from paper_2608_12235_b300 import inputs

pytestmark = pytest.mark.gpu

N = 1_000_000
SKIN = dict(skin_abs=100.0, skin_s=0.02)   # the benchmark's list settings


@pytest.fixture(scope="module")
def rcp():
    import torch
    assert torch.cuda.is_available(), "the CUDA path needs a GPU"
    from paper_2608_12235_b300 import build, rcp as R
    build.build()
    R.load()
    return R


@pytest.fixture(scope="module")
def D0():
    return inputs.lognormal(N, 2.0, 5e5)


def _sigma0(orc, D0, cfg):
    m = orc.moments(D0)
    return cfg.skin_abs * ((cfg.lr_x * orc.kappa0(D0, 1.0, 0.05)) * (m[2] / m[1]))


def plant_near_contact(orc, x, D0, kappa, rng):
    """Move chosen partner spheres j onto the surface of chosen spheres i, at
    an overlap delta_ij from a log-uniform range [1e-6, 1e-3]: returns the new
    positions (binary64, wrapped into the unit box) and the planted (i, j)."""
    x = x.copy()
    order = np.argsort(D0, kind="stable")
    small, large = order[:4000], order[-40:]
    pairs = []
    # largest spheres against the smallest ones; smallest against their class;
    # random spheres against random partners
    for a in range(20):
        pairs.append((int(large[-1 - a]), int(small[a])))
    for a in range(20):
        pairs.append((int(small[20 + 2 * a]), int(small[21 + 2 * a])))
    rnd = rng.choice(np.setdiff1d(np.arange(N), np.concatenate([small[:100], large])), 40, replace=False)
    for a in range(20):
        pairs.append((int(rnd[2 * a]), int(rnd[2 * a + 1])))
    for i, j in pairs:
        delta = 10.0 ** rng.uniform(-6.0, -3.0)
        d = kappa * 0.5 * (D0[i] + D0[j])
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        x[j] = np.mod(x[i] + u * (d * (1.0 - delta)), 1.0)
    return x, pairs


def _compare(rcp, orc, D0, x, k, precision, term_scale, grad_check, sums_check, rows_to_report=()):
    p = rcp.Packing(D0, box=1.0, seed=0, precision=precision, **SKIN)
    p.set_positions(x, k)
    rp, col = p.neighbors()
    s0 = _sigma0(orc, D0, p.cfg)
    orp, ocol = orc.list_grid(x, D0, 1.0, k, p.cfg.skin_s, s0)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol), "neighbour list differs"
    lens = np.diff(rp)
    out = {"entries": int(col.size), "longest_row": int(lens.max()), "rows_over_1024": int((lens > 1024).sum())}
    for mu in (0.0, 0.013):
        E, g, dk, md = p.energy_grad(mu)
        oE, og, odk, omd = orc.energy_grad(x, D0, 1.0, k, mu, rowptr=orp, col=ocol)
        if precision == rcp.RCP_FP64:
            assert E == oE and dk == odk and md == omd
            assert np.array_equal(g, og)
            continue
        out[f"E_rel_mu{mu}"] = abs(E - oE) / abs(oE)
        out[f"dEdk_rel_mu{mu}"] = abs(dk - odk) / abs(odk)
        out["maxdelta_rel"] = abs(md - omd) / omd
        out[f"sums_error_over_bound_mu{mu}"] = sums_check(E, oE, dk, odk, mu, k, D0, what="mixed, N = 1e6")
        assert abs(md - omd) <= 1e-5 * omd
        if mu == 0.0:
            scale = term_scale(x, D0, 1.0, k)
            out["grad_worst_error_over_bound"] = grad_check(g, og, scale, what="mixed, N = 1e6")
            err = np.abs(g - og)
            out["grad_max_abs_error"] = float(err.max())
            nz = scale[0] > 0.0
            out["grad_max_error_over_row_scale"] = float((err[nz].max(axis=1) / scale[0][nz]).max())
            for name, rows in rows_to_report:
                rows = np.asarray(rows)
                e = err[rows].max(axis=1)
                out[f"{name}_max_error_over_row_scale"] = float((e / np.maximum(scale[0][rows], 1e-300)).max())
    p.close()
    print(precision, out)
    return out


@pytest.mark.parametrize("phi", [0.3, 0.6])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_uniform_states(rcp, orc, D0, phi, precision, term_scale, grad_check, sums_check):
    x = orc.init_positions(0, N)
    k = orc.kappa0(D0, 1.0, phi)
    prec = rcp.RCP_FP64 if precision == "fp64" else rcp.RCP_MIXED
    order = np.argsort(D0, kind="stable")
    out = _compare(rcp, orc, D0, x, k, prec, term_scale, grad_check, sums_check,
                   rows_to_report=[("largest20", order[-20:]), ("smallest20", order[:20])])
    if phi == 0.6:
        assert out["rows_over_1024"] > 0   # the multi-window walk of the long rows is reached


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_planted_near_contact(rcp, orc, D0, precision, term_scale, grad_check, sums_check):
    x0 = orc.init_positions(0, N)
    k = orc.kappa0(D0, 1.0, 0.3)
    x, pairs = plant_near_contact(orc, x0, D0, k, np.random.default_rng(12))
    prec = rcp.RCP_FP64 if precision == "fp64" else rcp.RCP_MIXED
    rows = sorted({i for i, _ in pairs} | {j for _, j in pairs})
    _compare(rcp, orc, D0, x, k, prec, term_scale, grad_check, sums_check, rows_to_report=[("planted", rows)])
    if prec == rcp.RCP_MIXED:
        # the planted rows one by one against the oracle's brute-force row
        # (all N partners), so the list cannot hide a missed pair
        p = rcp.Packing(D0, box=1.0, seed=0, precision=prec, **SKIN)
        p.set_positions(x, k)
        E, g, dk, md = p.energy_grad(0.0)
        sc = term_scale(x, D0, 1.0, k)
        for i in rows[:40]:
            og, oe, ok, omd = orc.row_grad(x, D0, 1.0, k, int(i))
            assert omd > 0.0
            grad_check(g[i:i + 1], og[None, :], (sc[0][i:i + 1], sc[1][i:i + 1]), what=f"planted row {i}")
        p.close()
