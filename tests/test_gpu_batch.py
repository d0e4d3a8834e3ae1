"""Batched packings (one graph of batched kernels for all of them) against
their solo runs: bit-identical trajectories, independent stops."""
import numpy as np
import pytest

from paper_2608_12235_b300 import inputs

pytestmark = pytest.mark.gpu

SPECS = [(300, 0.5, 10.0, 1), (1000, 0.8, 50.0, 2), (2500, 0.3, 5.0, 3), (600, 1.0, 150.0, 4)]


@pytest.fixture(scope="module")
def rcp():
    import torch
    assert torch.cuda.is_available()
    from paper_2608_12235_b300 import build, rcp as R
    build.build()
    R.load()
    return R


def _packings(rcp, precision):
    return [rcp.Packing(inputs.lognormal(n, sig, S), seed=seed, precision=precision) for n, sig, S, seed in SPECS]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_solo(rcp, precision):
    solo = _packings(rcp, precision)
    for p in solo:
        p.run(max_iters=900, shrink=False)
    batch_packs = _packings(rcp, precision)
    b = rcp.Batch(batch_packs, autotune=False)
    res = b.run(max_iters=900, shrink=False)
    assert all(r.iters == 900 for r in res)
    for p, q in zip(solo, batch_packs):
        xs, ms, vs, ss = p.state()
        xb, mb, vb, sb = q.state()
        assert np.array_equal(xs, xb) and np.array_equal(ms, mb) and sb.kappa == ss.kappa
    b.close()
    for p in solo + batch_packs:
        p.close()


def test_batch_runs_every_packing_to_its_stop(rcp):
    specs = SPECS[:3]
    solo = [rcp.Packing(inputs.lognormal(n, sig, S), seed=seed) for n, sig, S, seed in specs]
    ref = [p.run() for p in solo]
    packs = [rcp.Packing(inputs.lognormal(n, sig, S), seed=seed) for n, sig, S, seed in specs]
    b = rcp.Batch(packs)
    res = b.run()
    for r, q in zip(res, ref):
        assert r.stopped and r.iters == q.iters and r.phi == q.phi and r.kappa_c == q.kappa_c
    b.close()
    for p in solo + packs:
        p.close()


def test_batch_autotune_mixed(rcp, orc, term_scale, grad_check, sums_check):
    """The autotuned batch runs, and each packing's evaluation under the
    tuned long-row threshold still matches the oracle (a threshold beyond
    what the short-row path can mark would drop overlaps silently)."""
    packs = _packings(rcp, 1)
    b = rcp.Batch(packs, autotune=True)
    res = b.run(max_iters=1500, shrink=False)
    lr, chunk = b.tuning()
    assert lr in (8, 16, 32) and chunk in (8, 16, 32, 64)
    assert all(r.iters == 1500 for r in res)
    b.close()
    for p, (n, sig, S, seed) in zip(packs, SPECS):
        D0 = inputs.lognormal(n, sig, S)
        x, _, _, s = p.state()
        E, g, dk, md = p.energy_grad(0.01)
        oE, og, odk, omd = orc.energy_grad(x, D0, 1.0, s.kappa, 0.01)
        sums_check(E, oE, dk, odk, 0.01, s.kappa, D0, what=f"tuned long_row {lr}")
        grad_check(g, og, term_scale(x, D0, 1.0, s.kappa), what=f"tuned long_row {lr}")
        p.close()
