"""Final packing fraction of the mixed path beside the binary64 path at
N = 1e5 (truncated power law P(D) ~ D^-3, S = 20, phi0 = 0.05), each run to
App. A's stopping criterion (largest overlap below 5e-4) and shrunk to
contact (Sec. II).

The binary64 path is the oracle's arithmetic bit for bit (checked here over a
200-iteration window at the same N, against the oracle itself).  A whole run
is chaotic in the rounding, so the mixed path's phi differs from the binary64
phi of the same seed by an amount of the order of the protocol's own
run-to-run scatter; the paper reports phi reproducible only to a few 1e-4
when merely the thread count changes (Data and code availability).  Measured
on B300 over seeds 0-4: phi_mixed - phi_fp64 = -1.51e-3 ... +1.28e-3, mean
-2.7e-4 (earlier builds of the mixed kernel: -2.03e-3 ... +1.12e-3), against
a binary64 seed-to-seed standard deviation of 1.4e-3.  The
bounds below are twice that scatter per seed and 1e-3 on the mean of five
seeds (about 3.5 standard errors of a five-seed mean); the 1e-4 per-seed
target of a single run is not met and is not asserted.
"""
import numpy as np
import pytest

from paper_2608_12235_b300 import inputs

pytestmark = pytest.mark.gpu

N = 100_000


@pytest.fixture(scope="module")
def rcp():
    import torch
    assert torch.cuda.is_available(), "the CUDA path needs a GPU"
    from paper_2608_12235_b300 import build, rcp as R
    build.build()
    R.load()
    return R


def test_fp64_window_bitexact_against_the_oracle_at_n1e5(rcp, orc):
    """200 iterations of the protocol from the seeded start: the same
    positions, bit for bit, on the GPU and in the oracle."""
    D0 = inputs.power_law(N, -3.0, 20.0)
    p = rcp.Packing(D0, box=1.0, seed=3)
    p.run(max_iters=200, shrink=False)
    x, _, _, s = p.state()
    p.close()
    with orc.threads(8):
        ref = orc.run(D0, seed=3, max_iters=200)
    assert s.t == 200
    assert np.array_equal(x, ref.x)


def test_mixed_phi_beside_fp64_at_n1e5(rcp):
    D0 = inputs.power_law(N, -3.0, 20.0)
    dphi, phi64 = [], []
    for seed in range(5):
        out = {}
        for prec in (rcp.RCP_MIXED, rcp.RCP_FP64):
            p = rcp.Packing(D0, box=1.0, seed=seed, precision=prec)
            r = p.run()
            p.close()
            assert r.stopped and r.max_delta < 5e-4
            out[prec] = r.phi
        dphi.append(out[rcp.RCP_MIXED] - out[rcp.RCP_FP64])
        phi64.append(out[rcp.RCP_FP64])
    scatter = float(np.std(phi64, ddof=1))
    print(f"phi(mixed) - phi(fp64) per seed: {dphi}; mean {np.mean(dphi):.2e}; fp64 seed scatter {scatter:.2e}")
    assert all(abs(d) < 2.8e-3 for d in dphi)
    assert abs(float(np.mean(dphi))) < 1e-3
