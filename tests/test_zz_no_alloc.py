"""The allocation-free evaluation entry point (rcp_energy_grad_noalloc).

It exists for callers that cannot allocate device memory (a memory pool
owned and fully reserved by another runtime, device memory partitioned once
at start-up, or an allocator held by another library).  This file is
collected last on purpose: if the check fails, a run that stops at the first
failure has already run every other test.  It passes alone in a fresh process
and after the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [3000, 300_000, 1 << 21])
def test_noalloc_matches_the_allocating_entry_point_twice_in_a_row(n):
    """Bit for bit against rcp_energy_grad, two calls in a row, at a size of
    one finishing block, at one that needs the chunked finish (more than 1024
    blocks of partials), and at the largest size the scratch holds."""
    import torch

    import oracle
    from paper_2608_12235_b300 import build, inputs, rcp

    assert torch.cuda.is_available()
    build.build()
    D0 = inputs.lognormal(n, 0.5, 10.0)
    x = oracle.init_positions(5, n)
    k = oracle.kappa0(D0, 1.0, 0.55)
    mu = 0.013
    p = rcp.Packing(D0, box=1.0, seed=5)
    p.set_positions(x, k)
    E, g, dk, md = p.energy_grad(mu)  # the existing, allocating entry point
    rp, col = p.neighbors()
    p.close()
    dev = torch.device("cuda", 0)
    xt = torch.tensor(x, dtype=torch.float64, device=dev)
    Dt = torch.tensor(D0, dtype=torch.float64, device=dev)
    rpt = torch.tensor(rp.astype(np.int32), device=dev)
    colt = torch.tensor(col.astype(np.int32), device=dev)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        Et = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        dkt = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        mdt = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        gt = torch.full((n, 3), np.nan, dtype=torch.float64, device=dev)
        rcp.rcp_energy_grad_noalloc(xt, Dt, 1.0, k, mu, rpt, colt, Et, gt, dkt, mdt, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        # binary64, same operations in the same order: identical results
        assert Et.item() == E, call
        assert dkt.item() == dk, call
        assert mdt.item() == md, call
        assert np.array_equal(gt.cpu().numpy(), g), call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_2608_12235_b300 import rcp

    dev = torch.device("cuda", 0)
    n = (1 << 21) + 1
    one = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(rcp.RcpError) as e:
        rcp.rcp_energy_grad_noalloc(one, torch.zeros(n, dtype=torch.float64, device=dev), 1.0, 1.0, 0.0,
                                    one, one, one, one, one, one)
    assert e.value.status == 5
