"""The torch.autograd binding: forward = fused energy kernel, hand-written
backward.  Checked against a torch autograd reference written with plain torch
operations and against central finite differences, at N = 64."""
import numpy as np
import pytest

from paper_2608_12235_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available()
    from paper_2608_12235_b300 import autograd, build, rcp
    build.build()
    rcp.load()
    return torch, rcp, autograd


def _ref_energy(torch, x, D0, L, kappa, mu):
    n = x.shape[0]
    i, j = torch.triu_indices(n, n, 1, device=x.device)
    dx = x[i] - x[j]
    dx = dx - L * torch.round(dx / L)
    r = torch.sqrt((dx * dx).sum(1))
    d = kappa * 0.5 * (D0[i] + D0[j])
    delta = 1 - r / d
    return 0.5 * torch.sum(torch.clamp(delta, min=0) ** 2) - mu * kappa * D0.sum()


def _state(orc, n=64, phi=0.2, seed=5):
    D0 = inputs.lognormal(n, 0.4, 4.0)
    return D0, orc.init_positions(seed, n), orc.kappa0(D0, 1.0, phi)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_autograd_matches_torch_reference(mods, orc, precision, tol):
    torch, rcp, ag = mods
    D0, x, k = _state(orc)
    p = rcp.Packing(D0, seed=5, precision=precision)
    dev = torch.device("cuda", 0)
    mu = 0.02
    xt = torch.tensor(x, dtype=torch.float64, device=dev, requires_grad=True)
    kt = torch.tensor(k, dtype=torch.float64, device=dev, requires_grad=True)
    E = ag.energy(xt, kt, p, mu)
    (3.0 * E).backward()
    xr = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    kr = torch.tensor(k, dtype=torch.float64, requires_grad=True)
    Er = _ref_energy(torch, xr, torch.tensor(D0), 1.0, kr, mu)
    (3.0 * Er).backward()
    assert abs(E.item() - Er.item()) <= tol * abs(Er.item())
    g, gr = xt.grad.cpu().numpy(), xr.grad.numpy()
    assert np.linalg.norm(g - gr) <= tol * np.linalg.norm(gr)
    assert abs(kt.grad.item() - kr.grad.item()) <= tol * abs(kr.grad.item())
    p.close()


def test_autograd_central_differences(mods, orc):
    torch, rcp, ag = mods
    D0, x, k = _state(orc, seed=9)
    p = rcp.Packing(D0, seed=9)
    dev = torch.device("cuda", 0)
    mu = 0.01
    xt = torch.tensor(x, dtype=torch.float64, device=dev, requires_grad=True)
    kt = torch.tensor(k, dtype=torch.float64, device=dev, requires_grad=True)
    ag.energy(xt, kt, p, mu).backward()
    g = xt.grad.cpu().numpy()
    h = 1e-7
    rng = np.random.default_rng(0)
    for _ in range(12):
        i, a = int(rng.integers(64)), int(rng.integers(3))
        if g[i, a] == 0.0:
            continue
        xp, xm = x.copy(), x.copy()
        xp[i, a] += h
        xm[i, a] -= h
        with torch.no_grad():
            Ep = ag.energy(torch.tensor(xp, device=dev), torch.tensor(k, dtype=torch.float64, device=dev), p, mu).item()
            Em = ag.energy(torch.tensor(xm, device=dev), torch.tensor(k, dtype=torch.float64, device=dev), p, mu).item()
        assert (Ep - Em) / (2 * h) == pytest.approx(g[i, a], rel=2e-5, abs=1e-6 * np.abs(g).max())
    hk = 1e-7 * k
    with torch.no_grad():
        Ep = ag.energy(torch.tensor(x, device=dev), torch.tensor(k + hk, dtype=torch.float64, device=dev), p, mu).item()
        Em = ag.energy(torch.tensor(x, device=dev), torch.tensor(k - hk, dtype=torch.float64, device=dev), p, mu).item()
    assert (Ep - Em) / (2 * hk) == pytest.approx(kt.grad.item(), rel=1e-5)
    p.close()


def test_autograd_gradcheck(mods, orc):
    torch, rcp, ag = mods
    D0, x, k = _state(orc, n=32, phi=0.15, seed=13)
    p = rcp.Packing(D0, seed=13)
    dev = torch.device("cuda", 0)
    xt = torch.tensor(x, dtype=torch.float64, device=dev, requires_grad=True)
    kt = torch.tensor(k, dtype=torch.float64, device=dev, requires_grad=True)
    assert torch.autograd.gradcheck(lambda a, b: ag.energy(a, b, p, 0.01), (xt, kt), eps=1e-7, atol=1e-5,
                                    rtol=1e-4)
    p.close()
