import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU runs of the whole protocol")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


def row_term_scale(orc, x, D0, L, kappa, d=3, eps=1.0, band=1e-8, wall_mask=(0, 0)):
    """Scales of the element-wise gradient tolerance of the mixed path, from
    the inputs alone (binary64, no value of the CUDA path):

      s_i = sum over the overlapping partners j of sphere i of the magnitude
            eps delta_ij / d_ij of its term of dE/dx_i (d_ij the mean of the
            two contact diameters: kappa D^0, or F for a frozen sphere);
      a_i = sum over the partners with |delta_ij| < band of eps 2 band / d_ij.

    The mixed path forms each pair term in binary32 from exactly represented
    displacements (a few roundings of 2^-24 each), so every term is within
    about 5e-7 of itself and a row's gradient component within that fraction
    of s_i (plus the compensated sum's own error): s_i is the floor where the
    terms of a row cancel (a sphere pushed evenly from all sides), which no
    bound relative to the small net gradient covers.  The mixed overlap also
    carries an absolute error (56-bit fixed-point positions, about 3e-11 of
    the smallest contact distance at S = 5e5, and the float-float d^2 - r^2):
    a pair within `band` of contact may count on one side and not on the
    other, which a_i allows for.

    wall_mask = (flat-wall mask, container): every wall a sphere meets is one
    more term of its row (eps delta / rad, rad its contact radius), with the
    same band term; bounded axes take the plain difference, not the minimum
    image."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, d)
    D0 = np.asarray(D0, dtype=np.float64)
    n = D0.size
    # the pairs with r < d (1 + 2 band): interaction radius kappa D (1/2 + band)
    mask, container = wall_mask
    caxes = list(range(d)) if container == 1 else ([0, 1] if container == 2 else [])
    periodic = np.array([not ((mask >> a) & 1) and a not in caxes for a in range(d)])
    rp, col = orc.list_grid(x, D0, L, kappa, band, 0.0, d=d, wall_mask=wall_mask)
    rows = np.repeat(np.arange(n), np.diff(rp))
    dx = x[rows] - x[col]
    dx -= np.where(periodic, L * np.rint(dx / L), 0.0)
    r = np.sqrt(np.sum(dx * dx, axis=1))
    size = np.where(D0 > 0.0, kappa * D0, -D0)   # a frozen sphere (D0 = -F) keeps its contact diameter F
    dd = 0.5 * (size[rows] + size[col])
    delta = 1.0 - r / dd
    t = np.where(delta > 0.0, eps * delta / dd, 0.0)
    a = np.where(np.abs(delta) < band, eps * 2.0 * band / dd, 0.0)
    s_row = np.bincount(rows, weights=t, minlength=n)
    a_row = np.bincount(rows, weights=a, minlength=n)
    rad = 0.5 * size
    gaps = [x[:, ax] for ax in range(d) if (mask >> ax) & 1] + [L - x[:, ax] for ax in range(d) if (mask >> ax) & 1]
    if caxes:
        gaps.append(0.5 * L - np.sqrt(np.sum((x[:, caxes] - 0.5 * L) ** 2, axis=1)))
    for h in gaps:
        dw = 1.0 - h / rad
        s_row += np.where(dw > 0.0, eps * dw / rad, 0.0)
        a_row += np.where(np.abs(dw) < band, eps * 2.0 * band / rad, 0.0)
    return s_row, a_row


def kappa_term_magnitude(orc, x, D0, L, kappa, d=3, eps=1.0, wall_mask=(0, 0)):
    """Sum over the overlapping pairs (each once) and wall contacts of
    eps delta (|1 - delta| + delta) / kappa, from the inputs alone (mobile
    spheres; binary64).  A mixed kappa term eps delta (1 - delta) / kappa is
    within a few 2^-24 of eps delta max(|1 - delta|, delta) / kappa: its
    product's roundings, and for a pair the rounding of delta carried into
    1 - delta.  The scale of dE/dkappa's error when its terms take both signs
    (a sphere past a wall, delta > 1, gives a negative term)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, d)
    D0 = np.asarray(D0, dtype=np.float64)
    n = D0.size
    mask, container = wall_mask
    caxes = list(range(d)) if container == 1 else ([0, 1] if container == 2 else [])
    periodic = np.array([not ((mask >> a) & 1) and a not in caxes for a in range(d)])
    rp, col = orc.list_grid(x, D0, L, kappa, 1e-8, 0.0, d=d, wall_mask=wall_mask)
    rows = np.repeat(np.arange(n), np.diff(rp))
    once = col > rows
    i, j = rows[once], col[once]
    dx = x[i] - x[j]
    dx -= np.where(periodic, L * np.rint(dx / L), 0.0)
    r = np.sqrt(np.sum(dx * dx, axis=1))
    mob = D0 > 0.0
    size = np.where(mob, kappa * D0, -D0)
    delta = 1.0 - r / (0.5 * (size[i] + size[j]))
    both = mob[i] | mob[j]
    total = float(np.sum(np.where((delta > 0.0) & both, eps * delta * (np.abs(1.0 - delta) + delta) / kappa, 0.0)))
    rad = 0.5 * size
    gaps = [x[:, a] for a in range(d) if (mask >> a) & 1] + [L - x[:, a] for a in range(d) if (mask >> a) & 1]
    if caxes:
        gaps.append(0.5 * L - np.sqrt(np.sum((x[:, caxes] - 0.5 * L) ** 2, axis=1)))
    for h in gaps:
        dw = 1.0 - h / rad
        total += float(np.sum(np.where((dw > 0.0) & mob, eps * dw * (np.abs(1.0 - dw) + dw) / kappa, 0.0)))
    return total


def assert_grad_close(g, og, scale, rel=1e-5, floor=1e-6, what=""):
    """Element-wise: |g - og| <= rel |og| + floor s_i + a_i, with (s, a) from
    row_term_scale.  Returns the largest ratio of an error to its bound
    (<= 1 passes)."""
    s, a = scale
    og = np.asarray(og)
    g = np.asarray(g).reshape(og.shape)
    bound = rel * np.abs(og) + (floor * np.asarray(s) + np.asarray(a))[:, None]
    err = np.abs(g - og)
    safe = np.where(bound > 0.0, bound, 1.0)
    ratio = np.where(bound > 0.0, err / safe, np.where(err > 0.0, np.inf, 0.0))
    worst = float(ratio.max()) if ratio.size else 0.0
    if worst > 1.0:
        i = int(np.unravel_index(np.argmax(ratio), ratio.shape)[0])
        raise AssertionError(f"{what} gradient row {i}: got {g[i]}, oracle {og[i]}, s_i {s[i]:.3e}, "
                             f"a_i {a[i]:.3e}, error/bound {worst:.3g}")
    return worst


@pytest.fixture(scope="session")
def grad_check():
    return assert_grad_close


def assert_sums_close(E, oE, dk, odk, mu, kappa, D0, rel=1e-6, what="", k_mag=None):
    """E and dE/dkappa of the mixed path against the oracle's.

    Eq. energy makes E the sum of the pair energies less mu kappa sum D_i^0,
    and dE/dkappa the sum of the pairs' kappa terms less mu sum D_i^0: each is
    the difference of two sums that nearly cancel where mu balances the
    overlaps (E can be 1 % of either sum).  The mixed path forms every pair's
    energy and kappa term in binary32 from exactly represented displacements
    (the overlap within a few roundings of 2^-24, its square within ~8e-7 of
    itself), adds them with compensated sums, and takes the mu terms in
    binary64, so its error is bounded relative to the magnitudes of the two
    sums, not to their difference:

      |E - oE|   <= rel (Se + mu kappa sum D0),  Se = oE + mu kappa sum D0,
      |dk - odk| <= rel (|Sk| + mu sum D0),      Sk = odk + mu sum D0,

    with Se and Sk from the oracle's binary64 values.  Where the kappa terms
    take both signs (a sphere past a wall: delta > 1), |Sk| no longer bounds
    their magnitudes; k_mag (kappa_term_magnitude) then stands in for it."""
    SD = float(np.sum(np.asarray(D0, dtype=np.float64)))
    muE, muK = mu * kappa * SD, mu * SD
    bE = rel * (abs(oE + muE) + muE)
    bK = rel * ((abs(odk + muK) if k_mag is None else max(abs(odk + muK), k_mag)) + muK)
    if not (abs(E - oE) <= bE and abs(dk - odk) <= bK):
        raise AssertionError(f"{what} E {E!r} vs {oE!r} (bound {bE:.3e}), dE/dkappa {dk!r} vs {odk!r} "
                             f"(bound {bK:.3e})")
    return max(abs(E - oE) / bE if bE > 0 else 0.0, abs(dk - odk) / bK if bK > 0 else 0.0)


@pytest.fixture(scope="session")
def sums_check():
    return assert_sums_close


@pytest.fixture(scope="session")
def kappa_mag(orc):
    return lambda *a, **k: kappa_term_magnitude(orc, *a, **k)


@pytest.fixture(scope="session")
def term_scale(orc):
    return lambda *a, **k: row_term_scale(orc, *a, **k)
