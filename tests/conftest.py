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


def row_term_scale(orc, x, D0, L, kappa, d=3, eps=1.0, band=1e-8):
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
    other, which a_i allows for."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, d)
    D0 = np.asarray(D0, dtype=np.float64)
    n = D0.size
    # the pairs with r < d (1 + 2 band): interaction radius kappa D (1/2 + band)
    rp, col = orc.list_grid(x, D0, L, kappa, band, 0.0, d=d)
    rows = np.repeat(np.arange(n), np.diff(rp))
    dx = x[rows] - x[col]
    dx -= L * np.rint(dx / L)
    r = np.sqrt(np.sum(dx * dx, axis=1))
    size = np.where(D0 > 0.0, kappa * D0, -D0)   # a frozen sphere (D0 = -F) keeps its contact diameter F
    dd = 0.5 * (size[rows] + size[col])
    delta = 1.0 - r / dd
    t = np.where(delta > 0.0, eps * delta / dd, 0.0)
    a = np.where(np.abs(delta) < band, eps * 2.0 * band / dd, 0.0)
    return np.bincount(rows, weights=t, minlength=n), np.bincount(rows, weights=a, minlength=n)


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


def assert_sums_close(E, oE, dk, odk, mu, kappa, D0, rel=1e-6, what=""):
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

    with Se and Sk from the oracle's binary64 values."""
    SD = float(np.sum(np.asarray(D0, dtype=np.float64)))
    muE, muK = mu * kappa * SD, mu * SD
    bE = rel * (abs(oE + muE) + muE)
    bK = rel * (abs(odk + muK) + muK)
    if not (abs(E - oE) <= bE and abs(dk - odk) <= bK):
        raise AssertionError(f"{what} E {E!r} vs {oE!r} (bound {bE:.3e}), dE/dkappa {dk!r} vs {odk!r} "
                             f"(bound {bK:.3e})")
    return max(abs(E - oE) / bE if bE > 0 else 0.0, abs(dk - odk) / bK if bK > 0 else 0.0)


@pytest.fixture(scope="session")
def sums_check():
    return assert_sums_close


@pytest.fixture(scope="session")
def term_scale(orc):
    return lambda *a, **k: row_term_scale(orc, *a, **k)
