"""Checks of the stored FP64 oracle values at full size against what the geometry and the paper fix.

The golden files (tests/golden/survey512_order4.json, large512_bisector6.json) hold the oracle's
multipoles of the 512^3 workloads.  Without re-running the oracle (an hour of CPU), three things
can be checked independently of it:

* the mode and lag counts and the mean |k|, |r| of every bin, recounted here from the mesh
  geometry alone (k = 2 pi n / L over the full grid, n in the FFT labelling; lags = h j over the
  integer lag cube, j != 0; half-open bins);
* the monopole's independence of the line of sight (L_0 = 1: no wide-angle term at ell = 0,
  Sec. 2.1): the midpoint and bisector P_0 and xi_0 of the same catalog agree to rounding;
* the internal consistency of each file (finite values, shapes, the bins of its generator).
"""
import json
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FILES = {"survey512_order4.json": ("midpoint", "bisector"), "large512_bisector6.json": ("bisector",)}


def _load(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


def _k_bins(N, L, kedges):
    """Modes of the full N^3 grid per half-open |k| bin, and the sum of their |k|."""
    kf = 2.0 * math.pi / L
    n = np.fft.fftfreq(N, 1.0 / N)
    nb = len(kedges) - 1
    cnt = np.zeros(nb, np.int64)
    s = np.zeros(nb)
    n2yz = n[:, None] ** 2 + n[None, :] ** 2
    for ix in range(N):
        k = kf * np.sqrt(n[ix] ** 2 + n2yz).ravel()
        b = np.searchsorted(kedges, k, side="right") - 1
        ok = (b >= 0) & (b < nb)
        cnt += np.bincount(b[ok], minlength=nb)
        s += np.bincount(b[ok], weights=k[ok], minlength=nb)
    return cnt, s


def _r_bins(N, L, redges):
    """Non-zero lags h j of the integer lag cube per half-open |r| bin, and the sum of their |r|."""
    h = L / N
    jm = int(math.ceil(redges[-1] / h)) + 1
    assert 2 * jm + 1 <= N, "the lag cube must fit the mesh (minimal images)"
    j = np.arange(-jm, jm + 1)
    r = h * np.sqrt(j[:, None, None] ** 2 + j[None, :, None] ** 2 + j[None, None, :] ** 2).ravel()
    nb = len(redges) - 1
    b = np.searchsorted(redges, r, side="right") - 1
    ok = (b >= 0) & (b < nb) & (r > 0)
    return np.bincount(b[ok], minlength=nb), np.bincount(b[ok], weights=r[ok], minlength=nb)


@pytest.mark.parametrize("name", sorted(FILES))
def test_bin_geometry_recounted(name):
    g = _load(name)
    N, L = g["n_mesh"], g["catalog"]["box_len"]
    kedges, redges = np.array(g["kedges"]), np.array(g["redges"])
    kc, ks = _k_bins(N, L, kedges)
    rc, rs = _r_bins(N, L, redges)
    for los in FILES[name]:
        r = g["los"][los]
        np.testing.assert_array_equal(r["n_modes"], kc)
        np.testing.assert_array_equal(r["n_cells"], rc)
        # FP64 sums of up to ~6e6 magnitudes in two orders: n eps ~ 7e-10
        np.testing.assert_allclose(r["k_mean"], ks / kc, rtol=1e-9)
        np.testing.assert_allclose(r["r_mean"], rs / rc, rtol=1e-9)
        assert np.all(np.asarray(r["k_mean"]) >= kedges[:-1]) and np.all(np.asarray(r["k_mean"]) < kedges[1:])


def test_monopole_independent_of_line_of_sight():
    g = _load("survey512_order4.json")
    m, b = g["los"]["midpoint"], g["los"]["bisector"]
    for kind in ("pk", "xi"):
        a, c = np.asarray(m[kind][0]), np.asarray(b[kind][0])
        assert np.max(np.abs(a - c)) <= 1e-12 * np.max(np.abs(a)), kind
    # and the higher multipoles do depend on it (the line of sight matters at ell > 0)
    assert np.max(np.abs(np.asarray(m["pk"][1]) - np.asarray(b["pk"][1]))) > 1e-6 * np.max(np.abs(m["pk"][1]))


@pytest.mark.parametrize("name", sorted(FILES))
def test_golden_file_consistent(name):
    g = _load(name)
    nl = g["ell_max"] // 2 + 1
    nk, nr = len(g["kedges"]) - 1, len(g["redges"]) - 1
    for los in FILES[name]:
        r = g["los"][los]
        assert np.asarray(r["pk"]).shape == (nl, nk) and np.asarray(r["xi"]).shape == (nl, nr)
        assert np.all(np.isfinite(r["pk"])) and np.all(np.isfinite(r["xi"]))
        assert np.all(np.asarray(r["pk"])[0] > 0)              # P_0 of a clustered catalog
        assert r["oracle_wall_s"] > 0 and r["units"] > 0
    fp = g["catalog"]
    assert all(len(fp[k]) == 64 for k in ("gal_sha256", "ran_sha256", "ran_nbar_sha256"))
