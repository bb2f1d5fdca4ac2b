"""Pins of the oracle's FFT estimators (O3) against the pair sums (O1/O2) and
against properties the paper fixes.  Sizes are small so the pair loops finish
in seconds."""
import math

import numpy as np
import pytest

from oracle import estimators as E
from oracle import pairs as P
from synth import snapped_catalog, uniform_cube_catalog

N = 16
BOX = 1024.0


def _geo(dist):
    """Dyadic box whose centre is ~dist from the observer along (1,1,1)/sqrt(3)."""
    c = round(dist / math.sqrt(3.0) / 64.0) * 64.0
    return np.array([c - BOX / 2] * 3)


def _kw(cat, N=N, assign=2, ell_max=4):
    return dict(N=N, box_lo=cat.box_lo, box_len=cat.box_len, assign=assign, ell_max=ell_max)


def _kedges(box_len, N, nb=6):
    return np.linspace(0.0, math.pi / (box_len / N), nb + 1)


REDGES = np.linspace(0.0, 400.0, 7)


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.fixture(scope="module")
def small_uniform():
    return uniform_cube_catalog(seed=7, n_gal=150, n_ran=600, side=500.0, distance=1000.0)


def test_midpoint_order0_equals_yamamoto(small_uniform):
    # Sec. 3.2: at alpha = 0 the midpoint estimator is the Yamamoto estimator
    c = small_uniform
    ke = _kedges(c.box_len, N)
    y = E.pk_multipoles(c.gal, c.ran, c.ran_nbar, los="yamamoto", order=0, kedges=ke, **_kw(c))
    m = E.pk_multipoles(c.gal, c.ran, c.ran_nbar, los="midpoint", order=0, kedges=ke, **_kw(c))
    assert _rel(m["pk"], y["pk"]) < 1e-12
    m = E.pk_multipoles(c.gal, c.ran, c.ran_nbar, los="midpoint_even", order=0, kedges=ke, **_kw(c))
    assert _rel(m["pk"], y["pk"]) < 1e-12
    y = E.xi_multipoles(c.gal, c.ran, c.ran_nbar, los="yamamoto", order=0, redges=REDGES, **_kw(c))
    m = E.xi_multipoles(c.gal, c.ran, c.ran_nbar, los="midpoint", order=0, redges=REDGES, **_kw(c))
    assert _rel(m["xi"], y["xi"]) < 1e-12


def test_monopole_independent_of_los(small_uniform):
    # L_0 = 1: the monopole carries no line of sight (Sec. 7.2, Fig. 3 caption)
    c = small_uniform
    ke = _kedges(c.box_len, N)
    ref = E.pk_multipoles(c.gal, c.ran, c.ran_nbar, los="yamamoto", order=0, kedges=ke, **_kw(c))
    refx = E.xi_multipoles(c.gal, c.ran, c.ran_nbar, los="yamamoto", order=0, redges=REDGES, **_kw(c))
    for los, K in (("midpoint", 2), ("midpoint", 3), ("midpoint_even", 4), ("bisector", 2), ("bisector", 4)):
        p = E.pk_multipoles(c.gal, c.ran, c.ran_nbar, los=los, order=K, kedges=ke, **_kw(c))
        assert _rel(p["pk"][0], ref["pk"][0]) < 1e-12
        x = E.xi_multipoles(c.gal, c.ran, c.ran_nbar, los=los, order=K, redges=REDGES, **_kw(c))
        assert _rel(x["xi"][0], refx["xi"][0]) < 1e-12
    np.testing.assert_array_equal(p["n_modes"], ref["n_modes"])


@pytest.fixture(scope="module")
def snapped():
    return snapped_catalog(seed=11, n_gal=70, N=N, box_lo=_geo(1500.0), box_len=BOX,
                           fill=0.4, n_ran=30)


@pytest.mark.parametrize("los,K", [("yamamoto", 0), ("midpoint", 2), ("midpoint", 3), ("bisector", 2),
                                   ("midpoint_even", 4)])
def test_pk_fft_equals_pairwise_series(snapped, los, K):
    # the convolution / relabelling steps of Secs. 3.2 and 5.2 are exact rewrites of the
    # truncated series summed pair by pair
    c = snapped
    ke = _kedges(c.box_len, N)
    o3 = E.pk_multipoles(c.gal, c.ran, c.ran_nbar, los=los, order=K, kedges=ke, **_kw(c))
    o2 = P.mesh_pk(c.gal, c.ran, c.ran_nbar, los=los, kedges=ke, series=K, **_kw(c))
    assert _rel(o3["pk"], o2["pk"]) < 1e-11
    np.testing.assert_array_equal(o3["n_modes"], o2["n_modes"])


@pytest.mark.parametrize("los,K", [("yamamoto", 0), ("midpoint", 2), ("midpoint", 4), ("bisector", 2),
                                   ("midpoint_even", 4)])
def test_xi_fft_equals_pairwise_series(snapped, los, K):
    c = snapped
    o3 = E.xi_multipoles(c.gal, c.ran, c.ran_nbar, los=los, order=K, redges=REDGES, **_kw(c))
    o2 = P.mesh_xi(c.gal, c.ran, c.ran_nbar, los=los, redges=REDGES, series=K, **_kw(c))
    assert _rel(o3["xi"], o2["xi"]) < 1e-11
    np.testing.assert_array_equal(o3["n_cells"], o2["n_cells"])


@pytest.mark.parametrize("los", ["yamamoto", "midpoint", "bisector"])
def test_particle_pairs_equal_mesh_pairs(snapped, los):
    # O1 == O2 for node-snapped CIC catalogs: each particle deposits on one node
    c = snapped
    o1 = P.particle_xi(c.gal, c.ran, c.ran_nbar, N=N, box_lo=c.box_lo, box_len=c.box_len,
                       ell_max=4, los=los, redges=REDGES)
    o2 = P.mesh_xi(c.gal, c.ran, c.ran_nbar, los=los, redges=REDGES, **_kw(c))
    assert _rel(o1["xi"], o2["xi"]) < 1e-12


def test_series_converge_to_exact_pair_sums():
    # truncation at higher K approaches the exact pairwise estimator (Secs. 3-6)
    c = snapped_catalog(seed=12, n_gal=80, N=N, box_lo=_geo(3000.0), box_len=BOX, fill=0.4)
    ke = _kedges(c.box_len, N)
    for los, Ks in (("midpoint", (0, 2, 4)), ("bisector", (0, 2, 4))):
        ex = P.mesh_pk(c.gal, None, None, los=los, kedges=ke, norm=0, **_kw(c))
        errs = [_rel(E.pk_multipoles(c.gal, None, None, los=los, order=K, kedges=ke, norm=0,
                                     **_kw(c))["pk"][1:], ex["pk"][1:]) for K in Ks]
        assert errs[0] > 5 * errs[1] > 25 * errs[2], (los, errs)
        exx = P.mesh_xi(c.gal, None, None, los=los, redges=REDGES, norm=0, **_kw(c))
        errs = [_rel(E.xi_multipoles(c.gal, None, None, los=los, order=K, redges=REDGES, norm=0,
                                     **_kw(c))["xi"][1:], exx["xi"][1:]) for K in Ks]
        assert errs[0] > 5 * errs[1] > 25 * errs[2], (los, errs)


def test_distant_observer_scaling():
    # Distant-observer limit (Sec. 2.1): every line of sight tends to the fixed one.
    # Moving the same catalog twice as far halves theta: the fixed LOS differs from
    # Yamamoto at O(theta) and Yamamoto from either pairwise LOS at O(theta^2).  The
    # midpoint and bisector directions differ by ((r2 - r1)/(r1 + r2)) phi/2 = O(theta^2)
    # for pairs at unequal distance, so their estimators separate at O(theta^2) too
    # (not O(theta^4) as the Sec. 2.1 footnote states).
    base = snapped_catalog(seed=13, n_gal=60, N=N, box_lo=np.zeros(3), box_len=BOX, fill=0.4)
    d = {}
    for dist in (4000.0, 8000.0):
        lo = _geo(dist)
        gal = base.gal.copy()
        gal[:, :3] += lo.astype(np.float32)
        kw = dict(N=N, box_lo=lo, box_len=BOX, assign=2, ell_max=2, norm=0)
        ke = _kedges(BOX, N)
        y = P.mesh_pk(gal, None, None, los="yamamoto", kedges=ke, **kw)["pk"][1]
        m = P.mesh_pk(gal, None, None, los="midpoint", kedges=ke, **kw)["pk"][1]
        b = P.mesh_pk(gal, None, None, los="bisector", kedges=ke, **kw)["pk"][1]
        f = E.pk_multipoles(gal, None, None, los="fixed", order=0, kedges=ke, **kw)["pk"][1]
        d[dist] = np.array([np.linalg.norm(f - y), np.linalg.norm(m - y),
                            np.linalg.norm(b - y), np.linalg.norm(m - b)])
    r = d[4000.0] / d[8000.0]
    assert 1.7 < r[0] < 2.3, r
    assert np.all((3.4 < r[1:]) & (r[1:] < 4.7)), r
