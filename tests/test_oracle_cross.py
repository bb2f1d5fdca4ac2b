"""Pins of the oracle's cross spectra of two tracers (delta_A from one catalog
pair, delta_B from another, A = sqrt(A_A A_B)).

- The FFT estimators equal the pair-by-pair evaluation of their truncated series
  over every (node of delta_A, node of delta_B) pair (``oracle.pairs`` with two
  densities), which holds only if both anchorings of the midpoint series are kept
  with weight 1/2 each and the bisector pairs F_A(-k) with F_B(k).
- One tracer given twice gives the auto spectrum.
- Polarisation: the auto spectrum of the union of two catalogs (raw sums, no
  randoms, so that painting is additive) is auto(A) + auto(B) + 2 cross(A, B); this
  fixes the factor 1/2 of the symmetrised estimator against the pinned auto one.
- Even ell are symmetric under A <-> B; the monopole carries no line of sight.
- The FKP-normalised cross spectrum does not change when every weight of one
  tracer (galaxies and randoms) is scaled: A_B scales as the square of the factor,
  which only sqrt(A_A A_B) absorbs.
"""
import math

import numpy as np
import pytest

from oracle import estimators as E
from oracle import pairs as P
from synth import snapped_catalog, uniform_cube_catalog

N = 16
BOX = 1024.0
REDGES = np.linspace(0.0, 400.0, 7)
LOS_K = [("yamamoto", 0), ("midpoint", 2), ("midpoint", 3), ("midpoint_even", 4), ("bisector", 2), ("bisector", 4)]


def _geo(dist):
    c = round(dist / math.sqrt(3.0) / 64.0) * 64.0
    return np.array([c - BOX / 2] * 3)


def _kedges(nb=6):
    return np.linspace(0.0, math.pi / (BOX / N), nb + 1)


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _kw(lo, ell_max=4, assign=2):
    return dict(N=N, box_lo=lo, box_len=BOX, assign=assign, ell_max=ell_max)


def _cross(b):
    return dict(gal_b=b.gal, ran_b=b.ran, ran_nbar_b=b.ran_nbar)


@pytest.fixture(scope="module")
def pair_snapped():
    lo = _geo(1500.0)
    a = snapped_catalog(seed=21, n_gal=70, N=N, box_lo=lo, box_len=BOX, fill=0.4, n_ran=30)
    b = snapped_catalog(seed=22, n_gal=50, N=N, box_lo=lo, box_len=BOX, fill=0.5, n_ran=40)
    b.gal[:, 3] = np.random.default_rng(3).uniform(0.5, 2.0, len(b.gal)).astype(np.float32)
    return lo, a, b


@pytest.fixture(scope="module")
def pair_uniform():
    a = uniform_cube_catalog(seed=31, n_gal=150, n_ran=600, side=500.0, distance=1000.0)
    b = uniform_cube_catalog(seed=32, n_gal=120, n_ran=500, side=500.0, distance=1000.0)
    return a, b


@pytest.mark.parametrize("los,K", LOS_K)
def test_cross_pk_fft_equals_pairwise_series(pair_snapped, los, K):
    lo, a, b = pair_snapped
    ke = _kedges()
    o3 = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, kedges=ke, **_kw(lo), **_cross(b))
    o2 = P.mesh_pk(a.gal, a.ran, a.ran_nbar, los=los, kedges=ke, series=K, **_kw(lo), **_cross(b))
    assert _rel(o3["pk"], o2["pk"]) < 1e-11
    np.testing.assert_array_equal(o3["n_modes"], o2["n_modes"])


@pytest.mark.parametrize("los,K", LOS_K)
def test_cross_xi_fft_equals_pairwise_series(pair_snapped, los, K):
    lo, a, b = pair_snapped
    o3 = E.xi_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, redges=REDGES, **_kw(lo), **_cross(b))
    o2 = P.mesh_xi(a.gal, a.ran, a.ran_nbar, los=los, redges=REDGES, series=K, **_kw(lo), **_cross(b))
    assert _rel(o3["xi"], o2["xi"]) < 1e-11


def test_one_anchor_would_not_match_the_pair_sums(pair_snapped):
    # the midpoint series anchored on the second galaxy only (the auto estimator's form with
    # delta_A conjugated and delta_B weighted) is a different truncation: it must not pass
    lo, a, b = pair_snapped
    ke = _kedges()
    g, ta, tb, A, _ = E._tracers(a.gal, a.ran, a.ran_nbar, b.gal, b.ran, b.ran_nbar, N, lo, BOX, 2, 1, False)
    one = E.g_fields(g, tb.delta, ta.D, 3, 4, tb.tr)
    both = E._cross_g_fields(g, ta, tb, 3, 4)
    diff = max(np.abs(one[k] - both[k]).max() for k in one if k[0] > 0)
    assert diff > 1e-6 * max(np.abs(v).max() for v in both.values())
    o2 = P.mesh_pk(a.gal, a.ran, a.ran_nbar, los="midpoint", kedges=ke, series=3, **_kw(lo), **_cross(b))
    o3 = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los="midpoint", order=3, kedges=ke, **_kw(lo), **_cross(b))
    assert _rel(o3["pk"], o2["pk"]) < 1e-11


@pytest.mark.parametrize("los,K", LOS_K + [("fixed", 0)])
def test_cross_of_one_tracer_is_auto(pair_uniform, los, K):
    a, _ = pair_uniform
    ke = _kedges()
    kw = _kw(a.box_lo)
    kw["box_len"] = a.box_len
    auto = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, kedges=ke, **kw)["pk"]
    cross = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, kedges=ke, **kw, **_cross(a))["pk"]
    assert _rel(cross, auto) < 1e-13
    auto = E.xi_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, redges=REDGES, **kw)["xi"]
    cross = E.xi_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, redges=REDGES, **kw, **_cross(a))["xi"]
    assert _rel(cross, auto) < 1e-13


@pytest.mark.parametrize("los,K", [("yamamoto", 0), ("midpoint", 3), ("midpoint_even", 2), ("bisector", 2)])
def test_polarisation_identity(pair_uniform, los, K):
    a, b = pair_uniform
    union = np.concatenate([a.gal, b.gal])
    kw = dict(N=N, box_lo=a.box_lo, box_len=a.box_len, assign=3, ell_max=4, los=los, order=K, norm=0,
              compensate=True)
    ke = _kedges()
    pa = E.pk_multipoles(a.gal, None, None, kedges=ke, **kw)["pk"]
    pb = E.pk_multipoles(b.gal, None, None, kedges=ke, **kw)["pk"]
    pu = E.pk_multipoles(union, None, None, kedges=ke, **kw)["pk"]
    pc = E.pk_multipoles(a.gal, None, None, kedges=ke, gal_b=b.gal, **kw)["pk"]
    assert _rel(pa + pb + 2.0 * pc, pu) < 1e-11
    xa = E.xi_multipoles(a.gal, None, None, redges=REDGES, **kw)["xi"]
    xb = E.xi_multipoles(b.gal, None, None, redges=REDGES, **kw)["xi"]
    xu = E.xi_multipoles(union, None, None, redges=REDGES, **kw)["xi"]
    xc = E.xi_multipoles(a.gal, None, None, redges=REDGES, gal_b=b.gal, **kw)["xi"]
    assert _rel(xa + xb + 2.0 * xc, xu) < 1e-11


@pytest.mark.parametrize("los,K", LOS_K)
def test_even_multipoles_symmetric_under_swap(pair_uniform, los, K):
    a, b = pair_uniform
    kw = dict(N=N, box_lo=a.box_lo, box_len=a.box_len, assign=2, ell_max=4, los=los, order=K)
    ke = _kedges()
    ab = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, kedges=ke, **kw, **_cross(b))["pk"]
    ba = E.pk_multipoles(b.gal, b.ran, b.ran_nbar, kedges=ke, **kw, **_cross(a))["pk"]
    assert _rel(ba, ab) < 1e-11
    ab = E.xi_multipoles(a.gal, a.ran, a.ran_nbar, redges=REDGES, **kw, **_cross(b))["xi"]
    ba = E.xi_multipoles(b.gal, b.ran, b.ran_nbar, redges=REDGES, **kw, **_cross(a))["xi"]
    assert _rel(ba, ab) < 1e-11


def test_cross_monopole_independent_of_los(pair_uniform):
    a, b = pair_uniform
    kw = dict(N=N, box_lo=a.box_lo, box_len=a.box_len, assign=2, ell_max=2)
    ke = _kedges()
    ref = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los="fixed", order=0, kedges=ke, **kw, **_cross(b))["pk"][0]
    refx = E.xi_multipoles(a.gal, a.ran, a.ran_nbar, los="fixed", order=0, redges=REDGES, **kw, **_cross(b))["xi"][0]
    for los, K in LOS_K:
        p = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, kedges=ke, **kw, **_cross(b))["pk"][0]
        assert _rel(p, ref) < 1e-12, los
        x = E.xi_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, redges=REDGES, **kw, **_cross(b))["xi"][0]
        assert _rel(x, refx) < 1e-12, los


def test_fkp_cross_invariant_under_weight_scale(pair_uniform):
    a, b = pair_uniform
    b3 = dict(gal_b=b.gal.copy(), ran_b=b.ran.copy(), ran_nbar_b=b.ran_nbar)
    b3["gal_b"][:, 3] *= 3.0
    b3["ran_b"][:, 3] *= 3.0
    kw = dict(N=N, box_lo=a.box_lo, box_len=a.box_len, assign=2, ell_max=2, los="midpoint", order=2)
    ke = _kedges()
    one = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, kedges=ke, **kw, **_cross(b))["pk"]
    three = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, kedges=ke, **kw, **b3)["pk"]
    assert _rel(three, one) < 1e-12
    raw1 = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, kedges=ke, norm=0, **kw, **_cross(b))["pk"]
    raw3 = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, kedges=ke, norm=0, **kw, **b3)["pk"]
    assert _rel(raw3, 3.0 * raw1) < 1e-12
    with pytest.raises(ValueError):
        E.xi_multipoles(a.gal, a.ran, a.ran_nbar, redges=REDGES, norm=2, **kw, **_cross(b))


def test_cross_series_converge_to_exact_pair_sums():
    lo = _geo(3000.0)
    a = snapped_catalog(seed=41, n_gal=80, N=N, box_lo=lo, box_len=BOX, fill=0.4)
    b = snapped_catalog(seed=42, n_gal=60, N=N, box_lo=lo, box_len=BOX, fill=0.4)
    ke = _kedges()
    kw = dict(N=N, box_lo=lo, box_len=BOX, assign=2, ell_max=4, norm=0, gal_b=b.gal)
    for los in ("midpoint", "bisector"):
        ex = P.mesh_pk(a.gal, None, None, los=los, kedges=ke, **kw)["pk"][1:]
        errs = [_rel(E.pk_multipoles(a.gal, None, None, los=los, order=K, kedges=ke, **kw)["pk"][1:], ex)
                for K in (0, 2, 4)]
        assert errs[0] > 5 * errs[1] > 25 * errs[2], (los, errs)
