"""Pins of the oracle's odd multipoles (ell = 1, 3) of cross spectra.

The series tables (phi, f, B) hold for odd ell as for even ell; their truncation
errors fall as eps^(K+1) and theta^(2 beta + 2) (checked here for ell = 1, 3).  An
odd multipole of P is the imaginary part of its shell mean (real densities make it
imaginary); xi_ell is real for every ell.

- One pair of particles on mesh nodes: the exact pairwise estimator is
  P_ell(k) = (2 ell + 1) mean_shell[L_ell(k.n) exp(-i k.Delta)] and
  xi_ell(r_b) = (2 ell + 1) L_ell(Delta.n) / N_b, written out here per mode and per
  lag; this fixes the sign of the odd multipoles and the direction of Delta.
- The FFT estimators equal the pair-by-pair evaluation of their truncated series
  over every (delta_A node, delta_B node) pair, which holds only with the signs
  (-1)^ell that relabelling the first-galaxy terms introduces.
- Odd multipoles change sign under A <-> B and vanish for one tracer; the midpoint
  series at K = 0 is the (two-endpoint) Yamamoto estimator; even multipoles do not
  change when odd ones are requested; the series approach the exact pair sums.
"""
import math

import numpy as np
import pytest

from oracle import estimators as E
from oracle import mesh
from oracle import pairs as P
from oracle.coeffs import bisector_series_ylm, shift_series_legendre, shift_series_ylm
from oracle.special import legendre_L, ylm
from synth import snapped_catalog

N = 16
BOX = 1024.0
REDGES = np.linspace(0.0, 400.0, 7)
LOS_K = [("yamamoto", 0), ("midpoint", 2), ("midpoint", 3), ("bisector", 2), ("bisector", 4)]


def _geo(dist):
    c = round(dist / math.sqrt(3.0) / 64.0) * 64.0
    return np.array([c - BOX / 2] * 3)


def _kedges(nb=6):
    return np.linspace(0.0, math.pi / (BOX / N), nb + 1)


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.fixture(scope="module")
def pair_snapped():
    lo = _geo(1500.0)
    a = snapped_catalog(seed=21, n_gal=70, N=N, box_lo=lo, box_len=BOX, fill=0.4, n_ran=30)
    b = snapped_catalog(seed=22, n_gal=50, N=N, box_lo=lo, box_len=BOX, fill=0.5, n_ran=40)
    b.gal[:, 3] = np.random.default_rng(3).uniform(0.5, 2.0, len(b.gal)).astype(np.float32)
    return lo, a, b


def _kw(lo, b=None, **extra):
    kw = dict(N=N, box_lo=lo, box_len=BOX, assign=2, ell_max=3, odd=True)
    if b is not None:
        kw.update(gal_b=b.gal, ran_b=b.ran, ran_nbar_b=b.ran_nbar)
    kw.update(extra)
    return kw


def test_series_tables_hold_for_odd_ell():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(40, 3))
    d = rng.normal(size=(40, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    for ell in (1, 3):
        for K in (0, 1, 2, 3):
            e = []
            for s in (0.04, 0.02):
                a = d * s * np.linalg.norm(A, axis=1)[:, None]
                y = max(abs(shift_series_ylm(ell, m, a, A, K) - ylm(ell, m, a + A)).max() for m in (-ell, 0, 1))
                mu = np.sum(a * (a + A), 1) / np.linalg.norm(a, axis=1) / np.linalg.norm(a + A, axis=1)
                f = abs(shift_series_legendre(ell, a, A, K) - legendre_L(ell, mu)).max()
                e.append((y, f))
            assert abs(math.log2(e[0][0] / e[1][0]) - (K + 1)) < 0.15, (ell, K, e)
            assert abs(math.log2(e[0][1] / e[1][1]) - (K + 1)) < 0.15, (ell, K, e)
        perp = np.cross(A, d)
        perp /= np.linalg.norm(perp, axis=1)[:, None]
        for bm in (0, 1, 2):
            e = []
            for th in (0.1, 0.05):
                r2 = (A / np.linalg.norm(A, axis=1)[:, None] * math.cos(th) + perp * math.sin(th)) * 2.0
                u = A / np.linalg.norm(A, axis=1)[:, None] + r2 / 2.0
                e.append(max(abs(bisector_series_ylm(ell, m, A, r2, bm) - ylm(ell, m, u)).max() for m in (0, 1, -ell)))
            assert abs(math.log2(e[0] / e[1]) - (2 * bm + 2)) < 0.15, (ell, bm, e)


@pytest.mark.parametrize("los", ["yamamoto", "midpoint", "bisector"])
def test_one_pair_closed_form(los):
    lo = _geo(1500.0)
    h = BOX / N
    ia, ib = np.array([6, 7, 5]), np.array([9, 6, 8])
    xa, xb = lo + ia * h, lo + ib * h

    def cat(x):
        return np.array([[*x, 1.0]], dtype=np.float32)

    kw = dict(N=N, box_lo=lo, box_len=BOX, assign=2, ell_max=3, los=los, norm=0, odd=True, gal_b=cat(xb))
    ke = _kedges()
    got = P.mesh_pk(cat(xa), None, None, kedges=ke, **kw)
    gx = P.mesh_xi(cat(xa), None, None, redges=REDGES, **kw)
    delta = (ib - ia) * h
    if los == "midpoint":
        ns = [xa + xb]
    elif los == "bisector":
        ns = [xa / np.linalg.norm(xa) + xb / np.linalg.norm(xb)]
    else:
        ns = [xb, xa]                            # the mean over the two endpoints
    kv, kmag = mesh.k_vectors(N, BOX), mesh.k_magnitude(N, BOX)
    phase = np.exp(-1j * (kv @ delta))
    kh = kv / np.where(kmag > 0, kmag, 1.0)[..., None]
    for ell in range(4):
        L = np.mean([legendre_L(ell, kh @ (n / np.linalg.norm(n))) for n in ns], axis=0)
        t = (2 * ell + 1) * L * phase
        t = t.real if ell % 2 == 0 else t.imag
        want = [t[(kmag >= a) & (kmag < b) & (kmag > 0)].mean() for a, b in zip(ke[:-1], ke[1:])]
        np.testing.assert_allclose(got["pk"][ell], want, rtol=1e-12, atol=1e-12)
        mu = [np.dot(delta, n) / np.linalg.norm(delta) / np.linalg.norm(n) for n in ns]
        b = np.searchsorted(REDGES, np.linalg.norm(delta), side="right") - 1
        want_x = np.zeros(len(REDGES) - 1)
        want_x[b] = (2 * ell + 1) * np.mean([legendre_L(ell, np.array(v)) for v in mu]) / gx["n_cells"][b]
        np.testing.assert_allclose(gx["xi"][ell], want_x, rtol=1e-12, atol=1e-14)
    assert abs(got["pk"][1]).max() > 0.1 and abs(gx["xi"][1]).max() > 0.0


@pytest.mark.parametrize("los,K", LOS_K)
def test_odd_fft_equals_pairwise_series(pair_snapped, los, K):
    lo, a, b = pair_snapped
    ke = _kedges()
    o3 = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, kedges=ke, **_kw(lo, b))["pk"]
    o2 = P.mesh_pk(a.gal, a.ran, a.ran_nbar, los=los, kedges=ke, series=K, **_kw(lo, b))["pk"]
    x3 = E.xi_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, redges=REDGES, **_kw(lo, b))["xi"]
    x2 = P.mesh_xi(a.gal, a.ran, a.ran_nbar, los=los, redges=REDGES, series=K, **_kw(lo, b))["xi"]
    for ell in range(4):
        assert _rel(o3[ell], o2[ell]) < 1e-11, (ell, "P")
        assert _rel(x3[ell], x2[ell]) < 1e-11, (ell, "xi")


@pytest.mark.parametrize("los,K", LOS_K + [("fixed", 0)])
def test_odd_antisymmetric_and_zero_for_one_tracer(pair_snapped, los, K):
    lo, a, b = pair_snapped
    ke = _kedges()
    ab = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, kedges=ke, **_kw(lo, b))["pk"]
    bb = dict(gal_b=a.gal, ran_b=a.ran, ran_nbar_b=a.ran_nbar)
    ba = E.pk_multipoles(b.gal, b.ran, b.ran_nbar, los=los, order=K, kedges=ke, **_kw(lo), **bb)["pk"]
    aa = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, kedges=ke, **_kw(lo), **bb)["pk"]
    for ell in range(4):
        sign = (-1) ** ell
        assert _rel(sign * ba[ell], ab[ell]) < 1e-11, ell
        if ell % 2:
            assert np.abs(aa[ell]).max() < 1e-11 * np.abs(aa[ell - 1]).max(), ell
    xab = E.xi_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, redges=REDGES, **_kw(lo, b))["xi"]
    xba = E.xi_multipoles(b.gal, b.ran, b.ran_nbar, los=los, order=K, redges=REDGES, **_kw(lo), **bb)["xi"]
    for ell in range(4):
        assert _rel((-1) ** ell * xba[ell], xab[ell]) < 1e-11, ell


def test_midpoint_order0_is_yamamoto_and_even_unchanged(pair_snapped):
    lo, a, b = pair_snapped
    ke = _kedges()
    y = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los="yamamoto", order=0, kedges=ke, **_kw(lo, b))["pk"]
    m = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los="midpoint", order=0, kedges=ke, **_kw(lo, b))["pk"]
    assert _rel(m, y) < 1e-12
    yx = E.xi_multipoles(a.gal, a.ran, a.ran_nbar, los="yamamoto", order=0, redges=REDGES, **_kw(lo, b))["xi"]
    mx = E.xi_multipoles(a.gal, a.ran, a.ran_nbar, los="midpoint", order=0, redges=REDGES, **_kw(lo, b))["xi"]
    assert _rel(mx, yx) < 1e-12
    for los, K in (("midpoint", 3), ("bisector", 2)):
        full = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, kedges=ke, **_kw(lo, b))["pk"]
        even = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los=los, order=K, kedges=ke,
                               **_kw(lo, b, ell_max=2, odd=False))["pk"]
        np.testing.assert_array_equal(full[[0, 2]], even)
    with pytest.raises(ValueError):
        E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los="midpoint_even", order=2, kedges=ke, **_kw(lo, b))
    with pytest.raises(ValueError):
        E.pk_multipoles(a.gal, a.ran, a.ran_nbar, los="midpoint", order=2, kedges=ke, **_kw(lo, b, odd=False))


def test_odd_series_converge_to_exact_pair_sums():
    lo = _geo(3000.0)
    a = snapped_catalog(seed=41, n_gal=80, N=N, box_lo=lo, box_len=BOX, fill=0.4)
    b = snapped_catalog(seed=42, n_gal=60, N=N, box_lo=lo, box_len=BOX, fill=0.4)
    ke = _kedges()
    kw = dict(N=N, box_lo=lo, box_len=BOX, assign=2, ell_max=3, norm=0, gal_b=b.gal, odd=True)
    for los in ("midpoint", "bisector"):
        ex = P.mesh_pk(a.gal, None, None, los=los, kedges=ke, **kw)["pk"][[1, 3]]
        errs = [_rel(E.pk_multipoles(a.gal, None, None, los=los, order=K, kedges=ke, **kw)["pk"][[1, 3]], ex)
                for K in (0, 2, 4)]
        assert errs[0] > 5 * errs[1] > 25 * errs[2], (los, errs)
