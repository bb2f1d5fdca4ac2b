"""The streamed loop order (oracle.streamed) against the plain estimators (oracle.estimators).

Both evaluate the same boxed estimators; the streamed order sums the midpoint transforms
product by product and the bisector bilinear form pair by pair, and evaluates only the binned
modes and lags.  They must agree to rounding (1e-12 relative to each multipole's largest
value), with identical mode and lag counts and mean magnitudes."""
import math

import numpy as np
import pytest

from oracle import estimators as E
from oracle import streamed as S
from synth import lognormal_cap_catalog


@pytest.fixture(scope="module")
def cap():
    return lognormal_cap_catalog(seed=11, n_gal=3000, ran_factor=5.0, gen_mesh=32)


def _close(a, b, tol=1e-12):
    a, b = np.asarray(a), np.asarray(b)
    for l in range(b.shape[0]):
        scale = np.max(np.abs(b[l]))
        assert np.max(np.abs(a[l] - b[l])) <= tol * scale, (l, np.max(np.abs(a[l] - b[l])) / scale)


@pytest.mark.parametrize("los,K,N,assign,comp", [("yamamoto", 0, 20, 2, False), ("yamamoto", 0, 16, 3, True),
                                                 ("midpoint", 2, 20, 2, False), ("midpoint", 4, 16, 3, True),
                                                 ("bisector", 2, 20, 2, False), ("bisector", 4, 16, 3, True)])
def test_streamed_equals_plain(cap, los, K, N, assign, comp):
    h = cap.box_len / N
    kedges = np.linspace(0.0, 0.8 * math.pi / h, 7)
    redges = np.linspace(0.0, 5 * h, 5)
    kw = dict(N=N, box_lo=cap.box_lo, box_len=cap.box_len, assign=assign, ell_max=4, los=los, order=K,
              compensate=comp)
    want_p = E.pk_multipoles(cap.gal, cap.ran, cap.ran_nbar, kedges=kedges, **kw)
    want_x = E.xi_multipoles(cap.gal, cap.ran, cap.ran_nbar, redges=redges, **kw)
    got = S.pk_xi_multipoles(cap.gal, cap.ran, cap.ran_nbar, kedges=kedges, redges=redges, block=3, **kw)
    _close(got["pk"], want_p["pk"])
    _close(got["xi"], want_x["xi"])
    np.testing.assert_array_equal(got["n_modes"], want_p["n_modes"])
    np.testing.assert_array_equal(got["n_cells"], want_x["n_cells"])
    np.testing.assert_array_equal(got["k_mean"], want_p["k_mean"])
    np.testing.assert_array_equal(got["r_mean"], want_x["r_mean"])


def test_streamed_one_statistic_and_stop(cap):
    N = 16
    h = cap.box_len / N
    kedges = np.linspace(0.0, math.pi / h, 5)
    kw = dict(N=N, box_lo=cap.box_lo, box_len=cap.box_len, assign=2, ell_max=2, los="bisector", order=2)
    only_p = S.pk_xi_multipoles(cap.gal, cap.ran, cap.ran_nbar, kedges=kedges, **kw)
    assert "xi" not in only_p
    _close(only_p["pk"], E.pk_multipoles(cap.gal, cap.ran, cap.ran_nbar, kedges=kedges, **kw)["pk"])
    seen = []

    def stop_after_two(kind, done, total):
        if kind == "unit":
            seen.append((done, total))
            if done == 2:
                raise S.Stop
    with pytest.raises(S.Stop):
        S.pk_xi_multipoles(cap.gal, cap.ran, cap.ran_nbar, kedges=kedges, progress=stop_after_two, **kw)
    assert seen == [(1, S.work_units("bisector", 2, 2)), (2, S.work_units("bisector", 2, 2))]
    with pytest.raises(ValueError):
        S.pk_xi_multipoles(cap.gal, cap.ran, cap.ran_nbar, kedges=kedges, **dict(kw, los="midpoint_even"))
