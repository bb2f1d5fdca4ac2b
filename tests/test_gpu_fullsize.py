"""Full-size checks in the benchmark's configuration (512^3 TSC, compensated,
survey-like catalog of 1e6 galaxies + 1e7 randoms, order 4, ell <= 4, the
paper's k and r bins).  The oracle cannot run the order-4 estimators at this
size in seconds, so the checks are (a) what the oracle computes exactly at full
size -- the monopole P_0 and xi_0 (L_0 = 1 makes them LOS-independent) and the
mode / lag-cell counts -- and (b) properties that hold at any size: the
monopole is the same for every LOS and order, and the midpoint estimator at
order 0 is the Yamamoto estimator."""
import numpy as np
import pytest

from parity import check_multipoles

pytestmark = pytest.mark.gpu

N = 512
KEDGES = np.round(np.arange(0.01, 0.2501, 0.01), 10)
REDGES = np.arange(10.0, 190.01, 10.0)


@pytest.fixture(scope="module")
def runs():
    import paper_2102_08384_gb300 as pkg
    from synth import lognormal_cap_catalog
    cat = lognormal_cap_catalog(seed=1, n_gal=1_000_000, ran_factor=10.0, gen_mesh=256)
    ctx = pkg.Context(0)
    out = {}
    for los, K in (("yamamoto", 0), ("midpoint", 0), ("midpoint", 4), ("bisector", 4)):
        p = pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=N, assign=3, ell_max=4, los=los,
                            order=K, compensate=True, precision=32)
        out[(los, K)] = ctx.pk_xi_multipoles(cat.gal, cat.ran, p, KEDGES, REDGES, ran_nbar=cat.ran_nbar)
    ctx.close()
    return cat, out


def test_monopole_same_for_every_los(runs):
    _, out = runs
    ref = out[("yamamoto", 0)]
    for key, r in out.items():
        check_multipoles(r["pk"][:1], ref["pk"][:1], "pk", label=f"{key} P0: ")
        check_multipoles(r["xi"][:1], ref["xi"][:1], "xi", label=f"{key} xi0: ")


def test_midpoint_order0_is_yamamoto(runs):
    _, out = runs
    check_multipoles(out[("midpoint", 0)]["pk"], out[("yamamoto", 0)]["pk"], "pk")
    check_multipoles(out[("midpoint", 0)]["xi"], out[("yamamoto", 0)]["xi"], "xi")


def test_monopole_and_counts_against_oracle(runs):
    from oracle import estimators as E
    cat, out = runs
    kw = dict(N=N, box_lo=cat.box_lo, box_len=cat.box_len, assign=3, ell_max=0, los="yamamoto", order=0,
              compensate=True)
    want_p = E.pk_multipoles(cat.gal, cat.ran, cat.ran_nbar, kedges=KEDGES, **kw)
    want_x = E.xi_multipoles(cat.gal, cat.ran, cat.ran_nbar, redges=REDGES, **kw)
    got = out[("bisector", 4)]
    np.testing.assert_array_equal(got["n_modes"], want_p["n_modes"])
    np.testing.assert_array_equal(got["n_cells"], want_x["n_cells"])
    np.testing.assert_allclose(got["k_mean"], want_p["k_mean"], rtol=1e-12)
    check_multipoles(got["pk"][:1], want_p["pk"], "pk", label="P0 vs oracle: ")
    check_multipoles(got["xi"][:1], want_x["xi"], "xi", label="xi0 vs oracle: ")
