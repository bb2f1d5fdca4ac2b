"""The large workload: 2e7 lognormal galaxies and 5e7 randoms in a 60-degree cap
over 600-2000 Mpc/h, 512^3 TSC, bisector line of sight at order 6 (the
memory-heaviest field set: 64 transforms), ell <= 4, FP32.

Every multipole at full size is compared bin by bin with the FP64 oracle values in
tests/golden/large512_bisector6.json (written by tests/golden/make_large512.py from
oracle.streamed), with the error stated per multipole; the order-6 bisector monopole is also
checked against the Yamamoto one (ell = 0 does not depend on the line of sight), and every
multipole against the plain oracle on a 1-in-50 subsample of the same catalog at 96^3."""
import hashlib
import json
import math
import os

import numpy as np
import pytest

from parity import check_multipoles, max_rel

pytestmark = pytest.mark.gpu
KEDGES = np.round(np.arange(0.01, 0.2501, 0.01), 10)
REDGES = np.arange(10.0, 190.01, 10.0)


@pytest.fixture(scope="module")
def pkg():
    import paper_2102_08384_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def big():
    from synth import lognormal_cap_catalog
    return lognormal_cap_catalog(seed=2, n_gal=20_000_000, ran_factor=2.5, half_angle_deg=60.0, r_min=600.0,
                                 r_max=2000.0, gen_mesh=256)


def test_order6_bisector_at_512(pkg, big):
    torch = pytest.importorskip("torch")
    g = torch.from_numpy(big.gal).cuda()
    r = torch.from_numpy(big.ran).cuda()
    rn = torch.from_numpy(big.ran_nbar).cuda()
    ctx = pkg.Context(0)
    out = {}
    for los, K in (("yamamoto", 0), ("bisector", 6)):
        p = pkg.make_params(box_lo=big.box_lo, box_len=big.box_len, n_mesh=512, assign=3, ell_max=4, los=los,
                            order=K, compensate=True, precision=32)
        out[los] = ctx.pk_xi_multipoles(g, r, p, KEDGES, REDGES, ran_nbar=rn)
    ctx.close()
    b, y = out["bisector"], out["yamamoto"]
    assert np.all(np.isfinite(b["pk"])) and np.all(np.isfinite(b["xi"]))
    assert np.all(b["n_modes"] > 0) and np.all(b["n_cells"] > 0)
    print("order-6 bisector vs Yamamoto monopole, max rel:", max_rel(b["pk"][:1], y["pk"][:1], "pk"),
          max_rel(b["xi"][:1], y["xi"][:1], "xi"))
    check_multipoles(b["pk"][:1], y["pk"][:1], "pk", label="P0: ")
    check_multipoles(b["xi"][:1], y["xi"][:1], "xi", label="xi0: ")
    # the line of sight matters for ell > 0 at this opening angle
    assert np.abs(b["pk"][1] - y["pk"][1]).max() > 1e-3 * np.abs(y["pk"][1]).max()


def test_per_multipole_error_against_oracle(pkg, big):
    from oracle import estimators as E
    gal, ran, nb = big.gal[::50], big.ran[::50], big.ran_nbar[::50]
    N = 96
    kedges = np.linspace(0.0, math.pi / (big.box_len / N), 9)
    redges = np.linspace(0.0, 8 * big.box_len / N, 9)
    p = pkg.make_params(box_lo=big.box_lo, box_len=big.box_len, n_mesh=N, assign=3, ell_max=4, los="bisector",
                        order=6, compensate=True, precision=32)
    ctx = pkg.Context(0)
    got = ctx.pk_xi_multipoles(gal, ran, p, kedges, redges, ran_nbar=nb)
    ctx.close()
    kw = dict(N=N, box_lo=big.box_lo, box_len=big.box_len, assign=3, ell_max=4, los="bisector", order=6,
              compensate=True)
    want_p = E.pk_multipoles(gal, ran, nb, kedges=kedges, **kw)["pk"]
    want_x = E.xi_multipoles(gal, ran, nb, redges=redges, **kw)["xi"]
    print("FP32 bisector order 6 vs FP64 oracle, max relative error per multipole (ell = 0, 2, 4):",
          "P", max_rel(got["pk"], want_p, "pk"), "xi", max_rel(got["xi"], want_x, "xi"))
    check_multipoles(got["pk"], want_p, "pk", label="P: ")
    check_multipoles(got["xi"], want_x, "xi", label="xi: ")


GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "large512_bisector6.json")


def test_every_multipole_against_oracle_at_512(pkg, big):
    torch = pytest.importorskip("torch")
    with open(GOLD) as fh:
        gold = json.load(fh)
    fp = gold["catalog"]
    for k, a in (("gal_sha256", big.gal), ("ran_sha256", big.ran), ("ran_nbar_sha256", big.ran_nbar)):
        assert hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest() == fp[k], \
            f"the catalog generator changed ({k}): regenerate the golden file"
    kedges, redges = np.array(gold["kedges"]), np.array(gold["redges"])
    g, r, rn = (torch.from_numpy(a).cuda() for a in (big.gal, big.ran, big.ran_nbar))
    ctx = pkg.Context(0)
    try:
        p = pkg.make_params(box_lo=big.box_lo, box_len=big.box_len, n_mesh=gold["n_mesh"], assign=3,
                            ell_max=gold["ell_max"], los="bisector", order=gold["order"], compensate=True,
                            precision=32, norm=1)
        got = ctx.pk_xi_multipoles(g, r, p, kedges, redges, ran_nbar=rn)
    finally:
        ctx.close()
    want = gold["los"]["bisector"]
    print("large workload, FP32 bisector order 6 at 512^3 vs FP64 oracle, max relative error per multipole "
          "(ell = 0, 2, 4): P", max_rel(got["pk"], want["pk"], "pk"), "xi", max_rel(got["xi"], want["xi"], "xi"))
    check_multipoles(got["pk"], want["pk"], "pk", label="P: ")
    check_multipoles(got["xi"], want["xi"], "xi", label="xi: ")
    np.testing.assert_array_equal(got["n_modes"], want["n_modes"])
    np.testing.assert_array_equal(got["n_cells"], want["n_cells"])
    # mean |k| and |r| of a bin: FP64 sums of up to 5.6e6 magnitudes in two different orders, whose
    # rounding is bounded by n eps = 5.6e6 x 1.1e-16 = 6e-10 relative
    np.testing.assert_allclose(got["k_mean"], want["k_mean"], rtol=1e-9)
    np.testing.assert_allclose(got["r_mean"], want["r_mean"], rtol=1e-9)
