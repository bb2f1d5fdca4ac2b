"""The 512^3 survey workload against the FP64 oracle, every multipole.

The benchmark's configuration -- the seed-1 lognormal cap (1e6 galaxies, 1e7 randoms), TSC
with compensation on a 512^3 mesh, order 4, ell = 0, 2, 4, P_ell on 0.01-0.25 h/Mpc and xi_ell
on 10-190 Mpc/h, midpoint and bisector lines of sight -- through the C ABI in FP32, compared
bin by bin with the FP64 oracle values in tests/golden/survey512_order4.json (written by
tests/golden/make_survey512.py from oracle.streamed).  Every FFT path a 512^3 FP32 request can
take is checked: the default (the library's z, y and x passes, the x pass running the midpoint
convolution's forward transform, product and inverse in one sweep), cuFFT 3D transforms, the
library's cluster plane pass, cuFFT plane transforms with the library's x pass, and cuFFT planes
plus cuFFT transforms along x; and the memory-bounded forms: midpoint g fields in ranges of 45
and bisector fields in blocks of 16.

Tolerances: 1e-5 relative on P_0 and xi_0; 1e-4 relative on ell = 2, 4 where
|X_ell| exceeds 1 % of the monopole scale, 1e-4 of that scale elsewhere."""
import hashlib
import json
import os

import numpy as np
import pytest

from parity import check_multipoles, max_rel

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "survey512_order4.json")


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def pkg():
    import paper_2102_08384_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def survey(gold):
    torch = pytest.importorskip("torch")
    from synth import lognormal_cap_catalog
    cat = lognormal_cap_catalog(seed=1, n_gal=1_000_000, ran_factor=10.0, half_angle_deg=30.0, r_min=800.0,
                                r_max=1600.0, gen_mesh=256)
    fp = gold["catalog"]
    got = {"gal_sha256": hashlib.sha256(np.ascontiguousarray(cat.gal).tobytes()).hexdigest(),
           "ran_sha256": hashlib.sha256(np.ascontiguousarray(cat.ran).tobytes()).hexdigest(),
           "ran_nbar_sha256": hashlib.sha256(np.ascontiguousarray(cat.ran_nbar).tobytes()).hexdigest()}
    for k, v in got.items():
        assert v == fp[k], f"the catalog generator changed ({k}): regenerate the golden file"
    dev = torch.device("cuda", 0)
    return cat, tuple(torch.from_numpy(a).to(dev) for a in (cat.gal, cat.ran, cat.ran_nbar))


CASES = [("midpoint", None, 0), ("bisector", None, 0), ("midpoint", 0, 0), ("bisector", 0, 0),
         ("midpoint", 1, 0), ("bisector", 1, 0), ("midpoint", 4, 0), ("bisector", 4, 0),
         ("midpoint", 5, 0), ("bisector", 5, 0), ("midpoint", None, 45), ("bisector", None, 16)]


@pytest.mark.parametrize("los,backend,chunk", CASES)
def test_survey512_every_multipole(pkg, gold, survey, los, backend, chunk):
    cat, (g, r, rn) = survey
    kedges, redges = np.array(gold["kedges"]), np.array(gold["redges"])
    ctx = pkg.Context(0)
    try:
        if backend is not None:
            ctx.set_fft_backend(backend)
        ctx.set_field_chunk(chunk)
        p = pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=gold["n_mesh"], assign=3,
                            ell_max=gold["ell_max"], los=los, order=gold["order"], compensate=True, precision=32,
                            norm=1)
        got = ctx.pk_xi_multipoles(g, r, p, kedges, redges, ran_nbar=rn)
    finally:
        ctx.close()
    want = gold["los"][los]
    label = f"{los} backend={backend} chunk={chunk}"
    print(label, "P max rel err per ell", max_rel(got["pk"], want["pk"], "pk"),
          "xi", max_rel(got["xi"], want["xi"], "xi"))
    check_multipoles(got["pk"], want["pk"], "pk", label=label + " P: ")
    check_multipoles(got["xi"], want["xi"], "xi", label=label + " xi: ")
    np.testing.assert_array_equal(got["n_modes"], want["n_modes"])
    np.testing.assert_array_equal(got["n_cells"], want["n_cells"])
    np.testing.assert_allclose(got["k_mean"], want["k_mean"], rtol=1e-12)
    np.testing.assert_allclose(got["r_mean"], want["r_mean"], rtol=1e-12)
