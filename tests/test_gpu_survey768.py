"""Meshes beyond 512^3 under a memory bound: the survey workload at 768^3.

At 768^3 a mesh slot is 1.82 GB: the resident midpoint field set of order 4 (161 slots, 293 GB)
does not fit the GPU, so the midpoint request runs its g fields in ranges, and the bisector its
fields in blocks.  Checked against the FP64 oracle (tests/golden/survey768_yamamoto.json, from
tests/golden/make_survey768.py):
* the Yamamoto estimator, every multipole, resident;
* the monopole of the midpoint (order 4, g fields in ranges of 24) and of the bisector (order 4,
  fields in blocks of 16): ell = 0 does not depend on the line of sight, so it equals the
  oracle's Yamamoto monopole;
and the bisector in blocks against the resident bisector on the same mesh, every multipole.
FP32 tolerances as in tests/parity.py."""
import hashlib
import json
import os

import numpy as np
import pytest

from parity import check_multipoles, max_rel

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "survey768_yamamoto.json")


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def runs(gold):
    torch = pytest.importorskip("torch")
    import paper_2102_08384_gb300 as pkg
    from synth import lognormal_cap_catalog
    cat = lognormal_cap_catalog(seed=1, n_gal=1_000_000, ran_factor=10.0, half_angle_deg=30.0, r_min=800.0,
                                r_max=1600.0, gen_mesh=256)
    assert hashlib.sha256(np.ascontiguousarray(cat.gal).tobytes()).hexdigest() == gold["catalog"]["gal_sha256"]
    assert hashlib.sha256(np.ascontiguousarray(cat.ran).tobytes()).hexdigest() == gold["catalog"]["ran_sha256"]
    dev = torch.device("cuda", 0)
    g, r, rn = (torch.from_numpy(a).to(dev) for a in (cat.gal, cat.ran, cat.ran_nbar))
    kedges, redges = np.array(gold["kedges"]), np.array(gold["redges"])
    ctx = pkg.Context(0)
    out = {}
    try:
        for label, los, K, chunk in (("yamamoto", "yamamoto", 0, 0), ("midpoint ranges", "midpoint", 4, 24),
                                     ("bisector blocks", "bisector", 4, 16), ("bisector", "bisector", 4, 0)):
            ctx.set_field_chunk(chunk)
            p = pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=768, assign=3, ell_max=4, los=los,
                                order=K, compensate=True, precision=32, norm=1)
            out[label] = ctx.pk_xi_multipoles(g, r, p, kedges, redges, ran_nbar=rn)
            torch.cuda.synchronize(dev)
    finally:
        ctx.set_field_chunk(0)
        ctx.close()
    return out


def test_yamamoto_768_every_multipole(gold, runs):
    got = runs["yamamoto"]
    print("yamamoto 768 P", max_rel(got["pk"], gold["pk"], "pk"), "xi", max_rel(got["xi"], gold["xi"], "xi"))
    check_multipoles(got["pk"], gold["pk"], "pk", label="yamamoto 768 P: ")
    check_multipoles(got["xi"], gold["xi"], "xi", label="yamamoto 768 xi: ")
    np.testing.assert_array_equal(got["n_modes"], gold["n_modes"])
    np.testing.assert_array_equal(got["n_cells"], gold["n_cells"])


@pytest.mark.parametrize("label", ["midpoint ranges", "bisector blocks", "bisector"])
def test_memory_bounded_monopole_768(gold, runs, label):
    got = runs[label]
    want_p, want_x = np.array(gold["pk"])[:1], np.array(gold["xi"])[:1]
    print(label, "P0", max_rel(got["pk"][:1], want_p, "pk"), "xi0", max_rel(got["xi"][:1], want_x, "xi"))
    check_multipoles(got["pk"][:1], want_p, "pk", label=f"{label} 768 P0: ")
    check_multipoles(got["xi"][:1], want_x, "xi", label=f"{label} 768 xi0: ")


def test_bisector_blocks_equal_resident_768(runs):
    a, b = runs["bisector blocks"], runs["bisector"]
    check_multipoles(a["pk"], b["pk"], "pk", label="bisector blocks vs resident P: ")
    check_multipoles(a["xi"], b["xi"], "xi", label="bisector blocks vs resident xi: ")
