"""Field sets under a memory bound (bym_set_field_chunk) against the resident
path and against the FP64 oracle.

Midpoint: H_{l m} (eq. FFT-midpoint) and the xi shell sums (eq.
xi-parity-all-estimator) are sums over the g fields, so any partition of the
fields into ranges gives the same estimator up to rounding order.  Bisector:
the bilinear sum of eq. bisector-pk-fft runs over field pairs, so summing the
pairs block pair by block pair gives it too."""
import math

import numpy as np
import pytest

from oracle import estimators as E
from parity import check_multipoles
from synth import lognormal_cap_catalog, uniform_cube_catalog

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2102_08384_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def cap():
    return lognormal_cap_catalog(seed=5, n_gal=30000, ran_factor=10.0, gen_mesh=64)


def _bins(cat, N):
    return np.linspace(0.0, math.pi / (cat.box_len / N), 11), np.linspace(0.0, 8 * cat.box_len / N, 9)


@pytest.mark.parametrize("los,K,N,chunk", [("midpoint", 4, 40, 16), ("midpoint", 4, 32, 45), ("midpoint", 3, 36, 7),
                                           ("midpoint_even", 4, 40, 10), ("midpoint", 2, 32, 1)])
def test_ranges_match_resident_fp32(pkg, cap, los, K, N, chunk):
    kedges, redges = _bins(cap, N)
    p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=N, ell_max=4, los=los, order=K, precision=32)
    ctx = pkg.Context(0)
    whole = ctx.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    ctx.set_field_chunk(chunk)
    parts = ctx.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    again = ctx.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    ctx.close()
    check_multipoles(parts["pk"], whole["pk"], "pk", label=f"{los} K={K} chunk={chunk} P: ")
    check_multipoles(parts["xi"], whole["xi"], "xi", label=f"{los} K={K} chunk={chunk} xi: ")
    np.testing.assert_array_equal(parts["n_modes"], whole["n_modes"])
    # the ranges leave nothing behind for the next request (FP32 painting atomics: equal up to summation order)
    check_multipoles(again["pk"], parts["pk"], "pk", label="repeat P: ")
    check_multipoles(again["xi"], parts["xi"], "xi", label="repeat xi: ")


@pytest.mark.parametrize("los,K", [("midpoint", 2), ("midpoint_even", 4)])
def test_ranges_match_oracle_fp64(pkg, los, K):
    cube = uniform_cube_catalog(seed=0, n_gal=4096, n_ran=40960, side=500.0, distance=1000.0)
    N = 32
    kedges = np.linspace(0.0, math.pi / (cube.box_len / N), 9)
    redges = np.linspace(0.0, 200.0, 9)
    p = pkg.make_params(box_lo=cube.box_lo, box_len=cube.box_len, n_mesh=N, ell_max=4, los=los, order=K,
                        precision=64, assign=3, compensate=True)
    ctx = pkg.Context(0)
    ctx.set_field_chunk(5)
    got = ctx.pk_xi_multipoles(cube.gal, cube.ran, p, kedges, redges, ran_nbar=cube.ran_nbar)
    ctx.close()
    kw = dict(N=N, box_lo=cube.box_lo, box_len=cube.box_len, assign=3, ell_max=4, los=los, order=K, compensate=True)
    want_p = E.pk_multipoles(cube.gal, cube.ran, cube.ran_nbar, kedges=kedges, **kw)
    want_x = E.xi_multipoles(cube.gal, cube.ran, cube.ran_nbar, redges=redges, **kw)
    check_multipoles(got["pk"], want_p["pk"], "pk", 1e-10, 1e-10, f"{los} P: ")
    check_multipoles(got["xi"], want_x["xi"], "xi", 1e-10, 1e-10, f"{los} xi: ")


def test_budget_turns_on_ranges(pkg, cap):
    # a budget below the resident footprint: the request still runs, in ranges
    N = 48
    kedges, redges = _bins(cap, N)
    p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=N, ell_max=4, los="midpoint", order=4,
                        precision=32)
    full = pkg.footprint(p, len(cap.gal), len(cap.ran))
    slot = N * N * (N + 4) * 4
    ctx = pkg.Context(0)
    whole = ctx.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    ctx.close()
    small = pkg.Context(0, hbm_budget_bytes=full - 100 * slot)
    parts = small.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    with pytest.raises(pkg.BymError) as ei:       # not even one field range fits
        tiny = pkg.Context(0, hbm_budget_bytes=10 * slot)
        try:
            tiny.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
        finally:
            tiny.close()
    assert ei.value.code == -3
    small.close()
    check_multipoles(parts["pk"], whole["pk"], "pk")
    check_multipoles(parts["xi"], whole["xi"], "xi")


# ---------------------------------------------------------------- bisector blocks
@pytest.mark.parametrize("K,N,block", [(4, 40, 16), (4, 32, 49), (2, 36, 5), (6, 32, 20), (2, 32, 1)])
def test_bisector_blocks_match_resident_fp32(pkg, cap, K, N, block):
    kedges, redges = _bins(cap, N)
    p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=N, ell_max=4, los="bisector", order=K,
                        precision=32, assign=3, compensate=True)
    ctx = pkg.Context(0)
    whole = ctx.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    pk_only = ctx.pk_multipoles(cap.gal, cap.ran, p, kedges, ran_nbar=cap.ran_nbar)
    ctx.set_field_chunk(block)
    parts = ctx.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    parts_pk = ctx.pk_multipoles(cap.gal, cap.ran, p, kedges, ran_nbar=cap.ran_nbar)
    ctx.close()
    check_multipoles(parts["pk"], whole["pk"], "pk", label=f"bisector K={K} block={block} P: ")
    check_multipoles(parts["xi"], whole["xi"], "xi", label=f"bisector K={K} block={block} xi: ")
    check_multipoles(parts_pk["pk"], pk_only["pk"], "pk", label=f"bisector K={K} block={block} P only: ")


def test_bisector_blocks_match_oracle_fp64(pkg):
    cube = uniform_cube_catalog(seed=0, n_gal=4096, n_ran=40960, side=500.0, distance=1000.0)
    N = 32
    kedges = np.linspace(0.0, math.pi / (cube.box_len / N), 9)
    redges = np.linspace(0.0, 200.0, 9)
    p = pkg.make_params(box_lo=cube.box_lo, box_len=cube.box_len, n_mesh=N, ell_max=4, los="bisector", order=2,
                        precision=64, assign=3, compensate=True)
    ctx = pkg.Context(0)
    ctx.set_field_chunk(7)       # 36 fields: blocks of 7, 7, 7, 7, 7, 1
    got = ctx.pk_xi_multipoles(cube.gal, cube.ran, p, kedges, redges, ran_nbar=cube.ran_nbar)
    ctx.close()
    kw = dict(N=N, box_lo=cube.box_lo, box_len=cube.box_len, assign=3, ell_max=4, los="bisector", order=2,
              compensate=True)
    want_p = E.pk_multipoles(cube.gal, cube.ran, cube.ran_nbar, kedges=kedges, **kw)
    want_x = E.xi_multipoles(cube.gal, cube.ran, cube.ran_nbar, redges=redges, **kw)
    check_multipoles(got["pk"], want_p["pk"], "pk", 1e-10, 1e-10, "bisector blocks P: ")
    check_multipoles(got["xi"], want_x["xi"], "xi", 1e-10, 1e-10, "bisector blocks xi: ")


def test_budget_turns_on_bisector_blocks(pkg, cap):
    N = 40
    kedges, redges = _bins(cap, N)
    p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=N, ell_max=4, los="bisector", order=4,
                        precision=32)
    full = pkg.footprint(p, len(cap.gal), len(cap.ran))      # 1 + 49 + 15 slots
    slot = N * N * (N + 4) * 4
    ctx = pkg.Context(0)
    whole = ctx.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    ctx.close()
    small = pkg.Context(0, hbm_budget_bytes=full - 25 * slot)  # room for blocks of 12 fields
    parts = small.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    small.close()
    check_multipoles(parts["pk"], whole["pk"], "pk")
    check_multipoles(parts["xi"], whole["xi"], "xi")
