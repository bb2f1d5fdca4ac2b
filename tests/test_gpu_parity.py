"""GPU parity: the library (through the C ABI) against the FP64 oracle, element by element.

Sizes are chosen so the oracle finishes in seconds while the meshes still span
many thread blocks and ragged warps (N = 40, 48 give half-spectrum rows of 21
and 25 modes)."""
import math

import numpy as np
import pytest

from oracle import estimators as E
from parity import check_multipoles, max_rel
from synth import lognormal_cap_catalog, snapped_catalog, uniform_cube_catalog

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2102_08384_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0)
    yield c
    c.close()


def _kedges(box_len, N, nb=16):
    return np.linspace(0.0, math.pi / (box_len / N), nb + 1)


def _oracle(cat, N, ell_max, los, K, kedges, redges, assign=2, compensate=False, norm=1, ran=True):
    kw = dict(N=N, box_lo=cat.box_lo, box_len=cat.box_len, assign=assign, ell_max=ell_max, los=los, order=K,
              compensate=compensate, norm=norm)
    r, rn = (cat.ran, cat.ran_nbar) if ran else (None, None)
    out = {}
    if kedges is not None:
        out["pk"] = E.pk_multipoles(cat.gal, r, rn, kedges=kedges, **kw)
    if redges is not None:
        out["xi"] = E.xi_multipoles(cat.gal, r, rn, redges=redges, **kw)
    return out


def _run(pkg, ctx, cat, N, ell_max, los, K, kedges, redges, precision, assign=2, compensate=False, norm=1,
         ran=True):
    p = pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=N, assign=assign, ell_max=ell_max,
                        los=los, order=K, compensate=compensate, precision=precision, norm=norm)
    r, rn = (cat.ran, cat.ran_nbar) if ran else (None, None)
    return ctx.pk_xi_multipoles(cat.gal, r, p, kedges, redges, ran_nbar=rn)


# ---------------------------------------------------------------- FP64, the small uniform-cube workload
@pytest.fixture(scope="module")
def cube():
    # 4096 galaxies + 40960 randoms in a 500 Mpc/h cube 1000 Mpc/h away, 1000 Mpc/h box (seed 0)
    return uniform_cube_catalog(seed=0, n_gal=4096, n_ran=40960, side=500.0, distance=1000.0)


@pytest.mark.parametrize("los,K", [("yamamoto", 0), ("midpoint", 2), ("midpoint", 0), ("bisector", 2)])
def test_fp64_uniform_cube_64(pkg, ctx, cube, los, K):
    N = 64
    kedges = _kedges(cube.box_len, N)
    redges = np.linspace(0.0, 100.0, 17)
    got = _run(pkg, ctx, cube, N, 2, los, K, kedges, redges, 64)
    want = _oracle(cube, N, 2, los, K, kedges, redges)
    check_multipoles(got["pk"], want["pk"]["pk"], "pk", 1e-10, 1e-10, f"{los} P: ")
    check_multipoles(got["xi"], want["xi"]["xi"], "xi", 1e-10, 1e-10, f"{los} xi: ")
    np.testing.assert_array_equal(got["n_modes"], want["pk"]["n_modes"])
    np.testing.assert_array_equal(got["n_cells"], want["xi"]["n_cells"])
    np.testing.assert_allclose(got["k_mean"], want["pk"]["k_mean"], rtol=1e-12)
    np.testing.assert_allclose(got["r_mean"], want["xi"]["r_mean"], rtol=1e-12)


# ---------------------------------------------------------------- FP32, survey-like catalogs
@pytest.fixture(scope="module")
def cap():
    return lognormal_cap_catalog(seed=1, n_gal=30000, ran_factor=10.0, gen_mesh=64)


@pytest.mark.parametrize("los,K,N", [
    ("yamamoto", 0, 48), ("midpoint", 4, 48), ("bisector", 4, 48),
    ("midpoint", 2, 40), ("bisector", 2, 40), ("midpoint", 3, 32), ("bisector", 6, 32),
    ("midpoint_even", 4, 40), ("midpoint_even", 2, 32),
])
def test_fp32_cap(pkg, ctx, cap, los, K, N):
    kedges = _kedges(cap.box_len, N, 12)
    redges = np.linspace(0.0, 8 * cap.box_len / N, 9)
    got = _run(pkg, ctx, cap, N, 4, los, K, kedges, redges, 32)
    want = _oracle(cap, N, 4, los, K, kedges, redges)
    print(los, K, N, "P rel err", max_rel(got["pk"], want["pk"]["pk"], "pk"),
          "xi rel err", max_rel(got["xi"], want["xi"]["xi"], "xi"))
    check_multipoles(got["pk"], want["pk"]["pk"], "pk", label=f"{los} K={K} N={N} P: ")
    check_multipoles(got["xi"], want["xi"]["xi"], "xi", label=f"{los} K={K} N={N} xi: ")
    np.testing.assert_array_equal(got["n_modes"], want["pk"]["n_modes"])


@pytest.mark.parametrize("los,K", [("midpoint", 4), ("bisector", 4)])
def test_fp32_repeatable(pkg, ctx, cap, los, K):
    # deterministic painting (fixed-point sums per tile) and shell sums (per-warp accumulators,
    # block totals added in block order): repeated FP32 requests agree bit for bit
    N = 48
    kedges = _kedges(cap.box_len, N, 12)
    redges = np.linspace(0.0, 8 * cap.box_len / N, 9)
    runs = [_run(pkg, ctx, cap, N, 4, los, K, kedges, redges, 32, assign=3, compensate=True) for _ in range(3)]
    for r in runs[1:]:
        for key in ("pk", "xi", "k_mean", "r_mean", "n_modes", "n_cells"):
            np.testing.assert_array_equal(r[key], runs[0][key], err_msg=key)


@pytest.mark.parametrize("los,K", [("yamamoto", 0), ("midpoint", 2), ("bisector", 4), ("midpoint_even", 4)])
def test_fp64_tsc_compensated(pkg, ctx, cap, los, K):
    N = 32
    kedges = _kedges(cap.box_len, N, 10)
    redges = np.linspace(0.0, 10 * cap.box_len / N, 6)
    got = _run(pkg, ctx, cap, N, 4, los, K, kedges, redges, 64, assign=3, compensate=True)
    want = _oracle(cap, N, 4, los, K, kedges, redges, assign=3, compensate=True)
    check_multipoles(got["pk"], want["pk"]["pk"], "pk", 1e-10, 1e-10, f"{los} P: ")
    check_multipoles(got["xi"], want["xi"]["xi"], "xi", 1e-10, 1e-10, f"{los} xi: ")


def test_xi_bins_beyond_half_box(pkg, ctx, cube):
    # the lag cube covers the whole periodic mesh when r_max exceeds half the box
    N = 32
    redges = np.linspace(0.0, 0.8 * cube.box_len, 9)
    p = pkg.make_params(box_lo=cube.box_lo, box_len=cube.box_len, n_mesh=N, ell_max=2, los="yamamoto",
                        precision=64)
    got = ctx.xi_multipoles(cube.gal, cube.ran, p, redges, ran_nbar=cube.ran_nbar)
    want = _oracle(cube, N, 2, "yamamoto", 0, None, redges)["xi"]
    check_multipoles(got["xi"], want["xi"], "xi", 1e-10, 1e-10)
    np.testing.assert_array_equal(got["n_cells"], want["n_cells"])


@pytest.mark.parametrize("ell_max", [0, 6])
def test_ell_max_range(pkg, ctx, cube, ell_max):
    N = 24
    kedges = _kedges(cube.box_len, N, 6)
    redges = np.linspace(0.0, 300.0, 5)
    got = _run(pkg, ctx, cube, N, ell_max, "yamamoto", 0, kedges, redges, 64)
    want = _oracle(cube, N, ell_max, "yamamoto", 0, kedges, redges)
    check_multipoles(got["pk"], want["pk"]["pk"], "pk", 1e-10, 1e-10)
    check_multipoles(got["xi"], want["xi"]["xi"], "xi", 1e-10, 1e-10)


# ---------------------------------------------------------------- edge cases
def test_no_randoms_raw(pkg, ctx):
    c = snapped_catalog(seed=3, n_gal=200, N=32, box_lo=np.array([512.0] * 3), box_len=1024.0, fill=0.4)
    N = 32
    kedges = _kedges(c.box_len, N, 8)
    redges = np.linspace(0.0, 300.0, 6)
    for los, K in (("yamamoto", 0), ("midpoint", 3), ("bisector", 2), ("midpoint_even", 4)):
        got = _run(pkg, ctx, c, N, 4, los, K, kedges, redges, 64, norm=0, ran=False)
        want = _oracle(c, N, 4, los, K, kedges, redges, norm=0, ran=False)
        check_multipoles(got["pk"], want["pk"]["pk"], "pk", 1e-10, 1e-10, f"{los}: ")
        check_multipoles(got["xi"], want["xi"]["xi"], "xi", 1e-10, 1e-10, f"{los}: ")


def test_empty_catalog_gives_zeros(pkg, ctx):
    N = 16
    p = pkg.make_params(box_lo=(100, 100, 100), box_len=400.0, n_mesh=N, ell_max=4, los="bisector", order=2,
                        norm=0)
    got = ctx.pk_xi_multipoles(np.zeros((0, 4), np.float32), None, p, _kedges(400.0, N, 4),
                               np.linspace(0, 100, 4))
    assert np.all(got["pk"] == 0) and np.all(got["xi"] == 0)
    assert got["n_modes"].sum() > 0


def test_out_of_box_is_an_error(pkg, ctx, cube):
    gal = cube.gal.copy()
    gal[7, 0] = cube.box_lo[0] - 1.0
    p = pkg.make_params(box_lo=cube.box_lo, box_len=cube.box_len, n_mesh=16, ell_max=2)
    with pytest.raises(pkg.BymError) as ei:
        ctx.pk_multipoles(gal, cube.ran, p, _kedges(cube.box_len, 16, 4), ran_nbar=cube.ran_nbar)
    assert ei.value.code == -2
    gal[7, 0] = np.nan
    with pytest.raises(pkg.BymError) as ei:
        ctx.pk_multipoles(gal, cube.ran, p, _kedges(cube.box_len, 16, 4), ran_nbar=cube.ran_nbar)
    assert ei.value.code == -2


def test_bad_arguments(pkg, ctx, cube):
    ke = _kedges(cube.box_len, 16, 4)
    for kw, code in ((dict(ell_max=3), -6), (dict(order=13, los="midpoint"), -6), (dict(n_mesh=15), -6),
                     (dict(order=6, los="midpoint_even"), -6),
                     (dict(assign=4), -1), (dict(precision=16), -1)):
        args = dict(box_lo=cube.box_lo, box_len=cube.box_len, n_mesh=16, ell_max=2)
        args.update(kw)
        with pytest.raises(pkg.BymError) as ei:
            ctx.pk_multipoles(cube.gal, cube.ran, pkg.make_params(**args), ke, ran_nbar=cube.ran_nbar)
        assert ei.value.code == code, kw
    p = pkg.make_params(box_lo=cube.box_lo, box_len=cube.box_len, n_mesh=16, ell_max=2)
    with pytest.raises(pkg.BymError):
        ctx.pk_multipoles(cube.gal, cube.ran, p, ke[::-1].copy(), ran_nbar=cube.ran_nbar)
    with pytest.raises(pkg.BymError):       # norm = 1 without nbar
        ctx.pk_multipoles(cube.gal, cube.ran, p, ke)


def test_device_pointers_match_host(pkg, ctx, cap):
    torch = pytest.importorskip("torch")
    N = 32
    kedges = _kedges(cap.box_len, N, 8)
    redges = np.linspace(0.0, 6 * cap.box_len / N, 5)
    p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=N, ell_max=4, los="bisector", order=2,
                        precision=64)
    host = ctx.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    g = torch.from_numpy(cap.gal).cuda()
    r = torch.from_numpy(cap.ran).cuda()
    rn = torch.from_numpy(cap.ran_nbar).cuda()
    dev = ctx.pk_xi_multipoles(g, r, p, kedges, redges, ran_nbar=rn)
    np.testing.assert_allclose(dev["pk"], host["pk"], rtol=1e-11, atol=1e-11 * np.abs(host["pk"]).max())
    np.testing.assert_allclose(dev["xi"], host["xi"], rtol=1e-11, atol=1e-11 * np.abs(host["xi"]).max())
