"""GPU parity of the LOS-independent extras against the FP64 oracle: the
random-random normalised xi_ell (norm=2), the shot-noise level of P_0 and
interlaced mass assignment."""
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
def ctx(pkg):
    c = pkg.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def cube():
    return uniform_cube_catalog(seed=0, n_gal=4096, n_ran=40960, side=500.0, distance=1000.0)


@pytest.mark.parametrize("los,K", [("yamamoto", 0), ("midpoint", 2), ("bisector", 2), ("midpoint_even", 2)])
def test_rr_normalised_fp64(pkg, ctx, cube, los, K):
    N = 32
    kedges = np.linspace(0.0, math.pi / (cube.box_len / N), 9)
    redges = np.linspace(0.0, 250.0, 11)
    p = pkg.make_params(box_lo=cube.box_lo, box_len=cube.box_len, n_mesh=N, ell_max=4, los=los, order=K,
                        precision=64, assign=3, compensate=True, norm=2)
    got = ctx.pk_xi_multipoles(cube.gal, cube.ran, p, kedges, redges, ran_nbar=cube.ran_nbar)
    kw = dict(N=N, box_lo=cube.box_lo, box_len=cube.box_len, assign=3, ell_max=4, los=los, order=K,
              compensate=True, norm=2)
    want_x = E.xi_multipoles(cube.gal, cube.ran, cube.ran_nbar, redges=redges, **kw)["xi"]
    want_p = E.pk_multipoles(cube.gal, cube.ran, cube.ran_nbar, kedges=kedges, **kw)["pk"]
    check_multipoles(got["xi"], want_x, "xi", 1e-10, 1e-10, f"{los} xi: ")
    check_multipoles(got["pk"], want_p, "pk", 1e-10, 1e-10, f"{los} P: ")


def test_rr_normalised_fp32_cap(pkg, ctx):
    cap = lognormal_cap_catalog(seed=2, n_gal=30000, ran_factor=10.0, gen_mesh=64)
    N = 40
    redges = np.linspace(0.0, 8 * cap.box_len / N, 9)
    p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=N, ell_max=4, los="midpoint", order=4,
                        precision=32, norm=2)
    got = ctx.xi_multipoles(cap.gal, cap.ran, p, redges, ran_nbar=cap.ran_nbar)
    want = E.xi_multipoles(cap.gal, cap.ran, cap.ran_nbar, N=N, box_lo=cap.box_lo, box_len=cap.box_len, assign=2,
                           ell_max=4, los="midpoint", order=4, redges=redges, norm=2)["xi"]
    check_multipoles(got["xi"], want, "xi", label="midpoint K=4 RR: ")


def test_rr_equals_fkp_for_node_filling_randoms(pkg, ctx):
    # randoms on every node, nbar V_cell = alpha_r: RR_0 = A V_cell in every bin
    N, lo, box = 16, np.array([512.0] * 3), 1024.0
    h = box / N
    idx = np.stack(np.meshgrid(*[np.arange(N)] * 3, indexing="ij"), -1).reshape(-1, 3)
    ran = np.concatenate([lo + idx * h, np.ones((len(idx), 1))], 1).astype(np.float32)
    rng = np.random.default_rng(3)
    gi = rng.integers(0, N, size=(300, 3))
    gal = np.concatenate([lo + gi * h, np.ones((300, 1))], 1).astype(np.float32)
    nbar = np.full(len(ran), 300 / box ** 3, np.float32)
    redges = np.linspace(0.0, 400.0, 6)
    out = {}
    for norm in (1, 2):
        p = pkg.make_params(box_lo=lo, box_len=box, n_mesh=N, ell_max=2, los="midpoint", order=2, precision=64,
                            norm=norm)
        out[norm] = ctx.xi_multipoles(gal, ran, p, redges, ran_nbar=nbar)["xi"]
    np.testing.assert_allclose(out[2], out[1], rtol=1e-11, atol=1e-11 * np.abs(out[1]).max())


@pytest.mark.parametrize("norm,with_ran", [(0, False), (0, True), (1, True), (2, True)])
def test_shot_noise(pkg, ctx, cube, norm, with_ran):
    gal = cube.gal.copy()
    gal[:, 3] = np.random.default_rng(1).uniform(0.5, 1.5, len(gal)).astype(np.float32)
    ran, rnb = (cube.ran, cube.ran_nbar) if with_ran else (None, None)
    p = pkg.make_params(box_lo=cube.box_lo, box_len=cube.box_len, n_mesh=32, norm=norm)
    got = ctx.shot_noise(gal, ran, p, ran_nbar=rnb)
    want = E.shot_noise(gal, ran, rnb, norm=norm)
    assert math.isclose(got, want, rel_tol=1e-12), (got, want)


def test_shot_noise_device_and_errors(pkg, ctx, cube):
    torch = pytest.importorskip("torch")
    p = pkg.make_params(box_lo=cube.box_lo, box_len=cube.box_len, n_mesh=32, norm=1)
    host = ctx.shot_noise(cube.gal, cube.ran, p, ran_nbar=cube.ran_nbar)
    dev = ctx.shot_noise(torch.from_numpy(cube.gal).cuda(), torch.from_numpy(cube.ran).cuda(), p,
                         ran_nbar=torch.from_numpy(cube.ran_nbar).cuda())
    assert math.isclose(dev, host, rel_tol=1e-12)
    bad = cube.gal.copy()
    bad[0, 1] = cube.box_lo[1] + 2 * cube.box_len
    with pytest.raises(pkg.BymError) as ei:
        ctx.shot_noise(bad, cube.ran, p, ran_nbar=cube.ran_nbar)
    assert ei.value.code == -2
    with pytest.raises(pkg.BymError) as ei:          # norm 2 without randoms
        ctx.xi_multipoles(cube.gal, None, pkg.make_params(box_lo=cube.box_lo, box_len=cube.box_len, n_mesh=16,
                                                          norm=2), np.linspace(0, 100, 3))
    assert ei.value.code == -1
    with pytest.raises(pkg.BymError) as ei:
        ctx.pk_multipoles(cube.gal, cube.ran, pkg.make_params(box_lo=cube.box_lo, box_len=cube.box_len, n_mesh=16,
                                                              norm=3), np.linspace(0, 0.1, 3), ran_nbar=cube.ran_nbar)
    assert ei.value.code == -1


# ---------------------------------------------------------------- interlacing
@pytest.mark.parametrize("los,K", [("yamamoto", 0), ("midpoint", 2), ("bisector", 2), ("midpoint_even", 2)])
def test_interlaced_fp64(pkg, ctx, cube, los, K):
    N = 32
    kedges = np.linspace(0.0, math.pi / (cube.box_len / N), 9)
    redges = np.linspace(0.0, 250.0, 11)
    p = pkg.make_params(box_lo=cube.box_lo, box_len=cube.box_len, n_mesh=N, ell_max=4, los=los, order=K,
                        precision=64, assign=3, compensate=True, interlace=True)
    got = ctx.pk_xi_multipoles(cube.gal, cube.ran, p, kedges, redges, ran_nbar=cube.ran_nbar)
    kw = dict(N=N, box_lo=cube.box_lo, box_len=cube.box_len, assign=3, ell_max=4, los=los, order=K,
              compensate=True, interlace=True)
    want_p = E.pk_multipoles(cube.gal, cube.ran, cube.ran_nbar, kedges=kedges, **kw)["pk"]
    want_x = E.xi_multipoles(cube.gal, cube.ran, cube.ran_nbar, redges=redges, **kw)["xi"]
    check_multipoles(got["pk"], want_p, "pk", 1e-10, 1e-10, f"{los} interlaced P: ")
    check_multipoles(got["xi"], want_x, "xi", 1e-10, 1e-10, f"{los} interlaced xi: ")


def test_interlaced_fp32_cap_and_errors(pkg, ctx):
    cap = lognormal_cap_catalog(seed=6, n_gal=30000, ran_factor=10.0, gen_mesh=64)
    N = 40
    kedges = np.linspace(0.0, math.pi / (cap.box_len / N), 11)
    redges = np.linspace(0.0, 8 * cap.box_len / N, 9)
    p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=N, ell_max=4, los="midpoint", order=4,
                        precision=32, assign=2, compensate=True, interlace=True)
    got = ctx.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    kw = dict(N=N, box_lo=cap.box_lo, box_len=cap.box_len, assign=2, ell_max=4, los="midpoint", order=4,
              compensate=True, interlace=True)
    check_multipoles(got["pk"], E.pk_multipoles(cap.gal, cap.ran, cap.ran_nbar, kedges=kedges, **kw)["pk"], "pk",
                     label="interlaced FP32 P: ")
    check_multipoles(got["xi"], E.xi_multipoles(cap.gal, cap.ran, cap.ran_nbar, redges=redges, **kw)["xi"], "xi",
                     label="interlaced FP32 xi: ")
    ctx.set_field_chunk(8)
    try:
        with pytest.raises(pkg.BymError) as ei:      # interlacing keeps every field resident
            ctx.pk_multipoles(cap.gal, cap.ran, p, kedges, ran_nbar=cap.ran_nbar)
        assert ei.value.code == -6
    finally:
        ctx.set_field_chunk(0)
