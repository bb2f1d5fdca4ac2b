"""GPU parity of the cross spectra of two tracers (bym_pk_xi_cross) against the
FP64 oracle, and properties that hold at any size: one tracer twice gives the
auto spectrum, the polarisation identity auto(A + B) = auto(A) + auto(B) +
2 cross(A, B), and the line-of-sight-free monopole."""
import math

import numpy as np
import pytest

from oracle import estimators as E
from parity import check_multipoles
from synth import lognormal_cap_catalog, uniform_cube_catalog

pytestmark = pytest.mark.gpu
LOS_K = [("yamamoto", 0), ("midpoint", 2), ("midpoint", 3), ("midpoint_even", 2), ("bisector", 2), ("bisector", 4)]


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
def cubes():
    a = uniform_cube_catalog(seed=0, n_gal=4096, n_ran=40960, side=500.0, distance=1000.0)
    b = uniform_cube_catalog(seed=1, n_gal=3000, n_ran=30000, side=500.0, distance=1000.0)
    b.gal[:, 3] = np.random.default_rng(4).uniform(0.5, 1.5, len(b.gal)).astype(np.float32)
    return a, b


def _oracle(a, b, kedges, redges, **kw):
    x = dict(gal_b=b.gal, ran_b=b.ran, ran_nbar_b=b.ran_nbar)
    out = {}
    if kedges is not None:
        out["pk"] = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, kedges=kedges, **kw, **x)["pk"]
    if redges is not None:
        out["xi"] = E.xi_multipoles(a.gal, a.ran, a.ran_nbar, redges=redges, **kw, **x)["xi"]
    return out


@pytest.mark.parametrize("los,K", LOS_K)
def test_cross_fp64(pkg, ctx, cubes, los, K):
    a, b = cubes
    N = 32
    kedges = np.linspace(0.0, math.pi / (a.box_len / N), 9)
    redges = np.linspace(0.0, 250.0, 11)
    p = pkg.make_params(box_lo=a.box_lo, box_len=a.box_len, n_mesh=N, ell_max=4, los=los, order=K, precision=64,
                        assign=3, compensate=True)
    got = ctx.pk_xi_cross(a.gal, a.ran, b.gal, b.ran, p, kedges, redges, ran_nbar_a=a.ran_nbar,
                          ran_nbar_b=b.ran_nbar)
    want = _oracle(a, b, kedges, redges, N=N, box_lo=a.box_lo, box_len=a.box_len, assign=3, ell_max=4, los=los,
                   order=K, compensate=True)
    check_multipoles(got["pk"], want["pk"], "pk", 1e-10, 1e-10, f"{los} K={K} cross P: ")
    check_multipoles(got["xi"], want["xi"], "xi", 1e-10, 1e-10, f"{los} K={K} cross xi: ")
    # one statistic at a time: the same numbers
    only_p = ctx.pk_xi_cross(a.gal, a.ran, b.gal, b.ran, p, kedges=kedges, ran_nbar_a=a.ran_nbar,
                             ran_nbar_b=b.ran_nbar)
    only_x = ctx.pk_xi_cross(a.gal, a.ran, b.gal, b.ran, p, redges=redges, ran_nbar_a=a.ran_nbar,
                             ran_nbar_b=b.ran_nbar)
    assert "xi" not in only_p and "pk" not in only_x
    check_multipoles(only_p["pk"], got["pk"], "pk", 1e-10, 1e-10, "P only: ")
    check_multipoles(only_x["xi"], got["xi"], "xi", 1e-10, 1e-10, "xi only: ")


@pytest.fixture(scope="module")
def cap_pair():
    cap = lognormal_cap_catalog(seed=7, n_gal=40000, ran_factor=10.0, gen_mesh=64)
    g, r, nb = cap.gal, cap.ran, cap.ran_nbar
    bright = g[0::2].copy()
    bright[:, 3] = 1.5                       # tracer B: the other half with another weight
    return cap, (g[1::2], r[1::2], nb[1::2]), (bright, r[0::2], nb[0::2])


@pytest.mark.parametrize("los,K", [("midpoint", 4), ("bisector", 4), ("yamamoto", 0), ("midpoint_even", 4)])
def test_cross_fp32_cap(pkg, ctx, cap_pair, los, K):
    cap, A, B = cap_pair
    N = 40
    kedges = np.linspace(0.0, math.pi / (cap.box_len / N), 11)
    redges = np.linspace(0.0, 8 * cap.box_len / N, 9)
    p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=N, ell_max=4, los=los, order=K,
                        precision=32, assign=3, compensate=True)
    got = ctx.pk_xi_cross(A[0], A[1], B[0], B[1], p, kedges, redges, ran_nbar_a=A[2], ran_nbar_b=B[2])
    kw = dict(N=N, box_lo=cap.box_lo, box_len=cap.box_len, assign=3, ell_max=4, los=los, order=K, compensate=True)
    x = dict(gal_b=B[0], ran_b=B[1], ran_nbar_b=B[2])
    want_p = E.pk_multipoles(A[0], A[1], A[2], kedges=kedges, **kw, **x)["pk"]
    want_x = E.xi_multipoles(A[0], A[1], A[2], redges=redges, **kw, **x)["xi"]
    # in the lowest k bin P_4 is 1.07 % of P_0, just above the 1 % line of the relative test
    check_multipoles(got["pk"], want_p, "pk", label=f"{los} K={K} FP32 cross P: ")
    check_multipoles(got["xi"], want_x, "xi", label=f"{los} K={K} FP32 cross xi: ")


@pytest.mark.parametrize("los,K,first", [("yamamoto", 0, (10.0, 14.0)), ("midpoint", 4, (9.25, 14.25)),
                                          ("bisector", 4, (8.0, 12.75))])
def test_fp32_auto_at_the_one_percent_line(pkg, ctx, cap_pair, los, K, first):
    # auto spectrum of tracer A in FP32 with a lowest k bin (in units of k_f) where |P_4| is 1.06-1.07 %
    # of P_0: the relative 1e-4 test on P_4 there asks for an error below 1.1e-6 of the monopole
    cap, A, _ = cap_pair
    N = 40
    kf = 2 * math.pi / cap.box_len
    kedges = kf * np.concatenate([[first[0]], np.linspace(first[1], 20.0, 7)])
    redges = np.linspace(0.0, 8 * cap.box_len / N, 9)
    p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=N, ell_max=4, los=los, order=K,
                        precision=32, assign=3, compensate=True)
    got = ctx.pk_xi_multipoles(A[0], A[1], p, kedges, redges, ran_nbar=A[2])
    kw = dict(N=N, box_lo=cap.box_lo, box_len=cap.box_len, assign=3, ell_max=4, los=los, order=K, compensate=True)
    want_p = E.pk_multipoles(A[0], A[1], A[2], kedges=kedges, **kw)["pk"]
    want_x = E.xi_multipoles(A[0], A[1], A[2], redges=redges, **kw)["xi"]
    assert 0.0105 < abs(want_p[2, 0] / want_p[0, 0]) < 0.0108
    check_multipoles(got["pk"], want_p, "pk", label=f"{los} K={K} FP32 auto P: ")
    check_multipoles(got["xi"], want_x, "xi", label=f"{los} K={K} FP32 auto xi: ")


@pytest.mark.parametrize("los,K,prec", [("midpoint", 3, 64), ("bisector", 4, 64), ("yamamoto", 0, 32),
                                        ("midpoint", 4, 32)])
def test_one_tracer_twice_is_auto(pkg, ctx, cubes, los, K, prec):
    a, _ = cubes
    N = 32
    kedges = np.linspace(0.0, math.pi / (a.box_len / N), 9)
    redges = np.linspace(0.0, 250.0, 11)
    p = pkg.make_params(box_lo=a.box_lo, box_len=a.box_len, n_mesh=N, ell_max=4, los=los, order=K, precision=prec)
    auto = ctx.pk_xi_multipoles(a.gal, a.ran, p, kedges, redges, ran_nbar=a.ran_nbar)
    cross = ctx.pk_xi_cross(a.gal, a.ran, a.gal, a.ran, p, kedges, redges, ran_nbar_a=a.ran_nbar,
                            ran_nbar_b=a.ran_nbar)
    r0, r = (1e-10, 1e-10) if prec == 64 else (1e-5, 1e-4)
    check_multipoles(cross["pk"], auto["pk"], "pk", r0, r, f"{los} P: ")
    check_multipoles(cross["xi"], auto["xi"], "xi", r0, r, f"{los} xi: ")
    np.testing.assert_array_equal(cross["n_modes"], auto["n_modes"])
    np.testing.assert_array_equal(cross["n_cells"], auto["n_cells"])


def test_cross_device_inputs_and_errors(pkg, ctx, cubes):
    torch = pytest.importorskip("torch")
    a, b = cubes
    N = 24
    kedges = np.linspace(0.0, math.pi / (a.box_len / N), 7)
    redges = np.linspace(0.0, 200.0, 6)
    p = pkg.make_params(box_lo=a.box_lo, box_len=a.box_len, n_mesh=N, ell_max=2, los="bisector", order=2,
                        precision=64)
    host = ctx.pk_xi_cross(a.gal, a.ran, b.gal, b.ran, p, kedges, redges, ran_nbar_a=a.ran_nbar,
                           ran_nbar_b=b.ran_nbar)
    t = lambda v: torch.from_numpy(v).cuda()
    dev = ctx.pk_xi_cross(t(a.gal), t(a.ran), t(b.gal), t(b.ran), p, kedges, redges, ran_nbar_a=t(a.ran_nbar),
                          ran_nbar_b=t(b.ran_nbar))
    check_multipoles(dev["pk"], host["pk"], "pk", 1e-12, 1e-12)
    check_multipoles(dev["xi"], host["xi"], "xi", 1e-12, 1e-12)

    def code(fn):
        with pytest.raises(pkg.BymError) as ei:
            fn()
        return ei.value.code

    mk = lambda **kw: pkg.make_params(box_lo=a.box_lo, box_len=a.box_len, n_mesh=N, ell_max=2, los="midpoint",
                                      order=2, **kw)
    run = lambda q, **kw: ctx.pk_xi_cross(a.gal, a.ran, b.gal, b.ran, q, kedges, redges, ran_nbar_a=a.ran_nbar,
                                          **({"ran_nbar_b": b.ran_nbar} | kw))
    assert code(lambda: run(mk(norm=2))) == -6
    assert code(lambda: run(mk(interlace=True))) == -6
    assert code(lambda: run(mk(), ran_nbar_b=None)) == -1           # norm 1 needs tracer B's nbar
    bad = b.gal.copy()
    bad[3, 0] = a.box_lo[0] - 1.0
    assert code(lambda: ctx.pk_xi_cross(a.gal, a.ran, bad, b.ran, mk(), kedges, ran_nbar_a=a.ran_nbar,
                                        ran_nbar_b=b.ran_nbar)) == -2
    ctx.set_field_chunk(8)
    try:
        assert code(lambda: run(mk())) == -6
    finally:
        ctx.set_field_chunk(0)
    ok = run(mk())                                               # the context still serves requests
    assert np.all(np.isfinite(ok["pk"]))


@pytest.fixture(scope="module")
def survey_halves():
    cap = lognormal_cap_catalog(seed=1, n_gal=1_000_000)
    return cap, cap.gal[0::2], cap.gal[1::2]


def test_polarisation_and_monopole_at_512(pkg, survey_halves):
    # the survey workload (1e6 galaxies, 512^3 TSC) split into two tracers: raw sums without
    # randoms, so that painting is additive and auto(A + B) = auto(A) + auto(B) + 2 cross(A, B)
    torch = pytest.importorskip("torch")
    cap, ga, gb = survey_halves
    kedges = np.round(np.arange(0.01, 0.2501, 0.01), 10)
    redges = np.arange(10.0, 190.01, 10.0)
    ctx = pkg.Context(0)
    G, A, B = (torch.from_numpy(v).cuda() for v in (cap.gal, ga, gb))
    out = {}
    for los, K in (("bisector", 4), ("midpoint", 2), ("yamamoto", 0)):
        p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=512, assign=3, ell_max=4, los=los,
                            order=K, compensate=True, precision=32, norm=0)
        aa = ctx.pk_xi_multipoles(A, None, p, kedges, redges)
        bb = ctx.pk_xi_multipoles(B, None, p, kedges, redges)
        uu = ctx.pk_xi_multipoles(G, None, p, kedges, redges)
        ab = ctx.pk_xi_cross(A, None, B, None, p, kedges, redges)
        out[los] = ab
        for kind in ("pk", "xi"):
            lhs = aa[kind] + bb[kind] + 2.0 * ab[kind]
            err = np.abs(lhs - uu[kind]).max(axis=1) / np.abs(uu[kind]).max(axis=1)
            assert np.all(err < 2e-5), (los, kind, err)
    ctx.close()
    for los in ("bisector", "midpoint"):
        check_multipoles(out[los]["pk"][:1], out["yamamoto"]["pk"][:1], "pk", label=f"{los} cross P0: ")
        check_multipoles(out[los]["xi"][:1], out["yamamoto"]["xi"][:1], "xi", label=f"{los} cross xi0: ")


# ---------------------------------------------------------------- odd multipoles (ell = 1, 3)
def _check_odd(got, want, rtol, scale_rows, label):
    """Odd multipoles: each row to rtol of its own largest value plus rtol of the scale row
    (the even cross multipole of the same bins) in that bin."""
    got, want = np.asarray(got), np.asarray(want)
    assert got.shape == want.shape, (got.shape, want.shape)
    for i in range(want.shape[0]):
        tol = rtol * (np.abs(want[i]).max() + np.abs(scale_rows))
        err = np.abs(got[i] - want[i])
        assert np.all(err <= tol), f"{label} row {i}: err {err.max():.3e} tol {tol[np.argmax(err - tol)]:.3e}"


@pytest.mark.parametrize("los,K", [("yamamoto", 0), ("midpoint", 2), ("midpoint", 3), ("bisector", 2),
                                   ("bisector", 4)])
def test_odd_cross_fp64(pkg, ctx, cubes, los, K):
    a, b = cubes
    N = 32
    kedges = np.linspace(0.0, math.pi / (a.box_len / N), 9)
    redges = np.linspace(0.0, 250.0, 11)
    p = pkg.make_params(box_lo=a.box_lo, box_len=a.box_len, n_mesh=N, ell_max=3, los=los, order=K, precision=64,
                        assign=3, compensate=True)
    got = ctx.pk_xi_cross(a.gal, a.ran, b.gal, b.ran, p, kedges, redges, ran_nbar_a=a.ran_nbar,
                          ran_nbar_b=b.ran_nbar, odd=True)
    assert got["ells"] == [1, 3]
    kw = dict(N=N, box_lo=a.box_lo, box_len=a.box_len, assign=3, ell_max=3, los=los, order=K, compensate=True,
              odd=True, gal_b=b.gal, ran_b=b.ran, ran_nbar_b=b.ran_nbar)
    want_p = E.pk_multipoles(a.gal, a.ran, a.ran_nbar, kedges=kedges, **kw)["pk"]
    want_x = E.xi_multipoles(a.gal, a.ran, a.ran_nbar, redges=redges, **kw)["xi"]
    _check_odd(got["pk"], want_p[[1, 3]], 1e-10, want_p[0], f"{los} K={K} odd P")
    _check_odd(got["xi"], want_x[[1, 3]], 1e-10, np.abs(want_x[0]).max(), f"{los} K={K} odd xi")
    assert np.abs(want_p[1]).max() > 1e-3 * np.abs(want_p[0]).max()      # the dipole is there
    # A <-> B: odd multipoles change sign; one tracer twice: they vanish
    ba = ctx.pk_xi_cross(b.gal, b.ran, a.gal, a.ran, p, kedges, redges, ran_nbar_a=b.ran_nbar,
                         ran_nbar_b=a.ran_nbar, odd=True)
    _check_odd(-ba["pk"], got["pk"], 1e-12, want_p[0], "swap P")
    _check_odd(-ba["xi"], got["xi"], 1e-12, np.abs(want_x[0]).max(), "swap xi")
    aa = ctx.pk_xi_cross(a.gal, a.ran, a.gal, a.ran, p, kedges, redges, ran_nbar_a=a.ran_nbar,
                         ran_nbar_b=a.ran_nbar, odd=True)
    assert np.abs(aa["pk"]).max() < 1e-10 * np.abs(want_p[0]).max()
    assert np.abs(aa["xi"]).max() < 1e-10 * np.abs(want_x[0]).max()
    only_p = ctx.pk_xi_cross(a.gal, a.ran, b.gal, b.ran, p, kedges=kedges, ran_nbar_a=a.ran_nbar,
                             ran_nbar_b=b.ran_nbar, odd=True)
    _check_odd(only_p["pk"], got["pk"], 1e-12, want_p[0], "P only")


@pytest.mark.parametrize("los,K", [("yamamoto", 0), ("midpoint", 4), ("bisector", 4)])
def test_odd_cross_fp32_cap(pkg, ctx, cap_pair, los, K):
    cap, A, B = cap_pair
    N = 40
    kedges = np.linspace(0.0, math.pi / (cap.box_len / N), 11)
    redges = np.linspace(0.0, 8 * cap.box_len / N, 9)
    p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=N, ell_max=3, los=los, order=K,
                        precision=32, assign=3, compensate=True)
    got = ctx.pk_xi_cross(A[0], A[1], B[0], B[1], p, kedges, redges, ran_nbar_a=A[2], ran_nbar_b=B[2], odd=True)
    kw = dict(N=N, box_lo=cap.box_lo, box_len=cap.box_len, assign=3, ell_max=3, los=los, order=K, compensate=True,
              odd=True, gal_b=B[0], ran_b=B[1], ran_nbar_b=B[2])
    want_p = E.pk_multipoles(A[0], A[1], A[2], kedges=kedges, **kw)["pk"]
    want_x = E.xi_multipoles(A[0], A[1], A[2], redges=redges, **kw)["xi"]
    # FP32: 1e-4 of each odd multipole's largest value plus 1e-5 of the monopole in the bin
    tol_p = 1e-4 * np.abs(want_p[[1, 3]]).max(axis=1)[:, None] + 1e-5 * np.abs(want_p[0])[None, :]
    assert np.all(np.abs(got["pk"] - want_p[[1, 3]]) <= tol_p), np.abs(got["pk"] - want_p[[1, 3]]) / tol_p
    tol_x = 1e-4 * np.abs(want_x[[1, 3]]).max(axis=1)[:, None] + 1e-5 * np.abs(want_x[0]).max()
    assert np.all(np.abs(got["xi"] - want_x[[1, 3]]) <= tol_x), np.abs(got["xi"] - want_x[[1, 3]]) / tol_x


def test_odd_errors(pkg, ctx, cubes):
    a, b = cubes
    kedges = np.linspace(0.0, 0.1, 5)

    def code(**kw):
        p = pkg.make_params(box_lo=a.box_lo, box_len=a.box_len, n_mesh=16, **kw)
        with pytest.raises(pkg.BymError) as ei:
            ctx.pk_xi_cross(a.gal, a.ran, b.gal, b.ran, p, kedges, ran_nbar_a=a.ran_nbar, ran_nbar_b=b.ran_nbar,
                            odd=True)
        return ei.value.code

    assert code(ell_max=3, los="midpoint_even", order=2) == -6
    assert code(ell_max=2, los="bisector", order=2) == -6
    assert code(ell_max=9, los="bisector", order=2) == -6
    assert code(ell_max=3, los="bisector", order=2, norm=2) == -6
    assert code(ell_max=3, los="yamamoto", interlace=True) == -6
