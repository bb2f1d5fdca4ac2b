"""Serving loop and batch runs: each result is the same alone and in the mix.

Requests of different mesh sizes, lines of sight, orders and precisions are
queued together on a serving loop with several slots (their work overlaps on
the GPU) and compared with the same request run alone through
bym_pk_xi_multipoles, within the parity tolerances."""
import math

import numpy as np
import pytest

from parity import check_multipoles
from synth import lognormal_cap_catalog

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2102_08384_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def cap():
    return lognormal_cap_catalog(seed=4, n_gal=20000, ran_factor=10.0, gen_mesh=64)


def _mix(pkg, cat):
    out = []
    for i, (N, los, K, prec) in enumerate([(32, "midpoint", 4, 32), (48, "bisector", 4, 32), (24, "yamamoto", 0, 64),
                                           (40, "midpoint", 2, 64), (64, "bisector", 2, 32), (32, "yamamoto", 0, 32),
                                           (56, "midpoint", 3, 32), (32, "bisector", 6, 64)]):
        p = pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=N, assign=2 + (i % 2), ell_max=4,
                            los=los, order=K, precision=prec, compensate=bool(i % 3 == 0))
        kedges = np.linspace(0.0, math.pi / (cat.box_len / N), 9)
        redges = np.linspace(0.0, 6 * cat.box_len / N, 6)
        out.append(dict(gal=cat.gal, ran=cat.ran, params=p, kedges=kedges, redges=redges, ran_nbar=cat.ran_nbar))
    return out


def _tol(prec):
    return (1e-5, 1e-4) if prec == 32 else (1e-10, 1e-10)


def test_results_same_alone_and_in_the_mix(pkg, cap):
    items = _mix(pkg, cap)
    ctx = pkg.Context(0)
    alone = [ctx.pk_xi_multipoles(it["gal"], it["ran"], it["params"], it["kedges"], it["redges"],
                                  ran_nbar=it["ran_nbar"]) for it in items]
    ctx.serve_start(n_slots=3)
    tickets = [ctx.submit(it["gal"], it["ran"], it["params"], it["kedges"], it["redges"], ran_nbar=it["ran_nbar"])
               for it in items]
    mixed = [ctx.wait(t) for t in tickets]
    stats = ctx.serve_stats()
    ctx.serve_stop()
    ctx.close()
    assert stats["count"] == len(items)
    assert stats["p99_s"] >= stats["p50_s"] > 0
    for it, a, m in zip(items, alone, mixed):
        # painting and shell sums do not depend on what else runs: the same bits alone and in the mix
        for key in ("pk", "xi", "k_mean", "r_mean", "n_modes", "n_cells"):
            np.testing.assert_array_equal(m[key], a[key], err_msg=f"{key} of {it['params'].los}")


def test_batch_run_matches_sequential(pkg, cap):
    items = _mix(pkg, cap)[:5]
    ctx = pkg.Context(0)
    seq = [ctx.pk_xi_multipoles(it["gal"], it["ran"], it["params"], it["kedges"], it["redges"],
                                ran_nbar=it["ran_nbar"]) for it in items]
    bat = ctx.batch_run(items)
    ctx.close()
    for it, a, b in zip(items, seq, bat):
        r0, r = _tol(it["params"].precision)
        check_multipoles(b["pk"], a["pk"], "pk", r0, r)
        check_multipoles(b["xi"], a["xi"], "xi", r0, r)


def test_admission_timeout_and_errors(pkg, cap):
    ctx = pkg.Context(0)
    small = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=32, ell_max=4, los="midpoint", order=2)
    fp = pkg.footprint(small, len(cap.gal), len(cap.ran))
    ctx.serve_start(n_slots=2, hbm_budget_bytes=int(1.5 * fp))
    big = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=256, ell_max=4, los="midpoint", order=4)
    kedges = np.linspace(0.0, 0.2, 5)
    with pytest.raises(pkg.BymError) as ei:          # can never fit the budget
        ctx.submit(cap.gal, cap.ran, big, kedges, ran_nbar=cap.ran_nbar)
    assert ei.value.code == -3
    # only one of two equal requests fits at a time: the second waits for memory
    t1 = ctx.submit(cap.gal, cap.ran, small, kedges, ran_nbar=cap.ran_nbar)
    t2 = ctx.submit(cap.gal, cap.ran, small, kedges, ran_nbar=cap.ran_nbar)
    with pytest.raises(pkg.BymError) as ei:
        ctx.wait(t2, timeout_s=0.0)
    assert ei.value.code == -5
    a = ctx.wait(t1)
    b = ctx.wait(t2)
    np.testing.assert_allclose(a["pk"], b["pk"], rtol=1e-5, atol=1e-5 * np.abs(a["pk"]).max())
    stats = ctx.serve_stats()
    assert stats["peak_hbm_bytes"] <= 1.5 * fp
    ctx.serve_reset_stats()
    assert ctx.serve_stats()["count"] == 0
    # a failing request reports its own error code
    bad = np.array(cap.gal, copy=True)
    bad[3, 0] = cap.box_lo[0] - 10.0
    t3 = ctx.submit(bad, cap.ran, small, kedges, ran_nbar=cap.ran_nbar)
    with pytest.raises(pkg.BymError) as ei:
        ctx.wait(t3)
    assert ei.value.code == -2
    ctx.serve_stop()
    ctx.close()


def test_autotune_keeps_results_and_caches(pkg, cap, tmp_path):
    ctx = pkg.Context(0)
    p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=48, ell_max=4, los="bisector", order=4)
    kedges = np.linspace(0.0, 0.3, 7)
    redges = np.linspace(0.0, 300.0, 6)
    ref = ctx.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    cache = str(tmp_path / "tune.txt")
    choice = ctx.autotune(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar, cache_path=cache)
    assert choice["source"] == "measured" and choice["fft_batch"] in (4, 8, 16)
    tuned = ctx.pk_xi_multipoles(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar)
    check_multipoles(tuned["pk"], ref["pk"], "pk")
    check_multipoles(tuned["xi"], ref["xi"], "xi")
    ctx.close()
    ctx2 = pkg.Context(0)
    again = ctx2.autotune(cap.gal, cap.ran, p, kedges, redges, ran_nbar=cap.ran_nbar, cache_path=cache)
    ctx2.close()
    assert again["source"] == "cache"
    assert {k: v for k, v in again.items() if k != "source"} == {k: v for k, v in choice.items() if k != "source"}


def test_batch_graph_matches_sequential(pkg, cap):
    # the mix (meshes, LOS, orders, precisions, compensation) plus a norm-2 item, as one CUDA graph
    items = _mix(pkg, cap)
    p2 = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=40, ell_max=4, los="midpoint", order=2,
                         precision=32, norm=2)
    items.append(dict(gal=cap.gal, ran=cap.ran, params=p2, kedges=np.linspace(0.0, 0.3, 7),
                      redges=np.linspace(0.0, 300.0, 6), ran_nbar=cap.ran_nbar))
    p3 = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=36, ell_max=4, los="bisector", order=2,
                         precision=64, interlace=True)
    items.append(dict(gal=cap.gal, ran=cap.ran, params=p3, kedges=np.linspace(0.0, 0.3, 7),
                      redges=np.linspace(0.0, 300.0, 6), ran_nbar=cap.ran_nbar))
    items = items + items[:3]            # repeated shapes reuse the warmed caches
    ctx = pkg.Context(0)
    seq = [ctx.pk_xi_multipoles(it["gal"], it["ran"], it["params"], it["kedges"], it["redges"],
                                ran_nbar=it["ran_nbar"]) for it in items]
    gr = ctx.batch_graph(items)
    again = ctx.batch_graph(items)       # a second graph on the same context
    ctx.close()
    for it, a, b, c in zip(items, seq, gr, again):
        r0, r = _tol(it["params"].precision)
        for out in (b, c):
            check_multipoles(out["pk"], a["pk"], "pk", r0, r)
            check_multipoles(out["xi"], a["xi"], "xi", r0, r)
            np.testing.assert_array_equal(out["n_modes"], a["n_modes"])


def test_batch_graph_reports_item_errors(pkg, cap):
    ctx = pkg.Context(0)
    p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=32, ell_max=4, los="bisector", order=2)
    bad = np.array(cap.gal, copy=True)
    bad[0, 2] = np.nan
    good = dict(gal=cap.gal, ran=cap.ran, params=p, kedges=np.linspace(0, 0.2, 5), ran_nbar=cap.ran_nbar)
    for items in ([good, dict(good, gal=bad)], [dict(good, gal=bad), good]):   # bad item captured / in warm-up
        with pytest.raises(pkg.BymError) as ei:
            ctx.batch_graph(items)
        assert ei.value.code == -2
    ctx.close()


def test_batch_plan_relaunch_follows_device_catalogs(pkg, cap):
    # a persistent captured batch: relaunching recomputes from the current device catalogs
    torch = pytest.importorskip("torch")
    g = torch.from_numpy(cap.gal).cuda()
    r = torch.from_numpy(cap.ran).cuda()
    rn = torch.from_numpy(cap.ran_nbar).cuda()
    items = []
    for N, los, K in ((32, "midpoint", 2), (48, "bisector", 4), (40, "yamamoto", 0)):
        p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=N, ell_max=4, los=los, order=K)
        items.append(dict(gal=g, ran=r, params=p, kedges=np.linspace(0.0, 0.3, 9), redges=np.linspace(0, 250, 6),
                          ran_nbar=rn))
    ctx = pkg.Context(0)
    plan = ctx.batch_plan(items)

    def seq():
        return [ctx.pk_xi_multipoles(it["gal"], it["ran"], it["params"], it["kedges"], it["redges"],
                                     ran_nbar=it["ran_nbar"]) for it in items]

    for _ in range(2):
        got = [dict((k, v.copy()) for k, v in o.items() if k != "ells") for o in plan.launch()]
        for a, b in zip(seq(), got):
            check_multipoles(b["pk"], a["pk"], "pk")
            check_multipoles(b["xi"], a["xi"], "xi")
        g[:, 3] = g[:, 3] * torch.linspace(0.5, 1.5, g.shape[0], device="cuda")   # new weights, same buffer
        torch.cuda.synchronize()
    plan.close()
    ctx.close()


def test_batch_plan_with_plane_backends_at_512(pkg, cap):
    # 512^3 items under the plane-transform backends (4: library x pass, 5: cuFFT along x): the
    # captured runs transform every plane, their warm-up the same, and results match a plain run
    N = 512
    kedges = np.linspace(0.0, 0.2, 6)
    redges = np.linspace(0.0, 150.0, 6)
    for mode in (4, 5):
        ctx = pkg.Context(0)
        ctx.set_fft_backend(mode)
        items = []
        for los, K in (("midpoint", 2), ("bisector", 2)):
            p = pkg.make_params(box_lo=cap.box_lo, box_len=cap.box_len, n_mesh=N, assign=3, ell_max=2, los=los,
                                order=K, compensate=True, precision=32)
            items.append(dict(gal=cap.gal, ran=cap.ran, ran_nbar=cap.ran_nbar, params=p, kedges=kedges,
                              redges=redges))
        seq = [ctx.pk_xi_multipoles(it["gal"], it["ran"], it["params"], kedges, redges, ran_nbar=it["ran_nbar"])
               for it in items]
        plan = ctx.batch_plan(items)
        got = plan.launch()
        plan.close()
        ctx.close()
        for a, b in zip(got, seq):
            check_multipoles(a["pk"], b["pk"], "pk", label=f"mode {mode} graph P: ")
            check_multipoles(a["xi"], b["xi"], "xi", label=f"mode {mode} graph xi: ")
