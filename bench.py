"""Benchmark: catalogs/s of the pairwise-LOS P_ell(k) + xi_ell(r) estimators on GB300.

One step = one survey-like catalog through the whole hot path: painting, field
generation, batched R2C/C2R transforms, k-space and lag-space contractions and
FP64 shell binning, for the midpoint AND the bisector line of sight, both P_ell
and xi_ell, ell <= 4, order 4 in theta, on a 512^3 TSC mesh.

Workload (synthetic stand-in for the paper's BOSS DR12 NGC Patchy mocks):
lognormal density with P(k) = 2e4 (k/0.1)^-1.5, Kaiser RSD (f = 0.7, b = 2)
along each galaxy's radial direction, 1e6 galaxies in a 30 degree cap over
800-1600 Mpc/h, 1e7 uniform randoms, FKP weights (P0 = 1e4), doubled bounding
box; k bins 0.01..0.25 h/Mpc (dk = 0.01), r bins 10..190 Mpc/h (dr = 10),
as in the paper's Sec. 7.2.  Inputs and fields (tens of GB) exceed the 129 MB
L2, so no explicit flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank processes its own catalogs (independent replicas,
weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "catalogs/s for P_ℓ,ξ_ℓ (ℓ≤4, order 4, 512³)"
N_MESH = 512
ORDER = 4
ELL_MAX = 4
KEDGES = np.round(np.arange(0.01, 0.2501, 0.01), 10)
REDGES = np.arange(10.0, 190.01, 10.0)
WORKLOAD = ("survey-like lognormal cap (30 deg, 800-1600 Mpc/h, 1e6 gal + 1e7 ran, FKP P0=1e4, "
            "Kaiser f=0.7 b=2), 512^3 TSC compensated, midpoint+bisector LOS, order 4, ell<=4, P_ell+xi_ell")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mesh", type=int, default=N_MESH, help="mesh size (512 is the benchmark workload)")
    ap.add_argument("--n-gal", type=int, default=1_000_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--los", default="midpoint,bisector", help="comma-separated LOS list (profiling runs)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving / batching leg")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--fft-backend", type=int, default=None, choices=[0, 1, 2, 3, 4, 5, 6],
                    help="force an FFT backend (bym_set_fft_backend) instead of the tuned choice (profiling runs)")
    ap.add_argument("--serve-requests", type=int, default=240)
    ap.add_argument("--order", type=int, default=ORDER, help="expansion order (4 is the benchmark; profiling runs)")
    ap.add_argument("--ell-max", type=int, default=ELL_MAX, help="largest multipole (4 is the benchmark; profiling runs)")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_catalog(seed, n_gal):
    from synth import lognormal_cap_catalog
    return lognormal_cap_catalog(seed=seed, n_gal=n_gal, ran_factor=10.0, half_angle_deg=30.0, r_min=800.0,
                                 r_max=1600.0, gen_mesh=256)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle baseline
def oracle_sample(cat, n_mesh_full, units=3):
    """Time the FP64 oracle on a bounded sample of the same workload and scale it.

    The oracle is oracle.streamed (the loop order that holds a few full grids; equal to the
    plain estimators to 1e-12), on the benchmark's own mesh, catalog, bins and order, for the
    midpoint and the bisector line of sight, P and xi together.  Sample: painting of every 10th
    object (scaled by 10: painting is linear in the objects), then for each line of sight the
    set-up (transform of delta, binned modes and lags) and its first `units` products (midpoint)
    or field pairs (bisector), scaled by the number of units the request visits.  The first
    midpoint products each need their own g function, so the linear scaling over-estimates the
    midpoint cost; the full oracle run that wrote tests/golden/survey512_order4.json is reported
    beside it (measured on the host that ran it)."""
    from oracle import mesh as M
    from oracle import streamed as S
    sub = slice(None, None, 10)
    t0 = time.perf_counter()
    M.density_mesh(cat.gal[sub], cat.ran[sub], n_mesh_full, cat.box_lo, cat.box_len, 3)
    t_paint = 10.0 * (time.perf_counter() - t0)
    parts = {}
    for los in ("midpoint", "bisector"):
        marks = {}
        t0 = time.perf_counter()

        def progress(kind, done, total):
            if kind == "setup":
                marks["setup"] = time.perf_counter() - t0
            elif kind == "unit":
                marks["total"] = total
                if done >= units:
                    marks["units"] = time.perf_counter() - t0 - marks["setup"]
                    raise S.Stop
        try:
            S.pk_xi_multipoles(cat.gal[sub], cat.ran[sub], cat.ran_nbar[sub], N=n_mesh_full, box_lo=cat.box_lo,
                               box_len=cat.box_len, assign=3, ell_max=ELL_MAX, los=los, order=ORDER, kedges=KEDGES,
                               redges=REDGES, compensate=True, norm=1, progress=progress)
        except S.Stop:
            pass
        per_unit = marks["units"] / units
        # the set-up painted every 10th object: count the full catalog's painting instead
        parts[los] = {"setup_s": marks["setup"], "per_unit_s": per_unit, "units": marks["total"],
                      "est_s": marks["setup"] - t_paint / 10.0 + t_paint + per_unit * marks["total"]}
    t_sample = t_paint / 10.0 + sum(v["setup_s"] + units * v["per_unit_s"] for v in parts.values())
    t_full = sum(v["est_s"] for v in parts.values())
    out = {"value": 1.0 / t_full, "unit": "catalogs/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": (f"FP64 oracle (oracle.streamed, numpy/scipy.fft, {os.cpu_count()} host cores) on the {n_mesh_full}^3 "
                      f"workload: painting of every 10th object x10 ({t_paint:.1f} s per catalog painting), then per LOS "
                      f"its set-up and first {units} units, scaled by the units it visits "
                      + ", ".join(f"{k}: {v['setup_s']:.1f} s + {v['per_unit_s']:.2f} s x {v['units']}"
                                  for k, v in parts.items())
                      + f" (set-ups include the 1/10 painting, replaced by the full one) -> {t_full:.0f} s per "
                      f"catalog ({t_sample:.0f} s sampled)"),
           "sample_seconds": t_sample}
    try:
        with open(os.path.join(ROOT, "tests", "golden", "survey512_order4.json")) as fh:
            g = json.load(fh)
        wall = sum(v["oracle_wall_s"] for v in g["los"].values())
        out["full_run_measured"] = {"seconds": wall, "catalogs_per_s": 1.0 / wall, "cores": g["host"]["cores"],
                                    "machine": g["host"]["machine"],
                                    "what": "the whole oracle run (both LOS, P and xi) that wrote the golden values"}
    except (OSError, KeyError, ValueError):
        pass
    return out


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    cat = make_catalog(1, args.n_gal)
    if args.warmup > 0:                    # warm-up: the oracle's coefficient tables (cached)
        from oracle import streamed as S
        S.midpoint_products(ORDER, ELL_MAX)
        S.bisector_pairs(ORDER, ELL_MAX)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):            # each step: a bounded sample (one unit per line of sight)
        vals.append(oracle_sample(cat, args.mesh, units=1))
    wall = time.perf_counter() - t0
    v = statistics.median([x["value"] for x in vals])
    cb = dict(vals[0])
    cb["value"] = v
    cb.pop("sample_seconds", None)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "catalogs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_mesh": args.mesh, "order": ORDER, "ell_max": ELL_MAX,
                       "parallelism": "host cores", "l2": "inputs larger than L2"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "catalogs/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0},
            "sample_wall_s": wall}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import paper_2102_08384_gb300 as pkg

    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    cat = make_catalog(1 + rank, args.n_gal)
    gal_d = torch.from_numpy(cat.gal).to(dev)
    ran_d = torch.from_numpy(cat.ran).to(dev)
    rnb_d = torch.from_numpy(cat.ran_nbar).to(dev)
    ctx = pkg.Context(local)
    if args.fft_backend is not None:
        ctx.set_fft_backend(args.fft_backend)
    params = [pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=args.mesh, assign=3,
                              ell_max=args.ell_max, los=los, order=args.order if los != "yamamoto" else 0,
                              compensate=True, precision=32, norm=1)
              for los in args.los.split(",")]
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream

    def step(g, r, rn):
        out = []
        for p in params:
            out.append(ctx.pk_xi_multipoles(g, r, p, KEDGES, REDGES, ran_nbar=rn, stream=sh))
        return out

    for _ in range(args.warmup):
        step(gal_d, ran_d, rnb_d)
    torch.cuda.synchronize(dev)
    tuned = {}
    if not args.no_autotune:
        for p in params:      # launch shapes for this workload (counted as warm-up, outside the timing)
            tuned[int(p.los)] = ctx.autotune(gal_d, ran_d, p, KEDGES, REDGES, ran_nbar=rnb_d)
    torch.cuda.synchronize(dev)

    # device-resident timed region
    pkg.lib().bym_profile_enable(ctx._h, 1)
    _read_profile(pkg, ctx, reset=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] or 0) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
    with ClockSampler(gpu_index) as cs:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step(gal_d, ran_d, rnb_d)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    prof = _read_profile(pkg, ctx, reset=True)
    pkg.lib().bym_profile_enable(ctx._h, 0)
    clocks = cs.summary()
    ms_max, value = replica_throughput(ms, args.steps, ws)

    # end to end: pinned host catalogs, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        g_h = torch.from_numpy(cat.gal).pin_memory().numpy()
        r_h = torch.from_numpy(cat.ran).pin_memory().numpy()
        rn_h = torch.from_numpy(cat.ran_nbar).pin_memory().numpy()
        step(g_h, r_h, rn_h)
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step(g_h, r_h, rn_h)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_e = _max_over_ranks(e0.elapsed_time(e1), ws)
        nl, nbk, nbr = args.ell_max // 2 + 1, len(KEDGES) - 1, len(REDGES) - 1
        h2d = len(params) * (g_h.nbytes + r_h.nbytes + rn_h.nbytes)
        d2h = len(params) * (8 * 8 + nl * nbk * 8 + nl * nbr * 8)
        e2e = {"value": ws * args.steps / (ms_e / 1000.0), "unit": "catalogs/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    if rank != 0:
        ctx.close()
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    roofline, kernels, launches = _roofline(prof, args.steps)
    line = {"metric": METRIC, "value": value, "unit": "catalogs/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_mesh": args.mesh, "order": args.order, "ell_max": args.ell_max,
                       "n_gal": int(len(cat.gal)), "n_ran": int(len(cat.ran)), "box_len": cat.box_len,
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": "inputs larger than L2 (catalog 176 MB, fields > 30 GB)",
                       "autotune": tuned or "off"},
            "e2e": e2e, "roofline": roofline, "gpu_launches": launches, "clocks": clocks, "kernels": kernels}
    if ws == 1 and not args.no_serve:
        perm = torch.randperm(gal_d.shape[0], device=dev)   # random order: any prefix covers the whole cap
        gal_p = gal_d[perm].contiguous()
        permr = torch.randperm(ran_d.shape[0], device=dev)
        ran_p, rnb_p = ran_d[permr].contiguous(), rnb_d[permr].contiguous()
        line["next_rows"] = next_rows_leg(pkg, torch, dev, cat, gal_d, ran_d, rnb_d, args.mesh)
        line["large_meshes"] = large_mesh_leg(pkg, torch, dev, cat, gal_d, ran_d, rnb_d)
        line["batch"] = batch_leg(pkg, torch, dev, cat, gal_p, ran_p, rnb_p)
        line["serving"] = serving_leg(pkg, torch, dev, cat, gal_p, ran_p, rnb_p, args.serve_requests)
    if ws == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(cat, args.mesh)
        cb.pop("sample_seconds", None)
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def _mock_subsets(torch, cat, gal_d, ran_d, rnb_d, rng, frac, half_angle_deg):
    """An uneven mock from the benchmark catalog: a random fraction of its galaxies and randoms
    (a fixed random order, so every prefix covers the whole cap) inside a narrower cap around
    the same pole; nbar and FKP weights are those of the full catalog (same density)."""
    pole = torch.tensor(cat.meta.get("pole", (1.0, 1.0, 1.0)), dtype=torch.float32, device=gal_d.device)
    pole = pole / pole.norm()
    cmin = math.cos(math.radians(half_angle_deg))
    out = []
    for x in (gal_d, ran_d):
        n = int(frac * x.shape[0])
        sub = x[:n]
        c = (sub[:, :3] @ pole) / sub[:, :3].norm(dim=1)
        out.append(c >= cmin)
    g = gal_d[: int(frac * gal_d.shape[0])][out[0]].contiguous()
    keep = out[1]
    r = ran_d[: int(frac * ran_d.shape[0])][keep].contiguous()
    rn = rnb_d[: int(frac * rnb_d.shape[0])][keep].contiguous()
    return g, r, rn


def next_rows_leg(pkg, torch, dev, cat, gal_d, ran_d, rnb_d, n_mesh, reps=2):
    """The benchmark catalog at the benchmark mesh through the extensions beyond the paper's
    boxed estimators (the library's FFT passes), each timed (CUDA events, after one warm-up run)
    beside its device footprint: the parity-even midpoint form; the midpoint g fields streamed in ranges of 45;
    the bisector fields in blocks of 16; xi normalised by the random-random count; interlacing; the
    cross spectra of two tracers (the catalog's even- and odd-numbered galaxies and randoms)."""
    ctx = pkg.Context(dev.index)
    ctx.set_fft_backend(6)        # the library's FFT passes: the path the autotuner picks for the step
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    halves = [(t[0::2].contiguous(), t[1::2].contiguous()) for t in (gal_d, ran_d, rnb_d)]
    # label, los, order, norm, field chunk (-1: interlaced), cross (2: its odd multipoles 1, 3)
    cases = [("midpoint_even order 4", "midpoint_even", 4, 1, 0, 0),
             ("midpoint order 4, g fields in ranges of 45", "midpoint", 4, 1, 45, 0),
             ("bisector order 4, fields in blocks of 16", "bisector", 4, 1, 16, 0),
             ("midpoint order 4, xi / RR (norm 2)", "midpoint", 4, 2, 0, 0),
             ("bisector order 4, interlaced", "bisector", 4, 1, -1, 0),
             ("bisector order 4, cross spectra of two tracers", "bisector", 4, 1, 0, 1),
             ("midpoint order 4, cross spectra of two tracers", "midpoint", 4, 1, 0, 1),
             ("bisector order 4, odd multipoles (1, 3) of the cross spectra", "bisector", 4, 1, 0, 2),
             ("midpoint order 4, odd multipoles (1, 3) of the cross spectra", "midpoint", 4, 1, 0, 2),
             ("yamamoto, odd multipoles (1, 3) of the cross spectra", "yamamoto", 0, 1, 0, 2)]
    out = {}
    for label, los, K, norm, chunk, cross in cases:
        il = chunk < 0                   # -1: interlaced, resident
        chunk = max(chunk, 0)
        odd = cross == 2
        p = pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=n_mesh, assign=3,
                            ell_max=3 if odd else ELL_MAX, los=los, order=K, compensate=True, precision=32, norm=norm,
                            interlace=il)
        ctx.set_field_chunk(chunk)
        if cross:
            (ga, gb), (ra, rb), (na, nb) = halves

            def run():
                ctx.pk_xi_cross(ga, ra, gb, rb, p, KEDGES, REDGES, ran_nbar_a=na, ran_nbar_b=nb, stream=sh,
                                odd=odd)
        else:
            def run():
                ctx.pk_xi_multipoles(gal_d, ran_d, p, KEDGES, REDGES, ran_nbar=rnb_d, stream=sh)
        n_f = {"midpoint_even": 88, "midpoint": 145, "bisector": 49, "yamamoto": 15}[los]
        slot = n_mesh * n_mesh * (n_mesh + 4) * 4
        if odd:   # odd field sets (bisector J <= 5: 36, midpoint J - alpha odd: 110, Yamamoto: 10), 10 X / H slots
            slots = 2 + 2 * {"bisector": 36, "midpoint": 110, "yamamoto": 10}[los] + (0 if los == "yamamoto" else 10)
        elif chunk and los == "midpoint":
            slots = 2 + chunk + 15
        elif chunk:
            slots = 1 + 2 * chunk + 15
        elif il or cross:
            slots = 2 + 2 * n_f + 15
        else:
            slots = 1 + n_f + 15
        try:
            run()
        except pkg.BymError as e:        # e.g. a footprint beyond this device's memory
            out[label] = {"error": str(e), "mesh_slots": slots, "field_memory_gb": slots * slot / 1e9}
            continue
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        out[label] = {"ms_per_catalog": ms, "catalogs_per_s": 1000.0 / ms, "mesh_slots": slots,
                      "field_memory_gb": slots * slot / 1e9}
    ctx.set_field_chunk(0)
    ctx.close()
    return out


def large_mesh_leg(pkg, torch, dev, cat, gal_d, ran_d, rnb_d):
    """The benchmark catalog on 768^3 and 1024^3 meshes, where the resident order-4 field sets do
    not fit the GPU (midpoint 161 slots of 1.82 / 4.3 GB, bisector 65): the midpoint with its g fields
    in ranges and the bisector with its fields in blocks, beside the resident Yamamoto request; each
    timed once after a warm-up run (CUDA events), with its mesh slots and the largest relative
    difference of its monopole (P_0 and xi_0, which do not depend on the line of sight) from
    Yamamoto's.  FFTs: cuFFT plane transforms over the occupied planes and cuFFT along x."""
    out = {}
    ctx = pkg.Context(dev.index)
    ctx.set_fft_backend(5)
    stream = torch.cuda.current_stream(dev)
    try:
        for N, mchunk, bchunk in ((768, 24, 16), (1024, 16, 8)):
            slot = N * N * (N + 4) * 4
            res = {}
            for label, los, K, chunk, slots in (("yamamoto", "yamamoto", 0, 0, 16),
                                                (f"midpoint order 4, g fields in ranges of {mchunk}", "midpoint", 4,
                                                 mchunk, 2 + mchunk + 15),
                                                (f"bisector order 4, fields in blocks of {bchunk}", "bisector", 4,
                                                 bchunk, 1 + 2 * bchunk + 15)):
                ctx.set_field_chunk(chunk)
                p = pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=N, assign=3, ell_max=ELL_MAX,
                                    los=los, order=K, compensate=True, precision=32, norm=1)
                try:
                    ctx.pk_xi_multipoles(gal_d, ran_d, p, KEDGES, REDGES, ran_nbar=rnb_d)
                    torch.cuda.synchronize(dev)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    r = ctx.pk_xi_multipoles(gal_d, ran_d, p, KEDGES, REDGES, ran_nbar=rnb_d)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                except pkg.BymError as e:
                    res[label] = {"error": str(e), "mesh_slots": slots, "field_memory_gb": slots * slot / 1e9}
                    continue
                res[label] = {"ms_per_catalog": e0.elapsed_time(e1), "mesh_slots": slots,
                              "field_memory_gb": slots * slot / 1e9, "_r": r}
            ref = res.get("yamamoto", {}).get("_r")
            for v in res.values():
                r = v.pop("_r", None)
                if r is not None and ref is not None:
                    v["monopole_max_rel_diff_vs_yamamoto"] = float(max(
                        np.max(np.abs(r["pk"][0] - ref["pk"][0]) / np.abs(ref["pk"][0])),
                        np.max(np.abs(r["xi"][0] - ref["xi"][0])) / np.max(np.abs(ref["xi"][0]))))
            out[f"{N}^3"] = res
    finally:
        ctx.set_field_chunk(0)
        ctx.close()
    return out


def torch_lognormal_cap(torch, dev, seed, n_gal, half_angle_deg, r_min=800.0, r_max=1600.0, ran_factor=10.0,
                        pk_amp=2e4, pk_slope=-1.5, k0=0.1, f_growth=0.7, bias=2.0, P0=1e4, gen_mesh=128):
    """A survey-like mock on the device, by the recipe of synth.lognormal_cap_catalog (lognormal
    density from a power-law Gaussian field, Poisson counts in a spherical cap, Kaiser
    displacements along each galaxy's own line of sight, uniform-in-volume randoms, FKP weights,
    pole (1,1,1)/sqrt(3)); drawn with torch's generator, so the same recipe but other numbers.
    Returns device float32 (n, 4) galaxies and randoms, random nbar, box_lo and box_len."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    cos_max = math.cos(math.radians(half_angle_deg))
    sin_max = math.sin(math.radians(half_angle_deg))
    v_cap = 2 * math.pi * (1 - cos_max) * (r_max ** 3 - r_min ** 3) / 3.0
    nbar = n_gal / v_cap
    zlo = r_min * cos_max
    side = max(r_max - zlo, 2 * r_max * sin_max) * 1.02
    g_lo = torch.tensor([-side / 2, -side / 2, 0.5 * (zlo + r_max) - side / 2], dtype=torch.float64, device=dev)
    Ng, hg, kf = gen_mesh, side / gen_mesh, 2 * math.pi / side
    n1 = torch.fft.fftfreq(Ng, d=1.0 / Ng, device=dev, dtype=torch.float64)
    nz = torch.fft.rfftfreq(Ng, d=1.0 / Ng, device=dev, dtype=torch.float64)
    kx, ky, kz = (n1 * kf)[:, None, None], (n1 * kf)[None, :, None], (nz * kf)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    kk = torch.sqrt(k2)
    pk = torch.where(kk > 0, pk_amp * (torch.clamp(kk, min=1e-30) / k0) ** pk_slope, torch.zeros_like(kk))
    white = torch.randn((Ng, Ng, Ng), generator=g, device=dev, dtype=torch.float64)
    Gk = torch.fft.rfftn(white) * torch.sqrt(pk / hg ** 3)
    G = torch.fft.irfftn(Gk, s=(Ng, Ng, Ng))
    dln = torch.exp(G - G.var() / 2.0)
    counts = torch.poisson(nbar * hg ** 3 * dln, generator=g).to(torch.int64).ravel()
    cells = torch.repeat_interleave(torch.arange(Ng ** 3, device=dev), counts)
    ci = torch.stack([cells // (Ng * Ng), (cells // Ng) % Ng, cells % Ng], dim=1)
    pos = g_lo[None, :] + (ci + torch.rand(ci.shape, generator=g, device=dev, dtype=torch.float64)) * hg
    rr = torch.linalg.norm(pos, dim=1)
    keep = (rr >= r_min) & (rr <= r_max) & (pos[:, 2] >= rr * cos_max)
    pos, ci = pos[keep], ci[keep]
    inv_k2 = torch.where(k2 > 0, 1.0 / torch.clamp(k2, min=1e-30), torch.zeros_like(k2))
    dm_k = Gk / bias
    psi = torch.stack([torch.fft.irfftn(1j * kc * dm_k * inv_k2, s=(Ng, Ng, Ng))[ci[:, 0], ci[:, 1], ci[:, 2]]
                       for kc in (kx, ky, kz)], dim=1)
    rhat = pos / torch.linalg.norm(pos, dim=1, keepdim=True)
    pos = pos + f_growth * torch.sum(psi * rhat, dim=1, keepdim=True) * rhat
    n_ran = int(round(ran_factor * len(pos)))
    u = torch.rand(n_ran, generator=g, device=dev, dtype=torch.float64)
    rad = (r_min ** 3 + u * (r_max ** 3 - r_min ** 3)) ** (1.0 / 3.0)
    mu = cos_max + (1 - cos_max) * torch.rand(n_ran, generator=g, device=dev, dtype=torch.float64)
    ph = 2 * math.pi * torch.rand(n_ran, generator=g, device=dev, dtype=torch.float64)
    st = torch.sqrt(torch.clamp(1 - mu * mu, min=0.0))
    ran = torch.stack([st * torch.cos(ph), st * torch.sin(ph), mu], dim=1) * rad[:, None]
    pole = torch.tensor([1.0, 1.0, 1.0], dtype=torch.float64, device=dev) / math.sqrt(3.0)
    z = torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64, device=dev)
    v = torch.linalg.cross(z, pole)
    s_, c_ = torch.linalg.norm(v), torch.dot(z, pole)
    vx = torch.tensor([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]], dtype=torch.float64, device=dev)
    R = torch.eye(3, dtype=torch.float64, device=dev) + vx + vx @ vx * ((1 - c_) / s_ ** 2)
    pos, ran = pos @ R.T, ran @ R.T
    w = 1.0 / (1.0 + nbar * P0)
    gal = torch.cat([pos, torch.full((len(pos), 1), w, dtype=torch.float64, device=dev)], dim=1).float()
    rand = torch.cat([ran, torch.full((n_ran, 1), w, dtype=torch.float64, device=dev)], dim=1).float()
    lo = torch.minimum(rand[:, :3].min(0).values, gal[:, :3].min(0).values).double()
    hi = torch.maximum(rand[:, :3].max(0).values, gal[:, :3].max(0).values).double()
    extent = float((hi - lo).max())
    box_lo = (0.5 * (lo + hi) - extent).cpu().numpy()
    return gal.contiguous(), rand.contiguous(), torch.full((n_ran,), nbar, dtype=torch.float32, device=dev), \
        box_lo, 2.0 * extent


def _tune_shapes(ctx, items):
    """bym_autotune once per (mesh, LOS) of a request mix (the tuner's key, with the precision),
    on the mix's largest request of that shape; every later request of the shape on ctx, and on
    the serving slots and batch branches made from it, runs with the measured choice."""
    rep = {}
    for it in items:
        p = it["params"]
        key = (p.n_mesh, int(p.los))
        if key not in rep or it["gal"].shape[0] > rep[key]["gal"].shape[0]:
            rep[key] = it
    out = {}
    for key, it in sorted(rep.items()):
        t = ctx.autotune(it["gal"], it["ran"], it["params"], it["kedges"], it["redges"], ran_nbar=it["ran_nbar"])
        out[f"n{key[0]}_los{key[1]}"] = t.get("native_fft")
    return out


def batch_leg(pkg, torch, dev, cat, gal_d, ran_d, rnb_d, n_mocks=64, slots=4):
    """The batched workload: 64 independent lognormal mocks, seeds 100 + i, N_gal log-uniform in
    [2e5, 2e6], cap half-angles uniform in [10, 60] degrees over 800-1600 Mpc/h, 10x randoms, meshes
    128, 192, 256, 384^3 in turn, midpoint for four mocks then bisector for four, order 4, ell <= 4,
    P and xi, FP32.  Run (a) one at a time, (b) as one batch through the 4-slot serving loop,
    (c) as one captured CUDA graph with 4 branches (captured once, then relaunched).  Launch shapes and
    FFT path of every (mesh, LOS) come from bym_autotune, run once per shape before any timing."""
    rng = np.random.default_rng(100)
    items = []
    t0 = time.perf_counter()
    for i in range(n_mocks):
        N = (128, 192, 256, 384)[i % 4]
        los = ("midpoint", "bisector")[(i // 4) % 2]     # every mesh with both LOS within 8 mocks
        n_gal = int(10 ** rng.uniform(math.log10(2e5), math.log10(2e6)))
        g, r, rn, box_lo, box_len = torch_lognormal_cap(torch, dev, 100 + i, n_gal, float(rng.uniform(10.0, 60.0)))
        p = pkg.make_params(box_lo=box_lo, box_len=box_len, n_mesh=N, assign=3, ell_max=ELL_MAX, los=los,
                            order=ORDER, compensate=True, precision=32, norm=1)
        items.append(dict(gal=g, ran=r, ran_nbar=rn, params=p, kedges=KEDGES, redges=REDGES))
    torch.cuda.synchronize(dev)
    t_gen = time.perf_counter() - t0
    ctx = pkg.Context(dev.index)
    t0 = time.perf_counter()
    tuned = _tune_shapes(ctx, items)       # launch shapes and FFT path per (mesh, LOS), like config 3 asks
    t_tune = time.perf_counter() - t0

    def alone(it):
        return ctx.pk_xi_multipoles(it["gal"], it["ran"], it["params"], it["kedges"], it["redges"],
                                    ran_nbar=it["ran_nbar"])

    for it in items[:8]:                   # kernels, plans and bin tables of every shape
        alone(it)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for it in items:
        alone(it)
    t_seq = time.perf_counter() - t0
    ctx.serve_start(n_slots=slots)
    ts = [ctx.submit(it["gal"], it["ran"], it["params"], it["kedges"], it["redges"], ran_nbar=it["ran_nbar"])
          for it in items[:8] for _ in range(slots)]   # every slot meets every shape
    for t in ts:
        ctx.wait(t)
    t0 = time.perf_counter()
    ts = [ctx.submit(it["gal"], it["ran"], it["params"], it["kedges"], it["redges"], ran_nbar=it["ran_nbar"])
          for it in items]
    for t in ts:
        ctx.wait(t)
    t_batch = time.perf_counter() - t0
    ctx.serve_stop()
    t0 = time.perf_counter()
    plan = ctx.batch_plan(items, n_streams=slots)
    t_capture = time.perf_counter() - t0
    plan.launch()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    plan.launch()
    t_graph = time.perf_counter() - t0
    plan.close()
    ctx.close()
    n_gal = [int(it["gal"].shape[0]) for it in items]
    return {"mocks": len(items),
            "mix": "64 independent lognormal mocks (seeds 100+i, generated on the device), 2e5-2e6 galaxies "
                   "log-uniform, 10-60 deg caps, 10x randoms; meshes 128/192/256/384^3 in turn, midpoint/bisector "
                   f"alternating, order 4, ell<=4, P_ell+xi_ell, FP32 ({min(n_gal)}-{max(n_gal)} galaxies)",
            "mock_generation_s": t_gen,
            "sequential_catalogs_per_s": len(items) / t_seq,
            "served_batch_catalogs_per_s": len(items) / t_batch,
            "graph_batch_catalogs_per_s": len(items) / t_graph,
            "graph_capture_s": t_capture, "branches": slots, "autotune_s": t_tune, "autotune": tuned}


def serving_leg(pkg, torch, dev, cat, gal_d, ran_d, rnb_d, n_req, slots=4):
    """A Poisson stream of requests at 0.8x the measured one-at-a-time capacity of the same mix:
    meshes 128, 256, 384, 512^3, a random LOS, order in {0, 2, 4, 6} (0 for Yamamoto), a
    random 10-100 % (log-uniform) of the galaxies and randoms; p50/p99 latency beside the
    catalogs/s of the stream and of the plain path."""
    rng = np.random.default_rng(3)
    items = []
    for i in range(n_req):
        N = int(rng.choice([128, 256, 384, 512]))
        los = str(rng.choice(["yamamoto", "midpoint", "bisector"]))
        K = 0 if los == "yamamoto" else int(rng.choice([0, 2, 4, 6]))
        frac = float(10 ** rng.uniform(-1, 0))
        g, r, rn = _mock_subsets(torch, cat, gal_d, ran_d, rnb_d, rng, frac, 30.0)
        p = pkg.make_params(box_lo=cat.box_lo, box_len=cat.box_len, n_mesh=N, assign=3, ell_max=ELL_MAX, los=los,
                            order=K, compensate=True, precision=32, norm=1)
        items.append(dict(gal=g, ran=r, ran_nbar=rn, params=p, kedges=KEDGES, redges=REDGES))
    ctx = pkg.Context(dev.index)
    tuned = _tune_shapes(ctx, items)

    def alone(it):
        return ctx.pk_xi_multipoles(it["gal"], it["ran"], it["params"], it["kedges"], it["redges"],
                                    ran_nbar=it["ran_nbar"])

    for it in items:                       # compile kernels, build plans and tables
        alone(it)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for it in items:
        alone(it)
    t_seq = time.perf_counter() - t0
    shapes = {}
    for it in items:                       # the smallest request of every shape warms every slot
        key = (it["params"].n_mesh, int(it["params"].los), it["params"].order)
        if key not in shapes or it["gal"].shape[0] < shapes[key]["gal"].shape[0]:
            shapes[key] = it
    ctx.serve_start(n_slots=slots)
    ts = [ctx.submit(it["gal"], it["ran"], it["params"], it["kedges"], it["redges"], ran_nbar=it["ran_nbar"])
          for it in shapes.values() for _ in range(slots)]
    for t in ts:
        ctx.wait(t)
    ctx.serve_reset_stats()                # the same (warm) slots take the stream
    rate = 0.8 * len(items) / t_seq
    gaps = rng.exponential(1.0 / rate, size=len(items))
    ts = []
    t0 = time.perf_counter()
    for it, gap in zip(items, gaps):
        time.sleep(gap)
        ts.append(ctx.submit(it["gal"], it["ran"], it["params"], it["kedges"], it["redges"], ran_nbar=it["ran_nbar"]))
    for t in ts:
        ctx.wait(t)
    t_stream = time.perf_counter() - t0
    st = ctx.serve_stats()
    ctx.serve_stop()
    ctx.close()
    return {"requests": len(items), "slots": slots,
            "mix": "meshes 128/256/384/512^3, random LOS, order in {0,2,4,6}, 10-100 % of the galaxies and randoms "
                   "(log-uniform), P_ell+xi_ell, FP32",
            "sequential_catalogs_per_s": len(items) / t_seq,
            "poisson_rate_per_s": rate, "poisson_catalogs_per_s": len(items) / t_stream,
            "p50_latency_s": st["p50_s"], "p99_latency_s": st["p99_s"],
            "run_p50_s": st["run_p50_s"], "run_p99_s": st["run_p99_s"], "mean_queue_s": st["mean_queue_s"],
            "peak_hbm_gb": st["peak_hbm_bytes"] / 1e9, "autotune": tuned}


def _read_profile(pkg, ctx, reset):
    import ctypes
    buf = ctypes.create_string_buffer(1 << 16)
    pkg.lib().bym_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t, ctypes.c_int]
    pkg.lib().bym_profile_read(ctx._h, buf, len(buf), int(reset))
    return json.loads(buf.value.decode() or "{}")


def _max_over_ranks(ms, ws):
    """Largest per-rank time: the whole job is as slow as its slowest replica."""
    if ws == 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(local_ms, steps, ws):
    """Whole-job catalogs/s of ws independent replicas that each ran `steps`
    catalogs: all catalogs over the slowest rank's time (weak scaling)."""
    ms_max = _max_over_ranks(local_ms, ws)
    return ms_max, ws * steps / (ms_max / 1000.0)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def _roofline(prof, steps):
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    kernels = {}
    ours_launches = 0
    for name, e in prof.items():
        gbs = e["bytes"] / (e["ms"] * 1e-3) / 1e9 if e["ms"] > 0 else None
        kernels[name] = {"launches": e["launches"], "ms_total": e["ms"],
                         "ms_per_step": e["ms"] / steps, "algorithmic_GBps": gbs,
                         "frac_of_" + src + "_hbm": (gbs / hbm) if gbs else None}
        if not name.startswith("cufft"):
            ours_launches += e["launches"]
    ours = {k: v for k, v in prof.items() if not k.startswith("cufft")}
    if not ours:
        return None, kernels, ours_launches
    top = max(ours, key=lambda k: ours[k]["ms"])
    e = ours[top]
    per_launch_bytes = e["bytes"] / e["launches"]
    per_launch_s = e["ms"] / e["launches"] * 1e-3
    ach = per_launch_bytes / per_launch_s / 1e9
    roof = {"kernel": top, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "peak_source": src, "traffic": _ncu_traffic(top), "algorithmic_bytes_per_launch": per_launch_bytes}
    return roof, kernels, ours_launches


# the source files that define each kernel the roofline may name (the library's FFT passes)
KERNEL_SOURCES = {k: ["fft512.cu", "fft512.h"] for k in
                  ("fft_native_x_convolve", "fft_native_x_fwd", "fft_native_x_inv", "fft_native_y_fwd",
                   "fft_native_y_inv", "fft_native_z_fwd", "fft_native_z_inv")}


def _ncu_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    taken on the kernel's current source (profiles/traffic.md lists kernel | bytes |
    hash of the kernel's source files, or of all library sources for other kernels)."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    try:
        import paper_2102_08384_gb300.build as b
        build_id = b.file_hash(KERNEL_SOURCES[kernel]) if kernel in KERNEL_SOURCES else b.source_hash()
    except Exception:
        return None
    for line in open(path):
        parts = [p.strip() for p in line.strip().strip("|").split("|")]
        if len(parts) >= 3 and parts[0] == kernel and parts[2] == build_id:
            try:
                return float(parts[1])
            except ValueError:
                return None
    return None


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
