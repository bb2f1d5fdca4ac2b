"""Write tests/golden/survey512_order4.json: FP64 oracle multipoles of the 512^3 survey workload.

The workload is the benchmark's: the seed-1 lognormal cap (1e6 galaxies and 1e7 randoms in a
30 degree cap over 800-1600 Mpc/h, FKP weights with P0 = 1e4, Kaiser f = 0.7, b = 2), painted
with TSC on a 512^3 mesh with compensation, P_ell(k) on the k bins 0.01-0.25 h/Mpc (dk = 0.01)
and xi_ell(r) on the r bins 10-190 Mpc/h (dr = 10), ell = 0, 2, 4, order 4, for the midpoint
(eq. FFT-midpoint, eq. xi-parity-all-estimator) and the bisector (eq. bisector-pk-fft, Sec. 6)
lines of sight, FKP normalisation.

Only ``oracle`` (its streamed loop order, pinned to the plain estimators) and the seeded
catalog generator ``synth`` are used.  The file also records a fingerprint of the catalog
(counts and SHA-256 of the float32 arrays) so that a test can refuse to compare against a
catalog generated differently, and the wall time of each line of sight with the host's core
count (the measured cost of the FP64 oracle on this workload).

Usage: python tests/golden/make_survey512.py [--mesh 512] [--out PATH]
"""
import argparse
import hashlib
import json
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import streamed  # noqa: E402
from synth import lognormal_cap_catalog  # noqa: E402

KEDGES = np.round(np.arange(0.01, 0.2501, 0.01), 10)
REDGES = np.arange(10.0, 190.01, 10.0)


def catalog():
    return lognormal_cap_catalog(seed=1, n_gal=1_000_000, ran_factor=10.0, half_angle_deg=30.0, r_min=800.0,
                                 r_max=1600.0, gen_mesh=256)


def fingerprint(cat):
    return {"n_gal": int(len(cat.gal)), "n_ran": int(len(cat.ran)),
            "gal_sha256": hashlib.sha256(np.ascontiguousarray(cat.gal).tobytes()).hexdigest(),
            "ran_sha256": hashlib.sha256(np.ascontiguousarray(cat.ran).tobytes()).hexdigest(),
            "ran_nbar_sha256": hashlib.sha256(np.ascontiguousarray(cat.ran_nbar).tobytes()).hexdigest(),
            "box_lo": [float(v) for v in cat.box_lo], "box_len": float(cat.box_len)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mesh", type=int, default=512)
    ap.add_argument("--out", default=os.path.join(ROOT, "tests", "golden", "survey512_order4.json"))
    args = ap.parse_args()
    cat = catalog()
    out = {"what": "FP64 oracle (oracle.streamed) P_ell and xi_ell, ell = 0, 2, 4, order 4, TSC compensated, "
                   "FKP normalisation, on the seed-1 survey-like lognormal cap",
           "n_mesh": args.mesh, "assign": 3, "compensate": True, "order": 4, "ell_max": 4, "norm": 1,
           "kedges": KEDGES.tolist(), "redges": REDGES.tolist(), "catalog": fingerprint(cat),
           "host": {"cores": os.cpu_count(), "machine": platform.machine(), "numpy": np.__version__},
           "los": {}}
    for los in ("midpoint", "bisector"):
        t0 = time.perf_counter()

        def progress(kind, done, total):
            if kind != "unit" or done % 25 == 0 or done == total:
                print(f"{los} {kind} {done}/{total} {time.perf_counter() - t0:.0f} s", flush=True)
        r = streamed.pk_xi_multipoles(cat.gal, cat.ran, cat.ran_nbar, N=args.mesh, box_lo=cat.box_lo,
                                      box_len=cat.box_len, assign=3, ell_max=4, los=los, order=4, kedges=KEDGES,
                                      redges=REDGES, compensate=True, norm=1, progress=progress)
        wall = time.perf_counter() - t0
        out["los"][los] = {"pk": r["pk"].tolist(), "k_mean": r["k_mean"].tolist(), "n_modes": r["n_modes"].tolist(),
                           "xi": r["xi"].tolist(), "r_mean": r["r_mean"].tolist(), "n_cells": r["n_cells"].tolist(),
                           "oracle_wall_s": wall, "units": streamed.work_units(los, 4, 4)}
        print(f"{los} done in {wall:.0f} s", flush=True)
    with open(args.out, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
