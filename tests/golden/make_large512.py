"""Write tests/golden/large512_bisector6.json: FP64 oracle multipoles of the large workload.

The workload: the seed-2 lognormal cap with 2e7 galaxies and 5e7 randoms (a 60 degree cap over
600-2000 Mpc/h, FKP weights with P0 = 1e4, Kaiser f = 0.7, b = 2), painted with TSC on a 512^3
mesh with compensation; the bisector line of sight at order 6 (beta <= 3, the 64 transforms of
J <= 7: eq. bisector-pk-fft, Sec. 6), ell = 0, 2, 4; P_ell(k) on the k bins 0.01-0.25 h/Mpc
(dk = 0.01) and xi_ell(r) on the r bins 10-190 Mpc/h (dr = 10); FKP normalisation.

Only ``oracle`` (its streamed loop order, pinned to the plain estimators) and the seeded catalog
generator ``synth`` are used.  The file records a fingerprint of the catalog (counts and SHA-256
of the float32 arrays), so that a test can refuse to compare against a catalog generated
differently, and the oracle's wall time with the host's core count.

Usage: python tests/golden/make_large512.py [--mesh 512] [--out PATH]
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
ORDER = 6


def catalog():
    return lognormal_cap_catalog(seed=2, n_gal=20_000_000, ran_factor=2.5, half_angle_deg=60.0, r_min=600.0,
                                 r_max=2000.0, gen_mesh=256)


def fingerprint(cat):
    return {"n_gal": int(len(cat.gal)), "n_ran": int(len(cat.ran)),
            "gal_sha256": hashlib.sha256(np.ascontiguousarray(cat.gal).tobytes()).hexdigest(),
            "ran_sha256": hashlib.sha256(np.ascontiguousarray(cat.ran).tobytes()).hexdigest(),
            "ran_nbar_sha256": hashlib.sha256(np.ascontiguousarray(cat.ran_nbar).tobytes()).hexdigest(),
            "box_lo": [float(v) for v in cat.box_lo], "box_len": float(cat.box_len)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mesh", type=int, default=512)
    ap.add_argument("--out", default=os.path.join(ROOT, "tests", "golden", "large512_bisector6.json"))
    args = ap.parse_args()
    cat = catalog()
    out = {"what": "FP64 oracle (oracle.streamed) P_ell and xi_ell, ell = 0, 2, 4, bisector order 6, TSC "
                   "compensated, FKP normalisation, on the seed-2 large lognormal cap",
           "n_mesh": args.mesh, "assign": 3, "compensate": True, "order": ORDER, "ell_max": 4, "norm": 1,
           "kedges": KEDGES.tolist(), "redges": REDGES.tolist(), "catalog": fingerprint(cat),
           "host": {"cores": os.cpu_count(), "machine": platform.machine(), "numpy": np.__version__},
           "los": {}}
    t0 = time.perf_counter()

    def progress(kind, done, total):
        if kind != "unit" or done % 50 == 0 or done == total:
            print(f"bisector {kind} {done}/{total} {time.perf_counter() - t0:.0f} s", flush=True)
    r = streamed.pk_xi_multipoles(cat.gal, cat.ran, cat.ran_nbar, N=args.mesh, box_lo=cat.box_lo,
                                  box_len=cat.box_len, assign=3, ell_max=4, los="bisector", order=ORDER,
                                  kedges=KEDGES, redges=REDGES, compensate=True, norm=1, progress=progress)
    wall = time.perf_counter() - t0
    out["los"]["bisector"] = {"pk": r["pk"].tolist(), "k_mean": r["k_mean"].tolist(),
                              "n_modes": r["n_modes"].tolist(), "xi": r["xi"].tolist(),
                              "r_mean": r["r_mean"].tolist(), "n_cells": r["n_cells"].tolist(),
                              "oracle_wall_s": wall, "units": streamed.work_units("bisector", ORDER, 4)}
    with open(args.out, "w") as fh:
        json.dump(out, fh, indent=1)
    print(f"bisector done in {wall:.0f} s; wrote {args.out}", flush=True)


if __name__ == "__main__":
    main()
