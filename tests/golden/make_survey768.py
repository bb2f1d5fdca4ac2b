"""Write tests/golden/survey768_yamamoto.json: FP64 oracle Yamamoto multipoles at 768^3.

The benchmark's seed-1 survey-like cap (1e6 galaxies, 1e7 randoms), TSC with compensation on a
768^3 mesh, P_ell(k) on 0.01-0.25 h/Mpc (dk = 0.01) and xi_ell(r) on 10-190 Mpc/h (dr = 10),
ell = 0, 2, 4, Yamamoto line of sight (eq. Yamamoto-estimator, eq. 2pcf-yama), FKP
normalisation.  The monopole does not depend on the line of sight, so it is also the expected
ell = 0 of the midpoint and bisector estimators on this mesh.  Only ``oracle`` (its streamed loop
order) and ``synth`` are used; the catalog fingerprint and the oracle's wall time are recorded.

Usage: python tests/golden/make_survey768.py [--out PATH]
"""
import argparse
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, HERE)

from make_survey512 import KEDGES, REDGES, catalog, fingerprint  # noqa: E402
from oracle import streamed  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "survey768_yamamoto.json"))
    args = ap.parse_args()
    cat = catalog()
    t0 = time.perf_counter()
    r = streamed.pk_xi_multipoles(cat.gal, cat.ran, cat.ran_nbar, N=768, box_lo=cat.box_lo, box_len=cat.box_len,
                                  assign=3, ell_max=4, los="yamamoto", order=0, kedges=KEDGES, redges=REDGES,
                                  compensate=True, norm=1)
    wall = time.perf_counter() - t0
    out = {"what": "FP64 oracle (oracle.streamed) Yamamoto P_ell and xi_ell, ell = 0, 2, 4, TSC compensated, FKP "
                   "normalisation, 768^3, on the seed-1 survey-like lognormal cap",
           "n_mesh": 768, "assign": 3, "compensate": True, "ell_max": 4, "norm": 1,
           "kedges": KEDGES.tolist(), "redges": REDGES.tolist(), "catalog": fingerprint(cat),
           "host": {"cores": os.cpu_count(), "machine": platform.machine(), "numpy": np.__version__},
           "pk": r["pk"].tolist(), "k_mean": r["k_mean"].tolist(), "n_modes": r["n_modes"].tolist(),
           "xi": r["xi"].tolist(), "r_mean": r["r_mean"].tolist(), "n_cells": r["n_cells"].tolist(),
           "oracle_wall_s": wall}
    with open(args.out, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", args.out, f"({wall:.0f} s)")


if __name__ == "__main__":
    main()
