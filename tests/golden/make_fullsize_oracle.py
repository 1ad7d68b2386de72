#!/usr/bin/env python3
"""Writes the oracle's exponents e_j = eta_j^dag (Mh^dag Mh - 1) eta_j at the benchmark's full-size
lattices into ``tests/golden/oracle_exponents_<lattice>.json``.

Calls only ``oracle/`` (and the seeded input generators of ``paper_1211_1214_gb300.synth``, which
hold none of the method's arithmetic).  Each entry is one noise vector of the benchmark's noise
stream (Philox seed 2, hit index h) at one target mass, computed by the oracle's five-solve chain
(Sec. 1; Eq. 3; Eq. 8 with N = 1): four CGNR block solves to relative residual 1e-13 and the CGNR
solve of D(m2) to 1e-12, all in FP64.  The file is updated after every entry, so a long run can
be stopped and resumed; entries already present are skipped.

    python tests/golden/make_fullsize_oracle.py --lattice 64x32^3 --hits 0 1 --masses 0.018 0.015 0.010
    python tests/golden/make_fullsize_oracle.py --lattice 48x24^3 --hits 0 --masses 0.015

One 64x32^3 entry takes about an hour on eight busy x86 host cores (a few minutes per CGNR solve
on sixteen idle Arm cores) and about 8 GB of memory.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the physics of the two paper-shaped lattices (Sec. 2: 48x24^3 with 6^4 blocks, 64x32^3 with 8^4)
LATTICES = {
    "64x32^3": dict(dims=(64, 32, 32, 32), l=8, eps=0.2, csw=1.9, m1=0.02),
    "48x24^3": dict(dims=(48, 24, 24, 24), l=6, eps=0.2, csw=1.9, m1=0.02),
}
SEED = 2  # noise seed of the benchmark's step 0 (hit offset 0)


def golden_path(name: str) -> str:
    return os.path.join(HERE, "oracle_exponents_%s.json" % "x".join(map(str, LATTICES[name]["dims"])))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", choices=list(LATTICES), required=True)
    ap.add_argument("--hits", type=int, nargs="+", required=True)
    ap.add_argument("--masses", type=float, nargs="+", required=True)
    ap.add_argument("--out", default=None, help="write here instead of tests/golden/ (copy it there after)")
    args = ap.parse_args()

    from oracle import core as oc
    from paper_1211_1214_gb300 import synth

    w = LATTICES[args.lattice]
    path = args.out or golden_path(args.lattice)
    doc = {"lattice": list(w["dims"]), "block": w["l"], "eps": w["eps"], "gauge_seed": 1, "csw": w["csw"],
           "m1": w["m1"], "noise_seed": SEED, "tol_block": 1e-13, "tol_outer": 1e-12,
           "what": "oracle exponents e = eta^dag (Mh^dag Mh - 1) eta, Mh = A(m2)^-1 A(m1), five FP64 CGNR solves; "
                   "eta = Philox noise (seed, hit) on supp P",
           "written_by": "tests/golden/make_fullsize_oracle.py", "entries": []}
    if os.path.exists(path):
        doc = json.load(open(path))
    have = {(round(e["m2"], 12), e["hit"]) for e in doc["entries"]}

    t0 = time.perf_counter()
    U = synth.gauge_field(w["dims"], w["eps"], seed=1)
    lat = oc.Lattice(w["dims"], (w["l"],) * 4, U, w["csw"])
    del U
    nP = len(lat.suppP_sites())
    print(f"lattice ready in {time.perf_counter() - t0:.0f} s, |supp P| = {nP} sites", flush=True)
    for h in args.hits:
        eta = None
        for m2 in args.masses:
            if (round(m2, 12), h) in have:
                continue
            if eta is None:
                eta = lat.unpack(oc.noise_packed(SEED, h, 1, 12 * nP)[0])
            t = time.perf_counter()
            res = lat.exponent(w["m1"], m2, eta, tol_block=1e-13, tol_outer=1e-12)
            dt = time.perf_counter() - t
            doc["entries"].append({"m2": m2, "hit": h, "e": res["e"], "cgnr_iters": res["iters"],
                                   "seconds": round(dt, 1)})
            doc["entries"].sort(key=lambda e: (e["m2"], e["hit"]))
            tmp = path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(doc, f, indent=1)
            os.replace(tmp, path)
            print(f"m2={m2} hit={h}: e={res['e']!r} iters={res['iters']} {dt:.0f} s", flush=True)


if __name__ == "__main__":
    main()
