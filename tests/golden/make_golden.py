"""Write tests/golden/oracle_2x2x2x4_ls4.json from the FP64 oracle alone.

The paper prints no worked numerical example of the domain-wall operator, so the stored values
here are regression fixtures of the oracle (itself pinned by tests/test_oracle_pins.py): if a
later change to the oracle's arithmetic moves any of them, the golden test fails and the change
has to name the reading of the operator that justifies it.

Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2203_06777_gb300 import synth  # noqa: E402

DIMS, LS, M5, MASS, BC = (2, 2, 2, 4), 4, 1.8, 0.01, (1, 1, 1, -1)
SAMPLES = [(0, 0, 0, 0, 0, 0, 0), (1, 1, 0, 1, 2, 3, 1), (3, 0, 1, 1, 3, 2, 2), (2, 1, 1, 0, 1, 1, 0)]


def sample(f):
    return [[float(f[i].real), float(f[i].imag)] for i in SAMPLES]


def main():
    U = synth.random_gauge(DIMS, seed=9001)
    psi = synth.random_spinor(DIMS, LS, seed=9002)
    out = {"dims": DIMS, "Ls": LS, "M5": M5, "mass": MASS, "bc": BC, "gauge_seed": 9001, "psi_seed": 9002,
           "samples_index": SAMPLES}
    d = oracle.dhop(DIMS, LS, BC, U, psi)
    dd = oracle.dhop(DIMS, LS, BC, U, psi, dag=True)
    mm = oracle.m(DIMS, LS, M5, MASS, BC, U, psi)
    mi = oracle.mooee(DIMS, LS, M5, MASS, psi, inverse=True)
    mdm = oracle.mdagm(DIMS, LS, M5, MASS, BC, U, psi)
    S, F, G = oracle.force(DIMS, LS, M5, MASS, BC, U, psi)
    out["dhop"] = {"norm2": oracle.norm2(d), "samples": sample(d)}
    out["dhop_dag"] = {"norm2": oracle.norm2(dd), "samples": sample(dd)}
    out["m"] = {"norm2": oracle.norm2(mm), "samples": sample(mm)}
    out["mooee_inv"] = {"norm2": oracle.norm2(mi), "samples": sample(mi)}
    out["mdagm"] = {"norm2": oracle.norm2(mdm)}
    out["force"] = {"S": S, "F_norm2": oracle.norm2(F), "G_norm2": oracle.norm2(G),
                    "F_000_mu3": [[float(z.real), float(z.imag)] for z in F[0, 0, 0, 0, 3].ravel()]}
    # pseudofermion action phi^+ (Mpc^+ Mpc)^-1 phi on the odd sites of the same spinor
    phi = psi * oracle.parity_mask(DIMS)[..., None, None, None]
    Spf, X, Fpf, Gpf, _ = oracle.pf_force(DIMS, LS, M5, MASS, BC, U, phi, tol=1e-14, maxiter=100000)
    out["pf_force"] = {"tol": 1e-14, "S": Spf, "X_norm2": oracle.norm2(X), "F_norm2": oracle.norm2(Fpf),
                       "G_norm2": oracle.norm2(Gpf)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_2x2x2x4_ls4.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
