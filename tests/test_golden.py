"""The oracle still reproduces its stored regression values (tests/golden/)."""
import json
import os

import numpy as np

from paper_2203_06777_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_golden_values(oracle_lib):
    with open(os.path.join(HERE, "golden", "oracle_2x2x2x4_ls4.json")) as fh:
        g = json.load(fh)
    dims, Ls, M5, mass, bc = tuple(g["dims"]), g["Ls"], g["M5"], g["mass"], tuple(g["bc"])
    U = synth.random_gauge(dims, seed=g["gauge_seed"])
    psi = synth.random_spinor(dims, Ls, seed=g["psi_seed"])
    idx = [tuple(i) for i in g["samples_index"]]
    fields = {
        "dhop": oracle_lib.dhop(dims, Ls, bc, U, psi),
        "dhop_dag": oracle_lib.dhop(dims, Ls, bc, U, psi, dag=True),
        "m": oracle_lib.m(dims, Ls, M5, mass, bc, U, psi),
        "mooee_inv": oracle_lib.mooee(dims, Ls, M5, mass, psi, inverse=True),
    }
    for name, f in fields.items():
        assert np.isclose(oracle_lib.norm2(f), g[name]["norm2"], rtol=1e-13)
        got = np.array([[f[i].real, f[i].imag] for i in idx])
        assert np.allclose(got, np.array(g[name]["samples"]), rtol=1e-12, atol=1e-13)
    assert np.isclose(oracle_lib.norm2(oracle_lib.mdagm(dims, Ls, M5, mass, bc, U, psi)), g["mdagm"]["norm2"],
                      rtol=1e-13)
    S, F, G = oracle_lib.force(dims, Ls, M5, mass, bc, U, psi)
    assert np.isclose(S, g["force"]["S"], rtol=1e-13)
    assert np.isclose(oracle_lib.norm2(F), g["force"]["F_norm2"], rtol=1e-12)
    assert np.isclose(oracle_lib.norm2(G), g["force"]["G_norm2"], rtol=1e-12)
    f0 = np.array([[z.real, z.imag] for z in F[0, 0, 0, 0, 3].ravel()])
    assert np.allclose(f0, np.array(g["force"]["F_000_mu3"]), rtol=1e-12, atol=1e-13)
    # the pseudofermion action and its force (an iterative solve to 1e-14: compared at 1e-10)
    phi = psi * oracle_lib.parity_mask(dims)[..., None, None, None]
    pf = g["pf_force"]
    Spf, X, Fpf, Gpf, _ = oracle_lib.pf_force(dims, Ls, M5, mass, bc, U, phi, tol=pf["tol"], maxiter=100000)
    assert np.isclose(Spf, pf["S"], rtol=1e-10)
    assert np.isclose(oracle_lib.norm2(X), pf["X_norm2"], rtol=1e-10)
    assert np.isclose(oracle_lib.norm2(Fpf), pf["F_norm2"], rtol=1e-10)
    assert np.isclose(oracle_lib.norm2(Gpf), pf["G_norm2"], rtol=1e-10)
