"""The spin tables of the float-float kernels against the gamma matrices (no GPU needed).

The float-float hopping and force kernels run one code path for every direction: the rank-2
projector (1 + S gamma_mu) is applied as h_k = psi_k + w_k psi_{p_k} (k = 0, 1) and the lower
spins are rebuilt as w'_j h_{q_j}, with w and w' read from two packed tables in
`csrc/ff_arith.cuh` (p = (3, 2) and q = (1, 0) for mu < 2, else (2, 3) and (0, 1)). This test
reads the tables from the source and checks that they reproduce (1 + S gamma_mu) row by row for
the chiral-basis gamma matrices of the operator's definition, both signs S, all four directions.
"""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2203_06777_gb300", "csrc", "ff_arith.cuh")

# chiral basis, mu = 0..3 <-> x, y, z, t
GAMMA = [
    np.array([[0, 0, 0, -1j], [0, 0, -1j, 0], [0, 1j, 0, 0], [1j, 0, 0, 0]]),
    np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]], dtype=complex),
    np.array([[0, 0, -1j, 0], [0, 0, 0, 1j], [1j, 0, 0, 0], [0, -1j, 0, 0]]),
    np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]], dtype=complex),
]
W = {0: 1, 1: -1, 2: 1j, 3: -1j}  # code -> multiplier; code ^ 1 negates


def table(name):
    text = open(SRC).read()
    m = re.search(name + r"\s*=\s*pack_w\(([^)]*)\)", text)
    assert m, f"{name} not found in {SRC}"
    codes = [int(v) for v in m.group(1).split(",")]
    assert len(codes) == 8
    return codes


def w(codes, mu, k, S):
    return W[codes[2 * mu + k] ^ (1 if S < 0 else 0)]


def test_gamma_basis_is_clifford():
    for a in range(4):
        for b in range(4):
            ac = GAMMA[a] @ GAMMA[b] + GAMMA[b] @ GAMMA[a]
            assert np.allclose(ac, 2 * np.eye(4) * (a == b))


@pytest.mark.parametrize("mu", [0, 1, 2, 3])
@pytest.mark.parametrize("S", [1, -1])
def test_projection_and_reconstruction_tables(mu, S):
    proj, recon = table("PROJ_W"), table("RECON_W")
    P = np.eye(4) + S * GAMMA[mu]
    p = (3, 2) if mu < 2 else (2, 3)
    q = (1, 0) if mu < 2 else (0, 1)
    e = np.eye(4)
    for k in (0, 1):  # upper rows: h_k = psi_k + w_k psi_{p_k}
        assert np.allclose(P[k], e[k] + w(proj, mu, k, S) * e[p[k]]), (mu, S, k)
    for j in (0, 1):  # lower rows: w'_j h_{q_j}
        assert np.allclose(P[2 + j], w(recon, mu, j, S) * P[q[j]]), (mu, S, j)
