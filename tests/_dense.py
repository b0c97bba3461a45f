"""Dense brute-force matrices of the domain-wall operator on tiny lattices (test pins).

Built independently of the oracle's stencil loops: every hop is a 12x12 Kronecker block
kron(spin projector, colour link) placed at (x, x +- mu) of a 12V x 12V matrix, and the fifth
dimension enters through Kronecker products with identities and with the Ls x Ls s-shift
matrices. Index order matches the canonical field layout psi[t,z,y,x,s,spin,colour].

The gamma matrices are typed out as explicit tables in the chiral basis (the convention the
operator is written in), not derived the way the oracle derives them.
"""
import numpy as np

GX = np.array([[0, 0, 0, -1j], [0, 0, -1j, 0], [0, 1j, 0, 0], [1j, 0, 0, 0]])
GY = np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]], dtype=complex)
GZ = np.array([[0, 0, -1j, 0], [0, 0, 0, 1j], [1j, 0, 0, 0], [0, -1j, 0, 0]])
GT = np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]], dtype=complex)
GAMMA = np.stack([GX, GY, GZ, GT])
G5 = np.diag([1.0, 1.0, -1.0, -1.0]).astype(complex)
I4 = np.eye(4, dtype=complex)


def lex(dims, c):
    lx, ly, lz, lt = dims
    return c[0] + lx * (c[1] + ly * (c[2] + lz * c[3]))


def all_coords(dims):
    lx, ly, lz, lt = dims
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    yield (x, y, z, t)


def dense_wilson_hop_4d(dims, bc, U, dag=False):
    """12V x 12V matrix of the 4D hopping term, index (site, spin, colour)."""
    V = int(np.prod(dims))
    H = np.zeros((12 * V, 12 * V), dtype=complex)
    Ucan = U.reshape(V, 4, 3, 3)  # canonical [t,z,y,x] flattens to the lexicographic site index
    sf = 1.0 if dag else -1.0  # forward projector (1 + sf gamma)
    for c in all_coords(dims):
        x = lex(dims, c)
        for mu in range(4):
            cf = list(c)
            cf[mu] = (c[mu] + 1) % dims[mu]
            cb = list(c)
            cb[mu] = (c[mu] - 1) % dims[mu]
            pf = bc[mu] if c[mu] == dims[mu] - 1 else 1
            pb = bc[mu] if c[mu] == 0 else 1
            xf, xb = lex(dims, cf), lex(dims, cb)
            H[12 * x:12 * x + 12, 12 * xf:12 * xf + 12] += pf * np.kron(I4 + sf * GAMMA[mu], Ucan[x, mu])
            H[12 * x:12 * x + 12, 12 * xb:12 * xb + 12] += pb * np.kron(I4 - sf * GAMMA[mu],
                                                                        Ucan[xb, mu].conj().T)
    return H


def dense_dhop(dims, Ls, bc, U, dag=False):
    """(12 V Ls)^2 matrix of Dhop (identity in s), index (site, s, spin, colour)."""
    V = int(np.prod(dims))
    H = dense_wilson_hop_4d(dims, bc, U, dag).reshape(V, 12, V, 12)
    D = np.einsum("aibj,st->asibtj", H, np.eye(Ls))
    n = V * Ls * 12
    return D.reshape(n, n)


def s_shift(Ls, k):
    """Ls x Ls matrix with ones at (s, s + k) for 0 <= s + k < Ls."""
    return np.eye(Ls, k=k)


def corner(Ls, r, c):
    e = np.zeros((Ls, Ls))
    e[r, c] = 1.0
    return e


def dense_mooee_site(Ls, M5, mass):
    """(4 Ls) x (4 Ls) matrix of Mooee on one site and colour, index (s, spin)."""
    Pp = 0.5 * (I4 + G5)
    Pm = 0.5 * (I4 - G5)
    K = (5.0 - M5) * np.eye(4 * Ls, dtype=complex)
    K -= np.kron(s_shift(Ls, 1), Pm)          # -P- psi_{s+1}
    K -= np.kron(s_shift(Ls, -1), Pp)         # -P+ psi_{s-1}
    K += mass * np.kron(corner(Ls, Ls - 1, 0), Pm)   # +m P- psi_0 at s = Ls-1
    K += mass * np.kron(corner(Ls, 0, Ls - 1), Pp)   # +m P+ psi_{Ls-1} at s = 0
    return K


def dense_mooee(dims, Ls, M5, mass):
    V = int(np.prod(dims))
    return np.kron(np.eye(V), np.kron(dense_mooee_site(Ls, M5, mass), np.eye(3)))


def dense_m(dims, Ls, M5, mass, bc, U):
    return dense_mooee(dims, Ls, M5, mass) - 0.5 * dense_dhop(dims, Ls, bc, U)


def parity_index(dims, Ls, parity):
    """Flat indices of the field components on sites of the given parity."""
    idx = []
    for c in all_coords(dims):
        if sum(c) % 2 == parity:
            base = lex(dims, c) * Ls * 12
            idx.extend(range(base, base + Ls * 12))
    return np.array(idx)


def dense_schur_odd(dims, Ls, M5, mass, bc, U):
    """Mpc = M_oo - M_oe M_ee^-1 M_eo taken directly from blocks of the dense M."""
    M = dense_m(dims, Ls, M5, mass, bc, U)
    e = parity_index(dims, Ls, 0)
    o = parity_index(dims, Ls, 1)
    Mee = M[np.ix_(e, e)]
    Meo = M[np.ix_(e, o)]
    Moe = M[np.ix_(o, e)]
    Moo = M[np.ix_(o, o)]
    return Moo - Moe @ np.linalg.solve(Mee, Meo), o
