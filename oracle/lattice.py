"""Lattice geometry, gamma matrices and momenta (test infrastructure; oracle).

Conventions (the paper fixes none of them; App. A only says the GPU code may use
another spin basis internally):
  * site lex(x,y,z,t) = x + X*(y + Y*(z + Z*t)); parity (x+y+z+t) mod 2, even = 0;
    checkerboard index = lex // 2 (needs X even).
  * field arrays are indexed [t][z][y][x]; mu = 0:x 1:y 2:z 3:t.
  * Euclidean hermitian chiral gamma matrices
        gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = 1,2,3 -> x,y,z)
        gamma_4 = [[0, 1], [1, 0]]                   (t)
        gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1).
  * Gamma_b = g1^b0 g2^b1 g3^b2 g4^b3 for bitmask b = 0..15 (Gamma_0 = 1).
  * momenta p = 2 pi n / L with n in Z^3, |n|^2 <= P, ordered nz, ny, nx
    (outer to inner), each ascending; the phase of site x is exp(-i p.x).
"""
from __future__ import annotations

import numpy as np

AXIS = {0: 3, 1: 2, 2: 1, 3: 0}  # mu -> array axis of a [t][z][y][x] field

_s1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_s2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_s3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = [
    _block(_Z2, -1j * _s1, 1j * _s1, _Z2),
    _block(_Z2, -1j * _s2, 1j * _s2, _Z2),
    _block(_Z2, -1j * _s3, 1j * _s3, _Z2),
    _block(_Z2, _I2, _I2, _Z2),
]
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=np.complex128)


def gamma_b(b: int) -> np.ndarray:
    """Gamma_b = g1^b0 g2^b1 g3^b2 g4^b3."""
    m = ID4.copy()
    for k in range(4):
        if (b >> k) & 1:
            m = m @ GAMMA[k]
    return m


GAMMAS16 = [gamma_b(b) for b in range(16)]


def coords(dims):
    """Integer coordinate arrays x, y, z, t, each of shape [T][Z][Y][X]."""
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return x, y, z, t


def lex_index(dims):
    X, Y, Z, T = dims
    x, y, z, t = coords(dims)
    return x + X * (y + Y * (z + Z * t))


def parity(dims):
    x, y, z, t = coords(dims)
    return (x + y + z + t) % 2


def cb_index(dims):
    """Index within its checkerboard: lex // 2."""
    return lex_index(dims) // 2


def momenta(p2max: int):
    """List of integer momenta n = (nx, ny, nz) with |n|^2 <= p2max."""
    m = int(np.floor(np.sqrt(p2max)))
    out = []
    for nz in range(-m, m + 1):
        for ny in range(-m, m + 1):
            for nx in range(-m, m + 1):
                if nx * nx + ny * ny + nz * nz <= p2max:
                    out.append((nx, ny, nz))
    return out
