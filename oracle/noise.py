"""Z4 noise for the stochastic trace estimator (test infrastructure; oracle).

Sec. 2.1 (Eqs. eq1, eq2) asks for noise entries from Z4 = {1, i, -1, -i} or
Z2 x iZ2 with E[eta] = 0 and E[eta eta^dagger] = 1.  Reading: entries are
(s1 + i s2)/sqrt(2) with independent random signs s1, s2 (Z2 x iZ2, which is Z4
rotated by pi/4), so |eta| = 1.  The option {1, i, -1, -i} takes the two bits
as a quadrant instead.

The paper draws the numbers with RANLUX on the host.  Here the noise is a
function of (seed, noise index r, site, spin, colour) through splitmix64
(Steele, Lea & Flood, OOPSLA 2014), written out below from its published
definition: state_n = seed + (n + 1) * 0x9E3779B97F4A7C15 (mod 2^64), then
z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
z ^= z >> 31.  Counter n = (r * V + lex) * 12 + 3 * spin + colour.
Bit 0 of the output gives s1 (0 -> +1), bit 1 gives s2.

Time dilution (Sec. 2.3): the noise space is split into subspaces and a source
fills one of them.  With the subspaces taken as sets of time slices, a source
keeps the entries of a full noise vector on the slices t = t0 (mod dt) and is
zero elsewhere: dt = T gives one slice per source, a smaller dt the coherent
sources of several far-apart slices.  The dt sources t0 = 0 .. dt-1 of one noise
vector sum to it (the direct sum of the subspaces).
"""
from __future__ import annotations

import numpy as np

from .lattice import lex_index

GOLDEN = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB


def splitmix64(seed: int, n: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (n.astype(np.uint64) + np.uint64(1)) * np.uint64(GOLDEN)
        z = z ^ (z >> np.uint64(30))
        z = z * np.uint64(MIX1)
        z = z ^ (z >> np.uint64(27))
        z = z * np.uint64(MIX2)
        z = z ^ (z >> np.uint64(31))
    return z


def z4_noise(dims, seed: int, r: int, quadrant: bool = False) -> np.ndarray:
    """Noise vector number r, complex128 [T][Z][Y][X][4][3]."""
    X, Y, Z, T = dims
    V = X * Y * Z * T
    lex = lex_index(dims).astype(np.uint64)
    a = np.arange(4, dtype=np.uint64)[:, None]
    c = np.arange(3, dtype=np.uint64)[None, :]
    n = (np.uint64(r) * np.uint64(V) + lex[..., None, None]) * np.uint64(12) + np.uint64(3) * a + c
    z = splitmix64(seed, n)
    b0 = (z & np.uint64(1)).astype(np.int64)
    b1 = ((z >> np.uint64(1)) & np.uint64(1)).astype(np.int64)
    if quadrant:
        q = b0 + 2 * b1
        return np.array([1, 1j, -1, -1j], dtype=np.complex128)[q]
    s1 = 1.0 - 2.0 * b0
    s2 = 1.0 - 2.0 * b1
    return (s1 + 1j * s2) / np.sqrt(2.0)


def time_diluted(eta: np.ndarray, t0: int, dt: int) -> np.ndarray:
    """eta ([T][Z][Y][X][4][3]) on the time slices t = t0 (mod dt), zero elsewhere (Sec. 2.3)."""
    T = eta.shape[0]
    if not (1 <= dt <= T and 0 <= t0 < dt):
        raise ValueError("need 1 <= dt <= T and 0 <= t0 < dt")
    out = np.zeros_like(eta)
    out[t0::dt] = eta[t0::dt]
    return out
