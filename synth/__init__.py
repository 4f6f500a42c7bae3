"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds input preparation only: SU(3) gauge links, random gauge
transformations and Gaussian test vectors.  It contains none of the method's
arithmetic (no Dirac operator, no noise of the stochastic estimator, no solver,
no contraction).  Both sides consume the arrays produced here; neither side
imports the other.

Layouts (C order, complex128):
  links   [T][Z][Y][X][mu][3][3]  mu = 0:x 1:y 2:z 3:t, U_mu(x) row-major
  su3     [T][Z][Y][X][3][3]
  spinor  [T][Z][Y][X][4][3]      spin-major, colour-minor

Random numbers: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) evaluated at counter n gives a 64-bit word;
the top 53 bits give a uniform in (0, 1]; Box-Muller turns pairs into normals.

Gauge links (the paper's B55.32 ensemble is not available, so links are
synthetic): per (site, mu) draw a 3x3 complex matrix A with independent
N(0, 1/2) real and imaginary parts, set H = (A + A^dagger)/2 minus its trace
part, and U = exp(i eps H), then re-unitarise (Gram-Schmidt of rows 0 and 1,
row 2 = conj(row0 x row1)) so that det U = 1 to rounding.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """splitmix64 output for state seed + (counter+1)*golden (uint64 wraparound)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _uniform(seed: int, counter: np.ndarray) -> np.ndarray:
    z = splitmix64(seed, counter)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normals(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normals (n even) from counters offset .. offset+n-1."""
    assert n % 2 == 0
    c = np.arange(offset, offset + n, dtype=np.uint64)
    u = _uniform(seed, c)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(n, dtype=np.float64)
    out[0::2] = r * np.cos(2.0 * np.pi * u2)
    out[1::2] = r * np.sin(2.0 * np.pi * u2)
    return out


def _mm(a, b):
    return np.einsum("nij,njk->nik", a, b, optimize=False)


def _expm_i_eps_h(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*h) for a stack of 3x3 hermitian h: scaling and squaring + Taylor."""
    n = h.shape[0]
    s = 4
    a = (1j * eps / (1 << s)) * h
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), (n, 3, 3))
    # Horner form of sum_{k<=12} a^k/k!
    out = eye + a / 12.0
    for k in range(11, 0, -1):
        out = eye + _mm(a, out) / k
    for _ in range(s):
        out = _mm(out, out)
    return out


def reunitarise(u: np.ndarray) -> np.ndarray:
    """Project a stack of near-unitary 3x3 matrices onto SU(3) via its rows."""
    r0 = u[:, 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=1, keepdims=True)
    r1 = u[:, 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=1)


def random_su3(n: int, eps: float, seed: int) -> np.ndarray:
    """n matrices exp(i eps H) with H random traceless hermitian (counter-seeded)."""
    g = normals(seed, 18 * n).reshape(n, 9, 2)
    a = ((g[..., 0] + 1j * g[..., 1]) / np.sqrt(2.0)).reshape(n, 3, 3)
    h = 0.5 * (a + np.conj(np.transpose(a, (0, 2, 1))))
    tr = np.trace(h, axis1=1, axis2=2).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)
    return reunitarise(_expm_i_eps_h(h, eps))


def gauge_links(dims, eps: float, seed: int) -> np.ndarray:
    """Synthetic SU(3) links, complex128 [T][Z][Y][X][4][3][3]; dims = (X, Y, Z, T)."""
    X, Y, Z, T = dims
    V = X * Y * Z * T
    u = np.empty((V * 4, 3, 3), dtype=np.complex128)
    chunk = 1 << 20
    for s in range(0, V * 4, chunk):
        e = min(V * 4, s + chunk)
        # counters of link l start at 18*l so each link's draws are fixed
        g = normals(seed, 18 * (e - s), offset=18 * s).reshape(e - s, 9, 2)
        a = ((g[..., 0] + 1j * g[..., 1]) / np.sqrt(2.0)).reshape(e - s, 3, 3)
        h = 0.5 * (a + np.conj(np.transpose(a, (0, 2, 1))))
        tr = np.trace(h, axis1=1, axis2=2).real / 3.0
        h = h - tr[:, None, None] * np.eye(3)
        u[s:e] = reunitarise(_expm_i_eps_h(h, eps))
    return u.reshape(T, Z, Y, X, 4, 3, 3)


def unit_links(dims) -> np.ndarray:
    X, Y, Z, T = dims
    u = np.zeros((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def gauge_transform_field(dims, seed: int, eps: float = 3.0) -> np.ndarray:
    """Random SU(3) field G(x), complex128 [T][Z][Y][X][3][3]."""
    X, Y, Z, T = dims
    return random_su3(X * Y * Z * T, eps, seed).reshape(T, Z, Y, X, 3, 3)


def gaussian_spinors(dims, n: int, seed: int) -> np.ndarray:
    """n complex Gaussian spinor fields, complex128 [n][T][Z][Y][X][4][3]."""
    X, Y, Z, T = dims
    cnt = n * X * Y * Z * T * 12
    g = normals(seed, 2 * cnt).reshape(cnt, 2)
    return ((g[:, 0] + 1j * g[:, 1]) / np.sqrt(2.0)).reshape(n, T, Z, Y, X, 4, 3)


def network_weights(n_layers: int, channels: int, seed: int, scale: float = 0.05, identity: float = 1.0) -> np.ndarray:
    """Initial weights of a parallel-transport network with channels 1 -> C -> ... -> C -> 1,
    complex64 concatenated per layer in the [9 terms][4 spin factors][C_out][C_in] layout:
    Gaussian entries of standard deviation scale / sqrt(36 C_in) per component, plus
    `identity` on the local unit-spin term from input channel 0 to output channel 0
    (the unused local spin factors 2, 3 stay zero)."""
    out = []
    cnt = 0
    for l in range(n_layers):
        ci = 1 if l == 0 else channels
        co = 1 if l == n_layers - 1 else channels
        n = 36 * co * ci
        g = normals(seed, 2 * n, offset=cnt).reshape(n, 2)
        cnt += 2 * n
        w = ((g[:, 0] + 1j * g[:, 1]) * scale / np.sqrt(2.0 * 36 * ci)).reshape(9, 4, co, ci)
        w[0, 2:] = 0.0
        w[0, 0, 0, 0] += identity
        out.append(w.ravel())
    return np.concatenate(out).astype(np.complex64)


# Configurations of the synthetic workloads: lattice (X, Y, Z, T), link
# smearing eps, hopping parameter kappa, twisted mass a*mu.  Link seeds are
# 1000 + id, noise seeds 2000 + id.
CONFIGS = {
    "tiny_4x4x4x4": dict(dims=(4, 4, 4, 4), eps=0.3, kappa=0.16, amu=0.01, id=0),
    "mixed_16x16x16x32": dict(dims=(16, 16, 16, 32), eps=0.4, kappa=0.161, amu=0.0055, id=1),
    "tsm_32x32x32x64": dict(dims=(32, 32, 32, 64), eps=0.4, kappa=0.1612, amu=0.0055, id=2),
    "learned_16x16x16x32": dict(dims=(16, 16, 16, 32), eps=0.4, kappa=0.161, amu=0.0055, id=3),
}


def config_links(name: str) -> np.ndarray:
    c = CONFIGS[name]
    return gauge_links(c["dims"], c["eps"], 1000 + c["id"])
