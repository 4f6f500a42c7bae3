"""Twisted-mass Wilson-Dirac operator, full and even-odd (test infrastructure; oracle).

App. A, Eq. (A.1): D_TM = D_W + i mu gamma_5 tau_3 for the degenerate doublet.
The kappa (hopping-parameter) normalisation implied by the kappa^2 of Eq. (A.2):

    M_f psi(x) = R_f psi(x) - kappa * D psi(x)
    D psi(x)   = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                          + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu) ]
    R_f        = 1 + 2 i kappa (a mu) f gamma_5,   f = +1 (u), -1 (d)

so that M_u - M_d = 4 i kappa a mu gamma_5 (Sec. 2.3's M_u - M_d = 2 i mu a gamma_5
in physical units, M_phys = M / (2 kappa)).  Hops that cross the time boundary
pick up the factor `bc` (-1: antiperiodic, the default reading; the paper does not
state its boundary conditions).

Even-odd (Eq. A.2, asymmetric): with D_eo = P_e D P_o and D_oe = P_o D P_e,
    Mhat = R_ee - kappa^2 D_eo R_oo^{-1} D_oe
    bhat = b_e + kappa D_eo R_oo^{-1} b_o
    psi_o = R_oo^{-1} (b_o + kappa D_oe psi_e)                         (Eq. A.4)
The printed right-hand sides of (A.2) and (A.4) lack kappa and carry a spurious
R_ee^{-1}; the forms above are the Schur complement of M, and the tests check
that they reproduce M psi = b on the full lattice.

Fields are full-lattice arrays [..., T, Z, Y, X, 4, 3]; even-odd vectors are
full-lattice arrays that vanish on the other parity.
"""
from __future__ import annotations

import numpy as np

from .lattice import GAMMA, GAMMA5, ID4, parity

_TAX = -6  # time axis of a [..., T, Z, Y, X, 4, 3] spinor field
_SAX = {0: -3, 1: -4, 2: -5, 3: -6}  # mu -> axis of a spinor field
_LAX = {0: 3, 1: 2, 2: 1, 3: 0}  # mu -> axis of the [T,Z,Y,X,...] link array


def spin(m: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a 4x4 spin matrix to every site."""
    return np.einsum("st,...tc->...sc", m, psi)


def colour(u: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply the 3x3 colour matrix field u [T,Z,Y,X,3,3] site by site."""
    return np.einsum("...ab,...sb->...sa", u, psi)


def dagger(u: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(u, -1, -2))


def shift_fwd(psi: np.ndarray, mu: int, bc: float) -> np.ndarray:
    """psi(x + mu), with the boundary factor on the hop T-1 -> 0."""
    out = np.roll(psi, -1, axis=_SAX[mu])
    if mu == 3:
        idx = [slice(None)] * out.ndim
        idx[_TAX] = -1
        out[tuple(idx)] *= bc
    return out


def shift_bwd(psi: np.ndarray, mu: int, bc: float) -> np.ndarray:
    """psi(x - mu), with the boundary factor on the hop 0 -> T-1."""
    out = np.roll(psi, 1, axis=_SAX[mu])
    if mu == 3:
        idx = [slice(None)] * out.ndim
        idx[_TAX] = 0
        out[tuple(idx)] *= bc
    return out


def link_bwd(links: np.ndarray, mu: int) -> np.ndarray:
    """U_mu(x - mu) as a [T,Z,Y,X,3,3] field."""
    return np.roll(links[..., mu, :, :], 1, axis=_LAX[mu])


def hop(links: np.ndarray, psi: np.ndarray, bc: float = -1.0, dag: bool = False) -> np.ndarray:
    """D psi (dag=False) or D^dagger psi = gamma_5 D gamma_5 psi (dag=True)."""
    s = 1.0 if dag else -1.0  # forward projector (1 + s gamma_mu)
    out = np.zeros_like(psi)
    for mu in range(4):
        fwd = colour(links[..., mu, :, :], shift_fwd(psi, mu, bc))
        bwd = colour(dagger(link_bwd(links, mu)), shift_bwd(psi, mu, bc))
        out += spin(ID4 + s * GAMMA[mu], fwd) + spin(ID4 - s * GAMMA[mu], bwd)
    return out


def twist_matrix(kappa: float, amu: float, f: int) -> np.ndarray:
    """R_f = 1 + 2 i kappa amu f gamma_5."""
    return ID4 + 2j * kappa * amu * f * GAMMA5


def twist(psi, kappa, amu, f):
    return spin(twist_matrix(kappa, amu, f), psi)


def twist_inv(psi, kappa, amu, f):
    return spin(np.linalg.inv(twist_matrix(kappa, amu, f)), psi)


def apply_m(links, psi, kappa, amu, f=1, bc=-1.0):
    """M_f psi = R_f psi - kappa D psi (Eq. A.1, kappa normalisation)."""
    return twist(psi, kappa, amu, f) - kappa * hop(links, psi, bc)


def apply_m_dag(links, psi, kappa, amu, f=1, bc=-1.0):
    """M_f^dagger psi = R_{-f} psi - kappa D^dagger psi."""
    return twist(psi, kappa, amu, -f) - kappa * hop(links, psi, bc, dag=True)


def wilson_a(links, psi, kappa, bc=-1.0):
    """A = (M_u + M_d)/2 = 1 - kappa D (the Wilson operator D_W of Sec. 2.3)."""
    return psi - kappa * hop(links, psi, bc)


def mask(dims, p: int) -> np.ndarray:
    """1 on sites of parity p, 0 elsewhere, broadcastable to a spinor field."""
    return (parity(dims) == p).astype(np.float64)[..., None, None]


def project(psi, dims, p):
    return psi * mask(dims, p)


def mhat(links, psi_e, kappa, amu, f=1, bc=-1.0, dims=None):
    """Mhat psi_e = R_ee psi_e - kappa^2 D_eo R_oo^{-1} D_oe psi_e (Eq. A.2)."""
    me, mo = mask(dims, 0), mask(dims, 1)
    t = twist_inv(mo * hop(links, me * psi_e, bc), kappa, amu, f)
    return me * (twist(psi_e, kappa, amu, f) - kappa * kappa * hop(links, mo * t, bc))


def mhat_dag(links, psi_e, kappa, amu, f=1, bc=-1.0, dims=None):
    """Mhat^dagger = R_ee^dagger - kappa^2 D_oe^dagger R_oo^{-dagger} D_eo^dagger."""
    me, mo = mask(dims, 0), mask(dims, 1)
    t = twist_inv(mo * hop(links, me * psi_e, bc, dag=True), kappa, amu, -f)
    return me * (twist(psi_e, kappa, amu, -f) - kappa * kappa * hop(links, mo * t, bc, dag=True))


def prep_source(links, b, kappa, amu, f=1, bc=-1.0, dims=None):
    """bhat_e = b_e + kappa D_eo R_oo^{-1} b_o."""
    me, mo = mask(dims, 0), mask(dims, 1)
    return me * (b + kappa * hop(links, mo * twist_inv(mo * b, kappa, amu, f), bc))


def reconstruct_odd(links, psi_e, b, kappa, amu, f=1, bc=-1.0, dims=None):
    """psi_o = R_oo^{-1} (b_o + kappa D_oe psi_e) (Eq. A.4, Schur-complement form)."""
    me, mo = mask(dims, 0), mask(dims, 1)
    return mo * twist_inv(mo * b + kappa * mo * hop(links, me * psi_e, bc), kappa, amu, f)


def dense_matrix(links, kappa, amu, f=1, bc=-1.0, which="M"):
    """The operator as a dense (12V x 12V) matrix, built column by column.

    which: "M" (M_f), "D" (hopping term), "A" (Wilson part 1 - kappa D).
    Column j is the operator applied to the j-th unit vector (site-major,
    then spin, then colour, matching the flattened [T,Z,Y,X,4,3] order).
    """
    shape = links.shape[:4] + (4, 3)
    n = int(np.prod(shape))
    cols = np.eye(n, dtype=np.complex128).reshape((n,) + shape)
    if which == "M":
        out = apply_m(links, cols, kappa, amu, f, bc)
    elif which == "D":
        out = hop(links, cols, bc)
    elif which == "A":
        out = wilson_a(links, cols, kappa, bc)
    else:
        raise ValueError(which)
    return out.reshape(n, n).T.copy()


def _site_shift(dims, site, mu, step):
    """Neighbour (t, z, y, x) of `site` one step along mu, and the time-boundary factor flag."""
    X, Y, Z, T = dims
    t, z, y, x = site
    crosses = False
    if mu == 0:
        x = (x + step) % X
    elif mu == 1:
        y = (y + step) % Y
    elif mu == 2:
        z = (z + step) % Z
    else:
        crosses = (t + step) >= T or (t + step) < 0
        t = (t + step) % T
    return (t, z, y, x), crosses


def apply_m_at(links, psi, site, kappa, amu, f=1, bc=-1.0):
    """(M_f psi)(x) at one site x = (t, z, y, x), from the definition (Eq. A.1):
    R_f psi(x) - kappa sum_mu [(1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)].
    Lets full-size fields be checked at sampled sites."""
    dims = (links.shape[3], links.shape[2], links.shape[1], links.shape[0])
    out = twist_matrix(kappa, amu, f) @ psi[site]
    for mu in range(4):
        fw, cf = _site_shift(dims, site, mu, +1)
        bw, cb = _site_shift(dims, site, mu, -1)
        u = links[site][mu]
        ub = links[bw][mu]
        pf = psi[fw] * (bc if cf else 1.0)
        pb = psi[bw] * (bc if cb else 1.0)
        out = out - kappa * ((ID4 - GAMMA[mu]) @ (pf @ u.T) + (ID4 + GAMMA[mu]) @ (pb @ np.conj(ub)))
    return out
