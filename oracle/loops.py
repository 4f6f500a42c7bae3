"""Loop contractions, estimators, momentum projection, HPE and TSM (test infrastructure; oracle).

Per site the paper forms the colour-traced Dirac outer product of the two
vectors it contracts (App. A, "Contraction kernels"):
    C_ab(x) = sum_c conj(xi_{a c}(x)) phi_{b c}(x),
from which the loop of any insertion X follows as
    l_X(x) = xi^dagger(x) X phi(x) = sum_ab X_ab C_ab(x).
Estimators (vectors for one noise eta and solution s = M_u^{-1} eta):
  standard       (xi, phi) = (eta, s)                    -> Tr[M_u^{-1} X]     (Eq. loopSt)
  one-end        (xi, phi) = (g5 s, s), factor -4 i kappa amu
                                                         -> Tr[(M_u^{-1}-M_d^{-1}) X]  (Eq. loopVv)
  generalised    (xi, phi) = (g5 s, g5 D_W s), factor 2  -> Tr[(M_u^{-1}+M_d^{-1}) X]  (Eq. loopStD)
  HPE remainder  (xi, phi) = (eta, (BH)^4 s)             -> Tr[X (BH)^4 M_u^{-1}]      (Eq. loopHPE1)
Factors are in the kappa normalisation of `operator`; Eq. (loopVv) prints
+2 i mu a on its left side, the resolvent identity (Eq. vvTrick) gives the minus
sign used here.

One-derivative insertions (App. A mentions a covariant-derivative kernel but
does not define it).  Reading: the symmetric covariant derivative
    l^mu_ab(x) = 1/4 [ xi^+(x) U_mu(x) phi(x+mu) - xi^+(x+mu) U_mu(x)^+ phi(x)
                     + xi^+(x-mu) U_mu(x-mu) phi(x) - xi^+(x) U_mu(x-mu)^+ phi(x-mu) ]_ab
with the same time-boundary factor as the operator.

Momentum projection (App. A, "Interfaces and workflow": FFT over space, then a
cut in p^2): L(t, p) = sum_{x vec} exp(-i p.x) C(x vec, t), p = 2 pi n / L.
"""
from __future__ import annotations

import numpy as np

from . import operator as op
from .lattice import GAMMA5, momenta


def bilinear(xi, phi):
    """C_ab(x) = sum_c conj(xi_ac(x)) phi_bc(x); shape [..., T, Z, Y, X, 4, 4]."""
    return np.einsum("...ac,...bc->...ab", np.conj(xi), phi)


def loop_from_c(c, x_matrix):
    """l_X = sum_ab X_ab C_ab."""
    return np.einsum("ab,...ab->...", x_matrix, c)


def g5(psi):
    return op.spin(GAMMA5, psi)


def derivative_bilinear(links, xi, phi, mu, bc=-1.0):
    """The symmetric covariant-derivative bilinear l^mu_ab(x) written term by term."""
    u = links[..., mu, :, :]
    ub = op.link_bwd(links, mu)
    t1 = bilinear(xi, op.colour(u, op.shift_fwd(phi, mu, bc)))
    t2 = bilinear(op.shift_fwd(xi, mu, bc), op.colour(op.dagger(u), phi))
    t3 = bilinear(op.shift_bwd(xi, mu, bc), op.colour(ub, phi))
    t4 = bilinear(xi, op.colour(op.dagger(ub), op.shift_bwd(phi, mu, bc)))
    return 0.25 * (t1 - t2 + t3 - t4)


def project_momenta(c, dims, p2max):
    """L[..., t, ip, ...] = sum_xyz exp(-2 pi i (nx x/X + ny y/Y + nz z/Z)) c[..., t, z, y, x, ...].

    `c` has site axes [t][z][y][x] followed by two trailing (Dirac) axes.
    """
    X, Y, Z, T = dims
    plist = momenta(p2max)
    z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    out = []
    for nx, ny, nz in plist:
        ph = np.exp(-2j * np.pi * (nx * x / X + ny * y / Y + nz * z / Z))
        out.append(np.einsum("zyx,...tzyxab->...tab", ph, c))
    return np.stack(out, axis=-3)


def pair(estimator, links, eta, s, kappa, amu, bc=-1.0):
    """The (xi, phi) pair of an estimator for noise eta and s = M_u^{-1} eta."""
    if estimator == "standard":
        return eta, s
    if estimator == "one_end":
        return g5(s), s
    if estimator == "gen_one_end":
        return g5(s), g5(op.wilson_a(links, s, kappa, bc))
    if estimator == "hpe":
        return eta, bh_power(links, s, kappa, amu, 4, bc)
    raise ValueError(estimator)


def prefactor(estimator, kappa, amu):
    return {"standard": 1.0, "one_end": -4j * kappa * amu, "gen_one_end": 2.0, "hpe": 1.0}[estimator]


def bh_apply(links, psi, kappa, amu, bc=-1.0, f=1):
    """B H psi with B = R_f^{-1}, H = -kappa D, so that M_f = B^{-1} + H (Eq. HPE)."""
    return op.twist_inv(-kappa * op.hop(links, psi, bc), kappa, amu, f)


def bh_power(links, psi, kappa, amu, k, bc=-1.0, f=1):
    for _ in range(k):
        psi = bh_apply(links, psi, kappa, amu, bc, f)
    return psi


def hpe_truncated_inverse(links, psi, kappa, amu, bc=-1.0, f=1):
    """(B - BHB + (BH)^2 B - (BH)^3 B) psi: the four exact terms of Eq. (HPE)."""
    b = op.twist_inv(psi, kappa, amu, f)
    out = b.copy()
    term = b
    for k in range(1, 4):
        term = bh_apply(links, term, kappa, amu, bc, f)
        out = out + ((-1) ** k) * term
    return out


def hpe_exact_site_block(links, kappa, amu, site, bc=-1.0, f=1):
    """12x12 diagonal block at `site` (t,z,y,x) of B - BHB + (BH)^2 B - (BH)^3 B, by brute force.

    Applies the truncated inverse to the 12 unit vectors supported on `site` and
    reads the result back at the same site; columns are (spin, colour) flattened.
    """
    shape = links.shape[:4] + (4, 3)
    cols = np.zeros((12,) + shape, dtype=np.complex128)
    for j in range(12):
        cols[(j,) + tuple(site) + (j // 3, j % 3)] = 1.0
    out = hpe_truncated_inverse(links, cols, kappa, amu, bc, f)
    blk = out[(slice(None),) + tuple(site)].reshape(12, 12)
    return blk.T.copy()


def hpe_exact_c(links, kappa, amu, site, bc=-1.0, f=1):
    """Exact HPE part in the C convention: C_ab = sum_c E[(b,c),(a,c)] (so l_X = Tr[X E])."""
    blk = hpe_exact_site_block(links, kappa, amu, site, bc, f).reshape(4, 3, 4, 3)
    e_spin = np.einsum("acbc->ab", blk)  # colour trace, E_ab
    return e_spin.T.copy()


def tsm_estimate(f_hp, f_lp_pair, f_lp_fresh):
    """Eq. (estiTSM) applied to a loop functional f:
    (1/N_HP) sum_r [f(s_r^HP) - f(s_r^LP)] + (1/N_LP) sum_j f(s_j^LP).
    The second sum is read as running over the N_LP fresh noise vectors j."""
    f_hp = np.asarray(f_hp)
    f_lp_pair = np.asarray(f_lp_pair)
    f_lp_fresh = np.asarray(f_lp_fresh)
    return (f_hp - f_lp_pair).mean(axis=0) + f_lp_fresh.mean(axis=0)


def tsm_error(f_hp, f_lp_pair, f_lp_fresh):
    """Standard error of the TSM estimate: sqrt(var(f_HP - f_LP)/N_HP + var(f_LP)/N_LP)."""
    d = np.asarray(f_hp) - np.asarray(f_lp_pair)
    lp = np.asarray(f_lp_fresh)
    return np.sqrt(d.var(axis=0, ddof=1) / d.shape[0] + lp.var(axis=0, ddof=1) / lp.shape[0])


def binary_storage_files(per_noise):
    """Base-2 storage of per-noise loop arrays (App. A, "Binary storage system").

    File k holds the sum of the 2^k noise vectors with indices 2^k - 1 .. 2^(k+1) - 2
    (File.1 = noise 0, File.2 = noise 1 + 2, File.4 = noise 3..6, ...).
    Returns {2^k: summed array} for every complete file.
    """
    files = {}
    k = 0
    start = 0
    n = len(per_noise)
    while start + (1 << k) <= n:
        files[1 << k] = np.sum(per_noise[start:start + (1 << k)], axis=0)
        start += 1 << k
        k += 1
    return files


def binary_storage_reconstruct(files, n):
    """Sum over a set of noise vectors whose size is n, from the files whose weights are n's set bits."""
    total = None
    for w, arr in files.items():
        if n & w:
            total = arr if total is None else total + arr
    return total


def free_field_inverse_trace(dims, kappa, amu, bc=-1.0):
    """Per-site Tr(M_u^{-1}) and Tr(gamma_5 M_u^{-1}) for unit links, from the momentum-space inverse.

    M(p) = A(p) + 2 i kappa sum_mu gamma_mu sin p_mu + 2 i kappa amu gamma_5,
    A(p) = 1 - 2 kappa sum_mu cos p_mu; p_mu = 2 pi n / L in space and
    (2 n + 1) pi / T in time for bc = -1.
    """
    X, Y, Z, T = dims
    tr1 = 0.0 + 0.0j
    tr5 = 0.0 + 0.0j
    tshift = 0.5 if bc < 0 else 0.0
    for nt in range(T):
        for nz in range(Z):
            for ny in range(Y):
                for nx in range(X):
                    p = (2 * np.pi * nx / X, 2 * np.pi * ny / Y, 2 * np.pi * nz / Z, 2 * np.pi * (nt + tshift) / T)
                    a = 1.0 - 2.0 * kappa * sum(np.cos(q) for q in p)
                    s2 = sum(np.sin(q) ** 2 for q in p)
                    den = a * a + 4 * kappa * kappa * s2 + 4 * kappa * kappa * amu * amu
                    tr1 += 4 * a / den
                    tr5 += 4 * (-2j * kappa * amu) / den
    V = X * Y * Z * T
    return 3 * tr1 / V, 3 * tr5 / V


