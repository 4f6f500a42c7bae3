"""Pins of the oracle's Dirac operator (CPU only): free field, gamma_5-hermiticity,
gauge covariance, explicit matrix elements, the even-odd Schur complement."""
import numpy as np
import pytest

import synth
from oracle import lattice
from oracle import operator as op

KAPPA, AMU = 0.16, 0.01


def _plane_wave(dims, n, u, bc=-1.0):
    """exp(i p.x) u with p_mu = 2 pi n_mu / L (space) and (2 n + 1) pi / T (time, bc=-1)."""
    X, Y, Z, T = dims
    x, y, z, t = lattice.coords(dims)
    shift = 0.5 if bc < 0 else 0.0
    p = (2 * np.pi * n[0] / X, 2 * np.pi * n[1] / Y, 2 * np.pi * n[2] / Z, 2 * np.pi * (n[3] + shift) / T)
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[..., None, None] * u[None, None, None, None], p


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (3, 1, 1, 2)])
def test_free_field_closed_form(n):
    dims = (4, 4, 6, 8)
    rng = np.random.default_rng(1)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    psi, p = _plane_wave(dims, n, u)
    links = synth.unit_links(dims)
    out = op.apply_m(links, psi, KAPPA, AMU, f=1)
    g = lattice.GAMMA
    mp = (1 - 2 * KAPPA * sum(np.cos(q) for q in p)) * np.eye(4) \
        + 2j * KAPPA * sum(g[m] * np.sin(p[m]) for m in range(4)) + 2j * KAPPA * AMU * lattice.GAMMA5
    expect, _ = _plane_wave(dims, n, mp @ u)
    assert np.abs(out - expect).max() < 1e-13


def test_flavour_relations():
    dims = (4, 2, 2, 4)
    links = synth.gauge_links(dims, 0.3, 5)
    psi = synth.gaussian_spinors(dims, 1, 6)[0]
    mu_ = op.apply_m(links, psi, KAPPA, AMU, 1)
    md_ = op.apply_m(links, psi, KAPPA, AMU, -1)
    assert np.allclose(mu_ - md_, 4j * KAPPA * AMU * op.spin(lattice.GAMMA5, psi), atol=1e-14)
    assert np.allclose(0.5 * (mu_ + md_), op.wilson_a(links, psi, KAPPA), atol=1e-14)


def test_gamma5_hermiticity_dense():
    dims = (4, 2, 2, 4)
    links = synth.gauge_links(dims, 0.5, 7)
    mu = op.dense_matrix(links, KAPPA, AMU, 1)
    md = op.dense_matrix(links, KAPPA, AMU, -1)
    g5 = np.kron(np.eye(mu.shape[0] // 12), np.kron(lattice.GAMMA5, np.eye(3)))
    assert np.abs(g5 @ mu @ g5 - md.conj().T).max() < 1e-14
    # the hopping-only adjoint used by Mhat^dagger
    psi = synth.gaussian_spinors(dims, 2, 8)
    lhs = np.vdot(psi[0], op.hop(links, psi[1]))
    rhs = np.vdot(op.hop(links, psi[0], dag=True), psi[1])
    assert abs(lhs - rhs) < 1e-12


def test_dense_matrix_elements():
    """Block (x, x+mu) of M is -kappa (1 - gamma_mu) U_mu(x); (x+mu, x) is -kappa (1 + gamma_mu) U_mu(x)^dagger."""
    dims = (4, 4, 2, 4)
    X, Y, Z, T = dims
    links = synth.gauge_links(dims, 0.3, 9)
    m = op.dense_matrix(links, KAPPA, AMU, 1)

    def idx(x, y, z, t):
        return 12 * (x + X * (y + Y * (z + Z * t)))

    site = (1, 2, 1, 0)
    x, y, z, t = site
    for mu, nb in [(0, (2, 2, 1, 0)), (1, (1, 3, 1, 0)), (3, (1, 2, 1, 1))]:
        u = links[t, z, y, x, mu]
        blk = m[idx(*site):idx(*site) + 12, idx(*nb):idx(*nb) + 12]
        assert np.allclose(blk, -KAPPA * np.kron(np.eye(4) - lattice.GAMMA[mu], u), atol=1e-15)
        blk2 = m[idx(*nb):idx(*nb) + 12, idx(*site):idx(*site) + 12]
        assert np.allclose(blk2, -KAPPA * np.kron(np.eye(4) + lattice.GAMMA[mu], u.conj().T), atol=1e-15)
    # the time hop T-1 -> 0 carries the antiperiodic factor
    top = (1, 2, 1, T - 1)
    u = links[T - 1, 1, 2, 1, 3]
    blk = m[idx(*top):idx(*top) + 12, idx(1, 2, 1, 0):idx(1, 2, 1, 0) + 12]
    assert np.allclose(blk, +KAPPA * np.kron(np.eye(4) - lattice.GAMMA[3], u), atol=1e-15)
    diag = m[idx(*site):idx(*site) + 12, idx(*site):idx(*site) + 12]
    assert np.allclose(diag, np.kron(np.eye(4) + 2j * KAPPA * AMU * lattice.GAMMA5, np.eye(3)))


def test_gauge_covariance():
    dims = (4, 4, 2, 4)
    links = synth.gauge_links(dims, 0.4, 11)
    g = synth.gauge_transform_field(dims, 12)
    lg = np.empty_like(links)
    for mu in range(4):
        gf = np.roll(g, -1, axis={0: 3, 1: 2, 2: 1, 3: 0}[mu])
        lg[..., mu, :, :] = g @ links[..., mu, :, :] @ np.conj(np.swapaxes(gf, -1, -2))
    psi = synth.gaussian_spinors(dims, 1, 13)[0]
    lhs = op.apply_m(lg, op.colour(g, psi), KAPPA, AMU)
    rhs = op.colour(g, op.apply_m(links, psi, KAPPA, AMU))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_even_odd_schur_complement():
    dims = (4, 4, 2, 4)
    links = synth.gauge_links(dims, 0.4, 14)
    b = synth.gaussian_spinors(dims, 1, 15)[0]
    psi_exact = np.linalg.solve(op.dense_matrix(links, KAPPA, AMU, 1), b.ravel()).reshape(b.shape)
    # the even part of the exact solution solves Mhat x = bhat ...
    pe = op.project(psi_exact, dims, 0)
    bhat = op.prep_source(links, b, KAPPA, AMU, 1, -1.0, dims)
    assert np.abs(op.mhat(links, pe, KAPPA, AMU, 1, -1.0, dims) - bhat).max() < 1e-12
    # ... and the odd reconstruction gives back the odd part
    po = op.reconstruct_odd(links, pe, b, KAPPA, AMU, 1, -1.0, dims)
    assert np.abs(po - op.project(psi_exact, dims, 1)).max() < 1e-12
    # Mhat^dagger is the adjoint of Mhat on the even sites
    v = op.project(synth.gaussian_spinors(dims, 2, 16), dims, 0)
    lhs = np.vdot(v[0], op.mhat(links, v[1], KAPPA, AMU, 1, -1.0, dims))
    rhs = np.vdot(op.mhat_dag(links, v[0], KAPPA, AMU, 1, -1.0, dims), v[1])
    assert abs(lhs - rhs) < 1e-12


def test_site_local_operator_matches_full_field():
    dims = (4, 4, 2, 6)
    links = synth.gauge_links(dims, 0.4, 17)
    psi = synth.gaussian_spinors(dims, 1, 18)[0]
    full = op.apply_m(links, psi, KAPPA, AMU, -1)
    for site in [(0, 0, 0, 0), (5, 1, 3, 2), (2, 0, 1, 3), (5, 1, 0, 0)]:
        assert np.abs(op.apply_m_at(links, psi, site, KAPPA, AMU, -1) - full[site]).max() < 1e-14
