"""Pins of the oracle's time dilution (Sec. 2.3): sources on the time slices t = t0 (mod dt),
single slices (dt = T) and coherent sources (several slices).  CPU only, dense 4x2x2x4."""
import numpy as np
import pytest

import synth
from oracle import lattice, loops, noise
from oracle import operator as op

KAPPA, AMU = 0.16, 0.01
DIMS = (4, 2, 2, 4)  # X, Y, Z, T
V = 64
T = DIMS[3]


@pytest.fixture(scope="module")
def dense():
    links = synth.gauge_links(DIMS, 0.3, 31)
    iu = np.linalg.inv(op.dense_matrix(links, KAPPA, AMU, 1))
    return dict(links=links, iu=iu)


def _site_op(x4):
    return np.kron(np.eye(V), np.kron(x4, np.eye(3)))


def _projector(t0, dt):
    """The oracle's time dilution as a matrix: its action on every unit vector."""
    n = 12 * V
    cols = [noise.time_diluted(e.reshape(DIMS[::-1] + (4, 3)), t0, dt).ravel() for e in np.eye(n, dtype=complex)]
    return np.array(cols).T


def _slice_of_component():
    """Time slice of every component of the flattened [T][Z][Y][X][4][3] vector (from the site coordinates)."""
    t = lattice.coords(DIMS)[3]
    return np.repeat(t.ravel(), 12)


@pytest.mark.parametrize("dt", [1, 2, 4])
def test_sources_partition_the_noise(dt):
    eta = noise.z4_noise(DIMS, 41, 3)
    parts = [noise.time_diluted(eta, t0, dt) for t0 in range(dt)]
    assert np.array_equal(sum(parts), eta)  # the subspaces form a direct sum
    ts = _slice_of_component().reshape(eta.shape)
    for t0, p in enumerate(parts):
        keep = ts % dt == t0
        assert np.array_equal(p[keep], eta[keep]) and not p[~keep].any()
    with pytest.raises(ValueError):
        noise.time_diluted(eta, dt, dt)


@pytest.mark.parametrize("t0,dt", [(1, 4), (0, 2), (1, 2)])
def test_projector_and_exact_expectation(dense, t0, dt):
    """E[(P eta)^+ X M^-1 P eta] = Tr[P X M^-1 P] = the sum of the site traces of X M^-1
    over the diluted slices, for every insertion (dense)."""
    p = _projector(t0, dt)
    assert np.allclose(p @ p, p) and np.allclose(p, p.conj().T)
    ts = _slice_of_component()
    assert np.array_equal(np.diag(p).real, (ts % dt == t0).astype(float))
    iu = dense["iu"]
    for xb in (0, 15, 11, 6):
        X = _site_op(lattice.GAMMAS16[xb])
        expect = np.trace(p.conj().T @ X @ iu @ p)
        blocks = X @ iu
        direct = sum(blocks[i, i] for i in range(12 * V) if ts[i] % dt == t0)
        assert abs(expect - direct) < 1e-12 * max(1.0, abs(direct))


def _exact_variance(a):
    """Var of eta^+ A eta over Z2 x iZ2 noise: sum of |A_ab|^2 over a != b
    (|eta_a| = 1 and E[eta_a^2] = 0 leave only the pairs (a, b) with themselves)."""
    return float((np.abs(a) ** 2).sum() - (np.abs(np.diag(a)) ** 2).sum())


@pytest.mark.parametrize("t0,dt", [(2, 4), (0, 2)])
def test_variance_of_the_slice_loop(dense, t0, dt):
    """The loop of slice t0 from diluted sources: sample variance over 400 sources matches
    the exact variance, which is below the undiluted one (the off-diagonal terms of the other
    slices are gone; Sec. 2.3)."""
    iu = dense["iu"]
    ts = _slice_of_component()
    on_t0 = np.diag((ts == t0).astype(complex))
    p = _projector(t0, dt)
    X = _site_op(lattice.GAMMAS16[0])
    var_dil = _exact_variance(on_t0 @ X @ iu @ p)
    var_full = _exact_variance(on_t0 @ X @ iu)
    assert var_dil < 0.8 * var_full
    n = 400
    f_dil, f_full = [], []
    for r in range(n):
        eta = noise.z4_noise(DIMS, 43, r)
        for src, f in ((noise.time_diluted(eta, t0, dt), f_dil), (eta, f_full)):
            s = (iu @ src.ravel()).reshape(src.shape)
            c = loops.bilinear(src, s)
            f.append(loops.loop_from_c(c, lattice.GAMMAS16[0])[t0].sum())
    f_dil, f_full = np.array(f_dil), np.array(f_full)
    assert abs(np.var(f_dil, ddof=1) / var_dil - 1) < 0.3
    assert abs(np.var(f_full, ddof=1) / var_full - 1) < 0.3
    exact = np.trace(on_t0 @ X @ iu)
    assert abs(f_dil.mean() - exact) < 4 * np.sqrt(var_dil / n)


def test_hpe_remainder_with_dilution(dense):
    """Time dilution combined with the HPE (Sec. 2.3 with Eq. HPE): the diluted remainder
    eta_S^+ X (BH)^4 s_S plus the exact orders 0-3 on the diluted slices has the expectation
    Tr over those slices of X M^-1 (dense: exact part from unit vectors)."""
    links, iu = dense["links"], dense["iu"]
    t0, dt = 1, 2
    p = _projector(t0, dt)
    n = 12 * V
    bh4 = np.array([loops.bh_power(links, e.reshape(DIMS[::-1] + (4, 3)), KAPPA, AMU, 4).ravel()
                    for e in np.eye(n, dtype=complex)]).T
    trunc = np.array([loops.hpe_truncated_inverse(links, e.reshape(DIMS[::-1] + (4, 3)), KAPPA, AMU).ravel()
                      for e in np.eye(n, dtype=complex)]).T
    for xb in (0, 15):
        X = _site_op(lattice.GAMMAS16[xb])
        remainder = np.trace(p.conj().T @ X @ bh4 @ iu @ p)
        exact_part = np.trace(p @ X @ trunc @ p)
        assert abs(remainder + exact_part - np.trace(p @ X @ iu @ p)) < 1e-10
