"""Pins of the oracle's solver, estimators, HPE, projection and TSM (CPU only)."""
import numpy as np
import pytest

import synth
from oracle import lattice, loops, noise, solver
from oracle import operator as op

KAPPA, AMU = 0.16, 0.01
SMALL = (4, 2, 2, 4)


@pytest.fixture(scope="module")
def small():
    links = synth.gauge_links(SMALL, 0.3, 21)
    mu = op.dense_matrix(links, KAPPA, AMU, 1)
    md = op.dense_matrix(links, KAPPA, AMU, -1)
    a = op.dense_matrix(links, KAPPA, AMU, 1, which="A")
    return dict(links=links, mu=mu, md=md, a=a, iu=np.linalg.inv(mu), id=np.linalg.inv(md))


def _site_op(x4, n_sites):
    """A spin matrix acting at every site, as a dense (12V x 12V) matrix."""
    return np.kron(np.eye(n_sites), np.kron(x4, np.eye(3)))


def test_cg_matches_dense_lu():
    dims = (4, 4, 2, 4)
    links = synth.gauge_links(dims, 0.3, 22)
    b = noise.z4_noise(dims, 5, 0)
    x_lu = solver.solve_dense(links, b, KAPPA, AMU)
    x_cg, iters, relres = solver.solve_eo(links, b, KAPPA, AMU, tol=1e-13)
    assert relres <= 1e-13 and iters > 10
    assert np.linalg.norm(x_cg - x_lu) / np.linalg.norm(x_lu) < 1e-9
    assert np.abs(op.apply_m(links, x_cg, KAPPA, AMU) - b).max() < 1e-10


def test_free_field_trace_closed_form():
    dims = (4, 2, 2, 4)
    links = synth.unit_links(dims)
    inv = np.linalg.inv(op.dense_matrix(links, KAPPA, AMU, 1))
    V = 64
    tr1 = np.trace(inv) / V
    tr5 = np.trace(_site_op(lattice.GAMMA5, V) @ inv) / V
    c1, c5 = loops.free_field_inverse_trace(dims, KAPPA, AMU)
    assert abs(tr1 - c1) < 1e-12 and abs(tr5 - c5) < 1e-12
    # gamma_mu traces vanish by symmetry
    for mu in range(4):
        assert abs(np.trace(_site_op(lattice.GAMMA[mu], V) @ inv)) < 1e-11


def test_resolvent_identities(small):
    """Eq. vvTrick and M_u + M_d = 2 D_W, exact on the dense matrices."""
    V = 64
    g5 = _site_op(lattice.GAMMA5, V)
    assert np.abs(small["iu"] - small["id"] + 4j * KAPPA * AMU * small["id"] @ g5 @ small["iu"]).max() < 1e-10
    assert np.abs(small["mu"] + small["md"] - 2 * small["a"]).max() < 1e-14


@pytest.mark.parametrize("xb", [0, 11, 15, 6])
def test_estimator_expectations_exact(small, xb):
    """E_eta[xi^+ X phi] = Tr[P^+ X Q] for xi = P eta, phi = Q eta; each estimator's
    expectation, times its factor, is the trace it is meant to give (dense)."""
    V = 64
    X = _site_op(lattice.GAMMAS16[xb], V)
    g5 = _site_op(lattice.GAMMA5, V)
    iu, id_, a = small["iu"], small["id"], small["a"]
    pairs = {
        "standard": (np.eye(iu.shape[0]), iu),
        "one_end": (g5 @ iu, iu),
        "gen_one_end": (g5 @ iu, g5 @ a @ iu),
    }
    targets = {
        "standard": np.trace(iu @ X),
        "one_end": np.trace((iu - id_) @ X),
        "gen_one_end": np.trace((iu + id_) @ X),
    }
    for est, (p, q) in pairs.items():
        e = np.trace(p.conj().T @ X @ q) * loops.prefactor(est, KAPPA, AMU)
        assert abs(e - targets[est]) < 1e-10 * max(1.0, abs(targets[est])), est


def test_estimator_pairs_match_matrices(small):
    """The oracle's (xi, phi) for a fixed noise are the dense matrices applied to eta."""
    links = small["links"]
    eta = noise.z4_noise(SMALL, 9, 0)
    s = (small["iu"] @ eta.ravel()).reshape(eta.shape)
    xi, phi = loops.pair("gen_one_end", links, eta, s, KAPPA, AMU)
    g5 = _site_op(lattice.GAMMA5, 64)
    assert np.allclose(phi.ravel(), g5 @ small["a"] @ s.ravel(), atol=1e-13)
    # D_W s = eta - 2 i kappa amu gamma_5 s (the site-local form the GPU uses)
    aw = op.wilson_a(links, s, KAPPA)
    assert np.allclose(aw, eta - 2j * KAPPA * AMU * loops.g5(s), atol=1e-12)


def test_stochastic_convergence(small):
    """Averages over Z4 noise approach the exact traces at O(1/sqrt(N)) (Eqs. eq2, loopSt, loopVv)."""
    n = 400
    eta = np.stack([noise.z4_noise(SMALL, 33, r) for r in range(n)])
    s = (small["iu"] @ eta.reshape(n, -1).T).T.reshape(eta.shape)
    V = 64
    for est, xb, target in [
        ("standard", 0, np.trace(small["iu"])),
        ("one_end", 15, np.trace((small["iu"] - small["id"]) @ _site_op(lattice.GAMMA5, V))),
    ]:
        xi, phi = loops.pair(est, small["links"], eta, s, KAPPA, AMU)
        c = loops.bilinear(xi, phi)
        f = loops.loop_from_c(c, lattice.GAMMAS16[xb]).reshape(n, -1).sum(1) * loops.prefactor(est, KAPPA, AMU)
        err = f.std(ddof=1) / np.sqrt(n)
        assert abs(f.mean() - target) < 4 * err + 1e-12, est
        # a factor-2 normalisation error in the noise would be many sigma away
        assert abs(0.5 * f.mean() - target) > 4 * err or abs(target) < 1e-9


def test_hpe_identity_dense(small):
    """Eq. (HPE): M^-1 = B - BHB + (BH)^2 B - (BH)^3 B + (BH)^4 M^-1."""
    links = small["links"]
    psi = synth.gaussian_spinors(SMALL, 1, 41)[0]
    minv_psi = (small["iu"] @ psi.ravel()).reshape(psi.shape)
    rhs = loops.hpe_truncated_inverse(links, psi, KAPPA, AMU) + loops.bh_power(links, minv_psi, KAPPA, AMU, 4)
    assert np.abs(rhs - minv_psi).max() < 1e-12


def test_hpe_exact_terms():
    dims = (4, 4, 4, 4)
    site = (1, 2, 3, 0)
    links = synth.gauge_links(dims, 0.4, 42)
    c_rand = loops.hpe_exact_c(links, KAPPA, AMU, site)
    c_unit = loops.hpe_exact_c(synth.unit_links(dims), KAPPA, AMU, (0, 0, 0, 0))
    # gauge independent (U U^dagger = 1): same on a random and on the unit field
    assert np.abs(c_rand - c_unit).max() < 1e-14
    # closed form: colour factor 3, B + kappa^2 B sum_mu [(1-g)B(1+g) + (1+g)B(1-g)] B
    b = np.linalg.inv(np.eye(4) + 2j * KAPPA * AMU * lattice.GAMMA5)
    s = sum((np.eye(4) - g) @ b @ (np.eye(4) + g) + (np.eye(4) + g) @ b @ (np.eye(4) - g) for g in lattice.GAMMA)
    e = 3 * (b + KAPPA ** 2 * b @ s @ b)
    assert np.abs(c_rand - e.T).max() < 1e-14
    # only Gamma = 1 and gamma_5 have a non-zero exact part (Sec. 2.5)
    for xb in range(16):
        val = loops.loop_from_c(c_rand, lattice.GAMMAS16[xb])
        if xb in (0, 15):
            assert abs(val) > 1e-3
        else:
            assert abs(val) < 1e-14


def test_hpe_exact_terms_need_extents_of_four():
    """With an extent of 2 two forward hops along that direction return to the site
    through two different links, so the brute-force exact part differs from the
    closed form (and from the unit-field value): the closed form holds for extents >= 4."""
    dims = (4, 4, 2, 4)
    links = synth.gauge_links(dims, 0.4, 43)
    c_rand = loops.hpe_exact_c(links, KAPPA, AMU, (0, 0, 0, 0))
    b = np.linalg.inv(np.eye(4) + 2j * KAPPA * AMU * lattice.GAMMA5)
    s = sum((np.eye(4) - g) @ b @ (np.eye(4) + g) + (np.eye(4) + g) @ b @ (np.eye(4) - g) for g in lattice.GAMMA)
    e = 3 * (b + KAPPA ** 2 * b @ s @ b)
    assert np.abs(c_rand - e.T).max() > 1e-3


def test_gauge_invariance_of_loops():
    dims = (4, 4, 2, 4)
    links = synth.gauge_links(dims, 0.4, 51)
    g = synth.gauge_transform_field(dims, 52)
    lg = np.empty_like(links)
    for mu in range(4):
        gf = np.roll(g, -1, axis={0: 3, 1: 2, 2: 1, 3: 0}[mu])
        lg[..., mu, :, :] = g @ links[..., mu, :, :] @ np.conj(np.swapaxes(gf, -1, -2))
    eta = noise.z4_noise(dims, 53, 0)
    s, _, _ = solver.solve_eo(links, eta, KAPPA, AMU, tol=1e-12)
    eta_g = op.colour(g, eta)
    s_g, _, _ = solver.solve_eo(lg, eta_g, KAPPA, AMU, tol=1e-12)
    assert np.abs(s_g - op.colour(g, s)).max() < 1e-8
    for est in ("standard", "one_end", "gen_one_end", "hpe"):
        a = loops.bilinear(*loops.pair(est, links, eta, s, KAPPA, AMU))
        b = loops.bilinear(*loops.pair(est, lg, eta_g, s_g, KAPPA, AMU))
        assert np.abs(a - b).max() < 1e-8, est
    for mu in range(4):
        a = loops.derivative_bilinear(links, loops.g5(s), s, mu)
        b = loops.derivative_bilinear(lg, loops.g5(s_g), s_g, mu)
        assert np.abs(a - b).max() < 1e-8


def test_derivative_bilinear_free_plane_waves():
    """Unit links, xi = e^{ipx} u, phi = e^{iqx} v:
    l^mu_ab(x) = (i/2)(sin p_mu + sin q_mu) e^{i(q-p)x} conj(u_a) v_b (colour summed)."""
    dims = (4, 4, 6, 8)
    X, Y, Z, T = dims
    x, y, z, t = lattice.coords(dims)
    links = synth.unit_links(dims)
    rng = np.random.default_rng(3)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    v = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))

    def wave(n):
        p = (2 * np.pi * n[0] / X, 2 * np.pi * n[1] / Y, 2 * np.pi * n[2] / Z, 2 * np.pi * (n[3] + 0.5) / T)
        return np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t)), p

    wp, p = wave((1, 0, 2, 1))
    wq, q = wave((0, 3, 1, 2))
    xi = wp[..., None, None] * u
    phi = wq[..., None, None] * v
    uv = np.einsum("ac,bc->ab", np.conj(u), v)
    for mu in range(4):
        got = loops.derivative_bilinear(links, xi, phi, mu)
        expect = 0.5j * (np.sin(p[mu]) + np.sin(q[mu])) * (np.conj(wp) * wq)[..., None, None] * uv
        assert np.abs(got - expect).max() < 1e-13


def test_projection_sign_and_order():
    dims = (4, 6, 4, 2)
    X, Y, Z, T = dims
    x, y, z, t = lattice.coords(dims)
    n0 = (1, -1, 1)
    field = np.exp(2j * np.pi * (n0[0] * x / X + n0[1] * y / Y + n0[2] * z / Z))
    c = field[..., None, None] * np.arange(16).reshape(4, 4)
    proj = loops.project_momenta(c, dims, 3)
    plist = lattice.momenta(3)
    for ip, n in enumerate(plist):
        expect = X * Y * Z * np.arange(16).reshape(4, 4) if n == n0 else 0.0
        assert np.abs(proj[:, ip] - expect).max() < 1e-11
    # p = 0 is the plain spatial sum
    rng = np.random.default_rng(4)
    c2 = rng.normal(size=(T, Z, Y, X, 4, 4))
    p0 = loops.project_momenta(c2, dims, 0)
    assert np.allclose(p0[:, 0], c2.sum(axis=(1, 2, 3)))


def test_tsm_unbiased_and_exact_algebra():
    """Eq. (estiTSM): with a deterministic truncated-CG LP map the estimator is unbiased
    over noise draws; with LP = HP the correction term vanishes."""
    dims = (2, 2, 2, 4)
    links = synth.gauge_links(dims, 0.3, 61)
    minv = np.linalg.inv(op.dense_matrix(links, KAPPA, AMU, 1))
    exact = np.trace(minv)

    def f_of(eta, s):
        return loops.loop_from_c(loops.bilinear(eta, s), np.eye(4)).sum()

    def lp(eta):
        return solver.solve_eo(links, eta, KAPPA, AMU, tol=3e-1)[0]

    n_hp, n_lp, trials = 4, 24, 30
    ests = []
    r = 0
    for _ in range(trials):
        hp_eta = [noise.z4_noise(dims, 71, r + i) for i in range(n_hp)]
        r += n_hp
        lp_eta = [noise.z4_noise(dims, 71, r + i) for i in range(n_lp)]
        r += n_lp
        f_hp = [f_of(e, (minv @ e.ravel()).reshape(e.shape)) for e in hp_eta]
        f_lpp = [f_of(e, lp(e)) for e in hp_eta]
        f_lpf = [f_of(e, lp(e)) for e in lp_eta]
        ests.append(loops.tsm_estimate(f_hp, f_lpp, f_lpf))
        # LP == HP: the estimator reduces to the plain mean of the fresh set
        assert abs(loops.tsm_estimate(f_hp, f_hp, f_lpf) - np.mean(f_lpf)) < 1e-12
    ests = np.array(ests)
    err = ests.std(ddof=1) / np.sqrt(trials)
    assert abs(ests.mean() - exact) < 4 * err
    # the truncated map alone is biased: its plain mean misses the exact trace
    f_lp_only = np.mean([f_of(noise.z4_noise(dims, 72, i), lp(noise.z4_noise(dims, 72, i))) for i in range(200)])
    assert abs(f_lp_only - exact) > abs(ests.mean() - exact)


def test_tsm_error_matches_the_spread_of_estimates():
    """Eq. estiTSM's standard error, var(f_HP - f_LP)/N_HP + var(f_LP)/N_LP, against the
    spread of the estimate over 4000 independent repetitions (correlated HP/LP pairs)."""
    rng = np.random.default_rng(7)
    reps, n_hp, n_lp = 4000, 12, 60
    f_hp = rng.normal(size=(reps, n_hp))
    f_pair = 0.9 * f_hp + 0.3 * rng.normal(size=(reps, n_hp))   # the LP map: correlated with HP
    f_lp = 0.9 * rng.normal(size=(reps, n_lp)) + 0.3 * rng.normal(size=(reps, n_lp))
    est = np.array([loops.tsm_estimate(f_hp[i], f_pair[i], f_lp[i]) for i in range(reps)])
    err = np.array([loops.tsm_error(f_hp[i], f_pair[i], f_lp[i]) for i in range(reps)])
    # exact: var(f_HP - f_LP) = 0.1^2 + 0.3^2, var(f_LP) = 0.9^2 + 0.3^2
    exact = np.sqrt((0.01 + 0.09) / n_hp + (0.81 + 0.09) / n_lp)
    assert abs(est.std(ddof=1) / exact - 1) < 0.05
    assert abs(np.sqrt(np.mean(err ** 2)) / exact - 1) < 0.05
    # a dropped 1/N factor or a swapped pair of terms would be far off
    assert abs(np.sqrt((0.1 / n_lp) + (0.9 / n_hp)) / exact - 1) > 0.3
