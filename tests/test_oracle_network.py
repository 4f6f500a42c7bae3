"""Pins of the oracle's parallel-transport network (CPU only): finite-difference
gradients, gauge equivariance, and a closed form built from the operator module."""
import numpy as np

import synth
from oracle import loops, network, noise
from oracle import operator as op

DIMS = (4, 2, 2, 4)
KAPPA, AMU = 0.16, 0.01


def _small_net(rng, c=3):
    return [network.init_layer(1, c, rng, 0.3), network.init_layer(c, c, rng, 0.3), network.init_layer(c, 1, rng, 0.3)]


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    links = synth.gauge_links(DIMS, 0.4, 81)
    weights = _small_net(rng)
    pairs = [(noise.z4_noise(DIMS, 5, r), synth.gaussian_spinors(DIMS, 1, 90 + r)[0]) for r in range(2)]
    _, grads = network.loss_and_grads(links, weights, pairs)
    h = 1e-6
    checked = 0
    for li, key, idx in [(0, "W0", (1, 0, 1)), (1, "Wf", (2, 0, 2, 3)), (1, "Wb", (3, 1, 1, 0)), (2, "W0", (0, 2, 0)),
                         (2, "Wf", (0, 0, 1, 1)), (1, "W0", (2, 1, 0))]:
        for part in (1.0, 1j):
            w_p = [{k: v.copy() for k, v in w.items()} for w in weights]
            w_m = [{k: v.copy() for k, v in w.items()} for w in weights]
            w_p[li][key][idx] += part * h
            w_m[li][key][idx] -= part * h
            lp, _ = network.loss_and_grads(links, w_p, pairs)
            lm, _ = network.loss_and_grads(links, w_m, pairs)
            fd = (lp - lm) / (2 * h)
            an = grads[li][key][idx].real if part == 1.0 else grads[li][key][idx].imag
            assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3), (li, key, idx, part, fd, an)
            checked += 1
    assert checked == 12


def test_residual_loss_gradients_match_finite_differences():
    """The residual loss |M N eta - eta|^2 / |eta|^2: Wirtinger gradients against central
    differences of the loss itself."""
    rng = np.random.default_rng(2)
    links = synth.gauge_links(DIMS, 0.4, 85)
    weights = _small_net(rng)
    etas = [noise.z4_noise(DIMS, 7, r) for r in range(2)]
    _, grads = network.residual_loss_and_grads(links, weights, etas, KAPPA, AMU)
    h = 1e-6
    for li, key, idx in [(0, "W0", (1, 0, 0)), (1, "Wf", (1, 2, 0, 1)), (1, "Wb", (0, 0, 2, 3)), (2, "Wb", (3, 0, 1, 2))]:
        for part in (1.0, 1j):
            w_p = [{k: v.copy() for k, v in w.items()} for w in weights]
            w_m = [{k: v.copy() for k, v in w.items()} for w in weights]
            w_p[li][key][idx] += part * h
            w_m[li][key][idx] -= part * h
            lp, _ = network.residual_loss_and_grads(links, w_p, etas, KAPPA, AMU)
            lm, _ = network.residual_loss_and_grads(links, w_m, etas, KAPPA, AMU)
            fd = (lp - lm) / (2 * h)
            an = grads[li][key][idx].real if part == 1.0 else grads[li][key][idx].imag
            assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3), (li, key, idx, part, fd, an)


def test_residual_loss_vanishes_at_the_inverse_and_equals_the_solution_loss_weighted():
    """At N = M^-1 (dense, on a tiny lattice through a one-layer stand-in) the residual
    is zero; and for any map y the residual loss equals |M (y - s)|^2 / |eta|^2 with
    s = M^-1 eta (the solution error weighted by M)."""
    links = synth.gauge_links(DIMS, 0.4, 86)
    eta = noise.z4_noise(DIMS, 8, 0)
    m = op.dense_matrix(links, KAPPA, AMU, 1)
    s = np.linalg.solve(m, eta.ravel()).reshape(eta.shape)
    r = op.apply_m(links, s, KAPPA, AMU) - eta
    assert np.vdot(r, r).real / np.vdot(eta, eta).real < 1e-24
    y = synth.gaussian_spinors(DIMS, 1, 87)[0]
    r = op.apply_m(links, y, KAPPA, AMU) - eta
    e = op.apply_m(links, y - s, KAPPA, AMU)
    assert abs(np.vdot(r, r).real - np.vdot(e, e).real) < 1e-10 * np.vdot(e, e).real


def test_gauge_equivariance():
    rng = np.random.default_rng(1)
    links = synth.gauge_links(DIMS, 0.4, 82)
    g = synth.gauge_transform_field(DIMS, 83)
    lg = np.empty_like(links)
    for mu in range(4):
        gf = np.roll(g, -1, axis={0: 3, 1: 2, 2: 1, 3: 0}[mu])
        lg[..., mu, :, :] = g @ links[..., mu, :, :] @ np.conj(np.swapaxes(gf, -1, -2))
    weights = _small_net(rng)
    eta = noise.z4_noise(DIMS, 6, 0)
    out, _ = network.forward(links, weights, eta)
    out_g, _ = network.forward(lg, weights, op.colour(g, eta))
    assert np.abs(out_g - op.colour(g, out)).max() < 1e-13


def test_closed_form_neumann_layers():
    """Layers B, (1 - BH), (1 - BH), (1 - BH) give N = (1 - BH)^3 B (B = R^-1, H = -kappa D, Eq. HPE)."""
    dims = (4, 4, 2, 4)
    links = synth.gauge_links(dims, 0.4, 84)
    w = 2 * KAPPA * AMU
    a, b = 1.0 / (1 + w * w), -w / (1 + w * w)
    zero = lambda: {"W0": np.zeros((1, 1, 2), complex), "Wf": np.zeros((4, 1, 1, 4), complex),
                    "Wb": np.zeros((4, 1, 1, 4), complex)}
    lb = zero()
    lb["W0"][0, 0] = [a, 1j * b]
    lh = zero()
    lh["W0"][0, 0] = [1.0, 0.0]
    for mu in range(4):
        lh["Wf"][mu, 0, 0] = KAPPA * np.array([a, -a, 1j * b, -1j * b])
        lh["Wb"][mu, 0, 0] = KAPPA * np.array([a, a, 1j * b, 1j * b])
    eta = noise.z4_noise(dims, 7, 0)
    out, _ = network.forward(links, [lb, lh, lh, lh], eta)
    ref = op.twist_inv(eta, KAPPA, AMU, 1)
    for _ in range(3):
        ref = ref - loops.bh_apply(links, ref, KAPPA, AMU)
    assert np.abs(out - ref).max() < 1e-13


def test_loss_vanishes_at_exact_map():
    dims = (4, 4, 2, 4)
    links = synth.gauge_links(dims, 0.4, 85)
    rng = np.random.default_rng(2)
    weights = _small_net(rng)
    eta = noise.z4_noise(dims, 8, 0)
    out, _ = network.forward(links, weights, eta)
    loss, grads = network.loss_and_grads(links, weights, [(eta, out)])
    assert loss < 1e-28
    assert all(np.abs(v).max() < 1e-12 for gw in grads for v in gw.values())


def test_layer_adjoint_is_the_adjoint():
    """<y, L x> = <L^+ y, x> for the input gradient of every layer shape (1->C, C->C, C->1),
    and the chain over layers is the adjoint of the network."""
    rng = np.random.default_rng(7)
    links = synth.gauge_links(DIMS, 0.4, 85)
    weights = _small_net(rng, c=3)
    x = synth.gaussian_spinors(DIMS, 1, 91)
    y = synth.gaussian_spinors(DIMS, 1, 92)
    nx, _ = network.forward(links, weights, x[0])
    g = y
    for li in range(len(weights) - 1, -1, -1):
        cin = weights[li]["W0"].shape[1]
        _, g = network.layer_backward(links, weights[li], np.zeros((cin,) + x.shape[1:], dtype=np.complex128), g)
    lhs = np.vdot(y[0], nx)
    rhs = np.vdot(g[0], x[0])
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
