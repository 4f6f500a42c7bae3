"""Gauge-covariant parallel-transport convolution network (test infrastructure; oracle).

The paper has no learned component; this restates the network the learned
preconditioner uses so its kernels can be checked.  A layer maps C_in input
spinor fields x_i to C_out output fields

    y_o(x) = sum_i [ sum_b W0[o,i,b] L_b x_i(x)
                     + sum_mu sum_b Wf[mu,o,i,b] H_b(mu) U_mu(x) x_i(x+mu)
                     + sum_mu sum_b Wb[mu,o,i,b] H_b(mu) U_mu(x-mu)^+ x_i(x-mu) ]

with complex scalar weights, local spin factors L_b in {1, g5} and hop spin
factors H_b(mu) in {1, g_mu, g5, g5 g_mu}; hops across t = T-1 <-> 0 carry the
time-boundary factor.  Weights act on channels and spin only, never on colour,
so every layer commutes with gauge transformations:  U_mu(x) -> G(x) U_mu(x)
G(x+mu)^+, x_i -> G x_i implies y_o -> G y_o.  The network is a stack of layers
(1 -> C -> ... -> C -> 1 channels); with no nonlinearity it is a linear map, and
four layers reach four hops.

Training loss over pairs (eta_k, s_k): sum_k |N(eta_k) - s_k|^2 / |s_k|^2, or the
residual loss sum_k |M N(eta_k) - eta_k|^2 / |eta_k|^2 (no solution needed; it weighs
the error of N by M itself, i.e. every mode of M N - 1 alike).
Gradients use the Wirtinger convention: for a real loss L and complex weight w,
grad(w) = dL/d(conj w) * 2 = 2 sum (conj(input feature) * output gradient), where
the output gradient g = dL/d(conj y) = (y - s) / |s|^2.
"""
from __future__ import annotations

import numpy as np

from . import operator as op
from .lattice import GAMMA, GAMMA5, ID4

NB_LOCAL, NB_HOP = 2, 4


def local_spin(b):
    return [ID4, GAMMA5][b]


def hop_spin(b, mu):
    return [ID4, GAMMA[mu], GAMMA5, GAMMA5 @ GAMMA[mu]][b]


def init_layer(cin, cout, rng, scale=0.1):
    """Random complex weights of one layer: dict of W0 [o,i,2], Wf/Wb [4,o,i,4]."""
    def c(*shape):
        return scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / np.sqrt(2 * cin)
    return {"W0": c(cout, cin, NB_LOCAL), "Wf": c(4, cout, cin, NB_HOP), "Wb": c(4, cout, cin, NB_HOP)}


def transports(links, x, bc=-1.0):
    """Forward and backward parallel transports of channel fields x [C, T,Z,Y,X,4,3]:
    F[mu] = U_mu(x) x(x+mu), Bk[mu] = U_mu(x-mu)^+ x(x-mu)."""
    F = [op.colour(links[..., mu, :, :], op.shift_fwd(x, mu, bc)) for mu in range(4)]
    Bk = [op.colour(op.dagger(op.link_bwd(links, mu)), op.shift_bwd(x, mu, bc)) for mu in range(4)]
    return F, Bk


def layer_forward(links, w, x, bc=-1.0):
    """y [C_out, ...] from x [C_in, ...]: the definition term by term."""
    F, Bk = transports(links, x, bc)
    cout = w["W0"].shape[0]
    y = np.zeros((cout,) + x.shape[1:], dtype=np.complex128)
    for b in range(NB_LOCAL):
        sx = op.spin(local_spin(b), x)
        y += np.einsum("oi,i...->o...", w["W0"][:, :, b], sx)
    for mu in range(4):
        for b in range(NB_HOP):
            h = hop_spin(b, mu)
            y += np.einsum("oi,i...->o...", w["Wf"][mu, :, :, b], op.spin(h, F[mu]))
            y += np.einsum("oi,i...->o...", w["Wb"][mu, :, :, b], op.spin(h, Bk[mu]))
    return y


def _gram(feat, g):
    """2 sum over sites, spin and colour of conj(feat_i) g_o, as an [o, i] matrix."""
    return 2.0 * (g.reshape(g.shape[0], -1) @ np.conj(feat.reshape(feat.shape[0], -1)).T)


def layer_backward(links, w, x, g, bc=-1.0):
    """Given the layer input x and the output gradient g = dL/d(conj y), return
    (gradient of every weight, gradient of the input dL/d(conj x)).

    Weight gradients: grad W[o,i] = 2 sum_x (feature_i)^+ g_o.
    Input gradient: sum_o conj(W) (spin factor)^+ g_o, moved back by the adjoint
    transports: (U_mu(x) .(x+mu))^+ = U_mu(x-mu)^+ .(x-mu) and vice versa."""
    F, Bk = transports(links, x, bc)
    gw = {k: np.zeros_like(v) for k, v in w.items()}
    for b in range(NB_LOCAL):
        sx = op.spin(local_spin(b), x)
        gw["W0"][:, :, b] = _gram(sx, g)
    for mu in range(4):
        for b in range(NB_HOP):
            h = hop_spin(b, mu)
            gw["Wf"][mu, :, :, b] = _gram(op.spin(h, F[mu]), g)
            gw["Wb"][mu, :, :, b] = _gram(op.spin(h, Bk[mu]), g)
    cin = x.shape[0]
    gx = np.zeros((cin,) + x.shape[1:], dtype=np.complex128)
    for b in range(NB_LOCAL):
        m = np.einsum("oi,o...->i...", np.conj(w["W0"][:, :, b]), g)
        gx += op.spin(local_spin(b).conj().T, m)
    for mu in range(4):
        for b in range(NB_HOP):
            hd = hop_spin(b, mu).conj().T
            mf = op.spin(hd, np.einsum("oi,o...->i...", np.conj(w["Wf"][mu, :, :, b]), g))
            mb = op.spin(hd, np.einsum("oi,o...->i...", np.conj(w["Wb"][mu, :, :, b]), g))
            # adjoint of F[mu]: U_mu(x-mu)^+ m(x-mu); adjoint of Bk[mu]: U_mu(x) m(x+mu)
            gx += op.colour(op.dagger(op.link_bwd(links, mu)), op.shift_bwd(mf, mu, bc))
            gx += op.colour(links[..., mu, :, :], op.shift_fwd(mb, mu, bc))
    return gw, gx


def forward(links, weights, eta, bc=-1.0):
    """N(eta) for a single field eta [T,Z,Y,X,4,3]; returns output and layer inputs."""
    x = eta[None]
    inputs = []
    for w in weights:
        inputs.append(x)
        x = layer_forward(links, w, x, bc)
    return x[0], inputs


def loss_and_grads(links, weights, pairs, bc=-1.0):
    """Loss sum_k |N(eta_k) - s_k|^2 / |s_k|^2 and its Wirtinger gradients."""
    total = 0.0
    grads = [{k: np.zeros_like(v) for k, v in w.items()} for w in weights]
    for eta, s in pairs:
        out, inputs = forward(links, weights, eta, bc)
        ns = np.vdot(s, s).real
        d = out - s
        total += np.vdot(d, d).real / ns
        g = (d / ns)[None]
        for li in range(len(weights) - 1, -1, -1):
            gw, g = layer_backward(links, weights[li], inputs[li], g, bc)
            for k in gw:
                grads[li][k] += gw[k]
    return total, grads


def residual_loss_and_grads(links, weights, etas, kappa, amu, f=1, bc=-1.0):
    """Loss sum_k |M_f N(eta_k) - eta_k|^2 / |eta_k|^2 and its Wirtinger gradients.

    With r = M y - eta, y = N(eta), the output gradient is dL/d(conj y) = M^+ r / |eta|^2,
    which the layers propagate back exactly as for the solution loss."""
    total = 0.0
    grads = [{k: np.zeros_like(v) for k, v in w.items()} for w in weights]
    for eta in etas:
        out, inputs = forward(links, weights, eta, bc)
        ne = np.vdot(eta, eta).real
        r = op.apply_m(links, out, kappa, amu, f, bc) - eta
        total += np.vdot(r, r).real / ne
        g = (op.apply_m_dag(links, r, kappa, amu, f, bc) / ne)[None]
        for li in range(len(weights) - 1, -1, -1):
            gw, g = layer_backward(links, weights[li], inputs[li], g, bc)
            for k in gw:
                grads[li][k] += gw[k]
    return total, grads
